"""The autotuner (tile, poses per wave, initial bin capacity) on the GPU.

Whatever it picks, the Table I counts stay bit-exact against the oracle and the cost and
gradient within the parity tolerances; the pick is applied to the map, cached under its key,
and re-applied from the cache without timing. A capacity smaller than the busiest bin is grown
by the library in the untimed warm-up, so the recorded capacity is one that ran.
"""
from __future__ import annotations

import json

import numpy as np
import pytest

import cases
import checks
import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - the gpu marker is deselected on CPU
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1702_06813_gb300 as rm  # noqa: E402
from paper_1702_06813_gb300 import autotune  # noqa: E402
from paper_1702_06813_gb300 import build as rmbuild  # noqa: E402

rmbuild.build()


def _np(t):
    return t.detach().cpu().numpy()


def test_autotune_picks_caches_and_keeps_parity(tmp_path):
    c = cases.config1(seed=1400)
    mesh, cam = c["mesh"], c["cam"]
    r = cases.rng(41)
    poses = np.concatenate([np.stack([c["gt"], c["start"]]), synth.perturb_gauss(c["gt"], r, 0.1, 5.0, 6)])
    gm = rm.Map(mesh.vertices, mesh.faces, mesh.labels)
    try:
        scan = rm.Scan.make(rm.Intrinsics.from_camera(cam), *c["scan"])
        cache = str(tmp_path / "tune.json")
        best = autotune.autotune(gm, scan, poses, tiles=((32, 32), (16, 16)), waves=(4, 8),
                                 capacities=(8, 256), reps=1, cache=cache)
        cands = best["candidates"]
        assert len(cands) == 2 * 2 + 2
        assert {k["bin_capacity"] >= 8 for k in cands} == {True}
        # the 8-record start cannot hold the busiest bins of this view: the library grew it
        assert cands[4]["bin_capacity"] > 8
        t = gm.get_tuning()
        assert list(t["tile"]) == best["tile"] and t["wave_poses"] == best["wave_poses"]
        assert t["bin_capacity"] == best["bin_capacity"]
        with open(cache) as fh:
            table = json.load(fh)
        assert len(table) == 1 and next(iter(table.values()))["ms"] == best["ms"]
        # cached: applied again without timing
        gm.set_tuning(tile=(64, 32), wave_poses=1)
        again = autotune.autotune(gm, scan, poses, cache=cache)
        assert "candidates" not in again
        assert list(gm.get_tuning()["tile"]) == best["tile"]
        out = rm.cost_grad(gm, scan, poses)
        om = oracle.OracleMap(mesh.vertices, mesh.faces, mesh.labels)
        sd, sc = c["scan"]
        for k in range(len(poses)):
            o = om.cost(poses[k], cam, sd, sc)
            assert np.array_equal(_np(out["counts"])[k], o["counts"]), k
            e = float(_np(out["e_ls"])[k])
            assert abs(e - o["e_ls"]) <= 1e-5 * abs(o["e_ls"]) + 1e-12, k
            checks.close_elementwise(_np(out["grad"])[k], o["grad"], 1e-3, f"tuned_grad[{k}]", floor=1e-9)
    finally:
        gm.close()
