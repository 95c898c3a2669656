"""Parity at full size: the benchmark's workload in its launch configuration, and the
2M-triangle panoramic (ray-table) workload.

The 1M-triangle 640x480 room with 256 candidate poses, evaluated as the benchmark does (64x32
tiles, two waves of 128 poses), is checked against the oracle on every pose: Table I counts
exact, E_ls within 1e-5 relative, gradient and Gauss-Newton matrix within 1e-3 element by
element (tests/checks.py); the same for the ICP terms; the whole z-buffer of the first and last
pose of each wave bit for bit; and the persistent batch kernel on the same 256 poses equal to
the waves.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import checks
import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - the gpu marker is deselected on CPU
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1702_06813_gb300 as rm  # noqa: E402
from paper_1702_06813_gb300 import build as rmbuild  # noqa: E402

rmbuild.build()

EPS_REL_COST = 1e-5
EPS_REL_GRAD = 1e-3
SAMPLED = (0, 127, 128, 255)  # first and last pose of each 128-pose wave
POOL = ThreadPoolExecutor(max_workers=os.cpu_count() or 4)  # the oracle's C calls drop the GIL


def _np(t):
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module")
def head():
    w = synth.workload_headline(3000, 256)
    mesh, cam = w["mesh"], w["cam"]
    gm = rm.Map(mesh.vertices, mesh.faces, mesh.labels)
    gm.set_tuning(tile=(64, 32), wave_poses=128)
    om = oracle.OracleMap(mesh.vertices, mesh.faces, mesh.labels)
    intr = rm.Intrinsics.from_camera(cam)
    scan = rm.Scan.make(intr, *w["scan"])
    poses = torch.as_tensor(w["poses"].reshape(-1, 16), dtype=torch.float64, device="cuda")
    yield dict(w=w, gm=gm, om=om, intr=intr, scan=scan, poses=poses)
    gm.close()


def test_fullsize_cost_grad_all_poses(head):
    w = head["w"]
    g = rm.cost_grad(head["gm"], head["scan"], head["poses"])
    assert g["counts"].shape == (256, 6)
    o = head["om"].cost_batch(w["poses"], w["cam"], *w["scan"])
    counts, etab, els = _np(g["counts"]), _np(g["e_table"]), _np(g["e_ls"])
    for k in range(256):
        assert np.array_equal(counts[k], o["counts"][k]), k
        c = o["counts"][k]
        assert int(etab[k]) == int(c[1] + c[3] + c[5] - c[0] - c[2] - c[4]), k
        assert abs(float(els[k]) - o["e_ls"][k]) <= EPS_REL_COST * abs(o["e_ls"][k]), k
        checks.close_elementwise(_np(g["grad"])[k], o["grad"][k], EPS_REL_GRAD, f"head_grad[{k}]")
        checks.close_elementwise(_np(g["jtj"])[k], o["jtj"][k], EPS_REL_GRAD, f"head_jtj[{k}]")
    # the poses exercise the least-squares path on most pixels
    assert counts[:, :2].sum() > 0.5 * counts.sum()


def test_fullsize_render_bit_exact(head):
    w = head["w"]
    sel = list(SAMPLED)
    r = rm.render_depth(head["gm"], head["poses"][sel], head["intr"])
    for i, k in enumerate(sel):
        o = head["om"].render(w["poses"][k], w["cam"])
        ids, depth = _np(r["tri_id"][i]), _np(r["depth"][i])
        assert np.array_equal(ids, o["tri_id"]), f"{np.sum(ids != o['tri_id'])} pixels differ"
        hit = ~np.isnan(o["depth"])
        assert np.array_equal(np.isnan(depth), ~hit)
        assert np.array_equal(depth[hit].view(np.uint32), o["depth"][hit].view(np.uint32))


def test_fullsize_persistent_equals_waves(head):
    g = rm.cost_grad(head["gm"], head["scan"], head["poses"])
    b = rm.cost_grad_batch(head["gm"], scans=head["scan"], poses=head["poses"])
    for key in ("counts", "e_table", "e_ls", "grad", "jtj"):
        assert torch.equal(g[key], b[key]), key


def test_fullsize_lidar_render_and_cost():
    """The 2M-triangle terrain seen by the 1024x64 panoramic sensor (ray-table model) at its
    full size: the z-buffer at the true pose bit for bit, cost and gradient at the start pose
    (30 cm / 3 deg off) within the parity tolerances."""
    w = synth.workload_lidar()
    mesh, cam = w["mesh"], w["cam"]
    gm = rm.Map(mesh.vertices, mesh.faces, mesh.labels)
    om = oracle.OracleMap(mesh.vertices, mesh.faces, mesh.labels)
    intr = rm.Intrinsics.from_camera(cam)
    scan = rm.Scan.make(intr, *w["scan"])
    r = rm.render_depth(gm, w["gt"][None], intr)
    o = om.render(w["gt"], cam)
    ids, depth = _np(r["tri_id"][0]), _np(r["depth"][0])
    assert np.array_equal(ids, o["tri_id"]), f"{np.sum(ids != o['tri_id'])} pixels differ"
    hit = ~np.isnan(o["depth"])
    assert np.array_equal(depth[hit].view(np.uint32), o["depth"][hit].view(np.uint32))
    g = rm.cost_grad(gm, scan, w["start"][None])
    oc = om.cost(w["start"], cam, *w["scan"])
    assert np.array_equal(_np(g["counts"])[0], oc["counts"])
    assert abs(float(_np(g["e_ls"])[0]) - oc["e_ls"]) <= EPS_REL_COST * abs(oc["e_ls"])
    checks.close_elementwise(_np(g["grad"])[0], oc["grad"], EPS_REL_GRAD, "lidar2M_grad")
    checks.close_elementwise(_np(g["jtj"])[0], oc["jtj"], EPS_REL_GRAD, "lidar2M_jtj")
    gm.close()


def test_fullsize_icp_terms_all_poses(head):
    """ICP terms of the 256 poses in the benchmark's launch configuration (64x32 tiles, two
    128-pose waves), every pose against the oracle: association counts exact, sums within the
    ICP parity tolerances, J^T e and J^T J element by element."""
    w = head["w"]
    g = rm.icp_terms(head["gm"], head["scan"], head["poses"], tol=0.1)
    outs = list(POOL.map(lambda k: head["om"].icp_terms(w["poses"][k], w["cam"], *w["scan"], 0.1), range(256)))
    for k, o in enumerate(outs):
        assert int(_np(g["n_assoc"])[k]) == o["n_assoc"], k
        for key in ("cost_l1", "e2"):
            assert abs(float(_np(g[key])[k]) - o[key]) <= 1e-5 * abs(o[key]), (k, key)
        checks.close_elementwise(_np(g["jte"])[k], o["jte"], 1e-3, f"head_icp_jte[{k}]")
        checks.close_elementwise(_np(g["jtj"])[k], o["jtj"], 1e-4, f"head_icp_jtj[{k}]")
    # poses far off the true one may associate nothing at this tolerance; most associate
    assert sum(o["n_assoc"] > 1000 for o in outs) > 200


def test_fullsize_dfo_same_search_as_oracle(head):
    """The derivative-free search on the full-size room from 3 cm / 1.5 deg (the benchmark's
    start): the same scored poses, iterations and final Table I cost as the oracle's search."""
    w = head["w"]
    r = np.random.Generator(np.random.PCG64(3000 + 9))
    start = synth.perturb_fixed(w["gt"], r, 0.03, 1.5)
    pg, rep = rm.dfo_align(head["gm"], head["scan"], start, dfo=rm.dfo_params(nm_iters=60, cd_iters=40))
    po, orep = head["om"].dfo_align(start, w["cam"], *w["scan"], dfo=oracle.dfo_params(nm_iters=60, cd_iters=40))
    for key in ("evals", "nm_iters", "nm_shrinks", "cd_iters", "converged"):
        assert rep[key] == orep[key], (key, rep, orep)
    assert rep["e_table_final"] == orep["e_table"]
    assert np.allclose(pg, po, rtol=0, atol=1e-9)
