"""Bounded device waits return a status, through the C ABI.

Every wait in the kernels (a bulk copy's mbarrier, the batch kernel's work queue) gives up
after a cycle budget and sets a bit that the host turns into RM_ETIMEOUT; nothing traps or
hangs. The tuning field wait_log2 shortens that budget to 2^wait_log2 cycles. With 16
cycles the first wait on any bulk copy, and any idle wait for work in the batch kernel, runs
out (a short budget polls the barrier with non-blocking tests, so that the budget, not the
hardware's suspend window, bounds the wait); a copy still in flight is drained with the
default budget before its block leaves. The call must return RM_ETIMEOUT, and the next call
with the default budget must succeed and give the same numbers as before.
"""
from __future__ import annotations

import pytest

import cases
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - the gpu marker is deselected on CPU
    pytest.skip("no CUDA device", allow_module_level=True)

import numpy as np  # noqa: E402

import paper_1702_06813_gb300 as rm  # noqa: E402
from paper_1702_06813_gb300 import _native as N  # noqa: E402
from paper_1702_06813_gb300 import build as rmbuild  # noqa: E402

rmbuild.build()


@pytest.fixture(scope="module")
def c1():
    c = cases.config1(seed=1000)
    gm = rm.Map(c["mesh"].vertices, c["mesh"].faces, c["mesh"].labels)
    scan = rm.Scan.make(rm.Intrinsics.from_camera(c["cam"]), *c["scan"])
    r = cases.rng(77)
    poses = np.stack([c["start"]] + [synth.perturb_fixed(c["gt"], r, 0.1, 3.0) for _ in range(3)])
    yield dict(c, gm=gm, scan=scan, poses=poses)
    gm.close()


def _same(a, b):
    for key in ("counts", "e_table", "e_ls", "grad", "jtj"):
        assert torch.equal(a[key], b[key]), key


def _timed_out(gm, fn):
    """fn() under a 16-cycle wait budget must fail with RM_ETIMEOUT; the budget is restored
    whatever happens."""
    gm.set_tuning(wait_log2=4)
    try:
        assert gm.get_tuning()["wait_log2"] == 4
        with pytest.raises(N.RenderMapError) as e:
            fn()
        assert e.value.status == N.RM_ETIMEOUT, e.value
    finally:
        gm.set_tuning()


def test_wave_wait_runs_out_then_recovers(c1):
    gm = c1["gm"]
    before = rm.cost_grad(gm, c1["scan"], c1["poses"])
    _timed_out(gm, lambda: rm.cost_grad(gm, c1["scan"], c1["poses"]))
    _same(rm.cost_grad(gm, c1["scan"], c1["poses"]), before)


def test_batch_kernel_wait_runs_out_then_recovers(c1):
    gm = c1["gm"]
    poses = torch.as_tensor(c1["poses"].reshape(-1, 16), dtype=torch.float64, device="cuda")
    before = rm.cost_grad_batch(gm, scans=c1["scan"], poses=poses)
    _timed_out(gm, lambda: rm.cost_grad_batch(gm, scans=c1["scan"], poses=poses))
    _same(rm.cost_grad_batch(gm, scans=c1["scan"], poses=poses), before)
    # and the LM batch after a timed-out one
    _timed_out(gm, lambda: rm.align_batch(gm, [(c1["scan"], c1["start"])], max_iters=3))
    p1, _, st = rm.align_batch(gm, [(c1["scan"], c1["start"])], max_iters=3)
    p2, _ = rm.align(gm, c1["scan"], c1["start"], max_iters=3)
    assert np.array_equal(p1[0], p2)


def test_single_pose_loop_wait_runs_out_then_recovers(c1):
    gm = c1["gm"]
    before = rm.align(gm, c1["scan"], c1["start"], max_iters=3)[0]
    _timed_out(gm, lambda: rm.align(gm, c1["scan"], c1["start"], max_iters=3))
    assert np.array_equal(rm.align(gm, c1["scan"], c1["start"], max_iters=3)[0], before)


def test_wait_log2_is_checked(c1):
    try:
        with pytest.raises(N.RenderMapError):
            c1["gm"].set_tuning(wait_log2=41)
        with pytest.raises(N.RenderMapError):
            c1["gm"].set_tuning(wait_log2=-1)
    finally:
        c1["gm"].set_tuning()
