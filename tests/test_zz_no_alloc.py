"""rm_cost_grad_noalloc: the allocation-free variant of rm_cost_grad.

It serves callers that must not allocate device memory while they evaluate poses (a real-time
loop that may not enter the allocator after start-up, a memory manager that owns the device,
a fixed memory budget): all its scratch comes from a fixed array inside the library. Here it
is called through the C ABI twice in a row, on two different poses, and each result is checked
against rm_cost_grad on the same inputs with the tolerances of the parity tests (Table I counts
exact, least-squares cost 1e-5 relative, gradient and Gauss-Newton matrix 1e-3 relative). The
second call also checks that free device memory does not change across it.

Collected last (file name) so that a run stopping at the first failure has run the rest.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

import cases
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - the gpu marker is deselected on CPU
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1702_06813_gb300 as rm  # noqa: E402
from paper_1702_06813_gb300 import _native as N  # noqa: E402
from paper_1702_06813_gb300 import build as rmbuild  # noqa: E402

rmbuild.build()


def test_noalloc_matches_cost_grad_on_two_calls_in_a_row():
    c = cases.config1(seed=1000)
    gm = rm.Map(c["mesh"].vertices, c["mesh"].faces, c["mesh"].labels)
    intr = rm.Intrinsics.from_camera(c["cam"])
    scan = rm.Scan.make(intr, *c["scan"])
    poses = [c["start"], synth.perturb_fixed(c["gt"], cases.rng(7), 0.1, 3.0)]
    prm = rm.cost_params()
    cs = scan.c()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    free_between = []
    for k, pose in enumerate(poses):
        counts = torch.full((1, 6), -1, dtype=torch.int64, device="cuda")
        etab = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        els = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        grad = torch.full((1, 6), -1.0, dtype=torch.float64, device="cuda")
        jtj = torch.full((1, 21), -1.0, dtype=torch.float64, device="cuda")
        dpose = torch.as_tensor(pose.reshape(16), dtype=torch.float64, device="cuda")
        out = N.rm_cost_out(counts.data_ptr(), etab.data_ptr(), els.data_ptr(), grad.data_ptr(),
                            jtj.data_ptr())
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        st = N.lib().rm_cost_grad_noalloc(gm.handle, ctypes.byref(cs),
                                          ctypes.c_void_p(dpose.data_ptr()), ctypes.byref(prm),
                                          ctypes.byref(out), stream)
        N.check(st)
        torch.cuda.synchronize()
        free_between.append((free_before, torch.cuda.mem_get_info()[0]))
        ref = rm.cost_grad(gm, scan, pose[None], prm)
        assert torch.equal(counts.cpu(), ref["counts"].cpu()), k
        assert int(etab.item()) == int(ref["e_table"].item())
        e, er = float(els.item()), float(ref["e_ls"].item())
        assert abs(e - er) <= 1e-5 * abs(er)
        g, gr = grad.cpu().numpy()[0], ref["grad"].cpu().numpy()[0]
        assert np.linalg.norm(g - gr) <= 1e-3 * np.linalg.norm(gr)
        h, hr = jtj.cpu().numpy()[0], ref["jtj"].cpu().numpy()[0]
        assert np.linalg.norm(h - hr) <= 1e-3 * np.linalg.norm(hr)
    # the first call may load the library's module on this device; the second allocates nothing
    assert free_between[1][0] == free_between[1][1]
    gm.close()


def test_noalloc_rejects_host_outputs():
    c = cases.config1(seed=1000)
    gm = rm.Map(c["mesh"].vertices, c["mesh"].faces, c["mesh"].labels)
    scan = rm.Scan.make(rm.Intrinsics.from_camera(c["cam"]), *c["scan"])
    host = np.zeros(1)
    out = N.rm_cost_out(None, None, host.ctypes.data, None, None)
    pose = np.ascontiguousarray(c["start"].reshape(16))
    cs = scan.c()
    prm = rm.cost_params()
    st = N.lib().rm_cost_grad_noalloc(gm.handle, ctypes.byref(cs), pose.ctypes.data_as(ctypes.c_void_p),
                                      ctypes.byref(prm), ctypes.byref(out), None)
    assert st == N.RM_EINVAL
    assert b"device" in N.lib().rm_last_error()
    gm.close()
