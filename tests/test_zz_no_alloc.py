"""rm_cost_grad_noalloc: the allocation-free variant of rm_cost_grad.

It serves callers that must not allocate device memory while they evaluate poses (a real-time
loop that may not enter the allocator after start-up, a memory manager that owns the device,
a fixed memory budget): all its scratch comes from a fixed array inside the library. Here it
is called through the C ABI twice in a row, on two different poses, and each result must
equal rm_cost_grad's on the same inputs bit for bit: both run the same kernels, and the
results do not depend on the bins' capacity or record order. The first pose is also checked
against the oracle with the parity tests' tolerances. Around the second call neither this
process's allocator (torch's reserved bytes) nor the device's free memory changes. The
benchmark's full-size room (1M triangles, 640x480) is checked the same way.

Collected last (file name) so that a run stopping at the first failure has run the rest.
"""
from __future__ import annotations

import ctypes

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
from paper_1702_06813_gb300 import _native as N  # noqa: E402
from paper_1702_06813_gb300 import build as rmbuild  # noqa: E402

rmbuild.build()


def _two_calls(mesh, cam, scan_np, poses):
    gm = rm.Map(mesh.vertices, mesh.faces, mesh.labels)
    intr = rm.Intrinsics.from_camera(cam)
    scan = rm.Scan.make(intr, *scan_np)
    prm = rm.cost_params()
    cs = scan.c()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    results = []
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
        reserved0 = torch.cuda.memory_reserved()
        free0 = torch.cuda.mem_get_info()[0]
        st = N.lib().rm_cost_grad_noalloc(gm.handle, ctypes.byref(cs),
                                          ctypes.c_void_p(dpose.data_ptr()), ctypes.byref(prm),
                                          ctypes.byref(out), stream)
        N.check(st)
        torch.cuda.synchronize()
        reserved1 = torch.cuda.memory_reserved()
        free1 = torch.cuda.mem_get_info()[0]
        ref = rm.cost_grad(gm, scan, pose[None], prm)
        got = {"counts": counts, "e_table": etab, "e_ls": els, "grad": grad, "jtj": jtj}
        for key in got:
            assert torch.equal(got[key], ref[key]), (k, key)
        results.append(({key: v.cpu().numpy()[0] for key, v in got.items()}, (reserved0, reserved1),
                        (free0, free1)))
    # the first call may load the library's module on this device; the second allocates nothing
    assert results[1][1][0] == results[1][1][1]
    assert results[1][2][0] == results[1][2][1]
    gm.close()
    return results


def _against_oracle(mesh, cam, scan_np, pose, got):
    om = oracle.OracleMap(mesh.vertices, mesh.faces, mesh.labels)
    o = om.cost(pose, cam, *scan_np)
    assert np.array_equal(got["counts"], o["counts"])
    assert int(got["e_table"]) == o["e_table"]
    assert abs(float(got["e_ls"]) - o["e_ls"]) <= 1e-5 * abs(o["e_ls"])
    checks.close_elementwise(got["grad"], o["grad"], 1e-3, "noalloc_grad")
    checks.close_elementwise(got["jtj"], o["jtj"], 1e-3, "noalloc_jtj")


def test_noalloc_matches_cost_grad_on_two_calls_in_a_row():
    c = cases.config1(seed=1000)
    poses = [c["start"], synth.perturb_fixed(c["gt"], cases.rng(7), 0.1, 3.0)]
    res = _two_calls(c["mesh"], c["cam"], c["scan"], poses)
    _against_oracle(c["mesh"], c["cam"], c["scan"], poses[0], res[0][0])


def test_noalloc_full_size_room():
    w = synth.workload_headline(3000, 2)
    res = _two_calls(w["mesh"], w["cam"], w["scan"], [w["poses"][0], w["poses"][1]])
    _against_oracle(w["mesh"], w["cam"], w["scan"], w["poses"][1], res[1][0])


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
