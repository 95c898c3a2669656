"""Vertex-position gradient (map refinement) on the GPU vs the CPU oracle, through the C ABI:
vertex by vertex within 1e-3 of the oracle's FP64 gradient (floor 1e-2 of the largest
vertex's, tests/checks.py; FP32 barycentrics and normals), summed over poses, for both camera
models; vertices the oracle leaves at zero are exactly zero."""
from __future__ import annotations

import dataclasses

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
from paper_1702_06813_gb300 import build as rmbuild  # noqa: E402

rmbuild.build()


def _close(g, o, rel=1e-3):
    assert (np.linalg.norm(o, axis=1) > 0).sum() > 100
    checks.close_rows(g, o, rel, "vertex_grad")


def test_vertex_grad_parity_pinhole():
    c = cases.config2(seed=2600, target_fo=40_000, target_fu=10_000)
    cam = dataclasses.replace(c["cam"], width=213, height=161, fx=175.0, fy=175.0, cx=106.5, cy=80.5)
    mesh = c["mesh"]
    sd, sc = synth.synth_scan(mesh, cam, c["gt"], cases.rng(26), sigma_rel=0.005, dropout=0.05)
    om = oracle.OracleMap(mesh.vertices, mesh.faces, mesh.labels)
    gm = rm.Map(mesh.vertices, mesh.faces, mesh.labels)
    scan = rm.Scan.make(rm.Intrinsics.from_camera(cam), sd, sc)
    poses = [c["start"], synth.perturb_fixed(c["gt"], cases.rng(27), 0.05, 2.0)]
    og = [om.vertex_grad(P, cam, sd, sc) for P in poses]
    for k, P in enumerate(poses):
        _close(rm.cost_grad_vertices(gm, scan, P[None]).cpu().numpy(), og[k])
    both = rm.cost_grad_vertices(gm, scan, np.stack(poses)).cpu().numpy()
    _close(both, og[0] + og[1])
    # host output through the ABI
    import ctypes
    from paper_1702_06813_gb300 import _native as N
    h = np.empty((mesh.vertices.shape[0], 3))
    pz = np.ascontiguousarray(poses[0], np.float64)
    st = N.lib().rm_cost_grad_vertices(gm.handle, ctypes.byref(scan.c()), pz.ctypes.data, 1,
                                       ctypes.byref(rm.cost_params()), h.ctypes.data, None)
    assert st == N.RM_OK
    _close(h, og[0])
    gm.close()


def test_vertex_grad_parity_raytable():
    w = synth.workload_lidar(seed=4400, target_fo=80_000, target_fu=30_000, n_panels=40)
    mesh, cam = w["mesh"], w["cam"]
    sd, sc = w["scan"]
    om = oracle.OracleMap(mesh.vertices, mesh.faces, mesh.labels)
    gm = rm.Map(mesh.vertices, mesh.faces, mesh.labels)
    scan = rm.Scan.make(rm.Intrinsics.from_camera(cam), sd, sc)
    _close(rm.cost_grad_vertices(gm, scan, w["start"][None]).cpu().numpy(),
           om.vertex_grad(w["start"], cam, sd, sc))
    gm.close()


def test_vertex_grad_sums_to_minus_pose_translation_gradient():
    """The GPU's own vertex and pose gradients satisfy the translation identity."""
    c = cases.config1(seed=2003)
    gm = rm.Map(c["mesh"].vertices, c["mesh"].faces, c["mesh"].labels)
    scan = rm.Scan.make(rm.Intrinsics.from_camera(c["cam"]), *c["scan"])
    g = rm.cost_grad_vertices(gm, scan, c["start"][None]).cpu().numpy()
    gp = rm.cost_grad(gm, scan, c["start"][None])["grad"].cpu().numpy()[0]
    want = -c["start"][:3, :3] @ gp[:3]
    assert np.linalg.norm(g.sum(0) - want) <= 2e-3 * np.linalg.norm(want)
    gm.close()
