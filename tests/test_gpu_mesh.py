"""Meshification of range images (Sec. IV.A) on the GPU vs the CPU oracle, and scan-to-scan
alignment against the mesh of a previous scan (Sec. V), through the C ABI.

Vertices, faces and labels must match the oracle bit for bit (the label decision is taken in
FP32 with the same operation order on both sides; the world transform in FP64, rounded once).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import cases
import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - the gpu marker is deselected on CPU
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1702_06813_gb300 as rm  # noqa: E402
from paper_1702_06813_gb300 import build as rmbuild  # noqa: E402

rmbuild.build()


def _np(t):
    return t.detach().cpu().numpy()


def _same_mesh(g, o):
    v, f, lab = o
    assert np.array_equal(_np(g["vertices"]).view(np.uint32), v.view(np.uint32))
    assert np.array_equal(_np(g["faces"]), f)
    assert np.array_equal(_np(g["labels"]), lab)


def _room_scans():
    c = cases.config2(seed=2500, target_fo=40_000, target_fu=10_000)
    cam = dataclasses.replace(c["cam"], width=213, height=161, fx=175.0, fy=175.0, cx=106.5, cy=80.5)
    r = cases.rng(25)
    out = []
    for k in range(2):
        pose = c["gt"] if k == 0 else synth.perturb_fixed(c["gt"], r, 0.2, 5.0)
        d, cl = synth.synth_scan(c["mesh"], cam, pose, r, sigma_rel=0.005, dropout=0.05, dropout_as_nan=(k == 1))
        out.append((pose, d, cl))
    return cam, out


@pytest.mark.parametrize("step", [1, 2, 3])
@pytest.mark.parametrize("max_edge", [0.1, 0.03])
def test_meshify_bit_exact_pinhole(step, max_edge):
    cam, scans = _room_scans()
    intr = rm.Intrinsics.from_camera(cam)
    fu_total = 0
    for pose, d, cl in scans:
        g = rm.meshify(rm.Scan.make(intr, d, cl), pose, max_range=cam.range_max, max_edge=max_edge, step=step)
        o = oracle.meshify(cam, d, cl, pose, cam.range_max, max_edge, step)
        _same_mesh(g, o)
        fu_total += int(o[2].sum())
    assert fu_total > 0


def test_meshify_bit_exact_raytable():
    w = synth.workload_lidar(seed=4200, target_fo=60_000, target_fu=20_000, n_panels=40)
    cam = w["cam"]
    d, cl = w["scan"]
    g = rm.meshify(rm.Scan.make(rm.Intrinsics.from_camera(cam), d, cl), w["gt"], max_range=cam.range_max,
                   max_edge=0.5)
    _same_mesh(g, oracle.meshify(cam, d, cl, w["gt"], cam.range_max, 0.5, 1))


def test_meshify_edge_cases_and_host_buffers():
    import ctypes
    from paper_1702_06813_gb300 import _native as N
    # a one-pixel-wide image has no 2x2 block
    cam = cases.small_pinhole(w=1, h=9)
    intr = rm.Intrinsics.from_camera(cam)
    g = rm.meshify(rm.Scan.make(intr, np.ones((9, 1), np.float32), np.zeros((9, 1), np.uint8)), np.eye(4), 4.0)
    assert g["faces"].shape == (0, 3) and g["vertices"].shape == (9, 3)
    # every pixel dead
    cam = cases.small_pinhole(w=17, h=11)
    intr = rm.Intrinsics.from_camera(cam)
    dead = np.full((11, 17), np.nan, np.float32)
    g = rm.meshify(rm.Scan.make(intr, dead, np.zeros((11, 17), np.uint8)), np.eye(4), 4.0)
    assert g["faces"].shape[0] == 0
    # host arrays in and out through the ABI
    cam, scans = _room_scans()
    pose, d, cl = scans[1]
    intr = rm.Intrinsics.from_camera(cam)
    d = np.ascontiguousarray(d, np.float32)
    cl = np.ascontiguousarray(cl, np.uint8)
    cs = N.rm_scan(intr.c(), d.ctypes.data, cl.ctypes.data)
    v = np.empty((cam.width * cam.height, 3), np.float32)
    cap = 2 * (cam.width - 1) * (cam.height - 1)
    f = np.empty((cap, 3), np.int32)
    lab = np.empty(cap, np.uint8)
    nf = ctypes.c_int64()
    pz = np.ascontiguousarray(pose, np.float64)
    prm = N.rm_meshify_params(cam.range_max, 0.1, 1, 0)
    st = N.lib().rm_meshify(ctypes.byref(cs), pz.ctypes.data, ctypes.byref(prm), v.ctypes.data, f.ctypes.data,
                            lab.ctypes.data, ctypes.byref(nf), None)
    assert st == N.RM_OK
    o = oracle.meshify(cam, d, cl, pose, cam.range_max, 0.1, 1)
    assert np.array_equal(v.view(np.uint32), o[0].view(np.uint32))
    assert np.array_equal(f[:nf.value], o[1]) and np.array_equal(lab[:nf.value], o[2])
    # bad parameters
    with pytest.raises(rm.RenderMapError):
        rm.meshify(rm.Scan.make(intr, d, cl), pose, max_range=-1.0)
    with pytest.raises(rm.RenderMapError):
        rm.meshify(rm.Scan.make(intr, d, cl), pose, max_range=4.0, step=0)


def _gap(P, Q):
    return (float(np.linalg.norm(P[:3, 3] - Q[:3, 3])),
            math.degrees(Rotation.from_matrix(P[:3, :3].T @ Q[:3, :3]).magnitude()))


def test_scan_to_scan_alignment():
    """Scan A meshed on the GPU becomes the map; scan B, taken 5 cm / 2 deg away, is aligned
    to it from A's pose by point-to-plane ICP (and by LM on the Table I surrogate), matching
    the oracle's run on the oracle's mesh."""
    c = cases.config1(seed=1800)
    mesh, cam = c["mesh"], c["cam"]
    r = cases.rng(5)
    A = synth.pose_from(c["gt"][:3, 3], 3.5, math.radians(35.0), 0.0)
    B = synth.perturb_fixed(A, r, 0.05, 2.0)
    sA = synth.synth_scan(mesh, cam, A, r, sigma_abs=0.005)
    sB = synth.synth_scan(mesh, cam, B, r, sigma_abs=0.005)
    intr = rm.Intrinsics.from_camera(cam)
    g = rm.meshify(rm.Scan.make(intr, *sA), A, max_range=cam.range_max)
    o = oracle.meshify(cam, sA[0], sA[1], A, cam.range_max, 0.1, 1)
    _same_mesh(g, o)
    gm = rm.Map(g["vertices"], g["faces"], g["labels"])
    om = oracle.OracleMap(*o)
    scanB = rm.Scan.make(intr, *sB)
    pg, rep = rm.icp_align(gm, scanB, A, tol=0.2, max_iters=30, step_tol=1e-5)
    po, orep = om.icp_align(A, cam, sB[0], sB[1], 0.2, 30, 1e-5)
    assert rep["converged"] == 1 and orep["converged"] == 1, (rep, orep)
    dt, da = _gap(pg, po)
    assert dt < 1e-4 and da < 2e-3, (dt, da)
    dt, da = _gap(pg, B)
    assert dt < 2e-3 and da < 0.05, (dt, da)
    pl, lrep = rm.align(gm, scanB, A, max_iters=50, step_tol=1e-7)
    dt, da = _gap(pl, B)
    assert dt < 0.02 and da < 0.3, (dt, da, lrep)
    gm.close()


def test_sequential_depth_image_alignment():
    """Sec. V's loop over a short trajectory: each scan meshed (downsampled by 2) at its
    estimated pose is the map for the next scan's ICP. Frames 1-3 move 4 cm / 1.5 deg each;
    the chained estimates stay within a few millimetres of the truth."""
    c = cases.config1(seed=1800)
    mesh, cam = c["mesh"], c["cam"]
    r = cases.rng(9)
    truth = [synth.pose_from(c["gt"][:3, 3], 3.5, math.radians(35.0), 0.0)]
    for _ in range(3):
        truth.append(synth.perturb_fixed(truth[-1], r, 0.04, 1.5))
    intr = rm.Intrinsics.from_camera(cam)
    scans = [rm.Scan.make(intr, *synth.synth_scan(mesh, cam, T, r, sigma_abs=0.003)) for T in truth]
    est, reps = rm.sequential_icp(scans, truth[0], max_range=cam.range_max, step=2)
    assert est.shape == (4, 4, 4) and len(reps) == 3
    for k in range(1, 4):
        dt, da = _gap(est[k], truth[k])
        assert dt < 0.01 and da < 0.3, (k, dt, da, reps[k - 1])
