"""Pins of the oracle's render-accelerated point-to-plane ICP (Sec. V) to things other than
itself (no GPU needed).

The association is projective: the map surface rendered at a pixel and the scan return of the
same pixel form a pair when both are occupied (FO) and their depths differ by less than the
tolerance. The residual is the distance of the scan point from the map surface's plane, and the
terms are J^T e and J^T J for the right-perturbation twist (rho, phi) of the camera pose.

Pins: closed forms for a fronto-parallel wall (count, C, residuals, every entry of J^T e and
J^T J), the association rules (strict tolerance, map labels, scan classes), finite differences
of the frozen point-to-plane cost (J^T e on noisy scans, J^T J where the residuals vanish) for
both camera models, and convergence of the alignment to the true pose on noise-free scans.
"""
from __future__ import annotations

import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import cases
import oracle
import synth


def packed(a, b):
    a, b = min(a, b), max(a, b)
    return 6 * a - a * (a - 1) // 2 + (b - a)


def _wall(labels=0, D=2.0):
    cam = cases.small_pinhole(w=32, h=24, f=30.0)
    v, f = cases.plane_grid(5, 5, (-20, -20, D), (40, 0, 0), (0, 40, 0))
    lab = np.full(len(f), labels, np.uint8) if np.isscalar(labels) else np.asarray(labels, np.uint8)
    return cam, oracle.OracleMap(v, f, lab)


def _pinhole_rays(cam):
    """Pixel-centre rays of a pinhole camera with unit z (the FP32 intrinsics widened)."""
    i = np.arange(cam.width, dtype=np.float64) + 0.5
    j = np.arange(cam.height, dtype=np.float64) + 0.5
    I, J = np.meshgrid(i, j)
    x = (I - np.float64(np.float32(cam.cx))) / np.float64(np.float32(cam.fx))
    y = (J - np.float64(np.float32(cam.cy))) / np.float64(np.float32(cam.fy))
    return x, y


@pytest.mark.parametrize("delta", [0.03, -0.045])
def test_icp_wall_closed_form(delta):
    """Camera facing a wall at 2 m, scan at 2 m + delta. With n = (0, 0, +-1) and r = (x, y, 1)
    the residual is the depth difference, and J = +-(0, 0, 1, p_y, -p_x, 0) with p the scan
    point, so every entry of J^T e and J^T J is a plain sum over the pixel grid."""
    cam, om = _wall()
    sd = np.full((cam.height, cam.width), 2.0 + delta, np.float32)
    sc = np.zeros_like(sd, np.uint8)
    out = om.icp_terms(np.eye(4), cam, sd, sc, tol=0.1)
    t = om.render(np.eye(4), cam)["depth"].astype(np.float64)   # within 2 ulp of 2 m
    assert np.all(np.abs(t - 2.0) <= 2 * np.spacing(np.float32(2.0)))
    d = np.float64(np.float32(2.0 + delta))
    N = cam.width * cam.height
    x, y = _pinhole_rays(cam)
    px, py = d * x, d * y
    dz = d - t
    assert out["n_assoc"] == N
    assert out["cost_l1"] == pytest.approx(np.sum(np.abs(dz)), rel=1e-12)
    assert out["e2"] == pytest.approx(np.sum(dz * dz), rel=1e-12)
    jte = np.array([0.0, 0.0, np.sum(dz), np.sum(dz * py), -np.sum(dz * px), 0.0])
    assert np.allclose(out["jte"], jte, rtol=1e-12, atol=1e-9 * np.abs(jte).max())
    H = np.zeros((6, 6))
    H[2, 2] = N
    H[2, 3] = H[3, 2] = np.sum(py)
    H[2, 4] = H[4, 2] = -np.sum(px)
    H[3, 3] = np.sum(py * py)
    H[4, 4] = np.sum(px * px)
    H[3, 4] = H[4, 3] = -np.sum(px * py)
    for a in range(6):
        for b in range(a, 6):
            assert out["jtj"][packed(a, b)] == pytest.approx(H[a, b], rel=1e-12, abs=1e-9 * N), (a, b)


def test_icp_association_rules():
    cam, om = _wall()
    eye = np.eye(4)
    t = om.render(eye, cam)["depth"]
    sc = np.zeros(t.shape, np.uint8)
    # beyond the tolerance: nothing associated
    out = om.icp_terms(eye, cam, np.full(t.shape, 2.15, np.float32), sc, tol=0.1)
    assert out["n_assoc"] == 0 and out["cost_l1"] == 0.0 and out["e2"] == 0.0
    assert np.all(out["jte"] == 0.0) and np.all(out["jtj"] == 0.0)
    # the tolerance is strict, decided on the FP32 difference t - d
    sd = np.full(t.shape, 2.0625, np.float32)
    dz32 = (t - sd).astype(np.float32)
    tol = float(np.abs(dz32).min())
    n_eq = int(np.sum(np.abs(dz32) < np.float32(tol)))
    assert om.icp_terms(eye, cam, sd, sc, tol=tol)["n_assoc"] == n_eq
    tol_up = float(np.nextafter(np.float32(tol), np.float32(1)))
    assert om.icp_terms(eye, cam, sd, sc, tol=tol_up)["n_assoc"] == int(np.sum(np.abs(dz32) < np.float32(tol_up)))
    # scan classes: FU and NaN pixels are never associated
    sd = np.full(t.shape, 2.02, np.float32)
    sc2 = sc.copy()
    sc2[:, :5] = 1
    sd2 = sd.copy()
    sd2[:3, :] = np.nan
    expect = int(np.sum((sc2 == 0) & ~np.isnan(sd2)))
    assert om.icp_terms(eye, cam, sd2, sc2, tol=0.1)["n_assoc"] == expect
    # map labels: only FO surfaces are associated (FU and UO faces are not)
    for lab in (1, 2):
        cam_, om_ = _wall(labels=lab)
        assert om_.icp_terms(eye, cam_, sd, sc, tol=0.1)["n_assoc"] == 0
    # a wall with mixed labels: exactly the pixels whose winning face is FO
    nf = 50
    mixed = (np.arange(nf) // 2 % 3 == 0).astype(np.uint8)  # two faces per cell
    cam_, om_ = _wall(labels=mixed)
    ids = om_.render(eye, cam_)["tri_id"]
    assert om_.icp_terms(eye, cam_, sd, sc, tol=0.1)["n_assoc"] == int(np.sum(mixed[ids] == 0))


def _fd_case(model):
    if model == "pinhole":
        c = cases.config1(seed=1600)
        return c["mesh"], c["cam"], c["start"], c["scan"]
    mesh = synth.room_mesh(1610)
    cam = cases.small_spherical(w=128, h=16)
    r = cases.rng(1611)
    gt = synth.room_pose(r, mesh)
    sd, sc = synth.synth_scan(mesh, cam, gt, r, sigma_abs=0.01)
    start = synth.perturb_fixed(gt, r, 0.03, 1.0)
    return mesh, cam, start, (sd, sc)


@pytest.mark.parametrize("model", ["pinhole", "spherical"])
def test_icp_jte_matches_frozen_fd(model):
    """J^T e is the gradient of the frozen point-to-plane cost 1/2 sum e^2 (associations, map
    points and normals held at the pose; scan points moved by the twist): central
    differences, Richardson-combined."""
    mesh, cam, pose, (sd, sc) = _fd_case(model)
    om = oracle.OracleMap(mesh.vertices, mesh.faces, mesh.labels)
    out = om.icp_terms(pose, cam, sd, sc, tol=0.1)
    assert out["n_assoc"] > 100
    assert om.icp_frozen(pose, cam, sd, sc, 0.1, np.zeros(6)) == pytest.approx(0.5 * out["e2"], rel=1e-12)

    def central(h):
        fd = np.zeros(6)
        for a in range(6):
            xi = np.zeros(6)
            xi[a] = h
            fd[a] = (om.icp_frozen(pose, cam, sd, sc, 0.1, xi)
                     - om.icp_frozen(pose, cam, sd, sc, 0.1, -xi)) / (2 * h)
        return fd

    fd = (4 * central(5e-5) - central(1e-4)) / 3
    assert np.linalg.norm(out["jte"] - fd) <= 1e-7 * np.linalg.norm(out["jte"])


@pytest.mark.parametrize("model", ["pinhole", "spherical"])
def test_icp_jtj_is_hessian_where_residuals_vanish(model):
    """On a scan rendered from the map itself every associated residual is zero, so the
    Hessian of the frozen cost at zero twist is exactly J^T J (four-point second
    differences)."""
    mesh, cam, pose, _ = _fd_case(model)
    fo = mesh.labels == 0
    om = oracle.OracleMap(mesh.vertices, mesh.faces[fo], mesh.labels[fo])
    sd, sc = cases.scan_from_render(om.render(pose, cam)["depth"], cam)
    out = om.icp_terms(pose, cam, sd, sc, tol=0.1)
    assert out["n_assoc"] == int(np.sum(sc == 0)) and out["e2"] == 0.0
    assert np.all(out["jte"] == 0.0)
    h = 1e-4
    f = lambda xi: om.icp_frozen(pose, cam, sd, sc, 0.1, xi)  # noqa: E731
    H = np.zeros((6, 6))
    E = np.eye(6) * h
    for a in range(6):
        for b in range(a, 6):
            H[a, b] = H[b, a] = (f(E[a] + E[b]) - f(E[a] - E[b]) - f(-E[a] + E[b]) + f(-E[a] - E[b])) / (4 * h * h)
    Hj = np.zeros((6, 6))
    for a in range(6):
        for b in range(a, 6):
            Hj[a, b] = Hj[b, a] = out["jtj"][packed(a, b)]
    assert np.linalg.norm(H - Hj) <= 1e-5 * np.linalg.norm(Hj)
    assert np.linalg.eigvalsh(Hj).min() > 0


@pytest.mark.parametrize("pitch_deg", [15.0, 25.0])
def test_icp_align_converges_noise_free(pitch_deg):
    """From 5 cm / 2 deg off, projective point-to-plane ICP on a noise-free scan of the
    room (tilted toward the floor so that every direction is constrained) returns to the
    true pose. The map depth is the FP32 z-buffer depth, so the steps settle at the FP32
    noise floor (about 1e-7 m here) within three iterations; step_tol sits above it."""
    c = cases.config1(seed=1500)
    mesh, cam = c["mesh"], c["cam"]
    gt = synth.pose_from(c["gt"][:3, 3], 0.7, math.radians(pitch_deg), 0.0)
    start = synth.perturb_fixed(gt, cases.rng(3), 0.05, 2.0)
    om = oracle.OracleMap(mesh.vertices, mesh.faces, mesh.labels)
    sd, sc = cases.scan_from_render(om.render(gt, cam)["depth"], cam)
    pose, rep = om.icp_align(start, cam, sd, sc, tol=0.2, max_iters=50, step_tol=1e-5)
    assert rep["converged"] == 1 and rep["iters"] <= 6
    assert np.linalg.norm(pose[:3, 3] - gt[:3, 3]) < 2e-6
    ang = Rotation.from_matrix(gt[:3, :3].T @ pose[:3, :3]).magnitude()
    assert math.degrees(ang) < 1e-4
    assert rep["n_assoc"] == int(np.sum(sc == 0))
    assert rep["cost_l1"] < 1e-6 * rep["n_assoc"]


def test_icp_empty_and_degenerate():
    cam = cases.small_pinhole()
    om = oracle.OracleMap(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32), np.zeros(0, np.uint8))
    sd = np.ones((cam.height, cam.width), np.float32)
    sc = np.zeros_like(sd, np.uint8)
    out = om.icp_terms(np.eye(4), cam, sd, sc, tol=0.1)
    assert out["n_assoc"] == 0 and np.all(out["jtj"] == 0.0)
    # nothing associated: the 6x6 system is singular, the alignment stops at once, unconverged
    pose, rep = om.icp_align(np.eye(4), cam, sd, sc, tol=0.1, max_iters=5)
    assert rep["converged"] == 0 and rep["iters"] == 0
    assert np.array_equal(pose, np.eye(4))


def test_icp_single_wall_is_degenerate():
    """Fig. 2's failure of point-only alignment: a view of one plane constrains only the
    depth and the two tilts, so J^T J is singular (rank 3) and no Gauss-Newton step is
    taken; the pose stays where it started."""
    cam, om = _wall()
    sd = np.full((cam.height, cam.width), 2.03, np.float32)
    sc = np.zeros_like(sd, np.uint8)
    out = om.icp_terms(np.eye(4), cam, sd, sc, tol=0.1)
    H = np.zeros((6, 6))
    for a in range(6):
        for b in range(a, 6):
            H[a, b] = H[b, a] = out["jtj"][packed(a, b)]
    assert np.linalg.matrix_rank(H) == 3
    pose, rep = om.icp_align(np.eye(4), cam, sd, sc, tol=0.1, max_iters=10)
    assert rep["converged"] == 0 and rep["iters"] == 0
    assert np.array_equal(pose, np.eye(4))


def test_icp_terms_are_rigidly_invariant():
    """Moving the world and the pose together by one rigid motion leaves the associations and
    the terms (all in the camera frame) unchanged, up to the FP32 rounding of the moved
    vertices."""
    c = cases.config1(seed=2400)
    mesh, cam = c["mesh"], c["cam"]
    sd, sc = c["scan"]
    G = synth.pose_from(np.array([12.0, -7.0, 3.0]), 1.1, 0.3, -0.2)
    v2 = (mesh.vertices.astype(np.float64) @ G[:3, :3].T + G[:3, 3]).astype(np.float32)
    a = oracle.OracleMap(mesh.vertices, mesh.faces, mesh.labels).icp_terms(c["start"], cam, sd, sc, 0.1)
    b = oracle.OracleMap(v2, mesh.faces, mesh.labels).icp_terms(G @ c["start"], cam, sd, sc, 0.1)
    assert abs(a["n_assoc"] - b["n_assoc"]) <= 1e-3 * a["n_assoc"]
    assert np.linalg.norm(a["jte"] - b["jte"]) <= 1e-3 * np.linalg.norm(a["jte"])
    assert np.linalg.norm(a["jtj"] - b["jtj"]) <= 1e-3 * np.linalg.norm(a["jtj"])


def test_associations_grow_with_the_tolerance():
    """A larger tolerance keeps every pair a smaller one makes (|Z_M - Z_1| < tol is monotone),
    and C grows with the pairs it adds."""
    c = cases.config1(seed=2500)
    om = oracle.OracleMap(c["mesh"].vertices, c["mesh"].faces, c["mesh"].labels)
    sd, sc = c["scan"]
    prev = None
    for tol in (0.0, 0.01, 0.03, 0.1, 0.3, 1.0):
        o = om.icp_terms(c["start"], c["cam"], sd, sc, tol)
        if prev is not None:
            assert o["n_assoc"] >= prev["n_assoc"] and o["cost_l1"] >= prev["cost_l1"]
        prev = o
    assert om.icp_terms(c["start"], c["cam"], sd, sc, 0.0)["n_assoc"] == 0
