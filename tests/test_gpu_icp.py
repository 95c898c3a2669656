"""Render-accelerated point-to-plane ICP (Sec. V) on the GPU vs the CPU oracle, through the
C ABI.

The association (which pixels pair up) is decided in FP32 on both sides from the same z-buffer
key and scan depth, so the association count must match bit for bit. The sums are FP32 per
tile on the GPU and FP64 in the oracle: C and sum e^2 within 1e-5 relative, J^T e within 1e-3
and J^T J within 1e-4, element by element (tests/checks.py). ICP alignments on both sides must end within
1e-5 m / 1e-3 deg of each other.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

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

EPS_REL_SUM = 1e-5
EPS_REL_JTE = 1e-3
EPS_REL_JTJ = 1e-4


def _np(t):
    return t.detach().cpu().numpy()


def _check_icp(g, o, k):
    assert int(_np(g["n_assoc"])[k]) == o["n_assoc"], k
    for key in ("cost_l1", "e2"):
        v = float(_np(g[key])[k])
        assert abs(v - o[key]) <= EPS_REL_SUM * abs(o[key]) + 1e-12, (key, k, v, o[key])
    gg, hh = _np(g["jte"])[k], _np(g["jtj"])[k]
    checks.close_elementwise(gg, o["jte"], EPS_REL_JTE, f"icp_jte[{k}]", floor=1e-9)
    checks.close_elementwise(hh, o["jtj"], EPS_REL_JTJ, f"icp_jtj[{k}]", floor=1e-9)


def _pose_gap(a, b):
    return (float(np.linalg.norm(a[:3, 3] - b[:3, 3])),
            math.degrees(Rotation.from_matrix(a[:3, :3].T @ b[:3, :3]).magnitude()))


@pytest.fixture(scope="module")
def room():
    """213x161 pinhole in a cluttered room with FU faces; noisy scan with NaN dropouts."""
    c = cases.config2(seed=2300, target_fo=60_000, target_fu=15_000)
    cam = dataclasses.replace(c["cam"], width=213, height=161, fx=175.0, fy=175.0, cx=106.5, cy=80.5)
    mesh = c["mesh"]
    r = cases.rng(23)
    sd, sc = synth.synth_scan(mesh, cam, c["gt"], r, sigma_rel=0.005, dropout=0.05, dropout_as_nan=True)
    om = oracle.OracleMap(mesh.vertices, mesh.faces, mesh.labels)
    gm = rm.Map(mesh.vertices, mesh.faces, mesh.labels)
    intr = rm.Intrinsics.from_camera(cam)
    yield dict(c, cam=cam, scan=(sd, sc), om=om, gm=gm, intr=intr, gscan=rm.Scan.make(intr, sd, sc))
    gm.close()


@pytest.mark.parametrize("tile", [(64, 32), (32, 32), (16, 16)])
def test_icp_terms_parity_pinhole(room, tile):
    room["gm"].set_tuning(tile=tile)
    r = cases.rng(41)
    poses = [room["gt"], room["start"], synth.perturb_fixed(room["gt"], r, 0.1, 3.0),
             synth.perturb_fixed(room["gt"], r, 0.3, 8.0)]
    sd, sc = room["scan"]
    for tol in (0.05, 0.25):
        g = rm.icp_terms(room["gm"], room["gscan"], np.stack(poses), tol=tol)
        for k, P in enumerate(poses):
            _check_icp(g, room["om"].icp_terms(P, room["cam"], sd, sc, tol), k)
        # about 40% of the pixels pair up at the true pose (FU frontier faces hide the rest)
        assert int(_np(g["n_assoc"])[0]) > 0.35 * sd.size
    room["gm"].set_tuning(tile=(0, 0))


def test_icp_terms_repeatable_and_wave_split(room):
    """The same poses give bit-identical terms whether evaluated alone, in one wave or split
    over several waves (fixed-order reductions)."""
    r = cases.rng(42)
    poses = np.stack([synth.perturb_fixed(room["gt"], r, 0.05, 2.0) for _ in range(9)])
    a = rm.icp_terms(room["gm"], room["gscan"], poses, tol=0.1)
    room["gm"].set_tuning(wave_poses=4)
    b = rm.icp_terms(room["gm"], room["gscan"], poses, tol=0.1)
    room["gm"].set_tuning(wave_poses=0)
    c = rm.icp_terms(room["gm"], room["gscan"], poses[3:4], tol=0.1)
    for key in a:
        assert torch.equal(a[key], b[key]), key
        assert torch.equal(a[key][3:4], c[key]), key


def test_icp_terms_edge_cases(room):
    sd, sc = room["scan"]
    # tolerance 0: nothing associated, all sums zero
    g = rm.icp_terms(room["gm"], room["gscan"], room["gt"][None], tol=0.0)
    assert int(_np(g["n_assoc"])[0]) == 0 and float(_np(g["e2"])[0]) == 0.0
    assert not _np(g["jtj"]).any()
    # no poses
    g = rm.icp_terms(room["gm"], room["gscan"], np.zeros((0, 4, 4)), tol=0.1)
    assert g["n_assoc"].shape == (0,)
    # a scan with no FO return
    fu = rm.Scan.make(room["intr"], sd, np.ones_like(sc))
    g = rm.icp_terms(room["gm"], fu, room["gt"][None], tol=0.1)
    assert int(_np(g["n_assoc"])[0]) == 0
    # an empty map
    em = rm.Map(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32), np.zeros(0, np.uint8))
    g = rm.icp_terms(em, room["gscan"], room["gt"][None], tol=0.1)
    assert int(_np(g["n_assoc"])[0]) == 0
    pose, rep = rm.icp_align(em, room["gscan"], room["gt"], tol=0.1, max_iters=4)
    assert rep["converged"] == 0 and rep["iters"] == 0 and rep["status"] == "RM_ENOTCONV"
    assert np.array_equal(pose, room["gt"])
    em.close()
    # a negative or NaN tolerance is an argument error
    with pytest.raises(rm.RenderMapError):
        rm.icp_terms(room["gm"], room["gscan"], room["gt"][None], tol=-1.0)
    with pytest.raises(rm.RenderMapError):
        rm.icp_terms(room["gm"], room["gscan"], room["gt"][None], tol=float("nan"))


def test_icp_single_wall_is_degenerate():
    """A view of one plane leaves J^T J singular on both sides: no step is taken."""
    cam = cases.small_pinhole(w=32, h=24, f=30.0)
    v, f = cases.plane_grid(5, 5, (-20, -20, 2.0), (40, 0, 0), (0, 40, 0))
    lab = np.zeros(len(f), np.uint8)
    gm = rm.Map(v, f, lab)
    sd = np.full((cam.height, cam.width), 2.03, np.float32)
    sc = np.zeros_like(sd, np.uint8)
    scan = rm.Scan.make(rm.Intrinsics.from_camera(cam), sd, sc)
    g = rm.icp_terms(gm, scan, np.eye(4)[None], tol=0.1)
    _check_icp(g, oracle.OracleMap(v, f, lab).icp_terms(np.eye(4), cam, sd, sc, 0.1), 0)
    pose, rep = rm.icp_align(gm, scan, np.eye(4), tol=0.1, max_iters=10)
    assert rep["converged"] == 0 and rep["iters"] == 0 and np.array_equal(pose, np.eye(4))
    gm.close()


def test_icp_terms_host_buffers_match_device(room):
    """Host (numpy) scan, poses and outputs through the same ABI give the same numbers."""
    import ctypes
    from paper_1702_06813_gb300 import _native as N
    sd, sc = room["scan"]
    sd = np.ascontiguousarray(sd, np.float32)
    sc = np.ascontiguousarray(sc, np.uint8)
    poses = np.ascontiguousarray(np.stack([room["gt"], room["start"]]), np.float64)
    cs = N.rm_scan(room["intr"].c(), sd.ctypes.data, sc.ctypes.data)
    na = np.zeros(2, np.int64)
    l1, e2 = np.zeros(2), np.zeros(2)
    g, h = np.zeros((2, 6)), np.zeros((2, 21))
    out = N.rm_icp_out(na.ctypes.data, l1.ctypes.data, e2.ctypes.data, g.ctypes.data, h.ctypes.data)
    st = N.lib().rm_icp_terms(room["gm"].handle, ctypes.byref(cs), poses.ctypes.data, 2, 0.1,
                              ctypes.byref(out), None)
    assert st == N.RM_OK
    d = rm.icp_terms(room["gm"], room["gscan"], poses, tol=0.1)
    assert np.array_equal(na, _np(d["n_assoc"]))
    assert np.array_equal(l1, _np(d["cost_l1"])) and np.array_equal(e2, _np(d["e2"]))
    assert np.array_equal(g, _np(d["jte"])) and np.array_equal(h, _np(d["jtj"]))


def test_icp_jte_matches_oracle_frozen_fd(room):
    """The GPU's J^T e against central differences of the oracle's frozen point-to-plane
    cost (independent of the oracle's own J^T e)."""
    sd, sc = room["scan"]
    pose = room["start"]
    g = _np(rm.icp_terms(room["gm"], room["gscan"], pose[None], tol=0.1)["jte"])[0]
    fd = np.zeros(6)
    h = 1e-5
    for a in range(6):
        xi = np.zeros(6)
        xi[a] = h
        fd[a] = (room["om"].icp_frozen(pose, room["cam"], sd, sc, 0.1, xi)
                 - room["om"].icp_frozen(pose, room["cam"], sd, sc, 0.1, -xi)) / (2 * h)
    checks.close_elementwise(g, fd, 1e-3, "icp_jte_vs_fd")


def test_icp_align_matches_oracle_pinhole(room):
    sd, sc = room["scan"]
    pg, rep = rm.icp_align(room["gm"], room["gscan"], room["start"], tol=0.2, max_iters=30, step_tol=1e-5)
    po, orep = room["om"].icp_align(room["start"], room["cam"], sd, sc, tol=0.2, max_iters=30, step_tol=1e-5)
    assert rep["converged"] == 1 and orep["converged"] == 1, (rep, orep)
    assert abs(rep["iters"] - orep["iters"]) <= 1, (rep, orep)
    dt, da = _pose_gap(pg, po)
    assert dt < 1e-5 and da < 1e-3, (dt, da, rep, orep)
    assert abs(rep["n_assoc"] - orep["n_assoc"]) <= 1e-3 * orep["n_assoc"]
    assert rep["cost_l1_final"] < rep["cost_l1_initial"]
    dgt, agt = _pose_gap(pg, room["gt"])
    assert dgt < 5e-3 and agt < 0.1, (dgt, agt)


def test_icp_align_noise_free_returns_to_true_pose():
    c = cases.config1(seed=1500)
    mesh, cam = c["mesh"], c["cam"]
    gt = synth.pose_from(c["gt"][:3, 3], 0.7, math.radians(25.0), 0.0)
    start = synth.perturb_fixed(gt, cases.rng(3), 0.05, 2.0)
    om = oracle.OracleMap(mesh.vertices, mesh.faces, mesh.labels)
    sd, sc = cases.scan_from_render(om.render(gt, cam)["depth"], cam)
    gm = rm.Map(mesh.vertices, mesh.faces, mesh.labels)
    scan = rm.Scan.make(rm.Intrinsics.from_camera(cam), sd, sc)
    pose, rep = rm.icp_align(gm, scan, start, tol=0.2, max_iters=50, step_tol=1e-5)
    assert rep["converged"] == 1 and rep["iters"] <= 6, rep
    dt, da = _pose_gap(pose, gt)
    assert dt < 1e-5 and da < 1e-3, (dt, da)
    gm.close()


@pytest.fixture(scope="module")
def lidar():
    w = synth.workload_lidar(seed=4100, target_fo=140_000, target_fu=60_000, n_panels=120)
    om = oracle.OracleMap(w["mesh"].vertices, w["mesh"].faces, w["mesh"].labels)
    gm = rm.Map(w["mesh"].vertices, w["mesh"].faces, w["mesh"].labels)
    intr = rm.Intrinsics.from_camera(w["cam"])
    yield dict(w, om=om, gm=gm, intr=intr, gscan=rm.Scan.make(intr, *w["scan"]))
    gm.close()


def test_icp_terms_parity_raytable(lidar):
    r = cases.rng(43)
    poses = [lidar["gt"], lidar["start"], synth.perturb_fixed(lidar["gt"], r, 0.5, 5.0)]
    sd, sc = lidar["scan"]
    g = rm.icp_terms(lidar["gm"], lidar["gscan"], np.stack(poses), tol=0.3)
    for k, P in enumerate(poses):
        _check_icp(g, lidar["om"].icp_terms(P, lidar["cam"], sd, sc, 0.3), k)


def test_icp_align_matches_oracle_raytable(lidar):
    """From 30 cm / 3 deg off, ICP on the panoramic scan converges in a handful of
    iterations on both sides, to the same pose."""
    sd, sc = lidar["scan"]
    pg, rep = rm.icp_align(lidar["gm"], lidar["gscan"], lidar["start"], tol=0.5, max_iters=30, step_tol=1e-5)
    po, orep = lidar["om"].icp_align(lidar["start"], lidar["cam"], sd, sc, tol=0.5, max_iters=30, step_tol=1e-5)
    assert rep["converged"] == 1 and orep["converged"] == 1, (rep, orep)
    dt, da = _pose_gap(pg, po)
    assert dt < 1e-5 and da < 1e-3, (dt, da, rep, orep)
    dgt, agt = _pose_gap(pg, lidar["gt"])
    assert dgt < 1e-3 and agt < 0.01, (dgt, agt)
