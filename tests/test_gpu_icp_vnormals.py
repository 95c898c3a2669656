"""Point-to-plane ICP with the map's points coloured by their normals (Sec. V, sequential
depth-image alignment steps 2-3) on the GPU vs the CPU oracle, through the C ABI.

With vertex normals attached (rm_map_set_vertex_normals), the normal of an associated pixel is
the blend of the seen triangle's vertex normals by the hit's barycentrics. The association
count must match the oracle bit for bit (the NaN rule included); C and sum e^2 within 1e-5;
J^T e within 1e-3 and J^T J within 1e-3 element by element: the GPU's barycentrics are FP32
(within the bound the visibility-buffer test derives), which moves a blended normal by up to
that error times the spread of the three vertex normals. Alignments run the same iterations
and end within 1e-4 m / 2e-3 deg of the oracle's (blended normals move with the pose, so the
steps need not shrink below the step tolerance), and the sequential loop with Eq. 2 normals
tracks a trajectory.
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


def _np(t):
    return t.detach().cpu().numpy()


def _smooth_vertex_normals(v, f):
    a, b, c = (v[f[:, k]].astype(np.float64) for k in range(3))
    n = np.cross(b - a, c - a)
    out = np.zeros((v.shape[0], 3))
    for k in range(3):
        np.add.at(out, f[:, k], n)
    return out / np.maximum(np.linalg.norm(out, axis=1, keepdims=True), 1e-300)


def _gap(P, Q):
    return (float(np.linalg.norm(P[:3, 3] - Q[:3, 3])),
            math.degrees(Rotation.from_matrix(P[:3, :3].T @ Q[:3, :3]).magnitude()))


def _check_icp(g, o, k, what):
    assert int(_np(g["n_assoc"])[k]) == o["n_assoc"], (what, k)
    for key in ("cost_l1", "e2"):
        v = float(_np(g[key])[k])
        assert abs(v - o[key]) <= 1e-5 * abs(o[key]) + 1e-12, (what, key, k, v, o[key])
    checks.close_elementwise(_np(g["jte"])[k], o["jte"], 1e-3, f"{what}_jte[{k}]", floor=1e-9)
    checks.close_elementwise(_np(g["jtj"])[k], o["jtj"], 1e-3, f"{what}_jtj[{k}]", floor=1e-9)


@pytest.fixture(scope="module")
def room():
    c = cases.config2(seed=2310, target_fo=60_000, target_fu=15_000)
    cam = dataclasses.replace(c["cam"], width=213, height=161, fx=175.0, fy=175.0, cx=106.5, cy=80.5)
    mesh = c["mesh"]
    r = cases.rng(31)
    sd, sc = synth.synth_scan(mesh, cam, c["gt"], r, sigma_rel=0.005, dropout=0.05, dropout_as_nan=True)
    vn = _smooth_vertex_normals(mesh.vertices, mesh.faces)
    om = oracle.OracleMap(mesh.vertices, mesh.faces, mesh.labels)
    gm = rm.Map(mesh.vertices, mesh.faces, mesh.labels)
    intr = rm.Intrinsics.from_camera(cam)
    yield dict(c, cam=cam, scan=(sd, sc), vn=vn, om=om, gm=gm, intr=intr, gscan=rm.Scan.make(intr, sd, sc))
    gm.close()


def test_vertex_normal_terms_match_oracle(room):
    gm, om = room["gm"], room["om"]
    vn = room["vn"]
    r = cases.rng(32)
    poses = [room["gt"], room["start"], synth.perturb_fixed(room["gt"], r, 0.1, 3.0)]
    sd, sc = room["scan"]
    face = rm.icp_terms(gm, room["gscan"], np.stack(poses), tol=0.1)
    # normals given in a camera frame: the library rotates them to the world frame
    F = synth.pose_from(np.array([1.0, 2.0, 0.5]), 0.8, 0.2, -0.1)
    gm.set_vertex_normals((vn @ F[:3, :3]).astype(np.float32), pose=F)
    try:
        g = rm.icp_terms(gm, room["gscan"], np.stack(poses), tol=0.1)
        for k, P in enumerate(poses):
            _check_icp(g, om.icp_terms(P, room["cam"], sd, sc, 0.1, vnormals=vn), k, "vn")
        # the blended normals differ from the planes, so the terms do too
        assert not torch.equal(g["jte"], face["jte"])
    finally:
        gm.set_vertex_normals(None)
    # detached: the face-normal terms again, bit for bit
    again = rm.icp_terms(gm, room["gscan"], np.stack(poses), tol=0.1)
    for key in ("n_assoc", "cost_l1", "e2", "jte", "jtj"):
        assert torch.equal(again[key], face[key]), key


def test_nan_vertex_normals_leave_pixels_unassociated(room):
    gm, om = room["gm"], room["om"]
    vn = room["vn"].copy()
    vn[cases.rng(33).choice(vn.shape[0], vn.shape[0] // 20, replace=False)] = np.nan
    sd, sc = room["scan"]
    gm.set_vertex_normals(vn.astype(np.float32))
    try:
        g = rm.icp_terms(gm, room["gscan"], room["start"][None], tol=0.1)
    finally:
        gm.set_vertex_normals(None)
    o = om.icp_terms(room["start"], room["cam"], sd, sc, 0.1, vnormals=vn)
    _check_icp(g, o, 0, "vn_nan")
    assert o["n_assoc"] < om.icp_terms(room["start"], room["cam"], sd, sc, 0.1)["n_assoc"]


def test_vertex_normal_alignment_matches_oracle(room):
    gm, om = room["gm"], room["om"]
    vn = room["vn"]
    cam = room["cam"]
    gt = synth.pose_from(room["gt"][:3, 3], 0.7, math.radians(25.0), 0.0)
    start = synth.perturb_fixed(gt, cases.rng(34), 0.05, 2.0)
    sd, sc = synth.synth_scan(room["mesh"], cam, gt, cases.rng(35), sigma_rel=0.005)
    scan = rm.Scan.make(room["intr"], sd, sc)
    gm.set_vertex_normals(vn.astype(np.float32))
    try:
        pg, rep = rm.icp_align(gm, scan, start, tol=0.2, max_iters=30, step_tol=1e-5)
        pb, reps, _ = rm.icp_align_batch(gm, [(scan, start)], tol=0.2, max_iters=30, step_tol=1e-5)
    finally:
        gm.set_vertex_normals(None)
    po, orep = om.icp_align(start, cam, sd, sc, 0.2, 30, 1e-5, vnormals=vn)
    # blended normals move with the pose, so the steps need not shrink below 1e-5: both sides
    # run the same iterations
    assert rep["iters"] == orep["iters"] and rep["converged"] == orep["converged"], (rep, orep)
    dt, da = _gap(pg, po)
    assert dt < 1e-4 and da < 2e-3, (dt, da)
    assert np.array_equal(pb[0], pg)  # the batch kernel takes the same normals
    dt, da = _gap(pg, gt)
    assert dt < 0.01 and da < 0.3, (dt, da)


def test_eq2_pipeline_step_matches_oracle():
    """One step of Sec. V's loop with Eq. 2 normals: scan A meshed at its pose (downsampled
    by 2), its metric Eq. 2 normals at the mesh's grid pixels as vertex normals, and scan B
    aligned to that map by ICP, on the GPU and on the oracle."""
    c = cases.config1(seed=1810)
    mesh, cam = c["mesh"], c["cam"]
    r = cases.rng(6)
    A = synth.pose_from(c["gt"][:3, 3], 3.5, math.radians(35.0), 0.0)
    B = synth.perturb_fixed(A, r, 0.04, 1.5)
    sA = synth.synth_scan(mesh, cam, A, r, sigma_abs=0.003)
    sB = synth.synth_scan(mesh, cam, B, r, sigma_abs=0.003)
    intr = rm.Intrinsics.from_camera(cam)
    scanA, scanB = rm.Scan.make(intr, *sA), rm.Scan.make(intr, *sB)
    # GPU: the sequential loop's first step
    est, reps = rm.sequential_icp([scanA, scanB], A, max_range=cam.range_max, step=2, normals="eq2")
    # oracle: the same pipeline from its own mesh and normals
    v, f, lab = oracle.meshify(cam, sA[0], sA[1], A, cam.range_max, 0.1, 2)
    nrm, _ = oracle.depth_normals(sA[0], sA[1], sigma=1.0, metric=True, fx=cam.fx, fy=cam.fy)
    vn = nrm[::2, ::2].reshape(-1, 3) @ A[:3, :3].T
    om = oracle.OracleMap(v, f, lab)
    po, orep = om.icp_align(A, cam, sB[0], sB[1], 0.2, 20, 1e-5, vnormals=vn)
    assert reps[0]["iters"] == orep["iters"], (reps[0], orep)
    dt, da = _gap(est[1], po)
    assert dt < 1e-4 and da < 2e-3, (dt, da)
    dt, da = _gap(est[1], B)
    assert dt < 5e-3 and da < 0.2, (dt, da)


@pytest.mark.parametrize("normals", ["face", "eq2"])
def test_sequential_alignment_both_normal_modes(normals):
    c = cases.config1(seed=1800)
    mesh, cam = c["mesh"], c["cam"]
    r = cases.rng(9)
    truth = [synth.pose_from(c["gt"][:3, 3], 3.5, math.radians(35.0), 0.0)]
    for _ in range(3):
        truth.append(synth.perturb_fixed(truth[-1], r, 0.04, 1.5))
    intr = rm.Intrinsics.from_camera(cam)
    scans = [rm.Scan.make(intr, *synth.synth_scan(mesh, cam, T, r, sigma_abs=0.003)) for T in truth]
    est, reps = rm.sequential_icp(scans, truth[0], max_range=cam.range_max, step=2, normals=normals)
    for k in range(1, 4):
        dt, da = _gap(est[k], truth[k])
        assert dt < 0.01 and da < 0.3, (normals, k, dt, da, reps[k - 1])
