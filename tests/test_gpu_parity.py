"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Visibility (triangle ids and depth keys) and Table I counts must match bit for bit; the
least-squares cost within 1e-5 relative; gradient and Gauss-Newton matrix within 1e-3
relative of the oracle's FP64 values, element by element (tests/checks.py); barycentrics
within a per-pixel bound derived from the FP32 depth and vertex rounding; LM poses within
1 mm / 0.01 deg.
"""
from __future__ import annotations

import dataclasses
import math

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

EPS_REL_COST = 1e-5
EPS_REL_GRAD = 1e-3


def _np(t):
    return t.detach().cpu().numpy()


def _same_render(gpu, orc):
    ids = _np(gpu["tri_id"])
    depth = _np(gpu["depth"])
    assert np.array_equal(ids, orc["tri_id"]), f"{np.sum(ids != orc['tri_id'])} pixels differ in tri id"
    both = ~np.isnan(orc["depth"])
    assert np.array_equal(np.isnan(depth), ~both)
    assert np.array_equal(depth[both].view(np.uint32), orc["depth"][both].view(np.uint32))


def _check_cost(g, o, k=0, grad=True):
    assert np.array_equal(_np(g["counts"])[k], o["counts"])
    assert int(_np(g["e_table"])[k]) == o["e_table"]
    e = float(_np(g["e_ls"])[k])
    assert abs(e - o["e_ls"]) <= EPS_REL_COST * abs(o["e_ls"]) + 1e-12
    if grad:
        checks.close_elementwise(_np(g["grad"])[k], o["grad"], EPS_REL_GRAD, f"grad[{k}]", floor=1e-9)
        checks.close_elementwise(_np(g["jtj"])[k], o["jtj"], EPS_REL_GRAD, f"jtj[{k}]", floor=1e-9)


@pytest.fixture(scope="module")
def c1():
    c = cases.config1(seed=1000)
    om = oracle.OracleMap(c["mesh"].vertices, c["mesh"].faces, c["mesh"].labels)
    gm = rm.Map(c["mesh"].vertices, c["mesh"].faces, c["mesh"].labels)
    intr = rm.Intrinsics.from_camera(c["cam"])
    scan = rm.Scan.make(intr, *c["scan"])
    return dict(c, om=om, gm=gm, intr=intr, gscan=scan)


# ---------------------------------------------------------------------------------------
# visibility
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("tile", [(64, 32), (32, 32), (32, 16), (16, 16)])
def test_render_bit_exact_config1(c1, tile):
    c1["gm"].set_tuning(tile=tile)
    r = cases.rng(5)
    poses = [c1["gt"], c1["start"]] + [synth.room_pose(r, c1["mesh"]) for _ in range(4)]
    g = rm.render_depth(c1["gm"], np.stack(poses), c1["intr"])
    for k, P in enumerate(poses):
        o = c1["om"].render(P, c1["cam"])
        _same_render({"tri_id": g["tri_id"][k], "depth": g["depth"][k]}, o)
    c1["gm"].set_tuning()


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_render_bit_exact_triangle_soup_with_near_cuts(seed):
    """Random camera-frame triangles (many cut by the near plane, some huge, some off
    screen) at an odd image size that leaves ragged tiles."""
    cam = cases.small_pinhole(w=75, h=53, f=50.0)
    vc, f = cases.random_tris(seed, 400)
    om = oracle.OracleMap(vc, f, np.zeros(len(f), np.uint8))
    o = om.render(np.eye(4), cam)
    assert o["stats"]["clipped"] > 0
    gm = rm.Map(vc, f, np.zeros(len(f), np.uint8))
    g = rm.render_depth(gm, np.eye(4)[None], rm.Intrinsics.from_camera(cam))
    _same_render({"tri_id": g["tri_id"][0], "depth": g["depth"][0]}, o)


@pytest.mark.parametrize("shape", [(16384, 3), (3, 16384)])
def test_render_and_cost_at_the_largest_image_side(shape):
    """The largest image side the ABI accepts (16384 pixels): one row of 256 tiles, or one
    column of 512. A tilted, jittered grid of 80k triangles (about 450 visible along the
    strip, FU faces among them) renders bit for bit and gives the oracle's Table I counts and
    adjoint at two poses; a wide-angle soup with near cuts renders bit for bit too."""
    w, h = shape
    cam = cases.small_pinhole(w=w, h=h, f=1500.0)
    intr = rm.Intrinsics.from_camera(cam)
    vg, fg = cases.plane_grid(200, 200, (-20.0, -20.0, 2.0), (40.0, 0.0, 3.0), (0.0, 40.0, 1.0),
                              jitter=0.3, seed=5)
    labels = (np.arange(len(fg)) % 4 == 0).astype(np.uint8)
    om = oracle.OracleMap(vg, fg, labels)
    gm = rm.Map(vg, fg, labels)
    o = om.render(np.eye(4), cam)
    hit = ~np.isnan(o["depth"])
    assert len(np.unique(o["tri_id"][hit])) > 300
    g = rm.render_depth(gm, np.eye(4)[None], intr)
    _same_render({"tri_id": g["tri_id"][0], "depth": g["depth"][0]}, o)
    r = cases.rng(22)
    sd = np.where(hit, o["depth"] * (1.0 + 0.01 * r.standard_normal(o["depth"].shape)), 4.0).astype(np.float32)
    sc = np.where(hit, (r.uniform(size=sd.shape) < 0.2).astype(np.uint8), np.uint8(1))
    sc[r.uniform(size=sd.shape) < 0.05] = 2
    scan = rm.Scan.make(intr, sd, sc)
    poses = [np.eye(4), synth.perturb_fixed(np.eye(4), r, 0.05, 2.0)]
    gc = rm.cost_grad(gm, scan, np.stack(poses))
    for k, P in enumerate(poses):
        _check_cost(gc, om.cost(P, cam, sd, sc), k)
    gm.close()
    vs, fs = cases.random_tris(21, 600)
    om = oracle.OracleMap(vs, fs, np.zeros(len(fs), np.uint8))
    o = om.render(np.eye(4), cam)
    assert o["stats"]["clipped"] > 0
    gm = rm.Map(vs, fs, np.zeros(len(fs), np.uint8))
    g = rm.render_depth(gm, np.eye(4)[None], intr)
    _same_render({"tri_id": g["tri_id"][0], "depth": g["depth"][0]}, o)
    gm.close()


@pytest.mark.parametrize("tile", [(64, 32), (32, 32), (32, 16), (16, 16)])
def test_render_exact_ties_lower_id_wins(tile):
    """Duplicated faces (same vertex order: equal inverse depth bit for bit) under shuffled ids,
    plus copies with rotated vertex order (near ties): ids and depth bit-exact, so the lower id
    wins every exact tie as in the oracle."""
    cam = cases.small_pinhole(w=75, h=53, f=50.0)
    v, f = cases.plane_grid(12, 9, (-2.0, -1.5, 3.0), (4.0, 0.0, 1.0), (0.0, 3.0, 0.5), jitter=0.3, seed=3)
    ff = np.concatenate([f, f, f[:, [1, 2, 0]]])[cases.rng(5).permutation(3 * len(f))]
    lab = np.zeros(len(ff), np.uint8)
    o = oracle.OracleMap(v, ff, lab).render(np.eye(4), cam)
    gm = rm.Map(v, ff, lab)
    gm.set_tuning(tile=tile)
    g = rm.render_depth(gm, np.eye(4)[None], rm.Intrinsics.from_camera(cam))
    _same_render({"tri_id": g["tri_id"][0], "depth": g["depth"][0]}, o)
    gm.close()


def test_render_watertight_plane_gpu():
    cam = cases.small_pinhole(w=96, h=72, f=70.0)
    v, f = cases.plane_grid(41, 29, (-4, -4, 1.0), (8, 0, 3.0), (0, 8, 2.0), jitter=0.2, seed=9)
    om = oracle.OracleMap(v, f, np.zeros(len(f), np.uint8))
    o = om.render(np.eye(4), cam, frags=True)
    assert np.all(o["frags"] == 1)
    gm = rm.Map(v, f, np.zeros(len(f), np.uint8))
    g = rm.render_depth(gm, np.eye(4)[None], rm.Intrinsics.from_camera(cam))
    _same_render({"tri_id": g["tri_id"][0], "depth": g["depth"][0]}, o)
    assert not np.isnan(_np(g["depth"])).any()


def check_barycentrics(om, pose, cam, keys, bg):
    """GPU FP32 barycentrics against the oracle's FP64 ones, pixel by pixel.

    The kernel takes the hit point as t32 * r, with t32 the z-buffer's FP32 depth, and
    camera-frame vertices transformed in FP32. Moving the hit point by d moves (b1, b2) by at
    most |d| / h_min, h_min being the triangle's smallest altitude; so the bound per pixel is
    (|t32 - t64| |r| + 16 u (|t r| + max |v| + X)) / h_min with u = 2^-24 and X the largest
    re-centred map coordinate (the FP32 pose matrix and map vertices round at that scale);
    16 u covers the vertex transform, the edge differences and the two cross products."""
    b64 = om.barycentrics(pose, cam, keys)
    t32, ids = oracle.decode(keys)
    hit = ids >= 0
    assert np.array_equal(np.isnan(bg[..., 0]), ~hit) and np.array_equal(np.isnan(bg[..., 1]), ~hit)
    t64 = om.depth_exact(pose, cam, keys)[hit]
    R, tr = pose[:3, :3], pose[:3, 3]
    w = (om.v.astype(np.float64)[om.faces[ids[hit]]] - tr) @ R
    if cam.model == "pinhole":
        jj, ii = np.nonzero(hit)
        r = np.stack([(ii + 0.5 - np.float32(cam.cx)) / np.float32(cam.fx),
                      (jj + 0.5 - np.float32(cam.cy)) / np.float32(cam.fy), np.ones(ii.size)], 1)
    else:
        r = cam.ray_table_f32().astype(np.float64)[hit]
    rn = np.linalg.norm(r, axis=1)
    e = [w[:, 1] - w[:, 0], w[:, 2] - w[:, 1], w[:, 0] - w[:, 2]]
    area2 = np.linalg.norm(np.cross(e[0], -e[2]), axis=1)
    hmin = area2 / np.max(np.stack([np.linalg.norm(x, axis=1) for x in e], 1), axis=1)
    u = 2.0 ** -24
    dist = (np.abs(t32[hit].astype(np.float64) - t64) * rn
            + 16 * u * (np.abs(t64) * rn + np.abs(w).max(axis=(1, 2)) + np.abs(om.vr).max()))
    bound = dist / hmin + 1e-6
    err = np.abs(bg[hit].astype(np.float64) - b64[hit]).max(axis=1)
    ratio = err / bound
    checks.WORST["bary"] = max(checks.WORST.get("bary", 0.0), float(ratio.max()))
    assert ratio.max() <= 1.0, (float(ratio.max()), float(err[np.argmax(ratio)]), float(bound[np.argmax(ratio)]))
    assert np.median(err) < 1e-4, float(np.median(err))


def test_render_barycentrics(c1):
    for P in (c1["gt"], c1["start"]):
        g = rm.render_depth(c1["gm"], P[None], c1["intr"], want_bary=True)
        o = c1["om"].render(P, c1["cam"])
        _same_render({"tri_id": g["tri_id"][0], "depth": g["depth"][0]}, o)
        check_barycentrics(c1["om"], P, c1["cam"], o["keys"], _np(g["bary"][0]))


def test_render_bin_overflow_retry(c1):
    """A tiny starting bin capacity overflows; the library grows it and the result is exact."""
    c1["gm"].set_tuning(tile=(32, 32), bin_capacity=8)
    g = rm.render_depth(c1["gm"], c1["gt"][None], c1["intr"])
    assert c1["gm"].get_tuning()["bin_capacity"] > 8
    o = c1["om"].render(c1["gt"], c1["cam"])
    _same_render({"tri_id": g["tri_id"][0], "depth": g["depth"][0]}, o)
    c1["gm"].set_tuning()


def test_render_empty_and_away():
    cam = cases.small_pinhole()
    intr = rm.Intrinsics.from_camera(cam)
    gm = rm.Map(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32), np.zeros(0, np.uint8))
    g = rm.render_depth(gm, np.eye(4)[None], intr)
    assert torch.isnan(g["depth"]).all() and (g["tri_id"] == -1).all()
    v, f = cases.plane_grid(3, 3, (-1, -1, -2.0), (2, 0, 0), (0, 2, 0))
    gm = rm.Map(v, f, np.zeros(len(f), np.uint8))
    g = rm.render_depth(gm, np.eye(4)[None], intr)
    assert torch.isnan(g["depth"]).all()


def test_render_one_pixel_image(c1):
    cam = dataclasses.replace(c1["cam"], width=1, height=1, cx=0.5, cy=0.5)
    g = rm.render_depth(c1["gm"], c1["gt"][None], rm.Intrinsics.from_camera(cam))
    o = c1["om"].render(c1["gt"], cam)
    _same_render({"tri_id": g["tri_id"][0], "depth": g["depth"][0]}, o)


# ---------------------------------------------------------------------------------------
# cost and adjoint
# ---------------------------------------------------------------------------------------

def test_cost_grad_parity_config1(c1):
    r = cases.rng(6)
    poses = [c1["gt"], c1["start"]] + [synth.perturb_fixed(c1["gt"], r, 0.1, 4.0) for _ in range(4)]
    sd, sc = c1["scan"]
    g = rm.cost_grad(c1["gm"], c1["gscan"], np.stack(poses))
    gc = rm.cost(c1["gm"], c1["gscan"], np.stack(poses))
    for k, P in enumerate(poses):
        o = c1["om"].cost(P, c1["cam"], sd, sc)
        _check_cost(g, o, k)
        _check_cost(gc, o, k, grad=False)


def test_cost_parity_weights_and_eps(c1):
    prm = rm.cost_params(eps=0.05, w_fofo=1.0, w_fofu=2.5, w_fufo=0.5)
    oprm = oracle.make_params(eps=0.05, w_fofo=1.0, w_fofu=2.5, w_fufo=0.5)
    sd, sc = c1["scan"]
    g = rm.cost_grad(c1["gm"], c1["gscan"], c1["start"][None], prm)
    o = c1["om"].cost(c1["start"], c1["cam"], sd, sc, params=oprm)
    _check_cost(g, o)


def test_cost_parity_with_fu_faces_and_nan_scan():
    c = cases.config2(seed=2200, target_fo=60_000, target_fu=15_000)
    cam = dataclasses.replace(c["cam"], width=213, height=161, fx=175.0, fy=175.0, cx=106.5, cy=80.5)
    mesh = c["mesh"]
    r = cases.rng(9)
    sd, sc = synth.synth_scan(mesh, cam, c["gt"], r, sigma_rel=0.005, dropout=0.05, dropout_as_nan=True)
    om = oracle.OracleMap(mesh.vertices, mesh.faces, mesh.labels)
    gm = rm.Map(mesh.vertices, mesh.faces, mesh.labels)
    scan = rm.Scan.make(rm.Intrinsics.from_camera(cam), sd, sc)
    poses = [c["gt"], c["start"], synth.perturb_fixed(c["gt"], r, 0.2, 5.0)]
    g = rm.cost_grad(gm, scan, np.stack(poses))
    tot = np.zeros(6, np.int64)
    for k, P in enumerate(poses):
        o = om.cost(P, cam, sd, sc)
        _check_cost(g, o, k)
        tot += o["counts"]
    assert np.all(tot > 0)   # every Table I outcome was exercised


def test_cost_grad_empty_batch_and_batch_of_one(c1):
    """No poses: empty outputs and no launch failure; a batch of one equals that pose inside a
    larger batch bit for bit."""
    g = rm.cost_grad(c1["gm"], c1["gscan"], np.zeros((0, 4, 4)))
    assert g["counts"].shape[0] == 0 and g["grad"].shape[0] == 0
    poses = np.stack([c1["gt"], c1["start"], c1["gt"]])
    gb = rm.cost_grad(c1["gm"], c1["gscan"], poses)
    g1 = rm.cost_grad(c1["gm"], c1["gscan"], poses[1:2])
    for key in ("counts", "e_table", "e_ls", "grad", "jtj"):
        assert torch.equal(gb[key][1:2], g1[key]), key
    assert torch.equal(gb["grad"][0], gb["grad"][2])


def test_cost_host_buffers_match_device(c1):
    """Host (numpy) scan and poses through the same ABI give the same numbers."""
    import ctypes
    from paper_1702_06813_gb300 import _native as N
    sd, sc = c1["scan"]
    intr = c1["intr"]
    scan = N.rm_scan(intr.c(), sd.ctypes.data, sc.ctypes.data)
    poses = np.ascontiguousarray(np.stack([c1["gt"], c1["start"]]))
    counts = np.zeros((2, 6), np.int64)
    etab = np.zeros(2, np.int64)
    els = np.zeros(2)
    grad = np.zeros((2, 6))
    jtj = np.zeros((2, 21))
    out = N.rm_cost_out(counts.ctypes.data, etab.ctypes.data, els.ctypes.data, grad.ctypes.data, jtj.ctypes.data)
    prm = rm.cost_params()
    N.check(N.lib().rm_cost_grad(c1["gm"].handle, ctypes.byref(scan), poses.ctypes.data_as(ctypes.c_void_p), 2,
                                 ctypes.byref(prm), ctypes.byref(out), None))
    g = rm.cost_grad(c1["gm"], c1["gscan"], poses)
    assert np.array_equal(counts, _np(g["counts"]))
    assert np.array_equal(els, _np(g["e_ls"]))
    assert np.array_equal(grad, _np(g["grad"]))


def test_batched_waves_equal_single_calls(c1):
    r = cases.rng(10)
    poses = np.stack([synth.perturb_fixed(c1["gt"], r, 0.1, 3.0) for _ in range(7)])
    c1["gm"].set_tuning(wave_poses=3)
    gb = rm.cost_grad(c1["gm"], c1["gscan"], poses)
    c1["gm"].set_tuning()
    for k in range(7):
        g1 = rm.cost_grad(c1["gm"], c1["gscan"], poses[k:k + 1])
        assert torch.equal(gb["counts"][k], g1["counts"][0])
        assert torch.equal(gb["e_ls"][k], g1["e_ls"][0])
        assert torch.equal(gb["grad"][k], g1["grad"][0])


def test_cost_grad_repeatable_across_bin_rounds_and_record_order(c1):
    """Bin record order depends on the order of setup's atomics, and a 64x32 tile of the
    160x120 view holds hundreds of records (several staging rounds); results must not depend
    on either: repeated calls and the batched kernel agree bit for bit."""
    r = cases.rng(11)
    poses = np.stack([c1["gt"], c1["start"]] + [synth.perturb_fixed(c1["gt"], r, 0.1, 3.0) for _ in range(6)])
    c1["gm"].set_tuning(tile=(64, 32))
    a = rm.cost_grad(c1["gm"], c1["gscan"], poses)
    b = rm.cost_grad(c1["gm"], c1["gscan"], poses)
    c1["gm"].set_tuning()
    p = rm.cost_grad_batch(c1["gm"], scans=c1["gscan"], poses=torch.as_tensor(poses))
    for key in ("counts", "e_table", "e_ls", "grad", "jtj"):
        assert torch.equal(a[key], b[key]), key
        assert torch.equal(a[key], p[key]), key
    sd, sc = c1["scan"]
    for k in range(len(poses)):
        _check_cost(a, c1["om"].cost(poses[k], c1["cam"], sd, sc), k)


def test_gradient_matches_oracle_frozen_fd(c1):
    """The GPU adjoint against central differences of the oracle's FP64 frozen cost."""
    sd, sc = c1["scan"]
    P = c1["start"]
    g = _np(rm.cost_grad(c1["gm"], c1["gscan"], P[None])["grad"])[0]
    h = 1e-5
    fd = np.zeros(6)
    for a in range(6):
        xi = np.zeros(6)
        xi[a] = h
        fd[a] = (c1["om"].cost_frozen(P, c1["cam"], sd, sc, xi) - c1["om"].cost_frozen(P, c1["cam"], sd, sc, -xi)) / (2 * h)
    checks.close_elementwise(g, fd, EPS_REL_GRAD, "grad_vs_fd")


def test_autograd_function(c1):
    P = c1["start"]
    sd, sc = c1["scan"]
    for xi0 in [np.zeros(6), np.array([0.01, -0.02, 0.015, 0.01, -0.005, 0.02])]:
        xi = torch.tensor(xi0, dtype=torch.float64, requires_grad=True)
        e = rm.RenderMapCost.apply(xi, P, c1["gm"], c1["gscan"], None)
        e.backward()
        # the oracle at the retracted pose, and FD through the oracle's frozen cost
        Pr = oracle.se3_right(P, xi0)
        o = c1["om"].cost(Pr, c1["cam"], sd, sc)
        assert abs(e.item() - o["e_ls"]) <= EPS_REL_COST * o["e_ls"]
        # exact chain rule: d e(P exp(xi))/d xi = J_r(xi)^T g(P exp(xi))
        g_or = o["grad"]
        _, jr = rm.pose_retract(P[None], xi0[None], with_jacobian=True)
        want = _np(jr[0]).T @ g_or
        checks.close_elementwise(_np(xi.grad), want, EPS_REL_GRAD, "autograd")


def test_retraction_and_right_jacobian():
    from scipy.spatial.transform import Rotation
    r = cases.rng(11)
    T = synth.pose_from(np.array([1.0, -2.0, 0.5]), 0.3, 0.1, -0.2)
    for _ in range(4):
        xi = r.normal(scale=0.4, size=6)
        out, jr = rm.pose_retract(T[None], xi[None], with_jacobian=True)
        assert np.allclose(_np(out[0]), oracle.se3_right(T, xi), atol=1e-12)
        # columns of J_r: exp(xi)^-1 exp(xi + h e_k) ~ exp(J_r h e_k)
        E0 = oracle.se3_right(np.eye(4), xi)
        for k in range(6):
            h = 1e-6
            d = np.zeros(6)
            d[k] = h
            D = np.linalg.inv(E0) @ oracle.se3_right(np.eye(4), xi + d)
            col = np.concatenate([D[:3, 3], Rotation.from_matrix(D[:3, :3]).as_rotvec()]) / h
            assert np.allclose(col, _np(jr[0])[:, k], atol=2e-5)


# ---------------------------------------------------------------------------------------
# Levenberg-Marquardt on the device
# ---------------------------------------------------------------------------------------

def _pose_gap(a, b):
    from scipy.spatial.transform import Rotation
    dt = np.linalg.norm(a[:3, 3] - b[:3, 3])
    da = math.degrees(Rotation.from_matrix(a[:3, :3].T @ b[:3, :3]).magnitude())
    return dt, da


def test_align_matches_oracle_config1(c1):
    sd, sc = c1["scan"]
    gt = synth.pose_from(c1["gt"][:3, 3], 0.7, math.radians(20.0), 0.0)
    start = synth.perturb_fixed(gt, cases.rng(12), 0.05, 2.0)
    # noisy scan of the world from the tilted pose
    sd, sc = synth.synth_scan(c1["mesh"], c1["cam"], gt, cases.rng(13), sigma_abs=0.01, dropout=0.05)
    scan = rm.Scan.make(c1["intr"], sd, sc)
    pg, rep = rm.align(c1["gm"], scan, start, max_iters=50, step_tol=1e-7)
    po, orep = c1["om"].align(start, c1["cam"], sd, sc, max_iters=50, step_tol=1e-7)
    dt, da = _pose_gap(pg, po)
    assert dt < 1e-3 and da < 1e-2, (dt, da, rep, orep)
    assert rep["e_ls_final"] < rep["e_ls_initial"]
    dgt, agt = _pose_gap(pg, gt)
    assert dgt < 0.01 and agt < 0.5


# ---------------------------------------------------------------------------------------
# ray-table (panoramic) camera
# ---------------------------------------------------------------------------------------

def _soup_around(seed, n=120):
    r = cases.rng(seed)
    c = r.normal(size=(n, 3))
    c /= np.linalg.norm(c, axis=1, keepdims=True)
    c *= r.uniform(2, 15, (n, 1))
    v = c[:, None, :] + r.normal(scale=1.0, size=(n, 3, 3)) * r.uniform(0.1, 3.0, (n, 1, 1))
    # a large ground triangle under the sensor (contains the down pole) and one over it
    v = np.concatenate([v, np.array([[[-40, 3, -40], [40, 3, -40], [0, 3, 60]],
                                     [[-30, -4, 30], [30, -4, 30], [0, -4, -50]]], float)])
    vc = v.reshape(-1, 3).astype(np.float32)
    return vc, np.arange(vc.shape[0], dtype=np.int32).reshape(-1, 3)


@pytest.mark.parametrize("seed", [21, 22, 23])
def test_raytable_render_bit_exact_soup(seed):
    cam = cases.small_spherical(w=96, h=16)
    vc, f = _soup_around(seed)
    om = oracle.OracleMap(vc, f, np.zeros(len(f), np.uint8))
    o = om.render(np.eye(4), cam)
    gm = rm.Map(vc, f, np.zeros(len(f), np.uint8))
    g = rm.render_depth(gm, np.eye(4)[None], rm.Intrinsics.from_camera(cam))
    _same_render({"tri_id": g["tri_id"][0], "depth": g["depth"][0]}, o)
    assert (~np.isnan(o["depth"])).mean() > 0.3


def test_raytable_closed_box_gpu():
    v, f = cases.closed_box((-6, -5, -2), (7, 4, 5), 0.9)
    cam = cases.small_spherical(w=128, h=24)
    om = oracle.OracleMap(v, f, np.zeros(len(f), np.uint8))
    pose = synth.pose_from(np.array([0.5, 0.3, 0.1]), 0.7, 0.05, 0.02)
    o = om.render(pose, cam)
    gm = rm.Map(v, f, np.zeros(len(f), np.uint8))
    g = rm.render_depth(gm, pose[None], rm.Intrinsics.from_camera(cam))
    _same_render({"tri_id": g["tri_id"][0], "depth": g["depth"][0]}, o)
    assert not torch.isnan(g["depth"]).any()


@pytest.fixture(scope="module")
def lidar():
    w = synth.workload_lidar(seed=4100, target_fo=140_000, target_fu=60_000, n_panels=120)
    om = oracle.OracleMap(w["mesh"].vertices, w["mesh"].faces, w["mesh"].labels)
    gm = rm.Map(w["mesh"].vertices, w["mesh"].faces, w["mesh"].labels)
    intr = rm.Intrinsics.from_camera(w["cam"])
    return dict(w, om=om, gm=gm, intr=intr, gscan=rm.Scan.make(intr, *w["scan"]))


def test_raytable_lidar_render_and_cost(lidar):
    r = cases.rng(31)
    poses = [lidar["gt"], lidar["start"], synth.perturb_fixed(lidar["gt"], r, 1.0, 10.0)]
    g = rm.render_depth(lidar["gm"], np.stack(poses), lidar["intr"], want_bary=True)
    gc = rm.cost_grad(lidar["gm"], lidar["gscan"], np.stack(poses))
    sd, sc = lidar["scan"]
    for k, P in enumerate(poses):
        o = lidar["om"].render(P, lidar["cam"])
        _same_render({"tri_id": g["tri_id"][k], "depth": g["depth"][k]}, o)
        check_barycentrics(lidar["om"], P, lidar["cam"], o["keys"], _np(g["bary"][k]))
        _check_cost(gc, lidar["om"].cost(P, lidar["cam"], sd, sc), k)


def test_raytable_align_matches_oracle(lidar):
    """From 30 cm / 3 deg the truncated surrogate gains inliers slowly: LM needs ~120
    iterations to meet step_tol here; both sides must converge to the same pose."""
    sd, sc = lidar["scan"]
    pg, rep = rm.align(lidar["gm"], lidar["gscan"], lidar["start"], max_iters=200, step_tol=1e-7)
    po, orep = lidar["om"].align(lidar["start"], lidar["cam"], sd, sc, max_iters=200, step_tol=1e-7)
    assert rep["converged"] == 1 and orep["converged"] == 1, (rep, orep)
    dt, da = _pose_gap(pg, po)
    assert dt < 1e-3 and da < 1e-2, (dt, da, rep, orep)
    dgt, agt = _pose_gap(pg, lidar["gt"])
    assert dgt < 0.05 and agt < 0.5, (dgt, agt)


@pytest.mark.parametrize("axis,span", [(0, 0.2), (2, 0.15), (5, 0.05)])
def test_cost_sweep_matches_oracle(c1, axis, span):
    """Fig. 7's sweep along one twist axis, evaluated as one batch on the device: Table I
    counts exact and the surrogate within 1e-5 at every sample."""
    c1["gm"].set_tuning()
    sd, sc = c1["scan"]
    g = rm.cost_sweep(c1["gm"], c1["gscan"], c1["start"], axis, span, 11)
    ts, outs = c1["om"].cost_sweep(c1["start"], c1["cam"], sd, sc, axis, span, 11)
    for k, o in enumerate(outs):
        _check_cost(g, o, k, grad=False)
    # the sweep's samples are the same poses as separate evaluations
    single = rm.cost(c1["gm"], c1["gscan"], rm.pose_retract(c1["start"][None], np.eye(6)[axis][None] * ts[0]))
    assert torch.equal(single["counts"][0], g["counts"][0])


def test_twist_grad_is_the_right_jacobian_chain_rule():
    """rm_twist_grad: scale * J_r(xi)^T g, with J_r from rm_pose_retract (itself checked
    against finite differences above), for device and host buffers."""
    import ctypes
    from paper_1702_06813_gb300 import _native as N
    r = cases.rng(12)
    xi = r.normal(scale=0.3, size=(5, 6))
    g = r.normal(size=(5, 6))
    s = r.uniform(0.5, 2.0, size=5)
    _, jr = rm.pose_retract(np.tile(np.eye(4), (5, 1, 1)), xi, with_jacobian=True)
    want = s[:, None] * np.einsum("krc,kr->kc", _np(jr), g)
    got = _np(rm.twist_grad(xi, g, s))
    assert np.allclose(got, want, rtol=1e-13, atol=1e-13)
    host = np.empty((5, 6))
    st = N.lib().rm_twist_grad(np.ascontiguousarray(xi).ctypes.data, np.ascontiguousarray(g).ctypes.data,
                               None, 5, host.ctypes.data, None)
    assert st == N.RM_OK
    assert np.allclose(host, want / s[:, None], rtol=1e-13, atol=1e-13)
