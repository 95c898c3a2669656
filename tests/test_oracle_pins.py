"""Pins of the CPU oracle to things other than itself (no GPU needed).

Each test fixes a value the paper prints (Table I), a closed form, an invariant or a brute-force
result, so that a dropped term, a wrong sign, a wrong index or a transposed operand anywhere in
the oracle fails at least one of them.
"""
from __future__ import annotations

import math
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import cases
import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
MAP_CLASS = {"FO": 0, "FU": 1, "UO": 2, "NaN": 3}
SCAN_CLASS = {"FO": 0, "FU": 1, "NaN": 2}
VALUE_OF_OUTCOME = {-1: 0, 0: -1, 1: +1, 2: -1, 3: +1, 4: -1, 5: +1}


# ---------------------------------------------------------------------------------------
# Table I (Sec. IV.B)
# ---------------------------------------------------------------------------------------

def _table1_rows():
    rows = []
    with open(os.path.join(GOLDEN, "table1.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if not line:
                continue
            parts = line.split()
            rows.append((parts[0], parts[1], np.float32(parts[2]), int(parts[3])))
    return rows


@pytest.mark.parametrize("mc,sc,dz,value", _table1_rows())
def test_table1_golden(mc, sc, dz, value):
    if sc == "NaN" or mc == "NaN":
        # ignored before the table is consulted (no surface / dead pixel)
        assert value == 0
        if mc == "NaN":
            assert oracle.table1(MAP_CLASS[mc], SCAN_CLASS[sc], float(dz)) == -1
        return
    oc = oracle.table1(MAP_CLASS[mc], SCAN_CLASS[sc], float(dz), float(np.float32(0.1)))
    assert VALUE_OF_OUTCOME[oc] == value


def test_table1_cost_pixels_match_golden():
    """The per-pixel path of the cost (not just the table function) reproduces Table I:
    a fronto-parallel wall split into FO and FU halves against hand-set scan pixels."""
    cam = cases.small_pinhole(w=16, h=8, f=8.0)
    # wall at z = 2 covering the view, left half FO, right half FU
    v, f = cases.plane_grid(2, 1, (-20, -20, 2.0), (40, 0, 0), (0, 40, 0))
    labels = np.array([0, 0, 1, 1], np.uint8)  # faces of cell 0 FO, cell 1 FU
    om = oracle.OracleMap(v, f, labels)
    pose = np.eye(4)
    r = om.render(pose, cam)
    assert np.all(r["depth"] == np.float32(2.0))
    lab = labels[r["tri_id"]]
    sd = np.full((cam.height, cam.width), 2.0, np.float32)
    sc = np.zeros((cam.height, cam.width), np.uint8)
    # column-wise cases: dz = 2 - d_s
    offs = [0.0, 0.05, -0.2, 0.3, 0.0, 0.5, -0.5, 0.0]
    classes = [0, 0, 0, 0, 1, 1, 1, 2]
    for j in range(cam.height):
        sd[j, :] = np.float32(2.0 - offs[j])
        sc[j, :] = classes[j]
    sd[sc == 2] = np.nan
    out = om.cost(pose, cam, sd, sc, per_pixel=True)
    for j in range(cam.height):
        for i in range(cam.width):
            mc = int(lab[j, i])
            dz = np.float32(np.float32(2.0) - sd[j, i])
            expect = 0 if sc[j, i] == 2 else VALUE_OF_OUTCOME[oracle.table1(mc, int(sc[j, i]), float(dz))]
            assert VALUE_OF_OUTCOME[int(out["outcome"][j, i])] == expect
    # golden spot checks, written from the table by hand
    name = {0: "FO", 1: "FU"}
    for j, want_fo, want_fu in [(0, -1, -1), (3, +1, +1), (4, +1, 0), (5, -1, 0), (6, +1, 0)]:
        fo_i, fu_i = 0, cam.width - 1
        assert name[int(lab[j, fo_i])] == "FO" and name[int(lab[j, fu_i])] == "FU"
        assert VALUE_OF_OUTCOME[int(out["outcome"][j, fo_i])] == want_fo
        assert VALUE_OF_OUTCOME[int(out["outcome"][j, fu_i])] == want_fu


# ---------------------------------------------------------------------------------------
# z-buffer visibility
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_zbuffer_bbox_equals_brute_force_pinhole(seed):
    cam = cases.small_pinhole()
    vc, f = cases.random_tris(seed, 60)
    kb, fb, sb = oracle.zbuffer(vc, f, cam, brute=True, frags=True)
    k, fr, s = oracle.zbuffer(vc, f, cam, brute=False, frags=True)
    assert sb.n_clipped > 0  # the near-plane path is exercised
    assert np.array_equal(kb, k)
    assert np.array_equal(fb, fr)


def test_zbuffer_exact_ties_lower_id_wins():
    """Every face of a jittered grid twice, with the same vertex order (so both copies give the
    same inverse depth bit for bit at every sample), under shuffled ids: the visible surface is
    the single mesh's, and at every pixel the lower of the two ids wins (the raster rule of
    equal depths)."""
    cam = cases.small_pinhole(w=75, h=53, f=50.0)
    v, f = cases.plane_grid(12, 9, (-2.0, -1.5, 3.0), (4.0, 0.0, 1.0), (0.0, 3.0, 0.5), jitter=0.3, seed=3)
    perm = cases.rng(5).permutation(2 * len(f))
    ff = np.concatenate([f, f])[perm]
    orig = perm % len(f)  # geometric face of each id
    one = oracle.OracleMap(v, f, np.zeros(len(f), np.uint8)).render(np.eye(4), cam)
    two = oracle.OracleMap(v, ff, np.zeros(len(ff), np.uint8)).render(np.eye(4), cam)
    hit = one["tri_id"] >= 0
    assert hit.sum() > 1000
    assert np.array_equal(two["tri_id"] >= 0, hit)
    assert np.array_equal(two["depth"][hit].view(np.uint32), one["depth"][hit].view(np.uint32))
    won = two["tri_id"][hit]
    assert np.array_equal(orig[won], one["tri_id"][hit])
    lower = np.full(len(f), np.iinfo(np.int64).max)
    np.minimum.at(lower, orig, np.arange(len(ff)))
    assert np.array_equal(won, lower[orig[won]])


@pytest.mark.parametrize("seed", [5, 6, 7])
def test_zbuffer_bounds_equal_brute_force_raytable(seed):
    cam = cases.small_spherical()
    r = cases.rng(seed)
    n = 80
    # triangles all around the sensor, some across the azimuth seam (-z), some over the poles
    c = r.normal(size=(n, 3))
    c /= np.linalg.norm(c, axis=1, keepdims=True)
    c *= r.uniform(2, 15, (n, 1))
    v = c[:, None, :] + r.normal(scale=1.0, size=(n, 3, 3)) * r.uniform(0.1, 3.0, (n, 1, 1))
    v = np.concatenate([v, np.array([[[-40, 3, -40], [40, 3, -40], [0, 3, 60]]], float)])  # ground under
    vc = v.reshape(-1, 3).astype(np.float32)
    f = np.arange(vc.shape[0], dtype=np.int32).reshape(-1, 3)
    kb, fb, _ = oracle.zbuffer(vc, f, cam, brute=True, frags=True)
    k, fr, _ = oracle.zbuffer(vc, f, cam, brute=False, frags=True)
    assert np.array_equal(kb, k)
    assert np.array_equal(fb, fr)
    assert (fb > 0).mean() > 0.3


@pytest.mark.parametrize("jitter", [0.0, 0.2])
def test_watertight_screen_filling_plane(jitter):
    """A tessellated plane covering the view covers every pixel exactly once (pre-z)."""
    cam = cases.small_pinhole(w=64, h=48, f=50.0)
    for origin, u, v in [((-3, -3, 2.0), (6, 0, 0), (0, 6, 0)),               # fronto-parallel
                         ((-4, -4, 1.0), (8, 0, 3.0), (0, 8, 2.0))]:           # oblique
        vw, f = cases.plane_grid(23, 17, origin, u, v, jitter=jitter, seed=11)
        _, fr, _ = oracle.zbuffer(vw, f, cam, frags=True)
        assert np.all(fr == 1)


def test_watertight_across_near_plane():
    """A floor crossing the near plane: covered exactly once where the exact hit lies beyond
    the near plane, never more than once anywhere."""
    cam = cases.small_pinhole(w=64, h=48, f=40.0, near=0.6)
    vw, f = cases.plane_grid(30, 30, (-6, 1.0, 0.05), (12, 0, 0), (0, 0.0, 12.0), jitter=0.2, seed=3)
    keys, fr, st = oracle.zbuffer(vw, f, cam, frags=True)
    assert st.n_clipped > 0
    assert fr.max() == 1
    j, i = np.meshgrid(np.arange(cam.height), np.arange(cam.width), indexing="ij")
    ry = (j + 0.5 - cam.cy) / cam.fy
    rx = (i + 0.5 - cam.cx) / cam.fx
    with np.errstate(divide="ignore"):
        z = np.where(ry > 0, 1.0 / ry, np.inf)   # floor y = 1: hit at z = 1 / ry
    x = rx * z
    inside = (z >= cam.near + 0.05) & (z <= 11.5) & (np.abs(x) <= 5.5)
    outside = (z < cam.near - 0.05) | (z > 12.6) | (np.abs(x) > 6.5)
    assert np.all(fr[inside] == 1)
    assert np.all(fr[outside] == 0)


def test_watertight_closed_box_from_inside_pinhole():
    v, f = cases.closed_box((-1.5, -1.2, -1.0), (1.7, 1.3, 1.4), 0.37)
    cam = cases.small_pinhole(w=64, h=48, f=30.0)
    om = oracle.OracleMap(v, f, np.zeros(len(f), np.uint8))
    for yaw in np.linspace(0, 2 * math.pi, 7, endpoint=False):
        pose = synth.pose_from(np.array([0.1, -0.05, 0.2]), yaw, 0.3, -0.2)
        r = om.render(pose, cam, frags=True)
        assert np.all(r["frags"] == 1)
        assert not np.isnan(r["depth"]).any()


def test_watertight_closed_box_from_inside_raytable():
    v, f = cases.closed_box((-6, -5, -2), (7, 4, 5), 0.9)
    cam = cases.small_spherical(w=128, h=24)
    om = oracle.OracleMap(v, f, np.zeros(len(f), np.uint8))
    pose = synth.pose_from(np.array([0.5, 0.3, 0.1]), 0.7, 0.05, 0.02)
    r = om.render(pose, cam, frags=True)
    assert np.all(r["frags"] == 1)
    assert not np.isnan(r["depth"]).any()


# ---------------------------------------------------------------------------------------
# depth: closed forms
# ---------------------------------------------------------------------------------------

def test_depth_fronto_parallel_wall_is_constant():
    cam = cases.small_pinhole(w=40, h=30, f=35.0)
    for D in [0.5, 1.0, 2.75, 7.3]:
        v, f = cases.plane_grid(9, 7, (-30, -30, D), (60, 0, 0), (0, 60, 0), jitter=0.2, seed=2)
        keys, _, _ = oracle.zbuffer(v, f, cam)
        depth, _ = oracle.decode(keys)
        # d = round(nz * D) then d / nz: at most one rounding step away from D each way
        assert np.all(np.abs(depth - np.float32(D)) <= 2 * np.spacing(np.float32(D)))


def test_depth_matches_analytic_ray_cast_of_room():
    """Contract FP32 depth and FP64 depth vs an independent analytic ray-box cast."""
    mesh = synth.room_mesh(7, n_boxes=0)
    cam = synth.cam_160x120()
    r = cases.rng(8)
    om = oracle.OracleMap(mesh.vertices, mesh.faces, mesh.labels)
    for _ in range(3):
        pose = synth.room_pose(r, mesh)
        out = om.render(pose, cam)
        d_ref, _ = synth.synth_scan(
            synth.Mesh(mesh.vertices, mesh.faces, mesh.labels, np.zeros((0, 2, 3)), mesh.room),
            dataclass_replace(cam, range_max=math.inf), pose, r)
        d64 = om.depth_exact(pose, cam, out["keys"])
        rel32 = np.abs(out["depth"].astype(np.float64) - d_ref) / d_ref
        rel64 = np.abs(d64 - d_ref) / d_ref
        assert np.nanmax(rel32) < 5e-6
        assert np.nanmax(rel64) < 1e-6   # the analytic cast is float32-rounded at the end
        assert not np.isnan(out["depth"]).any()


def packed(a, b):
    """Index of (a, b), a <= b, in the row-major packed upper triangle of a 6x6 matrix."""
    return a * 6 - a * (a - 1) // 2 + (b - a)


def dataclass_replace(obj, **kw):
    import dataclasses
    return dataclasses.replace(obj, **kw)


def test_depth_oblique_plane_closed_form():
    """Plane n.x = d seen from a known pose: depth = d_c / (n_c . r) at every pixel."""
    cam = cases.small_pinhole(w=50, h=40, f=45.0)
    n_w = np.array([0.3, -0.2, 1.0])
    n_w /= np.linalg.norm(n_w)
    d_w = 4.0
    # parametrise the plane
    u = np.cross(n_w, [0, 1.0, 0])
    u /= np.linalg.norm(u)
    w = np.cross(n_w, u)
    o = n_w * d_w - 20 * u - 20 * w
    v, f = cases.plane_grid(11, 13, o, 40 * u, 40 * w, jitter=0.2, seed=4)
    pose = synth.pose_from(np.array([0.2, 0.1, 0.3]), 0.0, 0.0, 0.0)
    pose[:3, :3] = Rotation.from_rotvec([0.1, -0.15, 0.05]).as_matrix()
    om = oracle.OracleMap(v, f, np.zeros(len(f), np.uint8))
    out = om.render(pose, cam)
    R, t = pose[:3, :3], pose[:3, 3]
    n_c = R.T @ n_w
    d_c = d_w - n_w @ t
    jj, ii = np.meshgrid(np.arange(cam.height), np.arange(cam.width), indexing="ij")
    ray = np.stack([(ii + 0.5 - cam.cx) / cam.fx, (jj + 0.5 - cam.cy) / np.float32(cam.fy),
                    np.ones_like(ii, float)], -1)
    ray[..., 1] = (jj + 0.5 - cam.cy) / np.float64(np.float32(cam.fy))
    ray[..., 0] = (ii + 0.5 - np.float64(np.float32(cam.cx))) / np.float64(np.float32(cam.fx))
    ray[..., 1] = (jj + 0.5 - np.float64(np.float32(cam.cy))) / np.float64(np.float32(cam.fy))
    closed = d_c / (ray @ n_c)
    assert not np.isnan(out["depth"]).any()
    assert np.max(np.abs(out["depth"] - closed) / closed) < 5e-6
    d64 = om.depth_exact(pose, cam, out["keys"])
    assert np.max(np.abs(d64 - closed) / closed) < 1e-6


def test_raytable_depth_is_range():
    """Panoramic model: a sphere-like closed box's depth is the Euclidean range along the ray."""
    v, f = cases.closed_box((-6, -5, -2), (7, 4, 5), 0.9)
    cam = cases.small_spherical(w=128, h=24)
    om = oracle.OracleMap(v, f, np.zeros(len(f), np.uint8))
    pose = np.eye(4)
    pose[:3, 3] = [0.5, 0.3, 0.1]
    out = om.render(pose, cam)
    rays = cam.ray_table_f32().astype(np.float64)
    # analytic exit distance from the box along the (unit) ray, in world = camera frame here
    lo, hi = np.array([-6, -5, -2.0]) - pose[:3, 3], np.array([7, 4, 5.0]) - pose[:3, 3]
    with np.errstate(divide="ignore"):
        t = np.minimum(np.where(rays > 0, hi / rays, np.inf), np.where(rays < 0, lo / rays, np.inf)).min(-1)
    assert np.max(np.abs(out["depth"] - t) / t) < 5e-6


# ---------------------------------------------------------------------------------------
# cost: zero at the true pose, wall slope, empty cases
# ---------------------------------------------------------------------------------------

def test_zero_cost_at_true_pose_noise_free():
    c = cases.config2(seed=2100, target_fo=40_000, target_fu=10_000)
    mesh, cam = c["mesh"], c["cam"]
    cam = dataclass_replace(cam, width=160, height=120, fx=131.25, fy=131.25, cx=80.0, cy=60.0)
    om = oracle.OracleMap(mesh.vertices, mesh.faces, mesh.labels)
    fo = mesh.labels == 0
    om_fo = oracle.OracleMap(mesh.vertices, mesh.faces[fo], mesh.labels[fo])
    r = cases.rng(77)
    seen = np.zeros(6, np.int64)
    for k in range(6):
        gt = c["gt"] if k == 0 else synth.room_pose(r, mesh)
        sd, sc = cases.scan_from_render(om_fo.render(gt, cam)["depth"], cam)
        out = om.cost(gt, cam, sd, sc, per_pixel=True)
        assert out["e_ls"] == 0.0
        assert np.all(out["counts"][[1, 3, 5]] == 0)
        n_active = int(np.sum(out["outcome"] >= 0))
        assert out["e_table"] == -n_active
        assert np.all(out["grad"] == 0.0)
        seen += out["counts"]
    assert seen[4] > 0      # FU frontier panels in front of FO surfaces are rewarded
    assert seen[2] > 0      # map FO beyond the range limit vs scan FU: rewarded


def test_wall_slope_and_cost_closed_form():
    """Camera facing a wall at 2 m, scan at 1.95 m: r = 0.05 everywhere, dt/d rho_z = -1."""
    cam = cases.small_pinhole(w=32, h=24, f=30.0)
    v, f = cases.plane_grid(5, 5, (-20, -20, 2.0), (40, 0, 0), (0, 40, 0))
    om = oracle.OracleMap(v, f, np.zeros(len(f), np.uint8))
    sd = np.full((cam.height, cam.width), 1.95, np.float32)
    sc = np.zeros_like(sd, np.uint8)
    out = om.cost(np.eye(4), cam, sd, sc, residual_exact=True)
    N = cam.width * cam.height
    r = 2.0 - np.float64(np.float32(1.95))
    assert out["counts"][0] == N
    assert out["e_ls"] == pytest.approx(0.5 * N * r * r, rel=1e-12)
    assert out["grad"][2] == pytest.approx(-N * r, rel=1e-12)
    assert out["grad"][0] == pytest.approx(0.0, abs=1e-12)
    assert out["grad"][1] == pytest.approx(0.0, abs=1e-12)
    # rotation about the optical axis leaves a fronto-parallel wall's depth unchanged
    assert out["grad"][5] == pytest.approx(0.0, abs=1e-12)
    # JtJ(rho_z, rho_z) = N
    assert out["jtj"][packed(2, 2)] == pytest.approx(N, rel=1e-12)
    assert out["jtj"][packed(0, 0)] == pytest.approx(0.0, abs=1e-12)


def test_empty_map_and_looking_away():
    cam = cases.small_pinhole()
    om = oracle.OracleMap(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32), np.zeros(0, np.uint8))
    out = om.render(np.eye(4), cam)
    assert np.isnan(out["depth"]).all() and np.all(out["tri_id"] == -1)
    v, f = cases.plane_grid(3, 3, (-1, -1, -2.0), (2, 0, 0), (0, 2, 0))   # behind the camera
    om = oracle.OracleMap(v, f, np.zeros(len(f), np.uint8))
    out = om.render(np.eye(4), cam)
    assert np.isnan(out["depth"]).all()
    sd = np.ones((cam.height, cam.width), np.float32)
    sc = np.zeros_like(sd, np.uint8)
    c = om.cost(np.eye(4), cam, sd, sc)
    assert c["e_table"] == 0 and c["e_ls"] == 0.0


# ---------------------------------------------------------------------------------------
# gradient: finite differences of the FP64 frozen-visibility cost
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("h", [1e-4, 1e-5])
def test_gradient_matches_frozen_fd(h):
    """Central differences of the FP64 frozen-visibility cost. The rotation components carry
    an O(h^2) truncation term, so at h = 1e-4 the h and h/2 differences are combined by
    Richardson extrapolation; at h = 1e-5 the plain central difference is used."""
    c = cases.config1(seed=1200)
    mesh, cam = c["mesh"], c["cam"]
    sd, sc = c["scan"]
    om = oracle.OracleMap(mesh.vertices, mesh.faces, mesh.labels)
    pose = c["start"]
    g = om.cost(pose, cam, sd, sc, residual_exact=True)["grad"]

    def central(step):
        fd = np.zeros(6)
        for a in range(6):
            xi = np.zeros(6)
            xi[a] = step
            fd[a] = (om.cost_frozen(pose, cam, sd, sc, xi) - om.cost_frozen(pose, cam, sd, sc, -xi)) / (2 * step)
        return fd

    fd = (4 * central(h / 2) - central(h)) / 3 if h >= 1e-4 else central(h)
    assert np.linalg.norm(g - fd) <= 1e-6 * np.linalg.norm(g)
    # the translation part of the step is linear in the depth's plane offset: tight agreement
    assert np.allclose(g[:3], central(h)[:3], rtol=1e-8, atol=0)


def test_frozen_cost_at_zero_twist_equals_cost():
    c = cases.config1(seed=1300)
    om = oracle.OracleMap(c["mesh"].vertices, c["mesh"].faces, c["mesh"].labels)
    sd, sc = c["scan"]
    e = om.cost(c["start"], c["cam"], sd, sc, residual_exact=True)["e_ls"]
    e0 = om.cost_frozen(c["start"], c["cam"], sd, sc, np.zeros(6))
    assert e0 == pytest.approx(e, rel=1e-12)


def test_jtj_is_outer_product_sum():
    """JtJ from the cost equals sum J J^T rebuilt from per-axis finite differences of the
    frozen residuals (rank and symmetry pin)."""
    c = cases.config1(seed=1400)
    om = oracle.OracleMap(c["mesh"].vertices, c["mesh"].faces, c["mesh"].labels)
    sd, sc = c["scan"]
    out = om.cost(c["start"], c["cam"], sd, sc, residual_exact=True)
    H = np.zeros((6, 6))
    q = 0
    for a in range(6):
        for b in range(a, 6):
            H[a, b] = H[b, a] = out["jtj"][q]
            q += 1
    ev = np.linalg.eigvalsh(H)
    assert ev.min() > 0
    # Gauss-Newton identity: for a small step xi, E(xi) ~ E + g.xi + 1/2 xi^T H xi
    xi = np.array([2e-4, -1e-4, 1.5e-4, 1e-4, -2e-4, 5e-5])
    e_xi = om.cost_frozen(c["start"], c["cam"], sd, sc, xi)
    pred = out["e_ls"] + out["grad"] @ xi + 0.5 * xi @ H @ xi
    assert abs(e_xi - pred) <= 1e-3 * abs(e_xi - out["e_ls"])


# ---------------------------------------------------------------------------------------
# SE(3) and pose matrix against library routines
# ---------------------------------------------------------------------------------------

def test_se3_exp_special_cases():
    T = np.eye(4)
    out = oracle.se3_right(T, [0.1, -0.2, 0.3, 0, 0, 0])
    assert np.allclose(out[:3, 3], [0.1, -0.2, 0.3], atol=1e-15)
    rv = np.array([0.0, 0.0, 0.7])
    out = oracle.se3_right(T, np.concatenate([[0, 0, 0], rv]))
    assert np.allclose(out[:3, :3], Rotation.from_rotvec(rv).as_matrix(), atol=1e-14)
    rv = np.array([0.3, -0.4, 0.2])
    out = oracle.se3_right(T, np.concatenate([[0, 0, 0], rv]))
    assert np.allclose(out[:3, :3], Rotation.from_rotvec(rv).as_matrix(), atol=1e-14)
    # right multiplication: T * exp
    T2 = synth.pose_from(np.array([1.0, 2.0, 0.5]), 0.4, 0.1, -0.2)
    out = oracle.se3_right(T2, np.concatenate([[0, 0, 0], rv]))
    assert np.allclose(out[:3, :3], T2[:3, :3] @ Rotation.from_rotvec(rv).as_matrix(), atol=1e-14)
    # translation part follows V(phi) rho; at small angle it tends to rho
    out = oracle.se3_right(T, [1, 0, 0, 0, 0, 1e-9])
    assert np.allclose(out[:3, 3], [1, 0, 0], atol=1e-8)


def test_pose_matrix_inverts_pose():
    T = synth.pose_from(np.array([3.0, -2.0, 1.5]), 1.1, 0.2, -0.1)
    c = np.array([0.25, -0.5, 1.0])
    M = oracle.pose_matrix(T, c).astype(np.float64)
    Tinv = np.linalg.inv(T)
    p = np.array([1.0, 0.5, 2.0])
    pc = Tinv[:3, :3] @ p + Tinv[:3, 3]
    assert np.allclose(M[:, :3] @ (p - c) + M[:, 3], pc, atol=1e-6)


# ---------------------------------------------------------------------------------------
# LM: converges to the true pose on a noise-free scan
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("pitch_deg", [15.0, 25.0])
def test_lm_converges_noise_free(pitch_deg):
    """From 5 cm / 2 deg off, LM on a noise-free scan returns to the true pose. The view is
    tilted toward the floor so that all six directions are constrained (a view of a single
    flat wall leaves in-plane motion free, for this cost as for any depth-only cost)."""
    c = cases.config1(seed=1500)
    mesh, cam = c["mesh"], c["cam"]
    gt = synth.pose_from(c["gt"][:3, 3], 0.7, math.radians(pitch_deg), 0.0)
    start = synth.perturb_fixed(gt, cases.rng(3), 0.05, 2.0)
    om = oracle.OracleMap(mesh.vertices, mesh.faces, mesh.labels)
    sd, sc = cases.scan_from_render(om.render(gt, cam)["depth"], cam)
    pose, rep = om.align(start, cam, sd, sc, max_iters=50)
    assert rep["converged"] == 1
    assert rep["e_ls_final"] < 1e-6 * rep["e_ls_initial"]
    assert rep["e_table_final"] == -cam.width * cam.height
    assert np.linalg.norm(pose[:3, 3] - gt[:3, 3]) < 1e-6
    ang = Rotation.from_matrix(gt[:3, :3].T @ pose[:3, :3]).magnitude()
    assert math.degrees(ang) < 1e-4


@pytest.mark.parametrize("seed", [0, 1])
def test_rigid_invariance_of_depth(seed):
    """Moving the world and the pose together by one rigid motion G leaves the depth image
    unchanged, up to the FP32 rounding of the moved vertices (the same surfaces are seen)."""
    c = cases.config1(seed=2100 + seed)
    mesh, cam = c["mesh"], c["cam"]
    r = cases.rng(2200 + seed)
    G = synth.pose_from(r.uniform(-20, 20, 3), r.uniform(-math.pi, math.pi), r.uniform(-0.5, 0.5),
                        r.uniform(-0.5, 0.5))
    v2 = (mesh.vertices.astype(np.float64) @ G[:3, :3].T + G[:3, 3]).astype(np.float32)
    pose = c["start"]
    a = oracle.OracleMap(mesh.vertices, mesh.faces, mesh.labels).render(pose, cam)
    b = oracle.OracleMap(v2, mesh.faces, mesh.labels).render(G @ pose, cam)
    hit = ~np.isnan(a["depth"])
    assert np.array_equal(hit, ~np.isnan(b["depth"]))
    same = a["tri_id"] == b["tri_id"]
    assert same.mean() > 0.995   # ties at shared edges may go either way after rounding
    assert np.all(np.abs(b["depth"][hit & same] - a["depth"][hit & same]) <= 1e-5 * a["depth"][hit & same])


def test_cost_sweep_wall_closed_form():
    """Fig. 7-style sweep along the optical axis in front of a wall seen at its true distance:
    at displacement t the map is t nearer, so every pixel has dz = -t: rewarded with
    E_ls = N t^2 / 2 while |t| <= eps, penalised with N eps^2 / 2 beyond."""
    cam = cases.small_pinhole(w=32, h=24, f=30.0)
    v, f = cases.plane_grid(5, 5, (-20, -20, 2.0), (40, 0, 0), (0, 40, 0))
    om = oracle.OracleMap(v, f, np.zeros(len(f), np.uint8))
    sd = np.full((cam.height, cam.width), 2.0, np.float32)
    sc = np.zeros_like(sd, np.uint8)
    N = cam.width * cam.height
    ts, outs = om.cost_sweep(np.eye(4), cam, sd, sc, axis=2, span=0.33, n=12)
    assert ts[0] == -0.33 and ts[-1] == 0.33
    for t, o in zip(ts, outs):
        if abs(t) < 0.1:
            assert o["e_table"] == -N, t
            assert o["e_ls"] == pytest.approx(0.5 * N * t * t, rel=1e-5), t
        else:
            assert o["e_table"] == N, t
            assert o["e_ls"] == pytest.approx(0.5 * N * np.float32(0.1) ** 2, rel=1e-6), t


def test_cost_sweep_minimum_at_true_pose():
    """On a noise-free scan the sweep's Table I cost is lowest at zero displacement, where every
    compared pixel is rewarded, along translation and rotation axes alike."""
    c = cases.config1(seed=2300, noise=0.0, dropout=0.0)
    mesh, cam = c["mesh"], c["cam"]
    fo = mesh.labels == 0
    om = oracle.OracleMap(mesh.vertices, mesh.faces, mesh.labels)
    sd, sc = cases.scan_from_render(oracle.OracleMap(mesh.vertices, mesh.faces[fo], mesh.labels[fo])
                                    .render(c["gt"], cam)["depth"], cam)
    for axis, span in ((0, 0.3), (4, 0.1)):
        ts, outs = om.cost_sweep(c["gt"], cam, sd, sc, axis=axis, span=span, n=9)
        e = [o["e_table"] for o in outs]
        assert ts[4] == 0.0 and e[4] == min(e) and e[4] == -int(np.sum(outs[4]["counts"]))
        assert e[0] > e[4] and e[-1] > e[4]
