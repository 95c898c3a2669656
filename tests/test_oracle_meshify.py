"""Pins of the oracle's meshification of a range image (Sec. IV.A, Fig. 5), no GPU needed.

Closed forms: the vertices of a wall seen head-on, the labels that the edge threshold and the
no-return rule give, the faces that dead pixels remove, the downsampled grid; and an invariant:
every quad projects onto the rectangle between its four pixel centres, so rendering the mesh
of a scan from the scan's own pose puts each interior pixel's own vertex under it and
reproduces the scan's depth there.
"""
from __future__ import annotations

import math

import numpy as np
import pytest
from scipy import ndimage

import cases
import oracle
import synth


def _wall_scan(cam, D):
    return (np.full((cam.height, cam.width), D, np.float32),
            np.zeros((cam.height, cam.width), np.uint8))


def _rays(cam):
    x = np.arange(cam.width, dtype=np.float32)
    y = np.arange(cam.height, dtype=np.float32)
    rx = (x + np.float32(0.5) - np.float32(cam.cx)) / np.float32(cam.fx)
    ry = (y + np.float32(0.5) - np.float32(cam.cy)) / np.float32(cam.fy)
    return np.meshgrid(rx, ry)


def test_wall_vertices_faces_and_labels():
    cam = cases.small_pinhole(w=32, h=24, f=30.0)   # fx 30, fy 33
    d, c = _wall_scan(cam, 2.0)
    v, f, lab = oracle.meshify(cam, d, c, np.eye(4), max_range=4.0, max_edge=0.1)
    RX, RY = _rays(cam)
    want = np.stack([2.0 * RX, 2.0 * RY, np.full_like(RX, 2.0)], -1).reshape(-1, 3)
    assert np.array_equal(v, want.astype(np.float32))
    nq = (cam.width - 1) * (cam.height - 1)
    assert f.shape == (2 * nq, 3) and np.all(lab == 0)
    # block (i, j) = (1, 2): triangles (v00, v10, v11) and (v00, v11, v01)
    W = cam.width
    q = 2 * (cam.width - 1) + 1
    v00 = 2 * W + 1
    assert f[2 * q].tolist() == [v00, v00 + 1, v00 + W + 1]
    assert f[2 * q + 1].tolist() == [v00, v00 + W + 1, v00 + W]
    # sides are 2/30 and 2/33 m, the diagonal 0.090 m: a 0.08 m limit marks every quad FU
    # through the diagonal alone, 0.065 m through the long side too
    sx, sy = 2.0 / 30.0, 2.0 / 33.0
    assert max(sx, sy) < 0.08 < math.hypot(sx, sy)
    _, _, lab = oracle.meshify(cam, d, c, np.eye(4), max_range=4.0, max_edge=0.08)
    assert np.all(lab == 1)
    _, _, lab = oracle.meshify(cam, d, c, np.eye(4), max_range=4.0, max_edge=0.095)
    assert np.all(lab == 0)


def test_pose_moves_vertices_to_world():
    cam = cases.small_pinhole(w=20, h=16, f=20.0)
    d, c = _wall_scan(cam, 1.5)
    pose = synth.pose_from(np.array([1.0, -2.0, 0.5]), 0.4, 0.2, -0.1)
    v0, f0, l0 = oracle.meshify(cam, d, c, np.eye(4), max_range=4.0)
    v, f, lab = oracle.meshify(cam, d, c, pose, max_range=4.0)
    want = v0.astype(np.float64) @ pose[:3, :3].T + pose[:3, 3]
    assert np.allclose(v, want, rtol=0, atol=1e-6)
    assert np.array_equal(f, f0) and np.array_equal(lab, l0)


def test_depth_step_is_free_unknown():
    """Left columns at 2 m, the rest at 3 m: the one column of quads across the step is FU."""
    cam = cases.small_pinhole(w=24, h=10, f=60.0)
    d = np.full((cam.height, cam.width), 2.0, np.float32)
    d[:, 9:] = 3.0
    c = np.zeros_like(d, np.uint8)
    _, f, lab = oracle.meshify(cam, d, c, np.eye(4), max_range=4.0)
    lab = lab[0::2].reshape(cam.height - 1, cam.width - 1)
    want = np.zeros_like(lab)
    want[:, 8] = 1
    assert np.array_equal(lab, want)


def test_no_return_and_dead_pixels():
    cam = cases.small_pinhole(w=30, h=22, f=40.0)
    r = np.random.Generator(np.random.PCG64(7))
    d, c = _wall_scan(cam, 2.5)
    nor = r.random(d.shape) < 0.04
    dead = (r.random(d.shape) < 0.03) & ~nor
    c[nor] = 1
    c[dead] = 2
    d[nor] = 123.0    # ignored: no-return pixels sit at max_range
    v, f, lab = oracle.meshify(cam, d, c, np.eye(4), max_range=4.0)
    RX, RY = _rays(cam)
    vv = v.reshape(cam.height, cam.width, 3)
    assert np.array_equal(vv[nor][:, 2], np.full(nor.sum(), 4.0, np.float32))
    assert np.array_equal(vv[nor][:, 0], (np.float32(4.0) * RX)[nor])
    assert np.all(vv[dead] == 0.0)   # parked at the sensor origin
    # quads keep iff none of their four pixels is dead, FU iff one is a no-return
    def quads(m):
        return m[:-1, :-1] | m[1:, :-1] | m[:-1, 1:] | m[1:, 1:]
    keep = ~quads(dead)
    assert f.shape[0] == 2 * keep.sum()
    assert np.array_equal(lab[0::2], quads(nor)[keep].astype(np.uint8))
    assert np.array_equal(lab[0::2], lab[1::2])
    used = np.unique(f)
    assert not np.isin(np.flatnonzero(dead.ravel()), used).any()


def test_downsampled_grid():
    cam = cases.small_pinhole(w=33, h=20, f=30.0)
    r = np.random.Generator(np.random.PCG64(8))
    d = r.uniform(1.0, 3.0, (cam.height, cam.width)).astype(np.float32)
    c = np.zeros_like(d, np.uint8)
    v1, _, _ = oracle.meshify(cam, d, c, np.eye(4), max_range=4.0, step=1)
    v2, f2, _ = oracle.meshify(cam, d, c, np.eye(4), max_range=4.0, step=2)
    Ws, Hs = (cam.width - 1) // 2 + 1, (cam.height - 1) // 2 + 1
    assert v2.shape == (Ws * Hs, 3) and f2.shape[0] == 2 * (Ws - 1) * (Hs - 1)
    assert np.array_equal(v2.reshape(Hs, Ws, 3), v1.reshape(cam.height, cam.width, 3)[::2, ::2])


@pytest.mark.parametrize("seed", [1, 2])
def test_render_of_meshed_scan_reproduces_scan(seed):
    """Render the mesh of a noise-free room scan (its farthest 40% of returns turned into
    no-returns, drawn at the maximal range R = the 60th depth percentile) from the scan's pose. Every quad projects onto the rectangle between its
    pixel centres, so at an interior pixel whose four incident quads are present the winner
    is one of its own vertex's triangles: the depth is the vertex's. Where the four quads are
    all FO, or all at the maximal range, that holds to FP32 rounding (steep FU quads across a
    discontinuity are sensitive to the 1/256-pixel snap, so they are left out)."""
    c = cases.config1(seed=1700 + seed, noise=0.0, dropout=0.0)
    cam = c["cam"]
    sd, sc = (a.copy() for a in c["scan"])
    R = np.float32(np.percentile(sd, 60))
    far = sd > R
    sd[far] = R
    sc[far] = 1
    v, f, lab = oracle.meshify(cam, sd, sc, c["gt"], max_range=float(R))
    om = oracle.OracleMap(v, f, lab)
    t = om.render(c["gt"], cam)["depth"]
    H, W = sd.shape
    q = lab[0::2].reshape(H - 1, W - 1)
    inner = np.zeros((H, W), bool)
    inner[1:-1, 1:-1] = True

    def around(m):
        out = np.zeros((H, W), bool)
        out[1:-1, 1:-1] = m[:-1, :-1] & m[1:, :-1] & m[:-1, 1:] & m[1:, 1:]
        return out

    fo = around(q == 0)
    assert fo.sum() > 0.3 * H * W
    assert np.all(np.abs(t[fo] - sd[fo]) <= 2e-6 * sd[fo])
    nr = inner & (sc == 1)
    nr[1:-1, 1:-1] &= ((sc[:-2, 1:-1] == 1) & (sc[2:, 1:-1] == 1) & (sc[1:-1, :-2] == 1) & (sc[1:-1, 2:] == 1)
                       & (sc[:-2, :-2] == 1) & (sc[2:, 2:] == 1) & (sc[:-2, 2:] == 1) & (sc[2:, :-2] == 1))
    assert nr.sum() > 100
    assert np.all(np.abs(t[nr] - R) <= 2e-6 * R)
    assert 0.05 < lab.mean() < 0.9


def test_raytable_vertices_lie_on_their_rays():
    """Panoramic (ray-table) scan at a constant range R: every vertex is R along its pixel's
    unit ray (so |v| = R), and no-returns sit at the maximal range along theirs."""
    cam = cases.small_spherical(w=64, h=12)
    R = 7.5
    d = np.full((cam.height, cam.width), R, np.float32)
    c = np.zeros_like(d, np.uint8)
    c[3, 10:20] = 1
    v, f, lab = oracle.meshify(cam, d, c, np.eye(4), max_range=40.0, max_edge=10.0)
    rays = cam.ray_table_f32().reshape(-1, 3).astype(np.float64)
    rng = np.where(c.ravel() == 1, 40.0, R)
    want = (np.float32(rng)[:, None] * rays.astype(np.float32)).astype(np.float32)
    assert np.array_equal(v, want)
    assert np.allclose(np.linalg.norm(v, axis=1), rng, rtol=1e-6)
    # every 2x2 block is kept (no dead pixels); only the blocks touching a no-return are FU
    assert f.shape[0] == 2 * (cam.width - 1) * (cam.height - 1)
    blk = lab[0::2].reshape(cam.height - 1, cam.width - 1)
    nr = c == 1
    touch = nr[:-1, :-1] | nr[1:, :-1] | nr[:-1, 1:] | nr[1:, 1:]
    assert np.array_equal(blk, touch.astype(np.uint8))


def test_step_equals_meshing_the_subsampled_image():
    """Meshing with step 2 is meshing the image of every other pixel with a camera whose
    pixels are twice as large (the same rays), face for face and label for label."""
    import dataclasses
    c = cases.config1(seed=1750, noise=0.005, dropout=0.05)
    cam = c["cam"]
    sd, sc = c["scan"]
    v2, f2, l2 = oracle.meshify(cam, sd, sc, c["gt"], cam.range_max, 0.1, 2)
    # the subsampled camera: pixel (i, j) of it is pixel (2i, 2j) of the original
    sub = dataclasses.replace(cam, width=(cam.width - 1) // 2 + 1, height=(cam.height - 1) // 2 + 1,
                              fx=cam.fx / 2, fy=cam.fy / 2, cx=(cam.cx + 0.5) / 2, cy=(cam.cy + 0.5) / 2)
    vs, fs, ls = oracle.meshify(sub, np.ascontiguousarray(sd[::2, ::2]), np.ascontiguousarray(sc[::2, ::2]),
                                c["gt"], cam.range_max, 0.1, 1)
    assert np.array_equal(f2, fs) and np.array_equal(l2, ls)
    assert np.allclose(v2, vs, rtol=0, atol=1e-5)
