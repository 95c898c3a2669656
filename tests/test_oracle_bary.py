"""Pins for the oracle's visibility-buffer barycentrics (Sec. IV z-buffer; the per-pixel
triangle id plus barycentrics of the visibility buffer).

orc_barycentrics returns, per covered pixel, (b1, b2) such that the pixel's ray meets the
winning triangle's plane at (1 - b1 - b2) v0 + b1 v1 + b2 v2 (vertices in face order). Each pin
fixes that definition from outside the function:
- the reconstructed point lies on the pixel's ray at the ray-plane hit, with vertices taken to
  the camera frame here in numpy (not by the oracle);
- a pixel centre placed exactly on vertex k gives vertex k's unit coordinates (catches swapped
  b1/b2 and wrong vertex order);
- for pinhole cameras the perspective-correct screen-space barycentrics (affine 2-D
  barycentrics of the projected vertices, divided by each vertex's depth, renormalised) agree;
- covered pixels lie inside their triangle up to the 1/256-pixel snap of the coverage rule.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from cases import config1, random_tris, rng, small_pinhole, small_spherical

KEY_EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)


def _rays64(cam):
    """Per-pixel ray exactly as the oracle's camera carries it (FP32 intrinsics or table)."""
    if cam.model == "pinhole":
        fx, fy, cx, cy = (float(np.float32(x)) for x in (cam.fx, cam.fy, cam.cx, cam.cy))
        j, i = np.meshgrid(np.arange(cam.height, dtype=np.float64),
                           np.arange(cam.width, dtype=np.float64), indexing="ij")
        return np.stack([(i + 0.5 - cx) / fx, (j + 0.5 - cy) / fy, np.ones_like(i)], -1)
    return cam.ray_table_f32().astype(np.float64)


def _camera_vertices(v, pose):
    """World vertices (FP32 values, taken exactly to FP64) in the camera frame of `pose`."""
    R = pose[:3, :3]
    t = pose[:3, 3]
    return (v.astype(np.float64) - t) @ R


def _check_reconstruction(om, pose, cam, keys, rel=1e-10):
    b = om.barycentrics(pose, cam, keys)
    hit = keys != KEY_EMPTY
    assert np.all(np.isnan(b[~hit]))
    assert np.all(np.isfinite(b[hit]))
    ids = (keys[hit] & np.uint64(0xFFFFFFFF)).astype(np.int64)
    w = _camera_vertices(om.v, pose)[om.faces[ids]]  # (n, 3 vertices, 3)
    r = _rays64(cam)[hit]
    b1, b2 = b[hit][:, 0], b[hit][:, 1]
    P = (1.0 - b1 - b2)[:, None] * w[:, 0] + b1[:, None] * w[:, 1] + b2[:, None] * w[:, 2]
    # ray-plane hit from the camera-frame plane through the three vertices
    n = np.cross(w[:, 1] - w[:, 0], w[:, 2] - w[:, 0])
    t = np.einsum("nk,nk->n", n, w[:, 0]) / np.einsum("nk,nk->n", n, r)
    H = t[:, None] * r
    scale = np.maximum(np.linalg.norm(H, axis=1), np.abs(w).max(axis=(1, 2)))
    err = np.linalg.norm(P - H, axis=1) / scale
    assert err.max() <= rel, (err.max(), int(np.argmax(err)))
    return b[hit], ids


def test_barycentrics_reconstruct_the_ray_plane_hit_config1():
    c = config1()
    om = oracle.OracleMap(c["mesh"].vertices, c["mesh"].faces, c["mesh"].labels)
    keys = om.render(c["start"], c["cam"])["keys"]
    assert (keys != KEY_EMPTY).sum() > 10000
    _check_reconstruction(om, c["start"], c["cam"], keys)


@pytest.mark.parametrize("seed", [11, 12])
def test_barycentrics_reconstruct_the_ray_plane_hit_raytable_soup(seed):
    cam = small_spherical()
    r = rng(seed)
    # a soup around the sensor (every direction), identity-free pose
    n = 300
    c = r.normal(size=(n, 3))
    c *= r.uniform(2.0, 9.0, (n, 1)) / np.linalg.norm(c, axis=1, keepdims=True)
    v = (c[:, None, :] + r.normal(scale=0.8, size=(n, 3, 3))).reshape(-1, 3).astype(np.float32)
    f = np.arange(3 * n, dtype=np.int32).reshape(n, 3)
    pose = synth.pose_from(np.array([0.3, -0.2, 0.1]), 0.4, 0.1, -0.05)
    om = oracle.OracleMap(v, f, np.zeros(n, np.uint8))
    keys = om.render(pose, cam)["keys"]
    assert (keys != KEY_EMPTY).sum() > 200
    _check_reconstruction(om, pose, cam, keys)


def test_pixel_centre_on_a_vertex_gives_its_unit_coordinates():
    # fx = fy = 64 and a principal point on the pixel grid make every ray component exact
    cam = synth.Camera("pinhole", 64, 48, fx=64.0, fy=64.0, cx=24.0, cy=20.0, near=0.1)
    # three pixel centres (i + 0.5, j + 0.5) and three depths; X = (i + 0.5 - cx) / fx * Z exact
    pix = [(40, 10), (8, 30), (50, 44)]
    Z = [2.0, 3.0, 1.5]
    v = np.array([[(i + 0.5 - 24.0) / 64.0 * z, (j + 0.5 - 20.0) / 64.0 * z, z]
                  for (i, j), z in zip(pix, Z)], np.float32)
    assert np.array_equal(v.astype(np.float64),
                          np.array([[(i + 0.5 - 24.0) / 64.0 * z, (j + 0.5 - 20.0) / 64.0 * z, z]
                                    for (i, j), z in zip(pix, Z)]))
    f = np.array([[0, 1, 2]], np.int32)
    om = oracle.OracleMap(v, f, np.zeros(1, np.uint8))
    pose = np.eye(4)
    keys = np.full((cam.height, cam.width), KEY_EMPTY, np.uint64)
    for (i, j) in pix:
        keys[j, i] = np.uint64(0)  # triangle 0 at these pixels (any depth word)
    b = om.barycentrics(pose, cam, keys)
    want = [(0.0, 0.0), (1.0, 0.0), (0.0, 1.0)]
    for (i, j), (w1, w2) in zip(pix, want):
        assert abs(b[j, i, 0] - w1) <= 1e-14 and abs(b[j, i, 1] - w2) <= 1e-14, (i, j, b[j, i])
    # a reordered face permutes the coordinates accordingly
    om2 = oracle.OracleMap(v, np.array([[2, 0, 1]], np.int32), np.zeros(1, np.uint8))
    b = om2.barycentrics(pose, cam, keys)
    want = [(1.0, 0.0), (0.0, 1.0), (0.0, 0.0)]  # vertex 0 is now the face's second corner
    for (i, j), (w1, w2) in zip(pix, want):
        assert abs(b[j, i, 0] - w1) <= 1e-14 and abs(b[j, i, 1] - w2) <= 1e-14, (i, j, b[j, i])


def _screen_space_bary(om, pose, cam, keys):
    """Perspective-correct barycentrics from 2-D affine ones of the projected vertices."""
    hit = keys != KEY_EMPTY
    ids = (keys[hit] & np.uint64(0xFFFFFFFF)).astype(np.int64)
    w = _camera_vertices(om.v, pose)[om.faces[ids]]
    fx, fy, cx, cy = (float(np.float32(x)) for x in (cam.fx, cam.fy, cam.cx, cam.cy))
    sx = fx * w[..., 0] / w[..., 2] + cx
    sy = fy * w[..., 1] / w[..., 2] + cy
    jj, ii = np.nonzero(hit)
    px, py = ii + 0.5, jj + 0.5

    def area(ax, ay, bx, by, qx, qy):
        return (bx - ax) * (qy - ay) - (by - ay) * (qx - ax)

    A = area(sx[:, 0], sy[:, 0], sx[:, 1], sy[:, 1], sx[:, 2], sy[:, 2])
    lam = np.stack([area(sx[:, 1], sy[:, 1], sx[:, 2], sy[:, 2], px, py),
                    area(sx[:, 2], sy[:, 2], sx[:, 0], sy[:, 0], px, py),
                    area(sx[:, 0], sy[:, 0], sx[:, 1], sy[:, 1], px, py)], 1) / A[:, None]
    # distance (pixels) of the sample from each edge, signed positive inside
    edge = [(1, 2), (2, 0), (0, 1)]
    elen = np.stack([np.hypot(sx[:, b] - sx[:, a], sy[:, b] - sy[:, a]) for a, b in edge], 1)
    dist = lam * np.abs(A)[:, None] / elen
    q = lam / w[..., 2]
    persp = q / q.sum(axis=1, keepdims=True)
    return persp, dist, hit


@pytest.mark.parametrize("case", ["config1", "soup"])
def test_barycentrics_equal_perspective_correct_screen_space(case):
    if case == "config1":
        c = config1()
        v, f, lab, pose, cam = (c["mesh"].vertices, c["mesh"].faces, c["mesh"].labels,
                                c["start"], c["cam"])
    else:
        v, f = random_tris(21, 600, zmin=0.5, zmax=6.0)
        f = f[(v[f][..., 2] > 0.2).all(axis=1)]  # screen projection needs every vertex in front
        lab, pose, cam = np.zeros(len(f), np.uint8), np.eye(4), small_pinhole()
    om = oracle.OracleMap(v, f, lab)
    keys = om.render(pose, cam)["keys"]
    persp, dist, hit = _screen_space_bary(om, pose, cam, keys)
    b = om.barycentrics(pose, cam, keys)[hit]
    assert np.abs(b[:, 0] - persp[:, 1]).max() <= 1e-8
    assert np.abs(b[:, 1] - persp[:, 2]).max() <= 1e-8
    # covered samples are inside their triangle up to the vertex snap (1/256 px per coordinate)
    assert dist.min() >= -2.0 / 256.0, dist.min()
    b0 = 1.0 - b[:, 0] - b[:, 1]
    inside = dist.min(axis=1) > 2.0 / 256.0
    assert inside.mean() > 0.5
    assert b0[inside].min() >= 0 and b[inside].min() >= 0
