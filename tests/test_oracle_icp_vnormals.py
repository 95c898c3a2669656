"""Pins of the oracle's point-to-plane ICP with the map's points coloured by their normals
(Sec. V, sequential depth-image alignment, steps 2-3), no GPU needed.

With vertex normals attached, the normal used at an associated pixel is the blend of the seen
triangle's three vertex normals by the hit's barycentrics (a rasteriser interpolating a vertex
attribute), rotated into the camera frame and normalised; a pixel whose blend is not finite
is not associated. Pins:
- every vertex carrying its own face's normal (a triangle soup) reproduces the face-normal
  terms;
- the normal at a single associated pixel equals the blend by perspective-correct screen-space
  barycentrics computed here (not by the oracle), under a rotated pose;
- a NaN vertex normal removes exactly the associated pixels of the triangles that use it;
- J^T e is the gradient of the frozen cost with the same normals (central differences);
- Eq. 2 normals of a meshed fronto-parallel wall, seen from a rotated pose, give the wall's
  face-normal terms.
"""
from __future__ import annotations

import numpy as np
import pytest

import cases
import oracle
import synth


def _soup(mesh):
    """The mesh with every triangle on its own three vertices."""
    v = mesh.vertices[mesh.faces].reshape(-1, 3).astype(np.float32)
    f = np.arange(v.shape[0], dtype=np.int32).reshape(-1, 3)
    return v, f


def _face_normals(v, f):
    a, b, c = (v[f[:, k]].astype(np.float64) for k in range(3))
    n = np.cross(b - a, c - a)
    return n / np.linalg.norm(n, axis=1, keepdims=True)


def _smooth_vertex_normals(v, f):
    """Area-weighted vertex normals (each vertex: the sum of its faces' cross products)."""
    a, b, c = (v[f[:, k]].astype(np.float64) for k in range(3))
    n = np.cross(b - a, c - a)
    out = np.zeros((v.shape[0], 3))
    for k in range(3):
        np.add.at(out, f[:, k], n)
    return out / np.maximum(np.linalg.norm(out, axis=1, keepdims=True), 1e-300)


def test_own_face_normals_give_the_face_terms():
    c = cases.config1(seed=1700)
    v, f = _soup(c["mesh"])
    om = oracle.OracleMap(v, f, c["mesh"].labels)
    sd, sc = c["scan"]
    vn = np.repeat(_face_normals(v, f), 3, axis=0)  # soup: vertex 3k + m belongs to face k
    a = om.icp_terms(c["start"], c["cam"], sd, sc, 0.1)
    b = om.icp_terms(c["start"], c["cam"], sd, sc, 0.1, vnormals=vn)
    assert a["n_assoc"] == b["n_assoc"] > 1000
    assert b["cost_l1"] == a["cost_l1"]
    assert b["e2"] == pytest.approx(a["e2"], rel=1e-12)
    assert np.allclose(b["jte"], a["jte"], rtol=1e-10, atol=1e-12 * np.abs(a["jte"]).max())
    assert np.allclose(b["jtj"], a["jtj"], rtol=1e-10, atol=1e-12 * np.abs(a["jtj"]).max())
    # a flipped sign on every normal changes nothing (e and J both flip)
    c2 = om.icp_terms(c["start"], c["cam"], sd, sc, 0.1, vnormals=-vn)
    assert np.allclose(c2["jte"], a["jte"], rtol=1e-10, atol=1e-12 * np.abs(a["jte"]).max())


def test_blended_normal_at_one_pixel():
    """One large triangle in front of a rotated camera with three different vertex normals; the
    scan has one FO return. J^T J's first block is n n^T and J^T e's first three entries are
    n e for that pixel's normal n."""
    cam = cases.small_pinhole(w=48, h=40, f=40.0)
    pose = synth.pose_from(np.array([0.2, -0.1, 0.3]), 0.3, 0.1, -0.2)
    R, t = pose[:3, :3], pose[:3, 3]
    # camera-frame triangle, taken to the world frame
    wc = np.array([[-1.5, -1.2, 3.0], [1.8, -0.9, 3.6], [0.1, 1.6, 2.7]])
    v = (wc @ R.T + t).astype(np.float32)
    f = np.array([[0, 1, 2]], np.int32)
    r = cases.rng(5)
    vn = r.normal(size=(3, 3))
    vn /= np.linalg.norm(vn, axis=1, keepdims=True)
    vn[:, 2] = -np.abs(vn[:, 2])  # all facing the same half-space, as a depth image's are
    om = oracle.OracleMap(v, f, np.zeros(1, np.uint8))
    rend = om.render(pose, cam)
    ii, jj = 25, 19
    assert rend["tri_id"][jj, ii] == 0
    sd = np.full((cam.height, cam.width), np.nan, np.float32)
    sc = np.full(sd.shape, 2, np.uint8)
    sd[jj, ii] = rend["depth"][jj, ii] + np.float32(0.02)
    sc[jj, ii] = 0
    out = om.icp_terms(pose, cam, sd, sc, 0.1, vnormals=vn)
    assert out["n_assoc"] == 1
    # perspective-correct barycentrics of the pixel centre from the projected vertices
    w = (v.astype(np.float64) - t) @ R
    fx, fy, cx, cy = (float(np.float32(x)) for x in (cam.fx, cam.fy, cam.cx, cam.cy))
    sx, sy = fx * w[:, 0] / w[:, 2] + cx, fy * w[:, 1] / w[:, 2] + cy
    px, py = ii + 0.5, jj + 0.5

    def area(a, b):
        return (sx[b] - sx[a]) * (py - sy[a]) - (sy[b] - sy[a]) * (px - sx[a])

    lam = np.array([area(1, 2), area(2, 0), area(0, 1)])
    lam /= lam.sum()
    q = lam / w[:, 2]
    bary = q / q.sum()
    n = R.T @ (bary @ vn)
    n /= np.linalg.norm(n)
    H = np.zeros((3, 3))
    k = 0
    for a in range(6):
        for b in range(a, 6):
            if a < 3 and b < 3:
                H[a, b] = H[b, a] = out["jtj"][k]
            k += 1
    assert np.allclose(H, np.outer(n, n), atol=1e-9)
    # e = (d - t)(n . r) with r = (x, y, 1)
    rr = np.array([(px - cx) / fx, (py - cy) / fy, 1.0])
    e = (np.float64(sd[jj, ii]) - np.float64(rend["depth"][jj, ii])) * (n @ rr)
    assert np.allclose(out["jte"][:3], n * e, atol=1e-12)


def test_nan_vertex_normal_drops_exactly_its_pixels():
    c = cases.config1(seed=1710)
    mesh = c["mesh"]
    om = oracle.OracleMap(mesh.vertices, mesh.faces, mesh.labels)
    sd, sc = c["scan"]
    vn = _smooth_vertex_normals(mesh.vertices, mesh.faces)
    base = om.icp_terms(c["start"], c["cam"], sd, sc, 0.1, vnormals=vn)
    face = om.icp_terms(c["start"], c["cam"], sd, sc, 0.1)
    assert base["n_assoc"] == face["n_assoc"] > 1000  # finite normals: the same pairs
    # associated pixels (the rule, evaluated here) and the triangles they see
    rend = om.render(c["start"], c["cam"])
    ids = rend["tri_id"]
    assoc = ((ids >= 0) & (sc == 0) & np.isfinite(sd)
             & (np.abs(rend["depth"] - sd) < np.float32(0.1)))
    assoc[ids >= 0] &= mesh.labels[ids[ids >= 0]] == 0
    assert int(assoc.sum()) == base["n_assoc"]
    seen = np.unique(ids[assoc])
    k = int(mesh.faces[seen[len(seen) // 2], 1])  # a vertex of a triangle that is seen
    bad = vn.copy()
    bad[k] = np.nan
    out = om.icp_terms(c["start"], c["cam"], sd, sc, 0.1, vnormals=bad)
    touches = np.zeros(ids.shape, bool)
    touches[ids >= 0] = (mesh.faces[ids[ids >= 0]] == k).any(axis=1)
    dropped = int((assoc & touches).sum())
    assert dropped > 0
    assert out["n_assoc"] == base["n_assoc"] - dropped


@pytest.mark.parametrize("model", ["pinhole", "spherical"])
def test_vertex_normal_jte_matches_frozen_fd(model):
    if model == "pinhole":
        c = cases.config1(seed=1720)
        mesh, cam, pose, (sd, sc) = c["mesh"], c["cam"], c["start"], c["scan"]
    else:
        mesh = synth.room_mesh(1730)
        cam = cases.small_spherical(w=128, h=16)
        r = cases.rng(1731)
        gt = synth.room_pose(r, mesh)
        sd, sc = synth.synth_scan(mesh, cam, gt, r, sigma_abs=0.01)
        pose = synth.perturb_fixed(gt, r, 0.03, 1.0)
    om = oracle.OracleMap(mesh.vertices, mesh.faces, mesh.labels)
    vn = _smooth_vertex_normals(mesh.vertices, mesh.faces)
    out = om.icp_terms(pose, cam, sd, sc, 0.1, vnormals=vn)
    assert out["n_assoc"] > 100
    assert om.icp_frozen(pose, cam, sd, sc, 0.1, np.zeros(6), vnormals=vn) == pytest.approx(0.5 * out["e2"], rel=1e-12)

    def central(h):
        fd = np.zeros(6)
        for a in range(6):
            xi = np.zeros(6)
            xi[a] = h
            fd[a] = (om.icp_frozen(pose, cam, sd, sc, 0.1, xi, vnormals=vn)
                     - om.icp_frozen(pose, cam, sd, sc, 0.1, -xi, vnormals=vn)) / (2 * h)
        return fd

    fd = (4 * central(5e-5) - central(1e-4)) / 3
    assert np.linalg.norm(out["jte"] - fd) <= 1e-7 * np.linalg.norm(out["jte"])


def test_eq2_normals_of_a_meshed_wall_give_the_face_terms():
    """A wall seen squarely from a rotated pose: its depth image is constant, so its Eq. 2
    normals are exactly (0, 0, -1) in the camera frame; taken to the world frame they are the
    wall's normal, and ICP against the wall's mesh (meshified from that image) with these
    vertex normals equals ICP with the face normals."""
    cam = cases.small_pinhole(w=40, h=32, f=36.0)
    pose = synth.pose_from(np.array([0.4, 0.2, 1.1]), 0.6, 0.0, 0.0)
    depth = np.full((cam.height, cam.width), 2.5, np.float32)
    cls = np.zeros(depth.shape, np.uint8)
    v, f, lab = oracle.meshify(cam, depth, cls, pose, 8.0, 0.1, 1)
    normals, _ = oracle.depth_normals(depth, cls, sigma=1.0, metric=True, fx=cam.fx, fy=cam.fy)
    inner = np.isfinite(normals).all(-1)
    assert inner.sum() > 0.7 * inner.size
    assert np.allclose(normals[inner], [0.0, 0.0, -1.0], atol=1e-12)
    vn = normals.reshape(-1, 3) @ pose[:3, :3].T  # camera frame -> world frame
    om = oracle.OracleMap(v, f, lab)
    start = synth.perturb_fixed(pose, cases.rng(3), 0.02, 0.5)
    sd = np.full(depth.shape, 2.5, np.float32) + np.float32(0.01)
    a = om.icp_terms(start, cam, sd, cls, 0.2)
    b = om.icp_terms(start, cam, sd, cls, 0.2, vnormals=vn)
    # border pixels of the image have no Eq. 2 normal: their triangles drop out
    assert 0 < b["n_assoc"] < a["n_assoc"]
    # on the kept pixels the blended normal is the wall's normal, so e and J match the face terms
    wn = _face_normals(v, f)
    assert np.allclose(np.abs(wn @ (-pose[:3, 2])), 1.0, atol=1e-6)
    face_vn = np.where(np.isfinite(vn), np.tile(-pose[:3, 2], (vn.shape[0], 1)), np.nan)
    c = om.icp_terms(start, cam, sd, cls, 0.2, vnormals=face_vn)
    assert c["n_assoc"] == b["n_assoc"]
    assert np.allclose(b["jte"], c["jte"], rtol=1e-9, atol=1e-12)
    assert np.allclose(b["jtj"], c["jtj"], rtol=1e-9, atol=1e-12)
