"""Pins of the oracle's vertex-position gradient of the least-squares surrogate (map
refinement, an extension of the adjoint), no GPU needed: central differences of the frozen-cell
cost with one vertex moved, the identity that moving every vertex by d is moving the camera by
-d (so the gradients sum to minus the pose gradient's translation part), and a wall's closed
form."""
from __future__ import annotations

import numpy as np
import pytest

import cases
import oracle


def test_vertex_gradient_matches_frozen_fd():
    c = cases.config1(seed=2000)
    om = oracle.OracleMap(c["mesh"].vertices, c["mesh"].faces, c["mesh"].labels)
    sd, sc = c["scan"]
    pose = c["start"]
    g = om.vertex_grad(pose, c["cam"], sd, sc)
    norms = np.linalg.norm(g, axis=1)
    assert (norms > 0).sum() > 50
    picks = np.argsort(-norms)[:4].tolist() + np.flatnonzero(norms > 0)[::97][:4].tolist()
    h = 1e-5
    for vk in picks:
        fd = np.zeros(3)
        for a in range(3):
            d = np.zeros(3)
            d[a] = h
            fd[a] = (om.cost_frozen_vertex(pose, c["cam"], sd, sc, vk, d)
                     - om.cost_frozen_vertex(pose, c["cam"], sd, sc, vk, -d)) / (2 * h)
        # the gradient weights its residual from the FP32 z-buffer depth, the frozen cost from
        # the FP64 re-intersection: they differ by ~1e-7 t out of residuals of centimetres
        assert np.linalg.norm(fd - g[vk]) <= 1e-4 * np.linalg.norm(g[vk]) + 1e-12, vk


@pytest.mark.parametrize("seed", [2001, 2002])
def test_vertex_gradients_sum_to_minus_pose_translation_gradient(seed):
    c = cases.config1(seed=seed)
    om = oracle.OracleMap(c["mesh"].vertices, c["mesh"].faces, c["mesh"].labels)
    sd, sc = c["scan"]
    pose = c["start"]
    g = om.vertex_grad(pose, c["cam"], sd, sc)
    gp = om.cost(pose, c["cam"], sd, sc)["grad"]
    want = -pose[:3, :3] @ gp[:3]
    assert np.allclose(g.sum(0), want, rtol=1e-9, atol=1e-9 * np.abs(want).max())


def test_wall_closed_form():
    """Wall at 2 m, scan at 1.95 m: r = 0.05 on every pixel and d t / d v_m = b_m along z, so
    the z-gradients sum to N r and the in-plane ones vanish."""
    cam = cases.small_pinhole(w=32, h=24, f=30.0)
    v, f = cases.plane_grid(5, 5, (-20, -20, 2.0), (40, 0, 0), (0, 40, 0))
    om = oracle.OracleMap(v, f, np.zeros(len(f), np.uint8))
    sd = np.full((cam.height, cam.width), 1.95, np.float32)
    sc = np.zeros_like(sd, np.uint8)
    g = om.vertex_grad(np.eye(4), cam, sd, sc)
    r = 2.0 - np.float64(np.float32(1.95))
    N = cam.width * cam.height
    assert np.all(g[:, :2] == 0.0)
    assert g[:, 2].sum() == pytest.approx(N * r, rel=1e-9)
