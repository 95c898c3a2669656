"""Pins of the oracle's derivative-free search (Nelder-Mead, then coordinate descent; Sec. IV.C),
no GPU needed.

The search is pinned on functions with known minima (a convex quadratic, an integer staircase
like the Table I cost), on the exact candidates of its first Nelder-Mead step, on its
evaluation accounting, and end to end on the Table I cost of a noise-free scan, whose minimum
is the true pose with every compared pixel rewarded.
"""
from __future__ import annotations

import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import cases
import oracle
import synth

SCALE = np.array([0.05, 0.05, 0.05, 0.035, 0.035, 0.035])


def test_quadratic_minimum():
    a = np.array([0.03, -0.02, 0.01, 0.02, -0.015, 0.005])
    w = np.array([1.0, 3.0, 0.5, 2.0, 1.0, 4.0])
    x, fb, rep = oracle.dfo_minimise(lambda X: ((X - a) ** 2 * w).sum(1), SCALE,
                                     oracle.dfo_params(nm_iters=200, cd_iters=200, cd_tol=1e-4))
    assert rep["converged"] == 1
    assert np.all(np.abs(x - a) <= 2e-4 * SCALE)
    assert fb <= ((np.zeros(6) - a) ** 2 * w).sum()


def test_staircase_minimum():
    """An integer-valued staircase (plateaus of width q): the search ends on the minimal
    plateau |x_k - a_k| < q_k."""
    a = np.array([0.021, -0.013, 0.04, -0.01, 0.017, 0.0])
    q = SCALE * 0.1
    f = lambda X: np.floor(np.abs(X - a) / q).sum(1)  # noqa: E731
    x, fb, rep = oracle.dfo_minimise(f, SCALE, oracle.dfo_params(nm_iters=100, cd_iters=100))
    assert fb == 0.0
    assert np.all(np.abs(x - a) < q)


def test_first_step_candidates_and_accounting():
    """The first batch is the simplex (origin, then nm_step * scale on each axis); the second is
    c + d, c + 2d, c + d/2, c - d/2 with c the mean of the best six and d = c - x_worst; every
    evaluated point is counted."""
    batches = []
    g = np.array([1.0, -2.0, 0.5, 3.0, -1.0, 2.5])

    def f(X):
        batches.append(X.copy())
        return X @ g

    prm = oracle.dfo_params(nm_iters=5, cd_iters=3, nm_step=1.0)
    x, fb, rep = oracle.dfo_minimise(f, SCALE, prm)
    s0 = batches[0]
    assert np.array_equal(s0[0], np.zeros(6))
    assert np.array_equal(s0[1:], np.diag(SCALE))
    vals = s0 @ g
    order = np.argsort(vals, kind="stable")
    c = sum(s0[i] for i in order[:6]) / 6.0
    d = c - s0[order[6]]
    want = np.stack([c + d, c + 2 * d, c + 0.5 * d, c - 0.5 * d])
    assert np.allclose(batches[1], want, rtol=0, atol=1e-15)
    n = sum(b.shape[0] for b in batches)
    assert rep["evals"] == n == 7 + 4 * rep["nm_iters"] + 6 * rep["nm_shrinks"] + 12 * rep["cd_iters"]
    assert [b.shape[0] for b in batches[-rep["cd_iters"]:]] == [12] * rep["cd_iters"]


def test_table1_search_reaches_true_pose_noise_free():
    c = cases.config1(seed=1900, noise=0.0, dropout=0.0)
    mesh, cam = c["mesh"], c["cam"]
    gt = synth.pose_from(c["gt"][:3, 3], 0.7, math.radians(25.0), 0.0)
    start = synth.perturb_fixed(gt, cases.rng(4), 0.03, 1.5)
    fo = mesh.labels == 0
    om = oracle.OracleMap(mesh.vertices, mesh.faces, mesh.labels)
    sd, sc = cases.scan_from_render(oracle.OracleMap(mesh.vertices, mesh.faces[fo], mesh.labels[fo])
                                    .render(gt, cam)["depth"], cam)
    e_start = om.cost(start, cam, sd, sc)["e_table"]
    pose, rep = om.dfo_align(start, cam, sd, sc, dfo=oracle.dfo_params(nm_iters=150, cd_iters=80))
    e_gt = om.cost(gt, cam, sd, sc)["e_table"]
    assert rep["e_table"] < e_start
    assert rep["e_table"] == om.cost(pose, cam, sd, sc)["e_table"]
    # the true pose rewards every compared pixel; the search closes 90% of the gap to it and
    # ends inside Table I's plateau (FO/FO pixels are rewarded anywhere within eps = 0.1 m,
    # so the cost does not single out the true pose more finely than that)
    assert rep["e_table"] - e_gt <= 0.1 * (e_start - e_gt)
    assert rep["e_table"] <= e_gt + 0.005 * abs(e_gt)
    assert np.linalg.norm(pose[:3, 3] - gt[:3, 3]) < 0.05
    assert math.degrees(Rotation.from_matrix(gt[:3, :3].T @ pose[:3, :3]).magnitude()) < 1.0


def test_search_depends_only_on_the_order_of_values():
    """Nelder-Mead and coordinate descent compare values only: adding a constant to the
    objective or scaling it by a positive factor leaves the whole search path unchanged. The
    objective is integer valued, like the Table I cost, so both changes are exact."""
    a = np.array([0.02, -0.01, 0.015, -0.02, 0.01, 0.005])
    w = np.array([1.0, 2.0, 0.5, 3.0, 1.0, 2.0])
    base = lambda X: np.floor(1e7 * ((X - a) ** 2 * w).sum(1))  # noqa: E731
    prm = oracle.dfo_params(nm_iters=40, cd_iters=30)
    x0, f0, r0 = oracle.dfo_minimise(base, SCALE, prm)
    x1, f1, r1 = oracle.dfo_minimise(lambda X: base(X) + 7.0, SCALE, prm)
    x2, f2, r2 = oracle.dfo_minimise(lambda X: 3.0 * base(X), SCALE, prm)
    assert np.array_equal(x0, x1) and np.array_equal(x0, x2)
    assert r0 == r1 == r2
    assert f1 == pytest.approx(f0 + 7.0) and f2 == pytest.approx(3.0 * f0)
