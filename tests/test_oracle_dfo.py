"""Pins of the oracle's derivative-free search (Nelder-Mead or Powell's method, then coordinate
descent; Sec. IV.C), no GPU needed.

The search is pinned on functions with known minima (a convex quadratic, rotated for Powell's
method, and an integer staircase like the Table I cost), on the exact candidates of its first
Nelder-Mead step and of Powell's first iterations (axis searches, the displacement search, the
replaced direction), on its evaluation accounting, on its invariance to adding a constant or
a positive factor, and end to end on the Table I cost of a noise-free scan, whose minimum is
the true pose with every compared pixel rewarded.
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


# ---------------------------------------------------------------------------------------
# Powell's conjugate-direction method (Sec. IV.C names it beside Nelder-Mead)
# ---------------------------------------------------------------------------------------

POWELL_A = [0.25, -0.25, 0.5, -0.5, 1.0, -1.0, 2.0, -2.0, 4.0, -4.0, 8.0, -8.0]


def test_powell_quadratic_minimum():
    """A convex quadratic with rotated axes (not separable in the twist coordinates)."""
    a = np.array([0.03, -0.02, 0.01, 0.02, -0.015, 0.005])
    R = Rotation.from_rotvec([0.3, -0.5, 0.2]).as_matrix()
    Q = np.zeros((6, 6))
    Q[:3, :3] = R.T @ np.diag([1.0, 5.0, 0.5]) @ R
    Q[3:, 3:] = R @ np.diag([2.0, 1.0, 4.0]) @ R.T
    u = lambda X: (X - a) / SCALE  # noqa: E731
    f = lambda X: np.einsum("nk,kl,nl->n", u(X), Q, u(X))  # noqa: E731
    prm = oracle.dfo_params(method="powell", powell_iters=200, powell_tol=1e-4, cd_iters=200, cd_tol=1e-4)
    x, fb, rep = oracle.dfo_minimise(f, SCALE, prm)
    assert rep["powell_iters"] >= 2 and rep["nm_iters"] == 0 and rep["converged"] == 1
    assert np.all(np.abs(x - a) <= 1e-3 * SCALE), (x - a) / SCALE


def test_powell_staircase_minimum():
    a = np.array([0.021, -0.013, 0.04, -0.01, 0.017, 0.0])
    q = SCALE * 0.1
    f = lambda X: np.floor(np.abs(X - a) / q).sum(1)  # noqa: E731
    x, fb, rep = oracle.dfo_minimise(f, SCALE, oracle.dfo_params(method="powell", cd_iters=100))
    assert fb == 0.0
    assert np.all(np.abs(x - a) < q)


def test_powell_candidates_and_direction_replacement():
    """f = 3 |u0 - 1| + |u1 - 1/2| in scaled units u = x / scale. The first batch is the origin;
    the axis searches take u0 = 1 (drop 3) and u1 = 1/2 (drop 1/2), the others do not move;
    the seventh batch searches x + a d along the displacement d = x - x0; the next iteration
    searches along d / |d|_scaled, which replaced axis 0 (the largest drop), then axis 1."""
    batches = []

    def f(X):
        batches.append(X.copy())
        u = X / SCALE
        return 3.0 * np.abs(u[:, 0] - 1.0) + np.abs(u[:, 1] - 0.5)

    prm = oracle.dfo_params(method="powell", powell_iters=2, powell_step=1.0, cd_iters=0)
    x, fb, rep = oracle.dfo_minimise(f, SCALE, prm)
    assert np.array_equal(batches[0], np.zeros((1, 6)))
    for i in range(6):
        want = np.zeros((12, 6))
        base = np.zeros(6)
        if i >= 1:
            base[0] = 1.0 * SCALE[0]
        if i >= 2:
            base[1] = 0.5 * SCALE[1]
        for m, am in enumerate(POWELL_A):
            want[m] = base + (am * 1.0) * np.eye(6)[i] * SCALE[i]
        assert np.array_equal(batches[1 + i], want), i
    x1 = np.zeros(6)
    x1[0], x1[1] = SCALE[0], 0.5 * SCALE[1]
    d = x1 - np.zeros(6)
    want = np.stack([x1 + (am * 1.0) * d for am in POWELL_A])
    assert np.array_equal(batches[7], want)
    # the displacement search cannot improve (x1 is the minimum); axis 0 is replaced by d / |d|
    n = math.sqrt(sum((d[k] / SCALE[k]) * (d[k] / SCALE[k]) for k in range(6)))
    dh = d / n
    want = np.stack([x1 + (am * 1.0) * dh for am in POWELL_A])
    assert np.array_equal(batches[8], want)
    assert np.array_equal(batches[9], np.stack([x1 + (am * 1.0) * np.eye(6)[1] * SCALE[1] for am in POWELL_A]))
    assert fb == 0.0 and np.array_equal(x, x1)
    assert rep["powell_iters"] == 2 and rep["cd_iters"] == 0
    assert rep["evals"] == sum(b.shape[0] for b in batches)


def test_powell_accounting_and_order_invariance():
    """Every batch after the first has 12 points and is counted; adding a constant or scaling
    by a positive factor leaves the path unchanged (the search compares values only)."""
    a = np.array([0.02, -0.01, 0.015, -0.02, 0.01, 0.005])
    w = np.array([1.0, 2.0, 0.5, 3.0, 1.0, 2.0])
    sizes = []

    def base(X):
        sizes.append(X.shape[0])
        return np.floor(1e7 * ((X - a) ** 2 * w).sum(1))

    prm = oracle.dfo_params(method="powell", powell_iters=25, cd_iters=20)
    x0, f0, r0 = oracle.dfo_minimise(base, SCALE, prm)
    assert sizes[0] == 1 and set(sizes[1:]) == {12}
    assert r0["evals"] == sum(sizes)
    x1, f1, r1 = oracle.dfo_minimise(lambda X: base(X) + 7.0, SCALE, prm)
    x2, f2, r2 = oracle.dfo_minimise(lambda X: 3.0 * base(X), SCALE, prm)
    assert np.array_equal(x0, x1) and np.array_equal(x0, x2)
    assert r0 == r1 == r2
    assert f1 == pytest.approx(f0 + 7.0) and f2 == pytest.approx(3.0 * f0)


def test_powell_table1_search_noise_free():
    c = cases.config1(seed=1900, noise=0.0, dropout=0.0)
    mesh, cam = c["mesh"], c["cam"]
    gt = synth.pose_from(c["gt"][:3, 3], 0.7, math.radians(25.0), 0.0)
    start = synth.perturb_fixed(gt, cases.rng(4), 0.03, 1.5)
    fo = mesh.labels == 0
    om = oracle.OracleMap(mesh.vertices, mesh.faces, mesh.labels)
    sd, sc = cases.scan_from_render(oracle.OracleMap(mesh.vertices, mesh.faces[fo], mesh.labels[fo])
                                    .render(gt, cam)["depth"], cam)
    e_start = om.cost(start, cam, sd, sc)["e_table"]
    e_gt = om.cost(gt, cam, sd, sc)["e_table"]
    pose, rep = om.dfo_align(start, cam, sd, sc, dfo=oracle.dfo_params(method="powell", powell_iters=20,
                                                                         cd_iters=60))
    assert rep["powell_iters"] >= 1
    assert rep["e_table"] == om.cost(pose, cam, sd, sc)["e_table"]
    # as for Nelder-Mead: 90% of the gap to the true pose closed, and the end inside Table I's
    # plateau (FO/FO pixels are rewarded anywhere within eps = 0.1 m of the scan)
    assert rep["e_table"] - e_gt <= 0.1 * (e_start - e_gt)
    assert rep["e_table"] <= e_gt + 0.005 * abs(e_gt)
    assert np.linalg.norm(pose[:3, 3] - gt[:3, 3]) < 0.1
