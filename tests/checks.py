"""Element-wise comparison of GPU sums against the oracle's FP64 values.

A gradient-type vector or matrix (pose gradient, Gauss-Newton matrix, ICP J^T e and J^T J,
vertex gradient) is compared element by element:

    |g_i - o_i| <= rel * max(|o_i|, tau * ||o||)

plus the aggregate |g - o| <= rel * ||o||. The floor tau * ||o|| exists because an element that
is the small difference of large per-pixel terms (a gradient component near a minimum, an
off-diagonal of J^T J) carries the FP32 rounding of those terms, which scales with the whole
sum rather than with the element; tau = 1e-2 puts that floor two decades below the largest
element, so a wrong sign, a dropped term or a swapped component still fails.
"""
from __future__ import annotations

import numpy as np

TAU = 1e-2

# worst ratio seen per label in this process (printed by the GPU suite's terminal summary)
WORST: dict[str, float] = {}


def close_elementwise(got, want, rel, what="", tau=TAU, floor=0.0):
    """Assert element-wise and aggregate closeness; returns the worst element ratio."""
    g = np.asarray(got, np.float64).ravel()
    o = np.asarray(want, np.float64).ravel()
    assert g.shape == o.shape, (what, g.shape, o.shape)
    assert np.all(np.isfinite(g)), what
    norm = float(np.linalg.norm(o))
    tol = rel * np.maximum(np.abs(o), tau * norm) + floor
    err = np.abs(g - o)
    ratio = err / np.where(tol > 0, tol, 1.0)
    ratio[tol == 0] = np.where(err[tol == 0] == 0, 0.0, np.inf)
    worst = float(ratio.max()) if ratio.size else 0.0
    key = what.split("[")[0] if what else "unnamed"
    WORST[key] = max(WORST.get(key, 0.0), worst)
    i = int(np.argmax(ratio)) if ratio.size else 0
    assert worst <= 1.0, (f"{what}: element {i} got {g[i]!r} want {o[i]!r} "
                          f"(|d| = {err[i]:.3g}, tol {tol[i]:.3g}, ||o|| = {norm:.3g})")
    assert np.linalg.norm(g - o) <= rel * norm + floor, (what, np.linalg.norm(g - o), norm)
    return worst


def close_rows(got, want, rel, what="", tau=TAU):
    """Per-row version for (n, k) arrays such as a vertex gradient: every row with a nonzero
    oracle value satisfies |g_v - o_v| <= rel * max(|o_v|, tau * max_u |o_u|), rows where the
    oracle is zero are zero on the GPU too, and the aggregate norm check holds."""
    g = np.asarray(got, np.float64)
    o = np.asarray(want, np.float64)
    assert g.shape == o.shape, (what, g.shape, o.shape)
    assert np.all(np.isfinite(g)), what
    on = np.linalg.norm(o, axis=1)
    err = np.linalg.norm(g - o, axis=1)
    nz = on > 0
    assert np.all(err[~nz] == 0), (what, int((err[~nz] > 0).sum()), "rows the oracle leaves at zero")
    tol = rel * np.maximum(on, tau * on.max())
    ratio = err[nz] / tol[nz]
    worst = float(ratio.max()) if ratio.size else 0.0
    key = what.split("[")[0] if what else "unnamed_rows"
    WORST[key] = max(WORST.get(key, 0.0), worst)
    i = int(np.flatnonzero(nz)[np.argmax(ratio)]) if ratio.size else 0
    assert worst <= 1.0, (f"{what}: row {i} got {g[i]} want {o[i]} (|d| = {err[i]:.3g}, "
                          f"tol {tol[i]:.3g}); {int((ratio > 1).sum())} of {ratio.size} rows over")
    assert np.linalg.norm(g - o) <= rel * np.linalg.norm(o), what
    return worst
