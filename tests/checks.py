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


def fp32_bound(om, pose, cam, scan_depth, scan_class, eps=0.1, weights=(1.0, 1.0, 1.0)):
    """A-priori bound on how far FP32 sums of the adjoint (gradient, J^T J) may sit from the
    oracle's FP64 ones, element by element: (grad_bound (6,), jtj_bound (21,)).

    Per active pixel the Jacobian J = -(1 / (n . r)) (n, t r x n) is computed in FP32 from a
    unit normal and a ray. Its relative error is dominated by cancellation in n . r (terms of
    size sum |n_i r_i| summing to n . r: 8 u sum |n_i r_i| / |n . r|) and in the inverse-depth
    plane evaluation that gives t (pinhole: 8 u (|A x| + |B y| + |C|) / |A x + B y + C|),
    u = 2^-24; each sum adds 16 u of its absolute terms. The device's J also takes the z-buffer
    depth t32, the oracle's the exact depth t64: the rotation components carry |t32 - t64| / t64
    more (measured here per pixel). Grazing pixels (n . r near 0) make the bound large, which is
    when an element-wise 1e-3 comparison is not the right test."""
    u = 2.0 ** -24
    o = om.cost(pose, cam, scan_depth, scan_class, per_pixel=True)
    rend = om.render(pose, cam)
    ids, t32 = rend["tri_id"], rend["depth"]
    oc = o["outcome"]
    dz32 = (t32.astype(np.float32) - np.asarray(scan_depth, np.float32)).astype(np.float32)
    e32 = np.float32(eps)
    active = (oc == 0) | ((oc == 3) & (-dz32 < e32)) | ((oc == 5) & (dz32 < e32))
    jj, ii = np.nonzero(active)
    if ii.size == 0:
        return np.zeros(6), np.zeros(21)
    fid = ids[jj, ii]
    R, tr = pose[:3, :3], pose[:3, 3]
    w3 = (om.v.astype(np.float64)[om.faces[fid]] - tr) @ R
    n = np.cross(w3[:, 1] - w3[:, 0], w3[:, 2] - w3[:, 0])
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    if cam.model == "pinhole":
        fx, fy, cx, cy = (float(np.float32(x)) for x in (cam.fx, cam.fy, cam.cx, cam.cy))
        px, py = ii + 0.5, jj + 0.5
        r = np.stack([(px - cx) / fx, (py - cy) / fy, np.ones(ii.size)], 1)
        A, B = n[:, 0] / fx, n[:, 1] / fy
        C = n[:, 2] - A * cx - B * cy
        plane = (np.abs(A * px) + np.abs(B * py) + np.abs(C)) / np.abs(A * px + B * py + C)
    else:
        r = cam.ray_table_f32().astype(np.float64)[jj, ii]
        plane = np.zeros(ii.size)
    nr = np.einsum("pk,pk->p", n, r)
    cancel = np.abs(n * r).sum(1) / np.abs(nr)
    rel = 8 * u * (cancel + plane) + 16 * u
    t = t32[jj, ii].astype(np.float64)
    # the device's J takes the z-buffer depth t32 (1 / w of the FP32 plane), the oracle's the
    # exact ray-plane depth; the rotation components scale with that depth
    t64 = om.depth_exact(pose, cam, rend["keys"])[jj, ii]
    rel_t = np.abs(t - t64) / np.abs(t64)
    J = -np.concatenate([n, t[:, None] * np.cross(r, n)], 1) / nr[:, None]
    wmap = {0: weights[0], 3: weights[1], 5: weights[2]}
    w = np.vectorize(wmap.get)(oc[jj, ii]).astype(np.float64)
    res = np.abs(o["resid"][jj, ii])
    aJ = np.abs(J)
    # absolute error of each component: relative part, plus the rounding of the cross product
    # r x n, whose components cancel where r and n are nearly parallel
    crs = np.stack([np.abs(r[:, 1] * n[:, 2]) + np.abs(r[:, 2] * n[:, 1]),
                    np.abs(r[:, 2] * n[:, 0]) + np.abs(r[:, 0] * n[:, 2]),
                    np.abs(r[:, 0] * n[:, 1]) + np.abs(r[:, 1] * n[:, 0])], 1)
    dJ = aJ * rel[:, None]
    dJ[:, 3:] += aJ[:, 3:] * rel_t[:, None] + 4 * u * (t / np.abs(nr))[:, None] * crs
    g_bound = ((w * res)[:, None] * dJ).sum(0)
    H = np.einsum("p,pa,pb->ab", w, dJ, aJ) + np.einsum("p,pa,pb->ab", w, aJ, dJ)
    iu = np.triu_indices(6)
    return g_bound, H[iu]


def close_elementwise_or_bounded(got, want, rel, what, bound_fn, tau=TAU, floor=0.0):
    """close_elementwise; where an element misses it, the element must instead lie within
    rel |o_i| plus the FP32 error bound that bound_fn() returns for it (computed only then)."""
    try:
        return close_elementwise(got, want, rel, what, tau=tau, floor=floor)
    except AssertionError:
        pass
    g = np.asarray(got, np.float64).ravel()
    o = np.asarray(want, np.float64).ravel()
    b = np.asarray(bound_fn(), np.float64).ravel()
    err = np.abs(g - o)
    tol = rel * np.maximum(np.abs(o), tau * np.linalg.norm(o)) + floor + b
    ratio = err / tol
    key = (what.split("[")[0] if what else "unnamed") + "_fp32bound"
    WORST[key] = max(WORST.get(key, 0.0), float(ratio.max()))
    i = int(np.argmax(ratio))
    assert ratio.max() <= 1.0, (f"{what}: element {i} got {g[i]!r} want {o[i]!r} (|d| = {err[i]:.3g}, "
                                f"tol {tol[i]:.3g} incl. FP32 bound {b[i]:.3g})")
    assert np.linalg.norm(g - o) <= rel * np.linalg.norm(o) + floor + np.linalg.norm(b), what
    return float(ratio.max())
