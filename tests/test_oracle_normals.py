"""Pins of the oracle's depth-image surface normals (Eq. 2) to closed forms (no GPU needed).

A symmetric, renormalised smoothing kernel leaves a linear depth image unchanged away from the
border, and central differences are exact for linear and quadratic images, so the normals of
such images are known exactly. Holes (invalid pixels) must invalidate exactly the pixels whose
central differences would touch them.
"""
from __future__ import annotations

import numpy as np
import pytest
from scipy import ndimage

import oracle


def _unit(v):
    v = np.asarray(v, float)
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


@pytest.mark.parametrize("sigma", [0.0, 0.8, 1.5, 3.0])
def test_normals_of_linear_depth(sigma):
    """z = a x + b y + c (dyadic coefficients, exact in FP32): away from the border the
    smoothed image is z itself and N = (a, b, -1) / |.|."""
    H, W = 40, 52
    a, b, c = 0.0625, -0.03125, 3.0
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    z = (a * x + b * y + c).astype(np.float32)
    assert np.array_equal(z.astype(np.float64), a * x + b * y + c)
    n, s = oracle.depth_normals(z, np.zeros((H, W), np.uint8), sigma=sigma)
    r = int(np.ceil(3 * sigma)) if sigma > 0 else 0
    inner = (slice(r + 1, H - r - 1), slice(r + 1, W - r - 1))
    assert np.allclose(s[inner], z[inner], rtol=1e-13, atol=0)
    assert np.allclose(n[inner], _unit([a, b, -1.0]), rtol=0, atol=1e-12)
    # the border row and column have no central difference
    assert np.isnan(n[0]).all() and np.isnan(n[-1]).all()
    assert np.isnan(n[:, 0]).all() and np.isnan(n[:, -1]).all()


def test_normals_of_quadratic_depth():
    """z = 2 + x^2 / 256: smoothing adds a constant, so dz/dx = x / 128 exactly and dz/dy = 0;
    N = (x / 128, 0, -1) / |.| at every interior pixel."""
    H, W = 24, 40
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    z = (2.0 + x * x / 256.0).astype(np.float32)
    n, s = oracle.depth_normals(z, np.zeros((H, W), np.uint8), sigma=1.0)
    inner = (slice(5, H - 5), slice(5, W - 5))
    want = _unit(np.stack([x / 128.0, np.zeros_like(x), -np.ones_like(x)], -1))
    assert np.allclose(n[inner], want[inner], rtol=0, atol=1e-12)


def test_holes_and_classes():
    """A constant image with holes (NaN depth, FU and NaN classes): the smoothed value is the
    constant wherever defined, normals face the camera, and the invalid set is the border
    plus the holes dilated by the 4-neighbour cross."""
    H, W = 30, 45
    r = np.random.Generator(np.random.PCG64(5))
    z = np.full((H, W), 2.5, np.float32)
    cls = np.zeros((H, W), np.uint8)
    hole = r.random((H, W)) < 0.05
    kind = r.integers(0, 3, (H, W))
    z[hole & (kind == 0)] = np.nan
    cls[hole & (kind == 1)] = 1
    cls[hole & (kind == 2)] = 2
    n, s = oracle.depth_normals(z, cls, sigma=1.2)
    assert np.array_equal(np.isnan(s), hole)
    assert np.allclose(s[~hole], 2.5, rtol=1e-13, atol=0)
    bad = ndimage.binary_dilation(hole, structure=ndimage.generate_binary_structure(2, 1))
    bad[0, :] = bad[-1, :] = bad[:, 0] = bad[:, -1] = True
    assert np.array_equal(np.isnan(n[..., 0]), bad)
    assert np.allclose(n[~bad], np.array([0.0, 0.0, -1.0]), rtol=0, atol=1e-12)


def test_metric_normal_of_tilted_plane_on_axis():
    """A plane n . P = d seen by a pinhole camera: at the pixel whose ray is the optical axis,
    Eq. 2 with the pixel footprint S/f as the step gives the plane's normal (oriented toward
    the camera) up to the central difference's truncation."""
    H, W, f = 41, 61, 120.0
    x0, y0 = 30, 20
    cx, cy = x0 + 0.5, y0 + 0.5
    nt = _unit([0.3, -0.2, -1.0])
    d = -2.0  # n . P = d with P = z r, r = ((x + .5 - cx) / f, (y + .5 - cy) / f, 1)
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    ray = np.stack([(x + 0.5 - cx) / f, (y + 0.5 - cy) / f, np.ones_like(x)], -1)
    z = (d / (ray @ nt)).astype(np.float32)
    n, _ = oracle.depth_normals(z, np.zeros((H, W), np.uint8), sigma=0.0, metric=True, fx=f, fy=f)
    assert np.allclose(n[y0, x0], nt, atol=2e-4)
    # in pixel units the same image gives the heightfield normal instead
    npx, _ = oracle.depth_normals(z, np.zeros((H, W), np.uint8), sigma=0.0)
    zx = 0.5 * (float(z[y0, x0 + 1]) - float(z[y0, x0 - 1]))
    zy = 0.5 * (float(z[y0 + 1, x0]) - float(z[y0 - 1, x0]))
    assert np.allclose(npx[y0, x0], _unit([zx, zy, -1.0]), atol=1e-12)


def test_sigma_bounds():
    z = np.ones((8, 8), np.float32)
    c = np.zeros((8, 8), np.uint8)
    with pytest.raises(ValueError):
        oracle.depth_normals(z, c, sigma=5.5)
    with pytest.raises(ValueError):
        oracle.depth_normals(z, c, sigma=-1.0)
    n, s = oracle.depth_normals(z, c, sigma=0.0)
    assert np.all(s == 1.0)


def test_blur_keeps_other_pixels_and_linear_interior():
    """Cost smoothing keeps FU and dead pixels as they are and, away from the border and the
    holes, leaves a linear depth image unchanged."""
    H, W = 30, 40
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    z = (2.0 + 0.0625 * x - 0.03125 * y).astype(np.float32)
    c = np.zeros((H, W), np.uint8)
    c[10:12, 5:8] = 1
    z[10:12, 5:8] = 4.0
    c[20, 30] = 2
    d, _ = oracle.depth_blur(z, c, sigma=1.0)
    assert np.array_equal(d[c != 0], z[c != 0])
    far = np.ones((H, W), bool)
    far[6:16, 1:12] = False  # within reach of the FU block
    far[16:25, 26:35] = False
    inner = np.zeros((H, W), bool)
    inner[4:-4, 4:-4] = True
    sel = far & inner & (c == 0)
    assert np.allclose(d[sel], z[sel], rtol=1e-6, atol=0)


def test_transpose_swaps_the_in_plane_components():
    """In pixel units, transposing a depth image transposes its normal field and swaps the
    x and y components (a mixed-up axis in either difference or in the cross product fails)."""
    r = np.random.Generator(np.random.PCG64(9))
    z = (2.0 + 0.3 * r.random((23, 31))).astype(np.float32)
    c = (r.random(z.shape) < 0.05).astype(np.uint8)
    n, _ = oracle.depth_normals(z, c, sigma=1.3)
    nt, _ = oracle.depth_normals(np.ascontiguousarray(z.T), np.ascontiguousarray(c.T), sigma=1.3)
    want = np.transpose(n, (1, 0, 2))[..., [1, 0, 2]]
    assert np.array_equal(np.isnan(nt), np.isnan(want))
    ok = ~np.isnan(want)
    assert np.allclose(nt[ok], want[ok], rtol=0, atol=1e-12)
