"""Depth-image surface normals (Eq. 2) on the GPU vs the CPU oracle, through the C ABI.

Which pixels have a normal (validity) must match exactly; the smoothed depth within 1e-5
relative and the unit normals within 5e-4 (FP32 smoothing and differences against FP64).
"""
from __future__ import annotations

import dataclasses

import numpy as np
import pytest

import cases
import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - the gpu marker is deselected on CPU
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1702_06813_gb300 as rm  # noqa: E402
from paper_1702_06813_gb300 import build as rmbuild  # noqa: E402

rmbuild.build()


def _np(t):
    return t.detach().cpu().numpy()


def _check(gn, gs, on, os_):
    gn, gs = _np(gn), _np(gs)
    assert np.array_equal(np.isnan(gs), np.isnan(os_))
    ok = ~np.isnan(os_)
    assert np.all(np.abs(gs[ok] - os_[ok]) <= 1e-5 * np.abs(os_[ok]))
    assert np.array_equal(np.isnan(gn), np.isnan(on))
    okn = ~np.isnan(on[..., 0])
    assert np.max(np.abs(gn[okn] - on[okn]), initial=0.0) <= 5e-4


@pytest.fixture(scope="module")
def scans():
    c = cases.config2(seed=2400, target_fo=40_000, target_fu=10_000)
    cam = dataclasses.replace(c["cam"], width=213, height=161, fx=175.0, fy=175.0, cx=106.5, cy=80.5)
    r = cases.rng(24)
    out = []
    for k in range(3):
        pose = c["gt"] if k == 0 else synth.perturb_fixed(c["gt"], r, 0.05, 2.0)
        out.append(synth.synth_scan(c["mesh"], cam, pose, r, sigma_rel=0.005, dropout=0.05,
                                    dropout_as_nan=(k == 2)))
    return cam, out


@pytest.mark.parametrize("sigma", [0.0, 1.0, 2.5, 5.0])
@pytest.mark.parametrize("metric", [False, True])
def test_depth_normals_parity(scans, sigma, metric):
    cam, sc = scans
    intr = rm.Intrinsics.from_camera(cam)
    d = np.stack([s[0] for s in sc])
    c = np.stack([s[1] for s in sc])
    gn, gs = rm.depth_normals(intr, d, c, sigma=sigma, metric=metric, want_smoothed=True)
    for k in range(len(sc)):
        on, os_ = oracle.depth_normals(d[k], c[k], sigma=sigma, metric=metric, fx=cam.fx, fy=cam.fy)
        _check(gn[k], gs[k], on, os_)
    assert (~torch.isnan(gn[..., 0])).float().mean() > 0.5


def test_depth_normals_edge_cases():
    cam = cases.small_pinhole(w=1, h=1)
    intr = rm.Intrinsics.from_camera(cam)
    n = rm.depth_normals(intr, np.ones((1, 1), np.float32), np.zeros((1, 1), np.uint8))
    assert torch.isnan(n).all()
    # no images
    cam = cases.small_pinhole(w=37, h=29)
    intr = rm.Intrinsics.from_camera(cam)
    n = rm.depth_normals(intr, np.zeros((0, 29, 37), np.float32), np.zeros((0, 29, 37), np.uint8))
    assert n.shape == (0, 29, 37, 3)
    # every pixel invalid
    n = rm.depth_normals(intr, np.full((29, 37), np.nan, np.float32), np.zeros((29, 37), np.uint8))
    assert torch.isnan(n).all()
    # sigma out of range, metric on a ray-table camera
    with pytest.raises(rm.RenderMapError):
        rm.depth_normals(intr, np.ones((29, 37), np.float32), np.zeros((29, 37), np.uint8), sigma=6.0)
    sph = rm.Intrinsics.from_camera(cases.small_spherical(w=64, h=8))
    with pytest.raises(rm.RenderMapError):
        rm.depth_normals(sph, np.ones((8, 64), np.float32), np.zeros((8, 64), np.uint8), metric=True)
    n = rm.depth_normals(sph, np.ones((8, 64), np.float32), np.zeros((8, 64), np.uint8))
    assert torch.allclose(n[1:-1, 1:-1], torch.tensor([0.0, 0.0, -1.0], device="cuda"))


def test_depth_normals_host_buffers(scans):
    """Host arrays in and out through the ABI equal the device path."""
    import ctypes
    from paper_1702_06813_gb300 import _native as N
    cam, sc = scans
    intr = rm.Intrinsics.from_camera(cam)
    d = np.ascontiguousarray(np.stack([s[0] for s in sc]), np.float32)
    c = np.ascontiguousarray(np.stack([s[1] for s in sc]), np.uint8)
    out = np.empty(d.shape + (3,), np.float32)
    ci = intr.c()
    st = N.lib().rm_depth_normals(ctypes.byref(ci), d.shape[0], d.ctypes.data, c.ctypes.data, 1.5, 1,
                                  out.ctypes.data, None, None)
    assert st == N.RM_OK
    g = _np(rm.depth_normals(intr, d, c, sigma=1.5, metric=True))
    assert np.array_equal(np.isnan(out), np.isnan(g))
    assert np.array_equal(out[~np.isnan(out)], g[~np.isnan(g)])


@pytest.mark.parametrize("sigma", [0.0, 1.0, 3.0])
def test_depth_blur_parity(scans, sigma):
    """Cost smoothing: FO returns take the smoothed depth (within 1e-5 relative of the
    oracle's), every other pixel keeps its input depth bit for bit; the blurred scan scores
    like any scan."""
    cam, sc = scans
    intr = rm.Intrinsics.from_camera(cam)
    for d, c in sc:
        g = rm.blur_scan(rm.Scan.make(intr, d, c), sigma=sigma)
        od, _ = oracle.depth_blur(d, c, sigma=sigma)
        gd = _np(g.depth)
        fo = (c == 0) & np.isfinite(d)
        assert np.all(np.abs(gd[fo] - od[fo]) <= 1e-5 * np.abs(od[fo]))
        assert np.array_equal(gd[~fo].view(np.uint32), d[~fo].view(np.uint32))
        assert torch.equal(g.cls, torch.as_tensor(c, device="cuda"))
        if sigma == 0.0:
            assert np.array_equal(gd.view(np.uint32), np.asarray(d, np.float32).view(np.uint32))
