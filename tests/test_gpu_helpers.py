"""Input helpers on the GPU vs the CPU oracle: scan classes of raw range images (bit for bit)
and poses of the paper's X (within FP64 rounding of sin and cos)."""
from __future__ import annotations

import ctypes
import math

import numpy as np
import pytest

import cases
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - the gpu marker is deselected on CPU
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1702_06813_gb300 as rm  # noqa: E402
from paper_1702_06813_gb300 import _native as N  # noqa: E402
from paper_1702_06813_gb300 import build as rmbuild  # noqa: E402

rmbuild.build()


def test_scan_from_range_bit_exact():
    r = np.random.Generator(np.random.PCG64(11))
    raw = r.uniform(-1.0, 6.0, (97, 131)).astype(np.float32)
    raw[r.random(raw.shape) < 0.05] = np.nan
    raw[r.random(raw.shape) < 0.03] = np.inf
    raw[r.random(raw.shape) < 0.03] = 0.0
    raw[0, :4] = [0.5, 4.0, np.nextafter(np.float32(4.0), np.float32(5)), np.nextafter(np.float32(0.5), np.float32(0))]
    cam = cases.small_pinhole(w=131, h=97)
    scan = rm.scan_from_range(rm.Intrinsics.from_camera(cam), raw, 0.5, 4.0)
    od, oc = oracle.scan_from_range(raw, 0.5, 4.0)
    gd, gc = scan.depth.cpu().numpy(), scan.cls.cpu().numpy()
    assert np.array_equal(gc, oc)
    assert np.array_equal(np.isnan(gd), np.isnan(od))
    assert np.array_equal(gd[~np.isnan(od)].view(np.uint32), od[~np.isnan(od)].view(np.uint32))
    assert set(np.unique(oc)) == {0, 1, 2}
    # host arrays through the ABI
    d = np.empty_like(raw)
    c = np.empty(raw.shape, np.uint8)
    assert N.lib().rm_scan_from_range(raw.ctypes.data, raw.size, 0.5, 4.0, d.ctypes.data, c.ctypes.data, None) == 0
    assert np.array_equal(c, oc)
    with pytest.raises(rm.RenderMapError):
        rm.scan_from_range(rm.Intrinsics.from_camera(cam), raw, 4.0, 0.5)


def test_pose_from_x_matches_oracle():
    r = np.random.Generator(np.random.PCG64(12))
    X = np.concatenate([r.normal(size=(50, 3)) * 10, r.uniform(-math.pi, math.pi, (50, 3))], 1)
    g = rm.pose_from_x(X).cpu().numpy()
    for k in range(50):
        assert np.allclose(g[k], oracle.pose_from_x(X[k]), rtol=0, atol=1e-14)
    out = np.empty((50, 16))
    Xc = np.ascontiguousarray(X)
    assert N.lib().rm_pose_from_x(Xc.ctypes.data, 50, out.ctypes.data, None) == 0
    assert np.array_equal(out.reshape(50, 4, 4), g)
