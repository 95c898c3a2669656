"""Pins of the oracle's input helpers: scan classes from a raw range image (Sec. IV.A, IV.B;
the reading rules in tests/golden/scan_classes.txt) and the pose of the paper's X (Eq. 1, read
as R = Rz Ry Rx), no GPU needed."""
from __future__ import annotations

import math
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
CLASS = {"FO": 0, "FU": 1, "NaN": 2}


def _rows():
    out = []
    for line in open(os.path.join(GOLDEN, "scan_classes.txt")):
        line = line.split("#")[0].strip()
        if line:
            raw, cls, depth = line.split()
            out.append((np.float32(raw), CLASS[cls], depth))
    return out


def test_scan_classes_golden():
    rows = _rows()
    raw = np.array([r[0] for r in rows], np.float32)
    d, c = oracle.scan_from_range(raw, 0.5, 4.0)
    for k, (r, cls, depth) in enumerate(rows):
        assert c[k] == cls, (r, c[k], cls)
        if depth == "max":
            assert d[k] == np.float32(4.0)
        elif depth == "nan":
            assert np.isnan(d[k])
        else:
            assert d[k] == np.float32(depth)


def test_pose_from_x_single_axes():
    for a in (0.3, -1.2, 2.9):
        T = oracle.pose_from_x([1.0, -2.0, 0.5, 0.0, 0.0, a])
        assert np.allclose(T[:3, :3], [[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1]],
                           atol=1e-15)
        assert np.array_equal(T[:3, 3], [1.0, -2.0, 0.5]) and np.array_equal(T[3], [0, 0, 0, 1])
        T = oracle.pose_from_x([0, 0, 0, a, 0.0, 0.0])
        assert np.allclose(T[:3, :3], [[1, 0, 0], [0, math.cos(a), -math.sin(a)], [0, math.sin(a), math.cos(a)]],
                           atol=1e-15)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_pose_from_x_is_rz_ry_rx(seed):
    r = np.random.Generator(np.random.PCG64(seed))
    X = np.concatenate([r.normal(size=3), r.uniform(-math.pi, math.pi, 3)])
    T = oracle.pose_from_x(X)
    # extrinsic rotations about x, then y, then z: R = Rz Ry Rx
    R = Rotation.from_euler("xyz", X[3:]).as_matrix()
    assert np.allclose(T[:3, :3], R, atol=1e-14)
    assert np.allclose(T[:3, :3] @ T[:3, :3].T, np.eye(3), atol=1e-14)
