"""The seeded synthetic inputs (stand-ins for the paper's RGB-D data): same seed, same
arrays; the recipe's shapes, counts and value ranges; scans that classify pixels by the
paper's no-return rule."""
from __future__ import annotations

import math

import numpy as np

import cases
import synth


def test_room_is_deterministic_and_sized():
    a = synth.room_mesh(1234)
    b = synth.room_mesh(1234)
    assert np.array_equal(a.vertices, b.vertices) and np.array_equal(a.faces, b.faces)
    assert np.array_equal(a.labels, b.labels)
    assert abs(a.n_tris - 20_000) <= 0.05 * 20_000 + 1000
    assert a.faces.min() >= 0 and a.faces.max() < a.vertices.shape[0]
    assert set(np.unique(a.labels)) <= {0, 1, 2}


def test_room_with_frontier_panels_has_fu_faces():
    m = synth.room_mesh(77, size=(10.0, 8.0, 3.0), n_boxes=40, n_slabs=4, target_fo=40_000,
                        target_fu=10_000, n_panels=20)
    frac = np.mean(m.labels == 1)
    assert 0.05 < frac < 0.5


def test_perturbations_have_the_requested_size():
    r = cases.rng(3)
    T = synth.pose_from(np.array([1.0, 2.0, 0.5]), 0.3, 0.1, -0.05)
    P = synth.perturb_fixed(T, r, 0.05, 2.0)
    assert abs(np.linalg.norm(P[:3, 3] - T[:3, 3]) - 0.05) < 1e-12
    c = (np.trace(T[:3, :3].T @ P[:3, :3]) - 1) / 2
    assert abs(math.degrees(math.acos(min(1.0, c))) - 2.0) < 1e-6
    G = synth.perturb_gauss(T, r, 0.1, 5.0, 2000)
    assert G.shape == (2000, 4, 4)
    # per-axis standard deviation of the displacement: 0.1 m (the candidate-pose recipe)
    sd = np.std(G[:, :3, 3] - T[:3, 3], axis=0)
    assert np.all((sd > 0.085) & (sd < 0.115)), sd


def test_scan_classes_follow_the_no_return_rule():
    c = cases.config1(seed=1000, noise=0.0, dropout=0.0)
    cam = c["cam"]
    d, cl = synth.synth_scan(c["mesh"], cam, c["gt"], cases.rng(5), dropout=0.2)
    fu = cl == 1
    assert fu.mean() > 0.1                       # dropout reads as "no return"
    assert np.all(d[fu] == np.float32(cam.range_max))
    fo = cl == 0
    assert np.all(d[fo] <= cam.range_max) and np.all(d[fo] > 0)
    d2, cl2 = synth.synth_scan(c["mesh"], cam, c["gt"], cases.rng(5), dropout=0.2, dropout_as_nan=True)
    dead = cl2 == 2                              # the same dropped pixels, now dead
    assert dead.mean() > 0.1 and np.all(fu[dead]) and np.all(np.isnan(d2[dead]))


def test_headline_workload_recipe():
    w = synth.workload_headline(3000, 8)
    assert w["mesh"].n_tris == 999_734
    assert w["cam"].width == 640 and w["cam"].height == 480 and w["cam"].fx == 525.0
    assert w["poses"].shape == (8, 4, 4)
    w2 = synth.workload_headline(3000, 8)
    assert np.array_equal(w["poses"], w2["poses"]) and np.array_equal(w["scan"][0], w2["scan"][0])
