"""Seeded test workloads built from the synth generators (shared by oracle and GPU tests)."""
from __future__ import annotations

import math

import numpy as np

import synth


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def config1(seed=1000, noise=0.01, dropout=0.05):
    """160x120 pinhole, ~20k FO triangles in a 5x4x3 m box room with 30 boxes."""
    mesh = synth.room_mesh(seed)
    cam = synth.cam_160x120()
    r = rng(seed + 1)
    gt = synth.room_pose(r, mesh)
    depth, cls = synth.synth_scan(mesh, cam, gt, r, sigma_abs=noise, dropout=dropout)
    start = synth.perturb_fixed(gt, r, 0.05, 2.0)
    return dict(mesh=mesh, cam=cam, gt=gt, scan=(depth, cls), start=start)


def config2(seed=2000, target_fo=400_000, target_fu=100_000):
    """640x480 Kinect-shaped pinhole, cluttered 10x8x3 m room, 20% FU faces."""
    mesh = synth.room_mesh(seed, size=(10.0, 8.0, 3.0), n_boxes=120, n_slabs=12,
                           target_fo=target_fo, target_fu=target_fu, n_panels=250)
    cam = synth.cam_kinect_640x480()
    r = rng(seed + 1)
    gt = synth.room_pose(r, mesh)
    depth, cls = synth.synth_scan(mesh, cam, gt, r, sigma_rel=0.005)
    start = synth.perturb_fixed(gt, r, 0.05, 2.0)
    return dict(mesh=mesh, cam=cam, gt=gt, scan=(depth, cls), start=start)


def scan_from_render(depth32, cam, ids=None, labels=None):
    """Noise-free observed scan from a z-buffer depth image (FO where the hit is within range,
    FU at range_max otherwise), as Sec. IV.A draws no-return pixels."""
    d = np.array(depth32, np.float32, copy=True)
    cls = np.zeros(d.shape, np.uint8)
    miss = ~(d <= cam.range_max)
    cls[miss] = 1
    d[miss] = np.float32(cam.range_max)
    return d, cls


def plane_grid(nu, nv, origin, u, v, jitter=0.0, seed=0):
    """Tessellated parallelogram with shared vertices; interior vertices jittered in-plane."""
    r = rng(seed)
    a = np.arange(nu + 1) / nu
    b = np.arange(nv + 1) / nv
    A, B = np.meshgrid(a, b, indexing="ij")
    if jitter:
        ja = r.uniform(-jitter, jitter, size=A.shape) / nu
        jb = r.uniform(-jitter, jitter, size=B.shape) / nv
        ja[0, :] = ja[-1, :] = 0
        jb[:, 0] = jb[:, -1] = 0
        A = A + ja
        B = B + jb
    P = (np.asarray(origin)[None, None] + A[..., None] * np.asarray(u)[None, None]
         + B[..., None] * np.asarray(v)[None, None])
    ii, jj = np.meshgrid(np.arange(nu), np.arange(nv), indexing="ij")
    q00 = (ii * (nv + 1) + jj).ravel()
    q10 = ((ii + 1) * (nv + 1) + jj).ravel()
    q11 = ((ii + 1) * (nv + 1) + jj + 1).ravel()
    q01 = (ii * (nv + 1) + jj + 1).ravel()
    f = np.empty((2 * q00.size, 3), np.int32)
    f[0::2] = np.stack([q00, q10, q11], 1)
    f[1::2] = np.stack([q00, q11, q01], 1)
    return P.reshape(-1, 3).astype(np.float32), f


def closed_box(lo, hi, cell):
    rects = synth.box_rects(np.asarray(lo, float), np.asarray(hi, float), synth.FO)
    v, f, _ = synth.tessellate(rects, cell)
    return v, f


def random_tris(seed, n, zmin=-1.0, zmax=6.0, spread=3.0, size=1.5):
    """Random camera-space triangles in front of (and some behind / across) the camera."""
    r = rng(seed)
    c = np.stack([r.uniform(-spread, spread, n), r.uniform(-spread, spread, n),
                  r.uniform(zmin, zmax, n)], 1)
    v = c[:, None, :] + r.normal(scale=size, size=(n, 3, 3)) * r.uniform(0.02, 1.0, (n, 1, 1))
    return v.reshape(-1, 3).astype(np.float32), np.arange(3 * n, dtype=np.int32).reshape(n, 3)


def small_pinhole(w=48, h=40, f=40.0, near=0.1):
    return synth.Camera("pinhole", w, h, fx=f, fy=f * 1.1, cx=w / 2 + 0.3, cy=h / 2 - 0.2, near=near,
                        range_min=0.0, range_max=8.0)


def small_spherical(w=96, h=16, near=0.5):
    return synth.Camera("spherical", w, h, az0=-math.pi, az_step=2 * math.pi / w,
                        el0=math.radians(15.0), el_step=math.radians(40.0) / (h - 1), near=near,
                        range_min=0.5, range_max=80.0)
