"""Seeded synthetic scenes shaped like the paper's Kinect (indoor) and Lidar (outdoor) workloads.

Conventions shared by every consumer of these arrays:

* World frame: metres, z up.
* Camera frame: x right, y down, z forward (pinhole); the same frame is used for the
  spherical (panoramic) model, where azimuth 0 / elevation 0 is +z, azimuth grows toward
  +x and elevation grows toward -y.
* A pose is a 4x4 float64 camera-to-world matrix T_wc (p_w = R p_c + t), row major.
* Face labels (Sec. IV.A, Fig. 3): 0 = free-occupied (FO), 1 = free-unknown (FU),
  2 = unknown-occupied (UO).
* Scan pixel classes (Sec. IV.B): 0 = FO (a return), 1 = FU (no return, drawn at the
  sensor's maximum range as Sec. IV.A prescribes), 2 = NaN (dead pixel).

All randomness comes from numpy's PCG64 seeded per call.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy.spatial.transform import Rotation

FO, FU, UO = 0, 1, 2
S_FO, S_FU, S_NAN = 0, 1, 2

# camera axes expressed in a body frame (x forward, y left, z up)
_R_BODY_CAM = np.array([[0.0, 0.0, 1.0], [-1.0, 0.0, 0.0], [0.0, -1.0, 0.0]])


@dataclasses.dataclass
class Mesh:
    vertices: np.ndarray  # (V, 3) float32, world
    faces: np.ndarray     # (T, 3) int32
    labels: np.ndarray    # (T,) uint8
    # solid world geometry used only to synthesise observed range images
    boxes: np.ndarray     # (B, 2, 3) float64 axis-aligned solids (lo, hi)
    room: np.ndarray | None = None   # (2, 3) inside-out box the sensor sits in, or None
    terrain: dict | None = None      # heightfield description, or None

    @property
    def n_tris(self) -> int:
        return int(self.faces.shape[0])

    @property
    def n_verts(self) -> int:
        return int(self.vertices.shape[0])


@dataclasses.dataclass
class Camera:
    model: str           # "pinhole" or "spherical"
    width: int
    height: int
    fx: float = 0.0
    fy: float = 0.0
    cx: float = 0.0
    cy: float = 0.0
    # spherical: azimuth of column i = az0 + az_step*(i+0.5); elevation of row j = el0 - el_step*j
    az0: float = 0.0
    az_step: float = 0.0
    el0: float = 0.0
    el_step: float = 0.0
    near: float = 0.1
    far: float = math.inf
    range_min: float = 0.0
    range_max: float = math.inf

    def rays(self) -> np.ndarray:
        """(H, W, 3) float64 ray per pixel centre in the camera frame.

        Pinhole rays are scaled to z = 1 (the ray parameter is z-depth); spherical rays are
        unit vectors (the ray parameter is range).
        """
        j, i = np.meshgrid(np.arange(self.height, dtype=np.float64),
                           np.arange(self.width, dtype=np.float64), indexing="ij")
        if self.model == "pinhole":
            return np.stack([(i + 0.5 - self.cx) / self.fx, (j + 0.5 - self.cy) / self.fy,
                             np.ones_like(i)], axis=-1)
        az = self.az0 + self.az_step * (i + 0.5)
        el = self.el0 - self.el_step * j
        return np.stack([np.cos(el) * np.sin(az), -np.sin(el), np.cos(el) * np.cos(az)], axis=-1)

    def ray_table_f32(self) -> np.ndarray:
        """Unit rays rounded to float32, (H, W, 3); the spherical model's calibration input."""
        return np.ascontiguousarray(self.rays().astype(np.float32))


# --------------------------------------------------------------------------------------
# poses
# --------------------------------------------------------------------------------------

def pose_from(position, yaw, pitch=0.0, roll=0.0) -> np.ndarray:
    """Camera-to-world pose of a sensor at `position` with body yaw/pitch/roll (radians)."""
    r_wb = Rotation.from_euler("ZYX", [yaw, pitch, roll]).as_matrix()
    t = np.eye(4)
    t[:3, :3] = r_wb @ _R_BODY_CAM
    t[:3, 3] = position
    return t


def perturb(pose: np.ndarray, trans: np.ndarray, rotvec: np.ndarray) -> np.ndarray:
    """pose * [Rot(rotvec), trans] (a perturbation expressed in the camera frame)."""
    d = np.eye(4)
    d[:3, :3] = Rotation.from_rotvec(rotvec).as_matrix()
    d[:3, 3] = trans
    return pose @ d


def perturb_fixed(pose, rng, trans_m, rot_deg):
    """Perturb by a random-direction translation of norm trans_m and a random-axis rotation."""
    u = rng.normal(size=3)
    u /= np.linalg.norm(u)
    a = rng.normal(size=3)
    a /= np.linalg.norm(a)
    return perturb(pose, u * trans_m, a * math.radians(rot_deg))


def perturb_gauss(pose, rng, sigma_m, sigma_deg, n):
    """n poses pose * [Rot(N(0, sigma_deg^2 I)), N(0, sigma_m^2 I)]."""
    out = np.empty((n, 4, 4))
    for k in range(n):
        out[k] = perturb(pose, rng.normal(scale=sigma_m, size=3),
                         rng.normal(scale=math.radians(sigma_deg), size=3))
    return out


# --------------------------------------------------------------------------------------
# tessellation
# --------------------------------------------------------------------------------------

def _rect_counts(rects, s):
    tot = 0
    for o, u, v, _ in rects:
        tot += 2 * max(1, math.ceil(np.linalg.norm(u) / s)) * max(1, math.ceil(np.linalg.norm(v) / s))
    return tot


def _solve_cell(rects, target):
    lo, hi = 1e-4, 100.0
    for _ in range(80):
        mid = math.sqrt(lo * hi)
        if _rect_counts(rects, mid) > target:
            lo = mid
        else:
            hi = mid
    return hi


def tessellate(rects, cell):
    """Grid-tessellate rectangles (origin o, edges u, v, label) with cells of about `cell` m."""
    vs, fs, ls = [], [], []
    base = 0
    for o, u, v, lab in rects:
        nu = max(1, math.ceil(np.linalg.norm(u) / cell))
        nv = max(1, math.ceil(np.linalg.norm(v) / cell))
        a = np.arange(nu + 1, dtype=np.float64) / nu
        b = np.arange(nv + 1, dtype=np.float64) / nv
        A, B = np.meshgrid(a, b, indexing="ij")
        p = o[None, None, :] + A[..., None] * u[None, None, :] + B[..., None] * v[None, None, :]
        vs.append(p.reshape(-1, 3))
        ii, jj = np.meshgrid(np.arange(nu), np.arange(nv), indexing="ij")
        q00 = (ii * (nv + 1) + jj).ravel()
        q10 = ((ii + 1) * (nv + 1) + jj).ravel()
        q11 = ((ii + 1) * (nv + 1) + jj + 1).ravel()
        q01 = (ii * (nv + 1) + jj + 1).ravel()
        f = np.empty((2 * q00.size, 3), dtype=np.int64)
        f[0::2] = np.stack([q00, q10, q11], axis=1)
        f[1::2] = np.stack([q00, q11, q01], axis=1)
        fs.append(f + base)
        ls.append(np.full(f.shape[0], lab, dtype=np.uint8))
        base += p.shape[0] * p.shape[1]
    V = np.concatenate(vs).astype(np.float32)
    F = np.concatenate(fs)
    L = np.concatenate(ls)
    # weld vertices with bit-identical float32 positions
    key = np.ascontiguousarray(V).view(np.dtype((np.void, 12))).ravel()
    _, first, inv = np.unique(key, return_index=True, return_inverse=True)
    order = np.argsort(first)
    remap = np.empty_like(order)
    remap[order] = np.arange(order.size)
    V = V[first[order]]
    F = remap[inv.ravel()][F].astype(np.int32)
    return np.ascontiguousarray(V), np.ascontiguousarray(F), L


def box_rects(lo, hi, label=FO):
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    dx, dy, dz = hi - lo
    ex, ey, ez = np.array([dx, 0, 0.0]), np.array([0, dy, 0.0]), np.array([0, 0, dz])
    return [
        (lo.copy(), ey, ex, label),                      # bottom
        (lo + ez, ex, ey, label),                        # top
        (lo.copy(), ex, ez, label),                      # y = lo
        (lo + ey, ez, ex, label),                        # y = hi
        (lo.copy(), ez, ey, label),                      # x = lo
        (lo + ex, ey, ez, label),                        # x = hi
    ]


def _inside_any(p, boxes, margin):
    for lo, hi in boxes:
        if np.all(p > lo - margin) and np.all(p < hi + margin):
            return True
    return False


def _room_boxes(rng, size, n_boxes, n_slabs):
    sx, sy, sz = size
    boxes = []
    for _ in range(n_boxes):
        d = rng.uniform(0.2, 1.0, size=3)
        if boxes and rng.uniform() < 0.25:
            # stack on an earlier box
            lo0, hi0 = boxes[rng.integers(len(boxes))]
            x = rng.uniform(lo0[0], max(lo0[0], hi0[0] - d[0] * 0.5))
            y = rng.uniform(lo0[1], max(lo0[1], hi0[1] - d[1] * 0.5))
            z = hi0[2]
        else:
            x = rng.uniform(0.0, sx - d[0])
            y = rng.uniform(0.0, sy - d[1])
            z = 0.0
        lo = np.array([x, y, z]) - np.array([sx, sy, 0.0]) / 2
        hi = lo + d
        hi[2] = min(hi[2], sz - 0.3)
        hi[0] = min(hi[0], sx / 2 - 0.01)
        hi[1] = min(hi[1], sy / 2 - 0.01)
        if np.all(hi > lo + 0.05):
            boxes.append((lo, hi))
    for _ in range(n_slabs):
        # tables: a thin top slab on four thin legs
        w, dpt, h = rng.uniform(1.0, 1.8), rng.uniform(0.6, 0.9), rng.uniform(0.7, 0.8)
        x = rng.uniform(-sx / 2 + 0.2, sx / 2 - 0.2 - w)
        y = rng.uniform(-sy / 2 + 0.2, sy / 2 - 0.2 - dpt)
        boxes.append((np.array([x, y, h - 0.04]), np.array([x + w, y + dpt, h])))
        for lx, ly in ((x, y), (x + w - 0.05, y), (x, y + dpt - 0.05), (x + w - 0.05, y + dpt - 0.05)):
            boxes.append((np.array([lx, ly, 0.0]), np.array([lx + 0.05, ly + 0.05, h - 0.04])))
    return boxes


def _frontier_panels(rng, size, boxes, n_panels):
    """FU interface panels: axis-aligned quads in free space 0.2-0.5 m in front of a wall."""
    sx, sy, sz = size
    rects = []
    for _ in range(n_panels):
        wall = rng.integers(4)
        w, h = rng.uniform(0.3, 1.0), rng.uniform(0.3, 1.0)
        off = rng.uniform(0.2, 0.5)
        z = rng.uniform(0.1, sz - 0.1 - h)
        if wall < 2:
            x = rng.uniform(-sx / 2 + 0.1, sx / 2 - 0.1 - w)
            y = (-sy / 2 + off) if wall == 0 else (sy / 2 - off)
            o, u, v = np.array([x, y, z]), np.array([w, 0, 0.0]), np.array([0, 0, h])
        else:
            y = rng.uniform(-sy / 2 + 0.1, sy / 2 - 0.1 - w)
            x = (-sx / 2 + off) if wall == 2 else (sx / 2 - off)
            o, u, v = np.array([x, y, z]), np.array([0, w, 0.0]), np.array([0, 0, h])
        rects.append((o, u, v, FU))
    return rects


def room_mesh(seed, size=(5.0, 4.0, 3.0), n_boxes=30, n_slabs=0, target_fo=20_000,
              target_fu=0, n_panels=0) -> Mesh:
    """Box room (inward walls) with axis-aligned clutter, grid-tessellated to ~target_fo FO
    triangles, plus ~target_fu FU frontier-panel triangles."""
    rng = np.random.Generator(np.random.PCG64(seed))
    size = np.asarray(size, np.float64)
    boxes = _room_boxes(rng, size, n_boxes, n_slabs)
    lo_r, hi_r = -size / 2 * np.array([1, 1, 0]), size / 2 * np.array([1, 1, 0]) + np.array([0, 0, size[2]])
    rects = box_rects(lo_r, hi_r, FO)
    for lo, hi in boxes:
        rects += box_rects(lo, hi, FO)
    cell = _solve_cell(rects, target_fo)
    V, F, L = tessellate(rects, cell)
    if target_fu > 0:
        prect = _frontier_panels(rng, size, boxes, n_panels)
        pcell = _solve_cell(prect, target_fu)
        V2, F2, L2 = tessellate(prect, pcell)
        F = np.concatenate([F, F2 + V.shape[0]]).astype(np.int32)
        V = np.concatenate([V, V2])
        L = np.concatenate([L, L2])
    return Mesh(vertices=np.ascontiguousarray(V), faces=np.ascontiguousarray(F),
                labels=np.ascontiguousarray(L), boxes=np.array([[lo, hi] for lo, hi in boxes]).reshape(-1, 2, 3),
                room=np.array([lo_r, hi_r]))


def room_pose(rng, mesh: Mesh, max_tilt_deg=10.0) -> np.ndarray:
    lo_r, hi_r = mesh.room
    for _ in range(10_000):
        p = np.array([rng.uniform(lo_r[0] + 0.6, hi_r[0] - 0.6),
                      rng.uniform(lo_r[1] + 0.6, hi_r[1] - 0.6),
                      rng.uniform(1.0, min(2.0, hi_r[2] - 0.4))])
        if not _inside_any(p, mesh.boxes, 0.4):
            break
    t = math.radians(max_tilt_deg)
    return pose_from(p, rng.uniform(-math.pi, math.pi), rng.uniform(-t, t), rng.uniform(-t, t))


# --------------------------------------------------------------------------------------
# observed range images (analytic ray cast of the world solids)
# --------------------------------------------------------------------------------------

def _cast_world(mesh: Mesh, origin, dirs):
    """Ray parameter of the first world surface hit along origin + t*dirs (inf if none)."""
    best = np.full(dirs.shape[:-1], np.inf)
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / dirs
        for lo, hi in mesh.boxes:
            t1 = (lo - origin) * inv
            t2 = (hi - origin) * inv
            tmin = np.nanmax(np.minimum(t1, t2), axis=-1)
            tmax = np.nanmin(np.maximum(t1, t2), axis=-1)
            hit = (tmax >= tmin) & (tmin > 0)
            best = np.where(hit & (tmin < best), tmin, best)
        if mesh.room is not None:
            lo, hi = mesh.room
            t1 = (lo - origin) * inv
            t2 = (hi - origin) * inv
            tmax = np.nanmin(np.maximum(t1, t2), axis=-1)
            best = np.where((tmax > 0) & (tmax < best), tmax, best)
    if mesh.terrain is not None:
        best = np.minimum(best, _cast_terrain(mesh.terrain, origin, dirs))
    return best


def synth_scan(mesh: Mesh, cam: Camera, pose: np.ndarray, rng, sigma_abs=0.0, sigma_rel=0.0,
               dropout=0.0, dropout_as_nan=False):
    """Observed range image of the world from `pose`: (depth float32 HxW, class uint8 HxW).

    No return beyond range_max, and dropped-out pixels, become FU at range_max (Sec. IV.A);
    returns closer than range_min are dead pixels (NaN)."""
    rays = cam.rays()
    dirs = rays @ pose[:3, :3].T
    t = _cast_world(mesh, pose[:3, 3], dirs)
    if sigma_abs or sigma_rel:
        t = t + rng.normal(size=t.shape) * (sigma_abs + sigma_rel * np.where(np.isfinite(t), t, 0.0))
    cls = np.full(t.shape, S_FO, np.uint8)
    far = ~(t <= cam.range_max)
    cls[far] = S_FU
    t = np.where(far, cam.range_max, t)
    if dropout > 0:
        drop = rng.uniform(size=t.shape) < dropout
        if dropout_as_nan:
            cls[drop] = S_NAN
        else:
            cls[drop] = S_FU
            t = np.where(drop, cam.range_max, t)
    close = (t < cam.range_min) & (cls == S_FO)
    cls[close] = S_NAN
    depth = t.astype(np.float32)
    depth[cls == S_NAN] = np.nan
    return np.ascontiguousarray(depth), np.ascontiguousarray(cls)


# --------------------------------------------------------------------------------------
# outdoor terrain (heightfield + extruded buildings)
# --------------------------------------------------------------------------------------

def _value_noise(terrain, x, y):
    h = np.zeros(np.broadcast(x, y).shape)
    for amp, freq, grid in terrain["octaves"]:
        gx = (x - terrain["x0"]) * freq
        gy = (y - terrain["y0"]) * freq
        ix = np.clip(np.floor(gx).astype(np.int64), 0, grid.shape[0] - 2)
        iy = np.clip(np.floor(gy).astype(np.int64), 0, grid.shape[1] - 2)
        fx = gx - ix
        fy = gy - iy
        sx = fx * fx * (3 - 2 * fx)
        sy = fy * fy * (3 - 2 * fy)
        g00 = grid[ix, iy]
        g10 = grid[ix + 1, iy]
        g01 = grid[ix, iy + 1]
        g11 = grid[ix + 1, iy + 1]
        h += amp * ((g00 * (1 - sx) + g10 * sx) * (1 - sy) + (g01 * (1 - sx) + g11 * sx) * sy)
    return h


def terrain_height(terrain, x, y):
    return _value_noise(terrain, x, y)


def _cast_terrain(terrain, origin, dirs):
    """Ray-march the heightfield (the world the terrain mesh samples), then bisect the first
    crossing of every ray (vectorised)."""
    shape = dirs.shape[:-1]
    d = dirs.reshape(-1, 3)
    tmax = terrain["max_range"]
    step = terrain["march_step"]
    best = np.full(d.shape[0], np.inf)
    alive = np.ones(d.shape[0], bool)
    t = step
    while t <= tmax and alive.any():
        idx = np.nonzero(alive)[0]
        p = origin[None, :] + t * d[idx]
        inside = (np.abs(p[:, 0]) <= terrain["half"]) & (np.abs(p[:, 1]) <= terrain["half"])
        below = inside & (p[:, 2] <= terrain_height(terrain, p[:, 0], p[:, 1]))
        hit = idx[below]
        if hit.size:
            a = np.full(hit.size, t - step)
            b = np.full(hit.size, t)
            for _ in range(30):
                m = 0.5 * (a + b)
                q = origin[None, :] + m[:, None] * d[hit]
                under = q[:, 2] <= terrain_height(terrain, q[:, 0], q[:, 1])
                b = np.where(under, m, b)
                a = np.where(under, a, m)
            best[hit] = 0.5 * (a + b)
            alive[hit] = False
        t += step
    return best.reshape(shape)


def terrain_mesh(seed, half=100.0, n_buildings=40, target_fo=1_400_000, target_fu=600_000,
                 n_panels=400) -> Mesh:
    """200x200 m heightfield terrain (6 octaves of value noise, +-3 m) plus extruded building
    boxes; FU frontier panels standing in free space near the buildings."""
    rng = np.random.Generator(np.random.PCG64(seed))
    octaves = []
    for o in range(6):
        freq = (2 ** o) / 50.0
        n = int(math.ceil(2 * half * freq)) + 2
        octaves.append((3.0 / (2 ** o) * 0.55, freq, rng.uniform(-1, 1, size=(n, n))))
    terrain = {"octaves": octaves, "x0": -half, "y0": -half, "half": half,
               "max_range": 120.0, "march_step": 0.25}
    boxes = []
    for _ in range(n_buildings):
        fx, fy = rng.uniform(5, 30, size=2)
        hgt = rng.uniform(3, 20)
        x = rng.uniform(-half + 2, half - 2 - fx)
        y = rng.uniform(-half + 2, half - 2 - fy)
        zb = float(np.min(terrain_height(terrain, np.array([x, x + fx, x, x + fx]),
                                         np.array([y, y, y + fy, y + fy])))) - 1.0
        boxes.append((np.array([x, y, zb]), np.array([x + fx, y + fy, zb + 1.0 + hgt])))
    # building walls + roofs
    rects = []
    for lo, hi in boxes:
        rects += box_rects(lo, hi, FO)[1:]
    # terrain grid cell solved jointly with the buildings' walls
    area_walls = sum(np.linalg.norm(u) * np.linalg.norm(v) for _, u, v, _ in rects)
    area_t = (2 * half) ** 2
    cell = math.sqrt(2 * (area_walls + area_t) / target_fo)
    n = max(2, int(round(2 * half / cell)))
    g = np.linspace(-half, half, n + 1)
    X, Y = np.meshgrid(g, g, indexing="ij")
    Z = terrain_height(terrain, X, Y)
    tv = np.stack([X, Y, Z], axis=-1).reshape(-1, 3)
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    q00 = (ii * (n + 1) + jj).ravel()
    q10 = ((ii + 1) * (n + 1) + jj).ravel()
    q11 = ((ii + 1) * (n + 1) + jj + 1).ravel()
    q01 = (ii * (n + 1) + jj + 1).ravel()
    tf = np.empty((2 * q00.size, 3), np.int64)
    tf[0::2] = np.stack([q00, q10, q11], 1)
    tf[1::2] = np.stack([q00, q11, q01], 1)
    V1, F1, L1 = tessellate(rects, cell)
    V = np.concatenate([tv.astype(np.float32), V1])
    F = np.concatenate([tf, F1 + tv.shape[0]])
    L = np.concatenate([np.zeros(tf.shape[0], np.uint8), L1])
    # FU frontier panels: vertical quads in free space 1-5 m in front of building walls
    prect = []
    for _ in range(n_panels):
        lo, hi = boxes[rng.integers(len(boxes))]
        side = rng.integers(4)
        w, h = rng.uniform(2, 8), rng.uniform(2, 6)
        off = rng.uniform(1, 5)
        z = rng.uniform(lo[2] + 1.0, max(lo[2] + 1.5, hi[2] - h))
        if side < 2:
            x = rng.uniform(lo[0], max(lo[0], hi[0] - w))
            y = lo[1] - off if side == 0 else hi[1] + off
            prect.append((np.array([x, y, z]), np.array([w, 0, 0.0]), np.array([0, 0, h]), FU))
        else:
            y = rng.uniform(lo[1], max(lo[1], hi[1] - w))
            x = lo[0] - off if side == 2 else hi[0] + off
            prect.append((np.array([x, y, z]), np.array([0, w, 0.0]), np.array([0, 0, h]), FU))
    if target_fu > 0 and prect:
        pcell = _solve_cell(prect, target_fu)
        V2, F2, L2 = tessellate(prect, pcell)
        F = np.concatenate([F, F2 + V.shape[0]])
        V = np.concatenate([V, V2])
        L = np.concatenate([L, L2])
    return Mesh(vertices=np.ascontiguousarray(V.astype(np.float32)),
                faces=np.ascontiguousarray(F.astype(np.int32)), labels=np.ascontiguousarray(L),
                boxes=np.array([[lo, hi] for lo, hi in boxes]).reshape(-1, 2, 3), room=None,
                terrain=terrain)


def workload_lidar(seed=4000, target_fo=1_400_000, target_fu=600_000, n_panels=400, noise=0.02):
    """Panoramic Lidar on a 200x200 m outdoor mesh: 1024 azimuths x 64 rings (+15..-25 deg),
    range 1-80 m, sigma 2 cm; the start pose is 30 cm / 3 deg off the true pose."""
    mesh = terrain_mesh(seed, target_fo=target_fo, target_fu=target_fu, n_panels=n_panels)
    cam = cam_lidar_1024x64()
    r = np.random.Generator(np.random.PCG64(seed + 1))
    gt = terrain_pose(r, mesh)
    depth, cls = synth_scan(mesh, cam, gt, r, sigma_abs=noise)
    start = perturb_fixed(gt, r, 0.30, 3.0)
    return dict(name="terrain-2M-lidar-1024x64", mesh=mesh, cam=cam, gt=gt, scan=(depth, cls),
                start=start)


def terrain_pose(rng, mesh: Mesh, height=1.8) -> np.ndarray:
    half = mesh.terrain["half"]
    for _ in range(10_000):
        xy = rng.uniform(-half * 0.6, half * 0.6, size=2)
        z = float(terrain_height(mesh.terrain, xy[0], xy[1])) + height
        p = np.array([xy[0], xy[1], z])
        if not _inside_any(p, mesh.boxes, 3.0):
            break
    return pose_from(p, rng.uniform(-math.pi, math.pi), 0.0, 0.0)


# --------------------------------------------------------------------------------------
# cameras of the five workloads
# --------------------------------------------------------------------------------------

def cam_160x120():
    return Camera("pinhole", 160, 120, fx=140.0, fy=140.0, cx=80.0, cy=60.0, near=0.1,
                  range_min=0.0, range_max=4.0)


def cam_kinect_640x480():
    return Camera("pinhole", 640, 480, fx=525.0, fy=525.0, cx=320.0, cy=240.0, near=0.5,
                  range_min=0.5, range_max=4.5)


def cam_320x240():
    return Camera("pinhole", 320, 240, fx=262.5, fy=262.5, cx=160.0, cy=120.0, near=0.1,
                  range_min=0.5, range_max=4.5)


def cam_lidar_1024x64():
    return Camera("spherical", 1024, 64, az0=-math.pi, az_step=2 * math.pi / 1024,
                  el0=math.radians(15.0), el_step=math.radians(40.0) / 63, near=1.0,
                  range_min=1.0, range_max=80.0)


# --------------------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------------------

def workload_headline(seed=3000, n_poses=256):
    """Candidate-pose batch on a 1M-triangle cluttered room (800k FO + 200k FU faces), one
    640x480 Kinect-shaped scan (fx = fy = 525, 0.5-4.5 m, noise 0.5% of depth) and n_poses
    poses drawn around the true pose with sigma 10 cm / 5 deg. The 40 frontier panels cover
    about a third of a view, so most pixels compare occupied surfaces (FO/FO)."""
    mesh = room_mesh(seed, size=(10.0, 8.0, 3.0), n_boxes=120, n_slabs=12, target_fo=800_000,
                     target_fu=200_000, n_panels=40)
    cam = cam_kinect_640x480()
    r = np.random.Generator(np.random.PCG64(seed + 1))
    gt = room_pose(r, mesh)
    depth, cls = synth_scan(mesh, cam, gt, r, sigma_rel=0.005)
    poses = perturb_gauss(gt, r, 0.10, 5.0, n_poses)
    return dict(name="room-1M-640x480-256poses", mesh=mesh, cam=cam, gt=gt, scan=(depth, cls),
                poses=poses)


def workload_tracking(seed=5000, n_agents=64, n_frames=200, target_fo=1_400_000,
                      target_fu=600_000, n_panels=400, speed=0.5, rate_hz=2.0):
    """Uneven tracking batch: n_agents walk seeded smooth trajectories (0.5 m/s, 2 Hz sensor
    rate, so 0.25 m per frame) over the outdoor mesh; agent a carries sensor a mod 3 in
    {160x120 pinhole, 640x480 pinhole, 1024x64 Lidar}. Returns the true camera poses per frame
    and agent; the observed scans are made per frame by the caller."""
    mesh = terrain_mesh(seed, target_fo=target_fo, target_fu=target_fu, n_panels=n_panels)
    r = np.random.Generator(np.random.PCG64(seed + 1))
    cams = [dataclasses.replace(cam_160x120(), range_max=40.0, near=0.3),
            dataclasses.replace(cam_kinect_640x480(), range_max=40.0, range_min=0.3, near=0.3),
            cam_lidar_1024x64()]
    step = speed / rate_hz
    poses = np.empty((n_frames, n_agents, 4, 4))
    kinds = np.arange(n_agents) % 3
    half = mesh.terrain["half"]
    for a in range(n_agents):
        for _ in range(1000):
            p0 = r.uniform(-half * 0.4, half * 0.4, size=2)
            if not _inside_any(np.array([p0[0], p0[1], 0.0]) * np.array([1, 1, 0]) +
                               np.array([0, 0, float(terrain_height(mesh.terrain, p0[0], p0[1]))]),
                               mesh.boxes, 3.0):
                break
        psi0, amp, ph = r.uniform(-math.pi, math.pi), r.uniform(0.1, 0.4), r.uniform(0, 2 * math.pi)
        h = 1.8 if kinds[a] == 2 else 1.5
        pitch = 0.0 if kinds[a] == 2 else math.radians(15.0)
        xy = p0.copy()
        for f in range(n_frames):
            psi = psi0 + amp * math.sin(2 * math.pi * f / 60.0 + ph)
            if f > 0:
                xy = xy + step * np.array([math.cos(psi), math.sin(psi)])
            z = float(terrain_height(mesh.terrain, xy[0], xy[1])) + h
            poses[f, a] = pose_from(np.array([xy[0], xy[1], z]), psi, pitch, 0.0)
    return dict(name=f"terrain-2M-tracking-{n_agents}x{n_frames}", mesh=mesh, cams=cams,
                kinds=kinds, poses=poses)
