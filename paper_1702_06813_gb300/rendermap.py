"""PyTorch-facing wrappers of the C ABI (include/rendermap.h).

Torch supplies device memory and the current CUDA stream; every step of the pose-cost path
runs in librendermap's kernels. Inputs may be numpy arrays or torch tensors (host or CUDA);
results come back as CUDA tensors unless ``host=True``.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass

import numpy as np
import torch

from . import _native as N
from ._native import check, lib

RM_PINHOLE, RM_RAYTABLE = N.RM_PINHOLE, N.RM_RAYTABLE
OUTCOMES = ("fofo_reward", "fofo_penalty", "fofu_reward", "fofu_penalty", "fufo_reward",
            "fufo_penalty")


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _dev_tensor(x, dtype, device="cuda"):
    if isinstance(x, torch.Tensor):
        return x.to(device=device, dtype=dtype).contiguous()
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device=device)


@dataclass
class Intrinsics:
    """Camera model of include/rendermap.h (pinhole, or a ray table for panoramic sensors)."""
    model: int
    width: int
    height: int
    fx: float = 0.0
    fy: float = 0.0
    cx: float = 0.0
    cy: float = 0.0
    az0: float = 0.0
    az_step: float = 0.0
    el0: float = 0.0
    el_step: float = 0.0
    near: float = 0.1
    far: float = math.inf
    rays: torch.Tensor | None = None  # (H, W, 3) float32 on the device for RM_RAYTABLE

    @staticmethod
    def from_camera(cam, device="cuda") -> "Intrinsics":
        """From any object with the attributes of synth.Camera."""
        model = RM_PINHOLE if cam.model == "pinhole" else RM_RAYTABLE
        rays = None
        if model == RM_RAYTABLE:
            rays = _dev_tensor(cam.ray_table_f32(), torch.float32, device)
        return Intrinsics(model, cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy, cam.az0,
                          cam.az_step, cam.el0, cam.el_step, cam.near, cam.far, rays)

    def c(self) -> N.rm_intrinsics:
        return N.rm_intrinsics(self.model, self.width, self.height, 0, self.fx, self.fy, self.cx,
                               self.cy, self.az0, self.az_step, self.el0, self.el_step, self.near,
                               self.far, None if self.rays is None else self.rays.data_ptr())


@dataclass
class Scan:
    """Observed scan Z_s of Eq. 1: per-pixel depth (float32) and class (uint8)."""
    intr: Intrinsics
    depth: torch.Tensor
    cls: torch.Tensor

    @staticmethod
    def make(intr: Intrinsics, depth, cls, device="cuda") -> "Scan":
        return Scan(intr, _dev_tensor(depth, torch.float32, device), _dev_tensor(cls, torch.uint8, device))

    def c(self) -> N.rm_scan:
        """The C view of this scan (rebuilt when the arrays or the intrinsics change)."""
        key = (self.depth.data_ptr(), self.cls.data_ptr(), id(self.intr), self.intr.width, self.intr.height)
        cached = self.__dict__.get("_c")
        if cached is None or cached[0] != key:
            cached = (key, N.rm_scan(self.intr.c(), self.depth.data_ptr(), self.cls.data_ptr()))
            self.__dict__["_c"] = cached
        return cached[1]


def cost_params(eps=0.1, w_fofo=1.0, w_fofu=1.0, w_fufo=1.0) -> N.rm_cost_params:
    return N.rm_cost_params(eps, w_fofo, w_fofu, w_fufo)


_DEFAULT_PARAMS = cost_params()


class Map:
    """A labelled triangle-mesh map (Sec. IV.A) resident on the GPU."""

    def __init__(self, vertices, faces, labels):
        v = np.ascontiguousarray(vertices.cpu().numpy() if isinstance(vertices, torch.Tensor) else vertices,
                                 dtype=np.float32).reshape(-1, 3)
        f = np.ascontiguousarray(faces.cpu().numpy() if isinstance(faces, torch.Tensor) else faces,
                                 dtype=np.int32).reshape(-1, 3)
        lab = np.ascontiguousarray(labels.cpu().numpy() if isinstance(labels, torch.Tensor) else labels,
                                   dtype=np.uint8).reshape(-1)
        if lab.shape[0] != f.shape[0]:
            raise ValueError("one label per face")
        h = ctypes.c_void_p()
        check(lib().rm_map_create(v.ctypes.data_as(ctypes.c_void_p), v.shape[0],
                                  f.ctypes.data_as(ctypes.c_void_p), lab.ctypes.data_as(ctypes.c_void_p),
                                  f.shape[0], ctypes.byref(h)))
        self._h = h
        self.n_vertices, self.n_faces = v.shape[0], f.shape[0]

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("map is closed")
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None:
            lib().rm_map_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def centre(self) -> np.ndarray:
        c = np.zeros(3)
        check(lib().rm_map_info(self.handle, None, None, c.ctypes.data_as(ctypes.c_void_p)))
        return c

    def set_tuning(self, tile=(0, 0), bin_capacity=0, wave_poses=0, async_status=False, wait_log2=0):
        t = N.rm_tuning(tile[0], tile[1], bin_capacity, wave_poses, int(async_status), int(wait_log2))
        check(lib().rm_map_set_tuning(self.handle, ctypes.byref(t)))

    def set_vertex_normals(self, normals, pose=None):
        """Per-vertex normals for the point-to-plane ICP (Sec. V step 3), (V, 3) in the frame of
        `pose` (camera-to-world, 4x4), or world-frame when pose is None; None detaches them."""
        if normals is None:
            check(lib().rm_map_set_vertex_normals(self.handle, None, None, _stream()))
            return
        n = _dev_tensor(normals, torch.float32).reshape(-1, 3).contiguous()
        if n.shape[0] != self.n_vertices:
            raise ValueError("one normal per map vertex")
        P = None if pose is None else np.ascontiguousarray(np.asarray(pose, np.float64).reshape(16))
        check(lib().rm_map_set_vertex_normals(self.handle, _ptr(n),
                                              None if P is None else P.ctypes.data_as(ctypes.c_void_p),
                                              _stream()))

    def profile(self, enable: bool):
        """Start (clearing the record) or stop per-kernel event timing on this map."""
        check(lib().rm_profile(self.handle, int(enable)))

    def profile_read(self) -> dict:
        """{kernel: (launches, total_ms)} recorded so far, plus the kernel launch count."""
        arr = (N.rm_kernel_time * 8)()
        n = ctypes.c_int32()
        launches = ctypes.c_int64()
        check(lib().rm_profile_read(self.handle, arr, 8, ctypes.byref(n), ctypes.byref(launches)))
        out = {arr[k].name.decode(): (arr[k].launches, arr[k].total_ms) for k in range(n.value)}
        return {"kernels": out, "launches": launches.value}

    def get_tuning(self) -> dict:
        t = N.rm_tuning()
        check(lib().rm_map_get_tuning(self.handle, ctypes.byref(t)))
        return {"tile": (t.tile_w, t.tile_h), "bin_capacity": t.bin_capacity,
                "wave_poses": t.wave_poses, "async_status": bool(t.async_status),
                "wait_log2": t.wait_log2}


def _poses(poses, device="cuda"):
    if (isinstance(poses, torch.Tensor) and poses.is_cuda and poses.dtype == torch.float64
            and poses.is_contiguous()):
        p = poses.view(-1, 16)
    else:
        p = _dev_tensor(poses, torch.float64, device).reshape(-1, 16)
    return p, p.shape[0]


def render_depth(m: Map, poses, intr: Intrinsics, want_id=True, want_bary=False):
    """R(Y) of Eq. 1 for each pose: depth (N,H,W) float32 NaN-for-miss, tri_id (N,H,W) int32,
    bary (N,H,W,2) float32."""
    p, n = _poses(poses)
    depth = torch.empty((n, intr.height, intr.width), dtype=torch.float32, device="cuda")
    ids = torch.empty_like(depth, dtype=torch.int32) if want_id else None
    bary = torch.empty((n, intr.height, intr.width, 2), dtype=torch.float32, device="cuda") if want_bary else None
    ci = intr.c()
    check(lib().rm_render_depth(m.handle, _ptr(p), n, ctypes.byref(ci), _ptr(depth), _ptr(ids),
                                _ptr(bary), _stream()))
    return {"depth": depth, "tri_id": ids, "bary": bary}


def _cost(fn, m, scan, poses, params, grad):
    p, n = _poses(poses)
    counts = torch.empty((n, 6), dtype=torch.int64, device="cuda")
    etab = torch.empty(n, dtype=torch.int64, device="cuda")
    els = torch.empty(n, dtype=torch.float64, device="cuda")
    g = torch.empty((n, 6), dtype=torch.float64, device="cuda") if grad else None
    h = torch.empty((n, 21), dtype=torch.float64, device="cuda") if grad else None
    out = N.rm_cost_out(counts.data_ptr(), etab.data_ptr(), els.data_ptr(),
                        None if g is None else g.data_ptr(), None if h is None else h.data_ptr())
    cs = scan.c()
    prm = params if params is not None else _DEFAULT_PARAMS
    check(fn(m.handle, ctypes.byref(cs), _ptr(p), n, ctypes.byref(prm), ctypes.byref(out), _stream()))
    res = {"counts": counts, "e_table": etab, "e_ls": els}
    if grad:
        res["grad"] = g
        res["jtj"] = h
    return res


def cost(m: Map, scan: Scan, poses, params=None):
    """Table I cost (counts per outcome and E_table) and the least-squares surrogate e_ls."""
    return _cost(lib().rm_cost, m, scan, poses, params, False)


def cost_grad(m: Map, scan: Scan, poses, params=None):
    """cost() plus d e_ls / d xi and the packed Gauss-Newton matrix."""
    return _cost(lib().rm_cost_grad, m, scan, poses, params, True)


def cost_grad_vertices(m: Map, scan: Scan, poses, params=None):
    """d e_ls / d (world vertex positions), summed over the poses: (V, 3) float64 on the device."""
    p, n = _poses(poses)
    g = torch.empty((m.n_vertices, 3), dtype=torch.float64, device="cuda")
    cs = scan.c()
    prm = params if params is not None else _DEFAULT_PARAMS
    check(lib().rm_cost_grad_vertices(m.handle, ctypes.byref(cs), _ptr(p), n, ctypes.byref(prm), _ptr(g),
                                      _stream()))
    return g


def cost_sweep(m: Map, scan: Scan, pose, axis, span, n, params=None):
    """Fig. 7's cost landscape along one camera-frame twist axis (0-2 metres, 3-5 radians):
    the Table I cost and the surrogate at n evenly spaced displacements in [-span, span]."""
    p, k = _poses(pose)
    if k != 1:
        raise ValueError("one pose")
    counts = torch.empty((n, 6), dtype=torch.int64, device="cuda")
    etab = torch.empty(n, dtype=torch.int64, device="cuda")
    els = torch.empty(n, dtype=torch.float64, device="cuda")
    out = N.rm_cost_out(counts.data_ptr(), etab.data_ptr(), els.data_ptr(), None, None)
    cs = scan.c()
    prm = params if params is not None else _DEFAULT_PARAMS
    check(lib().rm_cost_sweep(m.handle, ctypes.byref(cs), _ptr(p), int(axis), float(span), int(n), ctypes.byref(prm),
                              ctypes.byref(out), _stream()))
    return {"counts": counts, "e_table": etab, "e_ls": els}


def pose_retract(poses, twists, with_jacobian=False):
    """poses * exp(twists^) (and the SE(3) right Jacobians), computed on the device."""
    p, n = _poses(poses)
    t = _dev_tensor(twists, torch.float64).reshape(-1, 6)
    if t.shape[0] != n:
        raise ValueError("one twist per pose")
    out = torch.empty((n, 16), dtype=torch.float64, device="cuda")
    jr = torch.empty((n, 36), dtype=torch.float64, device="cuda") if with_jacobian else None
    check(lib().rm_pose_retract(_ptr(p), _ptr(t), n, _ptr(out), _ptr(jr), _stream()))
    out = out.reshape(n, 4, 4)
    return (out, jr.reshape(n, 6, 6)) if with_jacobian else out


def align(m: Map, scan: Scan, init_pose, params=None, max_iters=50, lambda0=1e-3, lambda_up=10.0,
          lambda_down=10.0, step_tol=1e-8):
    """Levenberg-Marquardt alignment on the device; returns (pose 4x4 float64 numpy, report)."""
    p, _ = _poses(init_pose)
    out = np.empty(16)
    rep = N.rm_align_report()
    lm = N.rm_align_params(max_iters, 0, lambda0, lambda_up, lambda_down, step_tol)
    cs = scan.c()
    prm = params if params is not None else cost_params()
    st = lib().rm_align(m.handle, ctypes.byref(cs), _ptr(p), ctypes.byref(prm), ctypes.byref(lm),
                        out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(rep), _stream())
    if st not in (N.RM_OK, N.RM_ENOTCONV):
        check(st)
    report = {f: getattr(rep, f) for f, _ in N.rm_align_report._fields_ if f != "reserved"}
    report["status"] = N.STATUS_NAMES[st]
    return out.reshape(4, 4), report


def blur_scan(scan: Scan, sigma=1.0) -> Scan:
    """The scan with its FO returns' depths Gaussian-smoothed (sigma pixels, over FO returns
    only) and every other pixel unchanged: cost smoothing (Sec. IV.C)."""
    intr = scan.intr
    out = torch.empty_like(scan.depth)
    ci = intr.c()
    check(lib().rm_depth_blur(ctypes.byref(ci), 1, _ptr(scan.depth), _ptr(scan.cls), float(sigma), _ptr(out),
                              _stream()))
    return Scan(intr, out, scan.cls)


def sequential_icp(scans, first_pose, max_range, step=2, max_edge=0.1, tol=0.2, max_iters=20,
                   step_tol=1e-5, normals="face", sigma=1.0):
    """Sequential depth-image alignment (Sec. V): each scan, downsampled by `step` and meshed
    at its pose, becomes the map the next scan is aligned to by point-to-plane ICP, starting
    from the previous pose. normals="eq2" takes the point-to-plane normals from the previous
    scan's Eq. 2 normals (metric, Gaussian sigma in pixels, pinhole scans) at the mesh's grid
    pixels, blended over each rendered triangle (the points rendered coloured by their normals,
    steps 2-3); normals="face" uses each mesh triangle's plane. Returns the (n, 4, 4) poses (the
    first is `first_pose`) and the per-step ICP reports. The meshes are built on the device;
    each becomes a Map through the host (rm_map_create)."""
    if normals not in ("face", "eq2"):
        raise ValueError("normals must be 'face' or 'eq2'")
    poses = [np.asarray(first_pose, dtype=np.float64).reshape(4, 4)]
    reports = []
    for k in range(1, len(scans)):
        prev = scans[k - 1]
        mesh = meshify(prev, poses[-1], max_range, max_edge=max_edge, step=step)
        m = Map(mesh["vertices"], mesh["faces"], mesh["labels"])
        try:
            if normals == "eq2":
                nrm = depth_normals(prev.intr, prev.depth, prev.cls, sigma=sigma, metric=True)
                st = max(int(step), 1)
                m.set_vertex_normals(nrm[::st, ::st].reshape(-1, 3), pose=poses[-1])
            pose, rep = icp_align(m, scans[k], poses[-1], tol=tol, max_iters=max_iters, step_tol=step_tol)
        finally:
            m.close()
        poses.append(pose)
        reports.append(rep)
    return np.stack(poses), reports


def dfo_params(nm_iters=60, cd_iters=60, nm_step=1.0, nm_tol=0.05, cd_step=0.25, cd_tol=0.01,
               scale_t=0.05, scale_r=0.0349, method="nm", powell_iters=30, powell_step=1.0,
               powell_tol=0.05) -> N.rm_dfo_params:
    """Derivative-free search settings; scales: 5 cm and 2 deg per unit. method "nm"
    (Nelder-Mead) or "powell" (Powell's method), then coordinate descent."""
    m = {"nm": 0, "powell": 1}[method]
    return N.rm_dfo_params(nm_iters, cd_iters, nm_step, nm_tol, cd_step, cd_tol, scale_t, scale_r, m,
                           powell_iters, powell_step, powell_tol)


def dfo_align(m: Map, scan: Scan, init_pose, params=None, dfo=None, gd_iters=0):
    """The paper's hybrid derivative-free alignment on the Table I cost (Sec. IV.C): optional
    initial gradient steps (Levenberg-Marquardt on the surrogate), then Nelder-Mead (or Powell's
    method, dfo_params(method="powell")) and coordinate descent, all on the device. Returns
    (pose 4x4 float64 numpy, report)."""
    start = init_pose
    gd = None
    if gd_iters > 0:
        start, gd = align(m, scan, init_pose, params=params, max_iters=gd_iters)
    p, _ = _poses(start)
    out = np.empty(16)
    rep = N.rm_dfo_report()
    prm = params if params is not None else _DEFAULT_PARAMS
    d = dfo if dfo is not None else dfo_params()
    cs = scan.c()
    st = lib().rm_dfo_align(m.handle, ctypes.byref(cs), _ptr(p), ctypes.byref(prm), ctypes.byref(d),
                            out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(rep), _stream())
    if st not in (N.RM_OK, N.RM_ENOTCONV):
        check(st)
    report = {f: getattr(rep, f) for f, _ in N.rm_dfo_report._fields_}
    report["status"] = N.STATUS_NAMES[st]
    if gd is not None:
        report["gd"] = gd
    return out.reshape(4, 4), report


def scan_from_range(intr: Intrinsics, rng, range_min, range_max) -> Scan:
    """A Scan from raw range images by the paper's rules: no reading -> FU at range_max,
    NaN or closer than range_min -> dead (Sec. IV.A, IV.B)."""
    r = _dev_tensor(rng, torch.float32)
    d = torch.empty_like(r)
    c = torch.empty(r.shape, dtype=torch.uint8, device="cuda")
    check(lib().rm_scan_from_range(_ptr(r), r.numel(), float(range_min), float(range_max), _ptr(d), _ptr(c),
                                   _stream()))
    return Scan(intr, d, c)


def pose_from_x(X):
    """(N, 4, 4) camera-to-world poses of X = (x, y, z, theta_x, theta_y, theta_z), R = Rz Ry Rx."""
    x = _dev_tensor(X, torch.float64).reshape(-1, 6)
    out = torch.empty((x.shape[0], 16), dtype=torch.float64, device="cuda")
    check(lib().rm_pose_from_x(_ptr(x), x.shape[0], _ptr(out), _stream()))
    return out.reshape(-1, 4, 4)


def icp_terms(m: Map, scan: Scan, poses, tol=0.1):
    """Point-to-plane ICP terms with projective association (Sec. V) for each pose:
    n_assoc (N,) int64, cost_l1 = C (N,), e2 (N,), jte (N,6) and jtj (N,21) float64."""
    p, n = _poses(poses)
    na = torch.empty(n, dtype=torch.int64, device="cuda")
    l1 = torch.empty(n, dtype=torch.float64, device="cuda")
    e2 = torch.empty(n, dtype=torch.float64, device="cuda")
    g = torch.empty((n, 6), dtype=torch.float64, device="cuda")
    h = torch.empty((n, 21), dtype=torch.float64, device="cuda")
    out = N.rm_icp_out(na.data_ptr(), l1.data_ptr(), e2.data_ptr(), g.data_ptr(), h.data_ptr())
    cs = scan.c()
    check(lib().rm_icp_terms(m.handle, ctypes.byref(cs), _ptr(p), n, float(tol), ctypes.byref(out),
                             _stream()))
    return {"n_assoc": na, "cost_l1": l1, "e2": e2, "jte": g, "jtj": h}


def icp_align(m: Map, scan: Scan, init_pose, tol=0.1, max_iters=30, step_tol=1e-5):
    """Point-to-plane ICP on the device; returns (pose 4x4 float64 numpy, report)."""
    p, _ = _poses(init_pose)
    out = np.empty(16)
    rep = N.rm_icp_report()
    prm = N.rm_icp_params(float(tol), int(max_iters), float(step_tol))
    cs = scan.c()
    st = lib().rm_icp_align(m.handle, ctypes.byref(cs), _ptr(p), ctypes.byref(prm),
                            out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(rep), _stream())
    if st not in (N.RM_OK, N.RM_ENOTCONV):
        check(st)
    report = {f: getattr(rep, f) for f, _ in N.rm_icp_report._fields_}
    report["status"] = N.STATUS_NAMES[st]
    return out.reshape(4, 4), report


def depth_normals(intr: Intrinsics, depth, cls, sigma=1.0, metric=False, want_smoothed=False):
    """Surface normals of depth images (Eq. 2): depth (N,H,W) or (H,W) float32 and class uint8
    -> normals (..., H, W, 3) float32, NaN where undefined (and the smoothed depth)."""
    d = _dev_tensor(depth, torch.float32)
    c = _dev_tensor(cls, torch.uint8)
    single = d.dim() == 2
    d = d.reshape(-1, intr.height, intr.width)
    c = c.reshape(-1, intr.height, intr.width)
    if c.shape != d.shape:
        raise ValueError("one class per depth pixel")
    n = d.shape[0]
    nrm = torch.empty((n, intr.height, intr.width, 3), dtype=torch.float32, device="cuda")
    sm = torch.empty((n, intr.height, intr.width), dtype=torch.float32, device="cuda") if want_smoothed else None
    ci = intr.c()
    check(lib().rm_depth_normals(ctypes.byref(ci), n, _ptr(d), _ptr(c), float(sigma), int(bool(metric)),
                                 _ptr(nrm), _ptr(sm), _stream()))
    if single:
        nrm = nrm[0]
        sm = sm[0] if sm is not None else None
    return (nrm, sm) if want_smoothed else nrm


def meshify(scan: Scan, pose, max_range, max_edge=0.1, step=1):
    """Labelled interface mesh of a range image seen from `pose` (Sec. IV.A): vertices
    (Hs*Ws, 3) float32, faces (F, 3) int32 and labels (F,) uint8, on the device."""
    p, n = _poses(pose)
    if n != 1:
        raise ValueError("one pose")
    intr = scan.intr
    st = max(int(step), 1)  # the library rejects step < 1
    Ws, Hs = (intr.width - 1) // st + 1, (intr.height - 1) // st + 1
    cap = 2 * (Ws - 1) * (Hs - 1)
    v = torch.empty((Ws * Hs, 3), dtype=torch.float32, device="cuda")
    f = torch.empty((max(cap, 1), 3), dtype=torch.int32, device="cuda")
    lab = torch.empty(max(cap, 1), dtype=torch.uint8, device="cuda")
    nf = ctypes.c_int64()
    prm = N.rm_meshify_params(float(max_range), float(max_edge), int(step), 0)
    cs = scan.c()
    check(lib().rm_meshify(ctypes.byref(cs), _ptr(p), ctypes.byref(prm), _ptr(v), _ptr(f), _ptr(lab),
                           ctypes.byref(nf), _stream()))
    return {"vertices": v, "faces": f[:nf.value], "labels": lab[:nf.value]}


class RenderMapCost(torch.autograd.Function):
    """e_ls(pose * exp(xi^)) as a differentiable function of the twist xi (6,) float64.

    forward: retraction and the fused render + Table I + least-squares + adjoint kernels;
    backward: grad_output * J_r(xi)^T g (rm_twist_grad), g the adjoint gradient at the
    retracted pose. Usage: RenderMapCost.apply(xi, pose, map, scan, params) -> scalar tensor.
    """

    @staticmethod
    def forward(ctx, xi, pose, m, scan, params=None):
        pose_t = _dev_tensor(pose, torch.float64).reshape(1, 16)
        xi_d = xi.detach().to(device="cuda", dtype=torch.float64).reshape(1, 6).contiguous()
        p = pose_retract(pose_t, xi_d)
        res = cost_grad(m, scan, p.reshape(1, 16), params)
        ctx.save_for_backward(res["grad"], xi_d)
        ctx.xi_device = xi.device
        return res["e_ls"][0].to(xi.device)

    @staticmethod
    def backward(ctx, grad_out):
        g, xi_d = ctx.saved_tensors
        return twist_grad(xi_d, g, grad_out)[0].to(ctx.xi_device), None, None, None, None


def twist_grad(twists, grads, scale=None):
    """scale_k * J_r(twists_k)^T grads_k on the device (rm_twist_grad): (n, 6) float64."""
    t = _dev_tensor(twists, torch.float64).reshape(-1, 6).contiguous()
    g = _dev_tensor(grads, torch.float64).reshape(-1, 6).contiguous()
    n = t.shape[0]
    if g.shape[0] != n:
        raise ValueError("one gradient per twist")
    sc = None
    if scale is not None:
        sc = _dev_tensor(scale, torch.float64).reshape(-1)
        sc = (sc.expand(n) if sc.numel() == 1 else sc).contiguous()
    out = torch.empty((n, 6), dtype=torch.float64, device="cuda")
    check(lib().rm_twist_grad(_ptr(t), _ptr(g), _ptr(sc), n, _ptr(out), _stream()))
    return out


def _problems(problems=None, scans=None, poses=None):
    """ctypes array of rm_problem from [(Scan, pose), ...], or from `scans` (one Scan, or one
    per problem) and `poses` (n x 4 x 4 or n x 16). The poses are laid out back to back in one
    device array (one copy in the library); the array is built from per-scan byte templates
    rather than field by field. Returns the array and the tensors it points into."""
    if problems is not None:
        scans = [sc for sc, _ in problems]
        poses = [ps for _, ps in problems]
    if isinstance(poses, torch.Tensor):
        P = poses.to(device="cuda", dtype=torch.float64).reshape(-1, 16).contiguous()
    elif all(isinstance(ps, torch.Tensor) for ps in poses):
        P = torch.stack([ps.reshape(16) for ps in poses]).to(device="cuda", dtype=torch.float64).contiguous()
    else:
        P = torch.as_tensor(np.stack([np.asarray(ps, dtype=np.float64).reshape(16) for ps in poses]),
                            device="cuda")
    n = P.shape[0]
    if isinstance(scans, Scan):
        scans = [scans] * n
    if len(scans) != n:
        raise ValueError("one scan per pose")
    rows, index = [], {}
    idx = np.empty(n, dtype=np.int64)
    for k, sc in enumerate(scans):
        j = index.get(id(sc))
        if j is None:
            j = index[id(sc)] = len(rows)
            t = N.rm_problem()
            t.scan = sc.c()
            rows.append(np.frombuffer(bytes(t), dtype=np.uint8))
        idx[k] = j
    size, off = ctypes.sizeof(N.rm_problem), N.rm_problem.pose.offset
    buf = np.stack(rows)[idx]
    ptrs = P.data_ptr() + 128 * np.arange(n, dtype=np.uint64)
    buf[:, off:off + 8] = ptrs.astype("<u8").view(np.uint8).reshape(n, 8)
    arr = (N.rm_problem * n).from_buffer_copy(np.ascontiguousarray(buf).reshape(n * size))
    return arr, [P, scans]


def cost_grad_batch(m: Map, problems=None, params=None, *, scans=None, poses=None):
    """cost_grad for [(Scan, pose), ...] that may differ in camera and size (or for `scans` and
    `poses` as in _problems): one persistent kernel launch. Returns the same dict as
    cost_grad, indexed by problem."""
    arr, keep = _problems(problems, scans, poses)
    n = len(arr)
    counts = torch.empty((n, 6), dtype=torch.int64, device="cuda")
    etab = torch.empty(n, dtype=torch.int64, device="cuda")
    els = torch.empty(n, dtype=torch.float64, device="cuda")
    g = torch.empty((n, 6), dtype=torch.float64, device="cuda")
    h = torch.empty((n, 21), dtype=torch.float64, device="cuda")
    out = N.rm_cost_out(counts.data_ptr(), etab.data_ptr(), els.data_ptr(), g.data_ptr(), h.data_ptr())
    prm = params if params is not None else cost_params()
    check(lib().rm_cost_grad_batch(m.handle, arr, n, ctypes.byref(prm), ctypes.byref(out), _stream()))
    del keep
    return {"counts": counts, "e_table": etab, "e_ls": els, "grad": g, "jtj": h}


def align_batch(m: Map, problems=None, params=None, max_iters=5, lambda0=1e-3, lambda_up=10.0,
                lambda_down=10.0, step_tol=1e-8, *, scans=None, poses=None):
    """LM for [(Scan, start pose), ...] (or `scans` and `poses` as in _problems) with every
    iteration of every problem in one persistent kernel launch. Returns (poses (n,4,4) numpy,
    list of reports, status name)."""
    arr, keep = _problems(problems, scans, poses)
    n = len(arr)
    out = np.empty((n, 16))
    reps = (N.rm_align_report * n)()
    lm = N.rm_align_params(max_iters, 0, lambda0, lambda_up, lambda_down, step_tol)
    prm = params if params is not None else cost_params()
    st = lib().rm_align_batch(m.handle, arr, n, ctypes.byref(prm), ctypes.byref(lm),
                              out.ctypes.data_as(ctypes.c_void_p), reps, _stream())
    if st not in (N.RM_OK, N.RM_ENOTCONV):
        check(st)
    del keep
    reports = [{f: getattr(r, f) for f, _ in N.rm_align_report._fields_ if f != "reserved"} for r in reps]
    return out.reshape(n, 4, 4), reports, N.STATUS_NAMES[st]


def icp_align_batch(m: Map, problems=None, tol=0.1, max_iters=10, step_tol=1e-5, *, scans=None, poses=None):
    """Point-to-plane ICP for [(Scan, start pose), ...] with every evaluation and step of every
    problem in one persistent kernel launch. Returns (poses (n,4,4) numpy, reports, status)."""
    arr, keep = _problems(problems, scans, poses)
    n = len(arr)
    out = np.empty((n, 16))
    reps = (N.rm_icp_report * n)()
    prm = N.rm_icp_params(float(tol), int(max_iters), float(step_tol))
    st = lib().rm_icp_align_batch(m.handle, arr, n, ctypes.byref(prm), out.ctypes.data_as(ctypes.c_void_p),
                                  reps, _stream())
    if st not in (N.RM_OK, N.RM_ENOTCONV):
        check(st)
    del keep
    reports = [{f: getattr(r, f) for f, _ in N.rm_icp_report._fields_} for r in reps]
    return out.reshape(n, 4, 4), reports, N.STATUS_NAMES[st]
