"""CPU oracle for the RenderMap pose-cost path (Ryde & Ding, arXiv 1702.06813).

TEST INFRASTRUCTURE ONLY. The tests, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg are the only code allowed to import this package; the product path never does.

The oracle is a plain C library (``rm_oracle.c``), compiled with ``-ffp-contract=off`` and
loaded through ctypes. It shares no code with the CUDA library. See ``rm_oracle.c`` for the
passages of the paper each function follows.

Parity status of each function (what pins it, see ``tests/test_oracle_pins.py``):
  * z-buffer visibility: brute force over every pixel and triangle, watertightness of
    tessellated planes and closed boxes, closed-form fronto-parallel and oblique planes;
  * FP32 depth: within a conditioning-scaled bound of the FP64 ray-plane depth
    (closed form d / (n . r));
  * Table I: the printed truth table with its boundary cases (``tests/golden/table1.txt``);
  * cost: zero least-squares cost and all-reward Table I at the true pose of a noise-free
    scan rendered by the oracle itself;
  * gradient: central finite differences of the FP64 frozen-visibility cost;
  * LM: convergence from a perturbed start to the true pose on noise-free scans;
  * point-to-plane ICP terms: closed forms for a fronto-parallel wall (association count,
    C, residuals, J^T e, J^T J), the association rules (tolerance, labels, scan classes),
    finite differences of the frozen point-to-plane cost (J^T e; J^T J where the residuals
    vanish); ICP alignment: convergence to the true pose on noise-free scans; with vertex
    normals: equal to the face-normal terms when every vertex carries its plane's normal,
    the blended normal at a single associated pixel against perspective-correct screen-space
    barycentrics, NaN normals removing exactly their triangles' pixels, finite differences;
  * barycentrics: the reconstructed hit lies on the pixel's ray, unit coordinates at the
    vertices, perspective-correct screen-space barycentrics (``tests/test_oracle_bary.py``);
  * depth-image normals (Eq. 2): closed forms for linear and quadratic depth images, a constant
    image with holes (values, and the invalid set as a dilation of the holes), the metric
    normal of a tilted plane at the principal point;
  * meshification: closed-form vertices and labels of a fronto-parallel wall, depth steps,
    no-return and dead pixels, face counts; rendering the mesh of a scan from the scan's own
    pose reproduces the scan's depths;
  * derivative-free search (Nelder-Mead or Powell's method, then coordinate descent): known
    minima of a convex (rotated) quadratic and an integer staircase, the exact candidates of
    the first steps, accounting, invariance under an added constant or a positive factor, a
    noise-free Table I search (``tests/test_oracle_dfo.py``);
  * vertex gradient: finite differences of the frozen cost with one vertex moved, the sum
    identity with the pose gradient, a wall's closed form (``tests/test_oracle_vgrad.py``);
  * input helpers: a golden table of raw readings, single-axis and Euler rotations
    (``tests/test_oracle_helpers.py``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sysconfig

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "librm_oracle.so")
_SRC = os.path.join(_HERE, "rm_oracle.c")

KEY_EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/librm_oracle.so (gcc, plain C99)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "rm_oracle.h"))):
        return _SO
    tmp = _SO + f".{os.getpid()}.tmp"
    base = ["gcc", "-std=gnu99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
            _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)
    os.replace(tmp, _SO)
    return _SO


class _Cam(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("pad_", ctypes.c_int32), ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float), ("az0", ctypes.c_float),
                ("az_step", ctypes.c_float), ("el0", ctypes.c_float), ("el_step", ctypes.c_float),
                ("near_m", ctypes.c_float), ("far_m", ctypes.c_float),
                ("rays", ctypes.POINTER(ctypes.c_float))]


class _Params(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_float), ("w_fofo", ctypes.c_float), ("w_fofu", ctypes.c_float),
                ("w_fufo", ctypes.c_float)]


class _Stats(ctypes.Structure):
    _fields_ = [("n_clipped", ctypes.c_int64), ("n_guard_culled", ctypes.c_int64),
                ("n_fragments", ctypes.c_int64)]


class _LM(ctypes.Structure):
    _fields_ = [("max_iters", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("lambda0", ctypes.c_double), ("lambda_up", ctypes.c_double),
                ("lambda_down", ctypes.c_double), ("step_tol", ctypes.c_double)]


class _LMReport(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("accepted", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("e_ls_initial", ctypes.c_double), ("e_ls_final", ctypes.c_double),
                ("e_table_initial", ctypes.c_int64), ("e_table_final", ctypes.c_int64)]


class _DfoParams(ctypes.Structure):
    _fields_ = [("nm_iters", ctypes.c_int32), ("cd_iters", ctypes.c_int32), ("nm_step", ctypes.c_double),
                ("nm_tol", ctypes.c_double), ("cd_step", ctypes.c_double), ("cd_tol", ctypes.c_double),
                ("scale_t", ctypes.c_double), ("scale_r", ctypes.c_double), ("method", ctypes.c_int32),
                ("powell_iters", ctypes.c_int32), ("powell_step", ctypes.c_double),
                ("powell_tol", ctypes.c_double)]


class _DfoReport(ctypes.Structure):
    _fields_ = [("evals", ctypes.c_int32), ("nm_iters", ctypes.c_int32), ("nm_shrinks", ctypes.c_int32),
                ("cd_iters", ctypes.c_int32), ("converged", ctypes.c_int32), ("powell_iters", ctypes.c_int32)]


_BATCH_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(ctypes.c_double))


def dfo_params(nm_iters=60, cd_iters=60, nm_step=1.0, nm_tol=0.05, cd_step=0.25, cd_tol=0.01,
               scale_t=0.05, scale_r=0.0349, method="nm", powell_iters=30, powell_step=1.0,
               powell_tol=0.05):
    """method: "nm" (Nelder-Mead) or "powell" (Powell's method), then coordinate descent."""
    m = {"nm": 0, "powell": 1}[method]
    return _DfoParams(nm_iters, cd_iters, nm_step, nm_tol, cd_step, cd_tol, scale_t, scale_r, m,
                      powell_iters, powell_step, powell_tol)


def dfo_minimise(f, scale, params=None):
    """The derivative-free search on a Python function of a (n, 6) batch of twists."""
    prm = params or dfo_params()

    def cb(_ctx, n, xi, out):
        x = np.ctypeslib.as_array(xi, shape=(n, 6)).copy()
        vals = np.asarray(f(x), dtype=np.float64)
        for i in range(n):
            out[i] = vals[i]
        return 0

    fn = _BATCH_FN(cb)
    x = np.zeros(6)
    fb = ctypes.c_double()
    rep = _DfoReport()
    st = lib().orc_dfo_core(fn, None, _p(_f64(scale)), ctypes.byref(prm), _p(x), ctypes.byref(fb),
                            ctypes.byref(rep))
    if st != 0:
        raise RuntimeError("orc_dfo_core failed")
    return x, fb.value, {f_: getattr(rep, f_) for f_, _ in _DfoReport._fields_}


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.orc_cost_frozen.restype = ctypes.c_double
        _lib.orc_icp_frozen.restype = ctypes.c_double
        _lib.orc_cost_frozen_vertex.restype = ctypes.c_double
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _pn(a):
    """Pointer of an optional array (NULL for None)."""
    return None if a is None else _p(a)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def make_cam(cam) -> tuple[_Cam, object]:
    """orc_cam from a synth.Camera; returns (struct, keep-alive ray table)."""
    c = _Cam()
    c.model = 0 if cam.model == "pinhole" else 1
    c.width, c.height = cam.width, cam.height
    c.fx, c.fy, c.cx, c.cy = cam.fx, cam.fy, cam.cx, cam.cy
    c.az0, c.az_step, c.el0, c.el_step = cam.az0, cam.az_step, cam.el0, cam.el_step
    c.near_m, c.far_m = cam.near, cam.far
    rays = None
    if c.model == 1:
        rays = cam.ray_table_f32()
        c.rays = rays.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    return c, rays


def make_params(eps=0.1, w_fofo=1.0, w_fofu=1.0, w_fufo=1.0) -> _Params:
    return _Params(eps, w_fofo, w_fofu, w_fufo)


def table1(map_class: int, scan_class: int, dz: float, eps: float = 0.1) -> int:
    return lib().orc_table1(int(map_class), int(scan_class), ctypes.c_float(dz), ctypes.c_float(eps))


def se3_right(T, xi):
    out = np.empty(16)
    lib().orc_se3_right(_p(_f64(T).reshape(16)), _p(_f64(xi)), _p(out))
    return out.reshape(4, 4)


def pose_matrix(T, centre):
    M = np.empty(12, np.float32)
    lib().orc_pose_matrix(_p(_f64(T).reshape(16)), _p(_f64(centre)), _p(M))
    return M.reshape(3, 4)


def transform(M, v):
    v = _f32(v)
    out = np.empty_like(v)
    lib().orc_transform(_p(_f32(M).reshape(12)), _p(v), ctypes.c_int64(v.shape[0]), _p(out))
    return out


def zbuffer(vc, faces, cam, brute=False, frags=False):
    """Z-buffer of camera-space vertices (no pose); returns (keys, frags or None, stats)."""
    c, keep = make_cam(cam)
    vc = _f32(vc)
    faces = np.ascontiguousarray(faces, np.int32)
    keys = np.empty((cam.height, cam.width), np.uint64)
    fr = np.empty((cam.height, cam.width), np.int32) if frags else None
    st = _Stats()
    lib().orc_zbuffer(_p(vc), _p(faces), ctypes.c_int64(faces.shape[0]), ctypes.byref(c), _p(keys),
                      _p(fr) if fr is not None else None, int(brute), ctypes.byref(st))
    del keep
    return keys, fr, st


def decode(keys):
    """(depth float32 with NaN, tri id int32 with -1) from a key image: the key's high word is
    the bitwise complement of the FP32 inverse depth w, and depth = 1 / w rounded to FP32."""
    empty = keys == KEY_EMPTY
    w = (~(keys >> np.uint64(32)).astype(np.uint32)).view(np.float32)
    with np.errstate(divide="ignore"):
        depth = np.float32(1.0) / w
    depth[empty] = np.nan
    ids = (keys & np.uint64(0xFFFFFFFF)).astype(np.int64).astype(np.int32)
    ids[empty] = -1
    return depth, ids


def depth_normals(depth, cls, sigma=1.0, metric=False, fx=1.0, fy=1.0):
    """Eq. 2 surface normals of a depth image: (normals (H, W, 3), smoothed depth (H, W))."""
    d = _f32(depth)
    c = np.ascontiguousarray(cls, np.uint8)
    H, W = d.shape
    n = np.empty((H, W, 3))
    s = np.empty((H, W))
    st = lib().orc_depth_normals(_p(d), _p(c), W, H, ctypes.c_double(sigma), int(metric),
                                 ctypes.c_double(fx), ctypes.c_double(fy), _p(n), _p(s))
    if st != 0:
        raise ValueError("bad sigma")
    return n, s


def meshify(cam, depth, cls, pose, max_range, max_edge=0.1, step=1):
    """Labelled mesh of a range image (Sec. IV.A): (vertices (Hs*Ws, 3) float32, faces (F, 3)
    int32, labels (F,) uint8)."""
    c, keep = make_cam(cam)
    d = _f32(depth)
    cl = np.ascontiguousarray(cls, np.uint8)
    Ws = (cam.width - 1) // step + 1 if cam.width > 0 else 0
    Hs = (cam.height - 1) // step + 1 if cam.height > 0 else 0
    v = np.empty((Hs * Ws, 3), np.float32)
    cap = max(2 * max(Hs - 1, 0) * max(Ws - 1, 0), 1)
    f = np.empty((cap, 3), np.int32)
    lab = np.empty(cap, np.uint8)
    nf = ctypes.c_int64()
    st = lib().orc_meshify(ctypes.byref(c), _p(d), _p(cl), _p(_f64(pose).reshape(16)),
                           ctypes.c_float(max_range), ctypes.c_float(max_edge), int(step), _p(v), _p(f),
                           _p(lab), ctypes.byref(nf))
    del keep
    if st != 0:
        raise ValueError("bad meshify parameters")
    return v, f[:nf.value].copy(), lab[:nf.value].copy()


def scan_from_range(rng, range_min, range_max):
    """(depth, class) of a raw range image by the no-return / dead-pixel rules."""
    r = _f32(rng)
    d = np.empty_like(r)
    c = np.empty(r.shape, np.uint8)
    lib().orc_scan_from_range(_p(r), ctypes.c_int64(r.size), ctypes.c_float(range_min),
                              ctypes.c_float(range_max), _p(d), _p(c))
    return d, c


def pose_from_x(X):
    """4x4 camera-to-world pose of X = (x, y, z, theta_x, theta_y, theta_z), R = Rz Ry Rx."""
    T = np.empty(16)
    lib().orc_pose_from_x(_p(_f64(X).reshape(6)), _p(T))
    return T.reshape(4, 4)


def depth_blur(depth, cls, sigma=1.0):
    """Cost smoothing: FO returns get their Eq. 2 smoothed depth, other pixels keep theirs."""
    _, s = depth_normals(depth, cls, sigma=sigma)
    d = np.array(depth, np.float32, copy=True)
    ok = ~np.isnan(s)
    d[ok] = s[ok]
    return d, s


class OracleMap:
    """The oracle's copy of a labelled triangle-mesh map (Sec. IV.A)."""

    def __init__(self, vertices, faces, labels):
        self.v = _f32(vertices).reshape(-1, 3)
        self.faces = np.ascontiguousarray(faces, np.int32).reshape(-1, 3)
        self.labels = np.ascontiguousarray(labels, np.uint8).reshape(-1)
        self.centre = np.empty(3)
        self.vr = np.empty_like(self.v)
        lib().orc_recentre(_p(self.v), ctypes.c_int64(self.v.shape[0]), _p(self.centre), _p(self.vr))

    @property
    def V(self):
        return ctypes.c_int64(self.v.shape[0])

    @property
    def T(self):
        return ctypes.c_int64(self.faces.shape[0])

    def render(self, pose, cam, brute=False, frags=False):
        c, keep = make_cam(cam)
        keys = np.empty((cam.height, cam.width), np.uint64)
        fr = np.empty((cam.height, cam.width), np.int32) if frags else None
        st = _Stats()
        lib().orc_render(_p(self.vr), self.V, _p(self.centre), _p(self.faces), self.T,
                         _p(_f64(pose).reshape(16)), ctypes.byref(c), _p(keys),
                         _p(fr) if fr is not None else None, int(brute), ctypes.byref(st))
        del keep
        depth, ids = decode(keys)
        return {"keys": keys, "depth": depth, "tri_id": ids, "frags": fr,
                "stats": {"clipped": st.n_clipped, "guard_culled": st.n_guard_culled,
                          "fragments": st.n_fragments}}

    def depth_exact(self, pose, cam, keys):
        c, keep = make_cam(cam)
        out = np.empty(keys.shape, np.float64)
        lib().orc_depth_exact(_p(self.v), _p(self.faces), _p(_f64(pose).reshape(16)), ctypes.byref(c),
                              _p(np.ascontiguousarray(keys)), _p(out))
        del keep
        return out

    def barycentrics(self, pose, cam, keys):
        c, keep = make_cam(cam)
        out = np.empty(keys.shape + (2,), np.float64)
        lib().orc_barycentrics(_p(self.v), _p(self.faces), _p(_f64(pose).reshape(16)),
                               ctypes.byref(c), _p(np.ascontiguousarray(keys)), _p(out))
        del keep
        return out

    def cost(self, pose, cam, scan_depth, scan_class, params=None, residual_exact=False,
             per_pixel=False):
        c, keep = make_cam(cam)
        prm = params or make_params()
        sd = _f32(scan_depth)
        sc = np.ascontiguousarray(scan_class, np.uint8)
        counts = np.zeros(6, np.int64)
        e = ctypes.c_double()
        g = np.zeros(6)
        h = np.zeros(21)
        oc = np.empty(sd.shape, np.int8) if per_pixel else None
        rs = np.empty(sd.shape, np.float64) if per_pixel else None
        lib().orc_cost(_p(self.v), _p(self.vr), self.V, _p(self.centre), _p(self.faces),
                       _p(self.labels), self.T, _p(_f64(pose).reshape(16)), ctypes.byref(c),
                       _p(sd), _p(sc), ctypes.byref(prm), int(residual_exact), _p(counts),
                       ctypes.byref(e), _p(g), _p(h), _p(oc) if oc is not None else None,
                       _p(rs) if rs is not None else None)
        del keep
        out = {"counts": counts, "e_table": int(counts[1] + counts[3] + counts[5]
                                               - counts[0] - counts[2] - counts[4]),
               "e_ls": e.value, "grad": g, "jtj": h}
        if per_pixel:
            out["outcome"] = oc
            out["resid"] = rs
        return out

    def cost_frozen(self, pose, cam, scan_depth, scan_class, xi, params=None):
        c, keep = make_cam(cam)
        prm = params or make_params()
        r = lib().orc_cost_frozen(_p(self.v), _p(self.vr), self.V, _p(self.centre), _p(self.faces),
                                  _p(self.labels), self.T, _p(_f64(pose).reshape(16)),
                                  ctypes.byref(c), _p(_f32(scan_depth)),
                                  _p(np.ascontiguousarray(scan_class, np.uint8)), ctypes.byref(prm),
                                  _p(_f64(xi)))
        del keep
        return r

    def align(self, pose0, cam, scan_depth, scan_class, params=None, max_iters=50,
              lambda0=1e-3, lambda_up=10.0, lambda_down=10.0, step_tol=1e-8):
        c, keep = make_cam(cam)
        prm = params or make_params()
        lm = _LM(max_iters, 0, lambda0, lambda_up, lambda_down, step_tol)
        rep = _LMReport()
        out = np.empty(16)
        lib().orc_align(_p(self.v), _p(self.vr), self.V, _p(self.centre), _p(self.faces),
                        _p(self.labels), self.T, _p(_f64(pose0).reshape(16)), ctypes.byref(c),
                        _p(_f32(scan_depth)), _p(np.ascontiguousarray(scan_class, np.uint8)),
                        ctypes.byref(prm), ctypes.byref(lm), _p(out), ctypes.byref(rep))
        del keep
        return out.reshape(4, 4), {f: getattr(rep, f) for f, _ in _LMReport._fields_ if f != "pad_"}

    def cost_sweep(self, pose, cam, scan_depth, scan_class, axis, span, n, params=None):
        """Fig. 7: the cost at pose exp(t_i e_axis^), t_i = -span + 2 span i / (n - 1)."""
        ts = [-span + 2.0 * span * i / (n - 1) for i in range(n)] if n > 1 else [0.0]
        out = []
        for t in ts:
            xi = np.zeros(6)
            xi[axis] = t
            out.append(self.cost(se3_right(pose, xi), cam, scan_depth, scan_class, params))
        return ts, out

    def cost_batch(self, poses, cam, scan_depth, scan_class, params=None):
        c, keep = make_cam(cam)
        prm = params or make_params()
        poses = _f64(poses).reshape(-1, 16)
        n = poses.shape[0]
        counts = np.zeros((n, 6), np.int64)
        e = np.zeros(n)
        g = np.zeros((n, 6))
        h = np.zeros((n, 21))
        threads = lib().orc_cost_batch(_p(self.v), _p(self.vr), self.V, _p(self.centre),
                                       _p(self.faces), _p(self.labels), self.T, _p(poses), n,
                                       ctypes.byref(c), _p(_f32(scan_depth)),
                                       _p(np.ascontiguousarray(scan_class, np.uint8)),
                                       ctypes.byref(prm), _p(counts), _p(e), _p(g), _p(h))
        del keep
        return {"counts": counts, "e_ls": e, "grad": g, "jtj": h, "threads": threads}

    def vertex_grad(self, pose, cam, scan_depth, scan_class, params=None):
        """d e_ls / d (world vertex positions), (V, 3)."""
        c, keep = make_cam(cam)
        prm = params or make_params()
        g = np.zeros((self.v.shape[0], 3))
        lib().orc_cost_vertex_grad(_p(self.v), _p(self.vr), self.V, _p(self.centre), _p(self.faces),
                                   _p(self.labels), self.T, _p(_f64(pose).reshape(16)), ctypes.byref(c),
                                   _p(_f32(scan_depth)), _p(np.ascontiguousarray(scan_class, np.uint8)),
                                   ctypes.byref(prm), _p(g))
        del keep
        return g

    def cost_frozen_vertex(self, pose, cam, scan_depth, scan_class, vk, delta, params=None):
        c, keep = make_cam(cam)
        prm = params or make_params()
        r = lib().orc_cost_frozen_vertex(_p(self.v), _p(self.vr), self.V, _p(self.centre), _p(self.faces),
                                         _p(self.labels), self.T, _p(_f64(pose).reshape(16)),
                                         ctypes.byref(c), _p(_f32(scan_depth)),
                                         _p(np.ascontiguousarray(scan_class, np.uint8)), ctypes.byref(prm),
                                         ctypes.c_int64(vk), _p(_f64(delta)))
        del keep
        return r

    def dfo_align(self, pose0, cam, scan_depth, scan_class, params=None, dfo=None):
        """Nelder-Mead (or Powell's method) then coordinate descent on the Table I cost
        (Sec. IV.C)."""
        c, keep = make_cam(cam)
        prm = params or make_params()
        d = dfo or dfo_params()
        out = np.empty(16)
        et = ctypes.c_int64()
        rep = _DfoReport()
        st = lib().orc_dfo_align(_p(self.v), _p(self.vr), self.V, _p(self.centre), _p(self.faces),
                                 _p(self.labels), self.T, _p(_f64(pose0).reshape(16)), ctypes.byref(c),
                                 _p(_f32(scan_depth)), _p(np.ascontiguousarray(scan_class, np.uint8)),
                                 ctypes.byref(prm), ctypes.byref(d), _p(out), ctypes.byref(et),
                                 ctypes.byref(rep))
        del keep
        if st != 0:
            raise RuntimeError("orc_dfo_align failed")
        r = {f_: getattr(rep, f_) for f_, _ in _DfoReport._fields_}
        r["e_table"] = et.value
        return out.reshape(4, 4), r

    def icp_terms(self, pose, cam, scan_depth, scan_class, tol, vnormals=None):
        """Point-to-plane ICP terms with projective association (Sec. V); vnormals (V, 3)
        world-frame vertex normals select the normal-coloured map (Sec. V step 3)."""
        c, keep = make_cam(cam)
        vn = None if vnormals is None else _f64(vnormals).reshape(-1, 3)
        na = ctypes.c_int64()
        l1 = ctypes.c_double()
        e2 = ctypes.c_double()
        g = np.zeros(6)
        h = np.zeros(21)
        lib().orc_icp_terms(_p(self.v), _p(self.vr), self.V, _p(self.centre), _p(self.faces),
                            _p(self.labels), _pn(vn), self.T, _p(_f64(pose).reshape(16)), ctypes.byref(c),
                            _p(_f32(scan_depth)), _p(np.ascontiguousarray(scan_class, np.uint8)),
                            ctypes.c_float(tol), ctypes.byref(na), ctypes.byref(l1),
                            ctypes.byref(e2), _p(g), _p(h))
        del keep
        return {"n_assoc": na.value, "cost_l1": l1.value, "e2": e2.value, "jte": g, "jtj": h}

    def icp_frozen(self, pose, cam, scan_depth, scan_class, tol, xi, vnormals=None):
        c, keep = make_cam(cam)
        vn = None if vnormals is None else _f64(vnormals).reshape(-1, 3)
        r = lib().orc_icp_frozen(_p(self.v), _p(self.vr), self.V, _p(self.centre), _p(self.faces),
                                 _p(self.labels), _pn(vn), self.T, _p(_f64(pose).reshape(16)),
                                 ctypes.byref(c), _p(_f32(scan_depth)),
                                 _p(np.ascontiguousarray(scan_class, np.uint8)),
                                 ctypes.c_float(tol), _p(_f64(xi)))
        del keep
        return r

    def icp_align(self, pose0, cam, scan_depth, scan_class, tol, max_iters=30, step_tol=1e-8,
                  vnormals=None):
        c, keep = make_cam(cam)
        vn = None if vnormals is None else _f64(vnormals).reshape(-1, 3)
        out = np.empty(16)
        it = ctypes.c_int()
        conv = ctypes.c_int()
        na = ctypes.c_int64()
        l1 = ctypes.c_double()
        lib().orc_icp_align(_p(self.v), _p(self.vr), self.V, _p(self.centre), _p(self.faces),
                            _p(self.labels), _pn(vn), self.T, _p(_f64(pose0).reshape(16)), ctypes.byref(c),
                            _p(_f32(scan_depth)), _p(np.ascontiguousarray(scan_class, np.uint8)),
                            ctypes.c_float(tol), int(max_iters), ctypes.c_double(step_tol), _p(out),
                            ctypes.byref(it), ctypes.byref(conv), ctypes.byref(na),
                            ctypes.byref(l1))
        del keep
        return out.reshape(4, 4), {"iters": it.value, "converged": conv.value,
                                   "n_assoc": na.value, "cost_l1": l1.value}
