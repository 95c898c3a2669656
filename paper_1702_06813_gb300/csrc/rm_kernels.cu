// rm_kernels.cu -- the pose-cost hot path on sm_103a.
//
// Per pose (one wave of poses at a time, blockIdx.y = pose within the wave):
//   k_pose_to_m   camera-to-world FP64 pose -> world-to-camera FP32 3x4 (Eq. 1's T(X) -> Y)
//   k_cull        per cluster of <= 64 triangles: bounding sphere against the view volume
//   k_setup       per visible cluster: camera-space vertices and their 1/256-px snapped
//                 projections, then per triangle: near-plane cut, cull, depth plane, append
//                 to the screen-tile bins
//   k_raster      one CTA per (pose, tile): bins staged into shared memory with bulk (TMA)
//                 copies, integer edge functions with the top-left rule, 64-bit
//                 depth|id z-test by shared-memory atomicMin (the z-buffer R(Y) of Sec. IV);
//                 then the fused epilogue: Table I per pixel (Sec. IV.B), the truncated
//                 least-squares residual, its pose Jacobian, and a fixed-order reduction;
//                 in ICP mode instead the projective association of each pixel's map
//                 surface with its scan return and the point-to-plane terms (Sec. V)
//   k_reduce      per pose: fixed-order sum of the per-tile partials
// k_lm_* and k_icp_* take the Levenberg-Marquardt and ICP steps between evaluations.
// k_persist runs the same phases for a batch of problems (and LM iterations) in one launch.
#include <cfloat>
#include <cmath>

#include "rm_kernels.cuh"

namespace rmk {

// ------------------------------------------------------------------ PTX helpers

__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *b, unsigned n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(n) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One-dimensional bulk copy global -> this CTA's shared memory, completion counted in bytes
// on `bar`. Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes,
                                         unsigned long long *bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try(unsigned long long *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Non-blocking test of a phase of `bar`.
__device__ __forceinline__ bool mbar_test(unsigned long long *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Default budget of a bounded device wait: about 2^31 cycles (~1 s at 2 GHz).
constexpr long long kWaitCycles = 1ll << 31;

// Bounded wait on a phase of `bar`: gives up after `budget` cycles (kWaitCycles when <= 0).
// try_wait may suspend the thread for a hardware-defined window, longer than a short budget;
// a shorter budget therefore polls with the non-blocking test instead.
__device__ __noinline__ bool mbar_wait(unsigned long long *bar, unsigned parity, long long budget) {
  if (budget <= 0) budget = kWaitCycles;
  const long long t0 = clock64();
  if (budget < kWaitCycles) {
    while (!mbar_test(bar, parity)) {
      if (clock64() - t0 > budget) return false;
    }
    return true;
  }
  while (!mbar_try(bar, parity)) {
    if (clock64() - t0 > budget) return false;
  }
  return true;
}

// ------------------------------------------------------------------ pose -> matrix

// M = inverse of (R, t - c) rounded to FP32: rotation R^T, translation -R^T (t - c), the
// translation summed in FP64 as ((r0 t0 + r1 t1) + r2 t2) without fused multiply-add.
__device__ __forceinline__ void pose_to_m(const double *T, double cx, double cy, double cz,
                                          float *M) {
  double t0 = __dsub_rn(T[3], cx), t1 = __dsub_rn(T[7], cy), t2 = __dsub_rn(T[11], cz);
  for (int i = 0; i < 3; ++i) {
    double r0 = T[i], r1 = T[4 + i], r2 = T[8 + i];
    double s = __dmul_rn(r0, t0);
    s = __dadd_rn(s, __dmul_rn(r1, t1));
    s = __dadd_rn(s, __dmul_rn(r2, t2));
    M[4 * i + 0] = __double2float_rn(r0);
    M[4 * i + 1] = __double2float_rn(r1);
    M[4 * i + 2] = __double2float_rn(r2);
    M[4 * i + 3] = __double2float_rn(-s);
  }
}

__global__ void k_pose_to_m(const double *poses, int n, double cx, double cy, double cz,
                            float *Ms) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) pose_to_m(poses + 16 * (long long)k, cx, cy, cz, Ms + 12 * (long long)k);
}

cudaError_t launch_pose_to_m(const double *poses, int n, double cx, double cy, double cz,
                             float *Ms, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_pose_to_m<<<(n + 127) / 128, 128, 0, s>>>(poses, n, cx, cy, cz, Ms);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ cluster culling

// A cluster is dropped only when its bounding sphere lies entirely outside the view volume
// that can hold a pixel sample: behind the near plane, beyond the far plane, or (pinhole)
// outside the side planes through image columns -2 and W+2 and rows -2 and H+2. The slack
// covers the FP32 error of transforming the sphere centre, so no triangle that the
// rasteriser would draw is ever dropped.
__device__ __forceinline__ bool cluster_visible(const DevCam &cam, const float *M, float4 sph) {
  const float3 c = xform(M, sph.x, sph.y, sph.z);
  const float r = sph.w;
  const float slack = 1e-4f * (1.0f + fabsf(c.x) + fabsf(c.y) + fabsf(c.z) + r);
  if (cam.model == 0) {
    if (c.z + r < cam.near_m - slack) return false;
    if (c.z - r > cam.far_m + slack) return false;
    // side planes X - a Z = 0 with a = (x_edge - cx) / fx, likewise for Y
    const float xl = -2.0f, xr = cam.W + 2.0f, yt = -2.0f, yb = cam.H + 2.0f;
    const float al = (xl - cam.cx) / cam.fx, ar = (xr - cam.cx) / cam.fx;
    const float at = (yt - cam.cy) / cam.fy, ab = (yb - cam.cy) / cam.fy;
    const float sx = cam.fx > 0.0f ? 1.0f : -1.0f, sy = cam.fy > 0.0f ? 1.0f : -1.0f;
    const float lim = r + slack;
    if (sx * (c.x - al * c.z) < -lim * sqrtf(1.0f + al * al)) return false;
    if (sx * (ar * c.z - c.x) < -lim * sqrtf(1.0f + ar * ar)) return false;
    if (sy * (c.y - at * c.z) < -lim * sqrtf(1.0f + at * at)) return false;
    if (sy * (ab * c.z - c.y) < -lim * sqrtf(1.0f + ab * ab)) return false;
    return true;
  }
  const float dist = sqrtf(c.x * c.x + c.y * c.y + c.z * c.z);
  if (dist + r < cam.near_m - slack) return false;
  if (dist - r > cam.far_m + slack) return false;
  if (dist <= r + slack) return true;  // the sensor is inside the sphere
  // elevation band of the rows (two rows of margin): the sphere subtends asin(r / dist)
  const float alpha = asinf(fminf(1.0f, (r + slack) / dist)) + 1e-4f;
  const float el_c = asinf(fmaxf(-1.0f, fminf(1.0f, -c.y / dist)));
  const float top = cam.el0 + 2.0f * cam.el_step;
  const float bot = cam.el0 - (cam.H + 1) * cam.el_step;
  if (el_c - alpha > top || el_c + alpha < bot) return false;
  return true;
}

// Reads of data that another CTA of the same (persistent) kernel may have written bypass L1.
__device__ __forceinline__ int ld_cg(const int *p) { return __ldcg(p); }
__device__ __forceinline__ bool skipped(const WaveArgs &a) { return a.skip && __ldcg(a.skip) != 0; }

// The pose matrix of pose q, read once per CTA (from L2: another CTA may have written it)
// into shared memory; every thread then copies it from there.
__device__ __forceinline__ void load_m_block(const WaveArgs &a, int q, float *sM) {
  if (threadIdx.x < 12) sM[threadIdx.x] = __ldcg(a.Ms + 12 * (long long)(a.wave_base + q) + threadIdx.x);
  __syncthreads();
}

// Clusters chunk*256 + threadIdx.x of pose q: test, and append the visible ones.
__device__ __forceinline__ void cull_block(const WaveArgs &a, int q, int chunk, float *sM) {
  load_m_block(a, q, sM);
  float M[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) M[k] = sM[k];
  int4 *vis = a.vis + (long long)q * a.n_clusters;
  const int c = chunk * blockDim.x + threadIdx.x;
  const bool keep = c < a.n_clusters && cluster_visible(a.cam, M, a.cl_sphere[c]);
  // warp-aggregated append
  const unsigned m = __ballot_sync(0xffffffffu, keep);
  if (m == 0) return;
  const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(&a.vis_count[q], __popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (keep) vis[base + __popc(m & ((1u << lane) - 1u))] = a.cl_info[c];  // setup needs no lookup
}

__global__ void __launch_bounds__(256) k_cull(WaveArgs a) {
  __shared__ float sM[12];
  if (skipped(a)) return;
  cull_block(a, blockIdx.y, blockIdx.x, sM);
}

// ------------------------------------------------------------------ triangle setup + binning

// Appends a snapped triangle piece (vertices in 1/256 px, inverse-depth plane, parent id) to
// the bins of every tile its sample bounding box overlaps, after normalising the winding so
// the doubled area is positive; zero-area pieces and pieces that cover no sample are dropped.
// Warp-collective: all 32 lanes call it, `valid` marks the lanes that hold a piece. The
// lanes append to the tiles their pieces overlap one tile per step; the
// lanes that target the same tile in a step take consecutive slots through one atomic add
// by their lowest lane, so a cluster's triangles, which mostly share a tile or two, cost
// a few atomics per step instead of one per triangle.
__device__ __forceinline__ void emit_piece_warp(bool valid, int x0, int y0, int x1, int y1,
                                                int x2, int y2, float Ai, float Bi, float Ci,
                                                unsigned id, const WaveArgs &a, int *counts,
                                                unsigned char *bins_b) {
  TriRec *bins = reinterpret_cast<TriRec *>(bins_b);
  const TileGeom &tg = a.tg;
  const int lane = threadIdx.x & 31;
  long long area = (long long)(x1 - x0) * (y2 - y0) - (long long)(y1 - y0) * (x2 - x0);
  if (area < 0) {
    int t = x1; x1 = x2; x2 = t;
    t = y1; y1 = y2; y2 = t;
  }
  const int W = a.cam.W, H = a.cam.H;
  const int xmin = min(x0, min(x1, x2)), xmax = max(x0, max(x1, x2));
  const int ymin = min(y0, min(y1, y2)), ymax = max(y0, max(y1, y2));
  const int i0 = max((xmin + 127) >> 8, 0), i1 = min((xmax - 128) >> 8, W - 1);
  const int j0 = max((ymin + 127) >> 8, 0), j1 = min((ymax - 128) >> 8, H - 1);
  valid = valid && area != 0 && i0 <= i1 && j0 <= j1;
  int tx0 = 0, nx = 0, ty0 = 0, nt = 0;
  if (valid) {
    tx0 = i0 / tg.tw;
    ty0 = j0 / tg.th;
    nx = i1 / tg.tw - tx0 + 1;
    nt = nx * (j1 / tg.th - ty0 + 1);
  }
  const int4 w0 = make_int4(x0, y0, x1, y1);
  const int4 w1 = make_int4(x2, y2, __float_as_int(Ai), __float_as_int(Bi));
  const int4 w2 = make_int4(__float_as_int(Ci), (int)id, 0, 0);
  for (int k = 0; __any_sync(0xffffffffu, k < nt); ++k) {
    const bool has = k < nt;
    const int tile = has ? (ty0 + k / nx) * tg.ntx + tx0 + k % nx : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, tile);
    const int leader = __ffs(peers) - 1;
    int base = 0;
    if (has && lane == leader) base = atomicAdd(&counts[tile], __popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (has) {
      const int slot = base + __popc(peers & ((1u << lane) - 1u));
      if (slot < tg.cap) {
        int4 *dst = reinterpret_cast<int4 *>(bins + (long long)tile * tg.cap + slot);
        dst[0] = w0;
        dst[1] = w1;
        dst[2] = w2;
      } else {
        atomicOr(a.status, kStatusOverflow);
      }
    }
  }
}

// Warp-collective append of a ray-table record to the bins of every tile its pixel rectangle
// r = (i0, i1, j0, j1) overlaps; `valid` marks the lanes that hold one. As for pinhole pieces,
// lanes that target the same tile in a step take consecutive slots with one atomic add.
__device__ __forceinline__ void emit_ray_warp(bool valid, const RayRec &rr, int4 r,
                                              const WaveArgs &a, int *counts,
                                              unsigned char *bins_b) {
  RayRec *bins = reinterpret_cast<RayRec *>(bins_b);
  const TileGeom &tg = a.tg;
  const int lane = threadIdx.x & 31;
  int tx0 = 0, nx = 0, ty0 = 0, nt = 0;
  if (valid) {
    tx0 = r.x / tg.tw;
    ty0 = r.z / tg.th;
    nx = r.y / tg.tw - tx0 + 1;
    nt = nx * (r.w / tg.th - ty0 + 1);
  }
  const int4 *src = reinterpret_cast<const int4 *>(&rr);
  int4 w3 = src[3];
  w3.z = r.x | (r.y << 16);
  w3.w = r.z | (r.w << 16);
  for (int k = 0; __any_sync(0xffffffffu, k < nt); ++k) {
    const bool has = k < nt;
    const int tile = has ? (ty0 + k / nx) * tg.ntx + tx0 + k % nx : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, tile);
    const int leader = __ffs(peers) - 1;
    int base = 0;
    if (has && lane == leader) base = atomicAdd(&counts[tile], __popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (has) {
      const int slot = base + __popc(peers & ((1u << lane) - 1u));
      if (slot < tg.cap) {
        int4 *dst = reinterpret_cast<int4 *>(bins + (long long)tile * tg.cap + slot);
        dst[0] = src[0];
        dst[1] = src[1];
        dst[2] = src[2];
        dst[3] = w3;
      } else {
        atomicOr(a.status, kStatusOverflowRay);
      }
    }
  }
}

// Ray-table triangle: contract side normals and inverse-depth normal, then a conservative
// pixel rectangle from the layout (azimuth from the vertices' smallest enclosing arc, full
// when a pole is inside; elevation from the vertices widened by the great-circle bulge
// bound z / cos(L/2), L the longest edge angle), a quarter-pixel margin (the FP32 angles
// are good to ~1e-6 rad and the table's rays lie within that margin of the layout), split
// at the seam into at most two rectangles (i0, i1, j0, j1), which are returned with their
// count. A triangle between pixel rays gets no rectangle; most far triangles of a panorama
// are such, so the record's plane is computed only once a rectangle exists.
__device__ __forceinline__ int setup_ray(const float3 v[3], const float4 u[3], const int gid[3],
                                         unsigned id, const DevCam &cam, RayRec &rr,
                                         int4 rect[2]) {
  const float3 c12 = cross_c(v[1], v[2]);
  const float det = dot_c(v[0].x, v[0].y, v[0].z, c12.x, c12.y, c12.z);
  if (det == 0.0f || det != det) return 0;
  float3 side[3];
  float sg[3];
  int sig = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int m = k == 2 ? 0 : k + 1;
    const bool lo_is_k = gid[k] < gid[m];
    side[k] = lo_is_k ? cross_c(v[k], v[m]) : cross_c(v[m], v[k]);
    sg[k] = (det > 0.0f ? 1.0f : -1.0f) * (lo_is_k ? 1.0f : -1.0f);
    if (sg[k] > 0.0f) sig |= 1 << k;
  }
  // ---- conservative pixel rectangle (any rounding; margins absorb it)
  // An edge plane keeps the up (down) direction out when sg side.y exceeds 1e-4 |side| (below
  // minus that): compared squared, sy^2 > 1e-8 |side|^2 with the sign of sy, no square root.
  bool has_up = true, has_dn = true;  // up = (0,-1,0), down = (0,1,0)
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float n2 = side[k].x * side[k].x + side[k].y * side[k].y + side[k].z * side[k].z;
    const float sy = sg[k] * side[k].y;
    const bool clear = sy * sy > 1e-8f * n2;
    if (clear && sy > 0.0f) has_up = false;
    if (clear && sy < 0.0f) has_dn = false;
  }
  float zmax = fmaxf(-u[0].y, fmaxf(-u[1].y, -u[2].y)), zmin = fminf(-u[0].y, fminf(-u[1].y, -u[2].y));
  const float cmin = fminf(u[0].x * u[1].x + u[0].y * u[1].y + u[0].z * u[1].z,
                           fminf(u[1].x * u[2].x + u[1].y * u[2].y + u[1].z * u[2].z,
                                 u[2].x * u[0].x + u[2].y * u[0].y + u[2].z * u[0].z));
  // half-angle cosine of the longest edge; its reciprocal square root widens the elevation
  // bounds (the directions are normalised approximately, which the margin absorbs)
  const float h2 = fmaxf(0.0f, 0.5f * (1.0f + cmin));
  if (h2 < 0.0025f) {
    zmax = 1.0f;
    zmin = -1.0f;
  } else {
    const float ich = rsqrtf(h2);
    if (zmax >= 0.0f) zmax = zmax * ich;
    if (zmin <= 0.0f) zmin = zmin * ich;
  }
  zmax = fminf(1.0f, zmax);
  zmin = fmaxf(-1.0f, zmin);
  if (has_up) zmax = 1.0f;
  if (has_dn) zmin = -1.0f;
  const float el_hi = asinf(zmax), el_lo = asinf(zmin);
  // approximate divisions: the margin absorbs their few-ulp error
  const int j0 = max(0, (int)ceilf(__fdividef(cam.el0 - el_hi, cam.el_step) - kRayMarginPx));
  const int j1 = min(cam.H - 1, (int)floorf(__fdividef(cam.el0 - el_lo, cam.el_step) + kRayMarginPx));
  if (j0 > j1) return 0;
  int nrect;
  if (has_up || has_dn) {
    rect[0] = make_int4(0, cam.W - 1, j0, j1);
    nrect = 1;
  } else {
    float s0 = u[0].w, s1 = u[1].w, s2 = u[2].w, t;
    if (s0 > s1) { t = s0; s0 = s1; s1 = t; }
    if (s1 > s2) { t = s1; s1 = s2; s2 = t; }
    if (s0 > s1) { t = s0; s0 = s1; s1 = t; }
    const float twopi = 6.28318530717958647692f;
    const float g01 = s1 - s0, g12 = s2 - s1, g20 = s0 + twopi - s2;
    float lo, hi;
    if (g20 >= g01 && g20 >= g12) { lo = s0; hi = s2; }
    else if (g01 >= g12) { lo = s1; hi = s0 + twopi; }
    else { lo = s2; hi = s1 + twopi; }
    const int ilo = (int)ceilf(__fdividef(lo - cam.az0, cam.az_step) - 0.5f - kRayMarginPx);
    const int ihi = (int)floorf(__fdividef(hi - cam.az0, cam.az_step) - 0.5f + kRayMarginPx);
    const int n = ihi - ilo + 1;
    if (n <= 0) return 0;
    if (n >= cam.W) {
      rect[0] = make_int4(0, cam.W - 1, j0, j1);
      nrect = 1;
    } else {
      int st = ilo % cam.W;
      if (st < 0) st += cam.W;
      if (st + n <= cam.W) {
        rect[0] = make_int4(st, st + n - 1, j0, j1);
        nrect = 1;
      } else {
        rect[0] = make_int4(st, cam.W - 1, j0, j1);
        rect[1] = make_int4(0, st + n - 1 - cam.W, j0, j1);
        nrect = 2;
      }
    }
  }
  rr.c0x = side[0].x; rr.c0y = side[0].y; rr.c0z = side[0].z;
  rr.c1x = side[1].x; rr.c1y = side[1].y; rr.c1z = side[1].z;
  rr.c2x = side[2].x; rr.c2y = side[2].y; rr.c2z = side[2].z;
  const PlaneN pl = plane_n(v[0], v[1], v[2]);
  rr.nix = __fdiv_rn(pl.nx, pl.d);
  rr.niy = __fdiv_rn(pl.ny, pl.d);
  rr.niz = __fdiv_rn(pl.nz, pl.d);
  rr.id = id;
  rr.sig = sig;
  rr.rect0 = rr.rect1 = 0;
  return nrect;
}

constexpr int kClusterMax = 64;  // vertices and triangles per cluster

// One warp per visible cluster: its vertices are transformed and snapped once into shared
// memory, then each lane sets up triangles (near-plane cut, culling, depth plane) and
// appends them to the screen-tile bins.
struct SetupSmem {
  float M[12];
  int nvis;
  float4 s_vc[8][kClusterMax];
  int2 s_vs[8][kClusterMax];
  int s_gid[8][kClusterMax];
  float4 s_dir[8][kClusterMax];  // ray table: unit direction and azimuth
};

template <int MODEL>
__device__ __forceinline__ void setup_block(const WaveArgs &a, int q, int worker, int nworkers,
                                            SetupSmem &sm) {
  float4(*s_vc)[kClusterMax] = sm.s_vc;
  int2(*s_vs)[kClusterMax] = sm.s_vs;
  int(*s_gid)[kClusterMax] = sm.s_gid;
  float4(*s_dir)[kClusterMax] = sm.s_dir;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) sm.nvis = ld_cg(&a.vis_count[q]);
  load_m_block(a, q, sm.M);
  float M[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) M[k] = sm.M[k];
  const int nvis = sm.nvis;
  const int4 *vis = a.vis + (long long)q * a.n_clusters;
  int *counts = a.counts + (long long)q * a.tg.ntiles;
  unsigned char *bins = a.bins + (long long)q * a.tg.ntiles * a.tg.cap * a.tg.rec_bytes;
  const int W = a.cam.W, H = a.cam.H;
  const float near_m = a.cam.near_m;
  constexpr bool raytable = MODEL != 0;  // one instantiation per camera model
  for (int ci = worker * 8 + warp; ci < nvis; ci += nworkers * 8) {
    const int4 info = __ldcg(&vis[ci]);  // vert offset, tri offset, nv, nt
    for (int k = lane; k < info.z; k += 32) {
      const float4 v = a.cl_pos[info.x + k];
      const int gv = __float_as_int(v.w);
      const float3 c = xform(M, v.x, v.y, v.z);
      int2 sv = make_int2(kSentinel, 1);  // behind the near plane
      if (raytable) {
        // the direction only bounds the rectangle: an approximate normalisation suffices
        const float n2 = c.x * c.x + c.y * c.y + c.z * c.z;
        const float inv = n2 > 0.0f ? rsqrtf(n2) : 0.0f;
        s_dir[warp][k] = make_float4(c.x * inv, c.y * inv, c.z * inv, atan2f(c.x, c.z));
      } else if (c.z >= near_m) {
        int xi, yi;
        sv = snap(a.cam, c.x, c.y, c.z, xi, yi) ? make_int2(xi, yi) : make_int2(kSentinel, 2);
      }
      s_vc[warp][k] = make_float4(c.x, c.y, c.z, 0.0f);
      s_vs[warp][k] = sv;
      s_gid[warp][k] = gv;
    }
    __syncwarp();
    if (raytable) {
      // every lane steps through the cluster's triangles together (warp-collective appends)
      for (int k0 = 0; k0 < info.w; k0 += 32) {
        const int k = k0 + lane;
        RayRec rr;
        int4 rect[2];
        int nrect = 0;
        if (k < info.w) {
          const uchar4 t = a.cl_tris[info.y + k];
          const unsigned id = (unsigned)a.cl_ids[info.y + k];
          const int loc[3] = {t.x, t.y, t.z};
          float3 v[3];
          float4 u[3];
          int gid[3];
#pragma unroll
          for (int m = 0; m < 3; ++m) {
            const float4 p = s_vc[warp][loc[m]];
            v[m] = make_float3(p.x, p.y, p.z);
            u[m] = s_dir[warp][loc[m]];
            gid[m] = s_gid[warp][loc[m]];
          }
          nrect = setup_ray(v, u, gid, id, a.cam, rr, rect);
        }
        emit_ray_warp(nrect > 0, rr, rect[0], a, counts, bins);
        if (__any_sync(0xffffffffu, nrect > 1)) emit_ray_warp(nrect > 1, rr, rect[1], a, counts, bins);
      }
      __syncwarp();
      continue;
    }
    // pinhole: every lane of the warp steps through the cluster's triangles together, so the
    // (at most two) pieces of a lane's triangle are appended by the warp-collective emitter
    for (int k0 = 0; k0 < info.w; k0 += 32) {
      const int k = k0 + lane;
      bool va = false, vb = false;
      int sx[4] = {0, 0, 0, 0}, sy[4] = {0, 0, 0, 0};
      float A = 0.0f, B = 0.0f, C = 0.0f;
      unsigned id = 0;
      if (k < info.w) {
        const uchar4 t = a.cl_tris[info.y + k];
        id = (unsigned)a.cl_ids[info.y + k];
        const int2 s0 = s_vs[warp][t.x], s1 = s_vs[warp][t.y], s2 = s_vs[warp][t.z];
        if (s0.x != kSentinel && s1.x != kSentinel && s2.x != kSentinel) {
          // all three in front of the near plane and inside the guard band
          const int xmin = min(s0.x, min(s1.x, s2.x)), xmax = max(s0.x, max(s1.x, s2.x));
          const int ymin = min(s0.y, min(s1.y, s2.y)), ymax = max(s0.y, max(s1.y, s2.y));
          if (max((xmin + 127) >> 8, 0) <= min((xmax - 128) >> 8, W - 1) &&
              max((ymin + 127) >> 8, 0) <= min((ymax - 128) >> 8, H - 1)) {
            const float4 p0 = s_vc[warp][t.x], p1 = s_vc[warp][t.y], p2 = s_vc[warp][t.z];
            const PlaneN pl = plane_n(make_float3(p0.x, p0.y, p0.z), make_float3(p1.x, p1.y, p1.z),
                                      make_float3(p2.x, p2.y, p2.z));
            fold_pinhole(a.cam, pl, A, B, C);
            sx[0] = s0.x; sy[0] = s0.y; sx[1] = s1.x; sy[1] = s1.y; sx[2] = s2.x; sy[2] = s2.y;
            va = true;
          }
        } else {
          // slow path: near-plane cut and/or guard band
          const int loc[3] = {t.x, t.y, t.z};
          int idx[3];
          float3 v[3];
          bool in[3];
          int nin = 0;
#pragma unroll
          for (int m = 0; m < 3; ++m) {
            const float4 p = s_vc[warp][loc[m]];
            v[m] = make_float3(p.x, p.y, p.z);
            idx[m] = s_gid[warp][loc[m]];
            in[m] = v[m].z >= near_m;
            nin += in[m];
          }
          // all behind, or all in front with a vertex beyond the guard band: nothing drawn
          if (nin != 0 && nin != 3) {
            const PlaneN pl = plane_n(v[0], v[1], v[2]);
            fold_pinhole(a.cam, pl, A, B, C);
            float3 poly[4];
            int n = 0;
#pragma unroll
            for (int m = 0; m < 3; ++m) {
              const int nx = (m + 1) % 3;
              if (in[m]) poly[n++] = v[m];
              if (in[m] != in[nx])
                poly[n++] = idx[m] < idx[nx] ? near_cut(v[m], v[nx], near_m) : near_cut(v[nx], v[m], near_m);
            }
            bool ok = true;
#pragma unroll
            for (int m = 0; m < 4; ++m)
              if (m < n) ok = ok && snap(a.cam, poly[m].x, poly[m].y, poly[m].z, sx[m], sy[m]);
            va = ok;
            vb = ok && n == 4;
          }
        }
      }
      emit_piece_warp(va, sx[0], sy[0], sx[1], sy[1], sx[2], sy[2], A, B, C, id, a, counts, bins);
      if (__any_sync(0xffffffffu, vb))
        emit_piece_warp(vb, sx[0], sy[0], sx[2], sy[2], sx[3], sy[3], A, B, C, id, a, counts, bins);
    }
    __syncwarp();
  }
}

// pinhole: six resident CTAs per SM (40 registers): setup is bound by the latency of its
// dependent loads, so more resident warps pay more than registers; the ray-table setup keeps
// a record and two rectangles per lane across its appends and gets 64 registers
template <int MODEL>
__global__ void __launch_bounds__(256, MODEL == 0 ? 6 : 4) k_setup(WaveArgs a) {
  __shared__ SetupSmem sm;
  if (skipped(a)) return;
  setup_block<MODEL>(a, blockIdx.y, blockIdx.x, gridDim.x, sm);
}

// ------------------------------------------------------------------ raster + epilogue

constexpr int kRecMaxPinhole = 192;  // bin records staged in shared memory per round (48 B)
constexpr int kRecMaxRay = 192;      // (64 B)

// Exact edge test with int32 operands and 64-bit products: E = dx (py - ya) - dy (px - xa),
// covered iff E > 0 or E == 0 on a top or left edge.
__device__ __forceinline__ bool edge_ok(int dx, int dy, int xa, int ya, int px, int py) {
  const long long E = (long long)dx * (py - ya) - (long long)dy * (px - xa);
  const bool top_left = dy < 0 || (dy == 0 && dx > 0);
  return E > 0 || (E == 0 && top_left);
}

constexpr int kRecFallback = 1 << 28;  // record keeps its snapped vertices (int64 edge tests)

// Per-record raster setup for one tile: clip the sample bounding box to the tile and turn
// each edge function into an exact int32 affine function of the pixel offset (di, dj) inside
// that rectangle, E = E0 + di*sx + dj*sy with the top-left bias folded into E0. Edges that
// hold on the whole rectangle become E = 0; a record whose rectangle misses one edge's half
// plane is dropped. Over the rectangle every value of E lies strictly between -(|ax| + |ay|)
// and |ax| + |ay| (ax, ay its extent along x and y), which is below 2^31 when
// 256 (|dx| + |dy|) (max(TW, TH) - 1) < 2^31: edges longer than that keep the record's
// vertices for the int64 test. Returns the rectangle's 2x2-quad count (0 = nothing).
template <int TW, int TH>
__device__ __forceinline__ int derive_rect(TriRec *rec, int4 *hdr, int k, int cnt, int ox,
                                           int oy, int xe, int ye) {
  constexpr int kEdgeMax = (TW > 32 || TH > 32) ? (1 << 17) : (1 << 18);
  static_assert(256ll * kEdgeMax * ((TW > TH ? TW : TH) - 1) < (1ll << 31), "int32 edge range");
  if (k >= cnt) return 0;
  TriRec &r = rec[k];
  const int xmin = min(r.x0, min(r.x1, r.x2)), xmax = max(r.x0, max(r.x1, r.x2));
  const int ymin = min(r.y0, min(r.y1, r.y2)), ymax = max(r.y0, max(r.y1, r.y2));
  const int i0 = max((xmin + 127) >> 8, ox), i1 = min((xmax - 128) >> 8, xe);
  const int j0 = max((ymin + 127) >> 8, oy), j1 = min((ymax - 128) >> 8, ye);
  if (i0 > i1 || j0 > j1) return 0;
  const int bw = i1 - i0 + 1, bh = j1 - j0 + 1;
  const int xs[3] = {r.x0, r.x1, r.x2}, ys[3] = {r.y0, r.y1, r.y2};
  const int px0 = 256 * i0 + 128, py0 = 256 * j0 + 128;
  int e0[3], sx[3], sy[3];
  bool fallback = false;
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const int nb = e == 2 ? 0 : e + 1;
    const int dx = xs[nb] - xs[e], dy = ys[nb] - ys[e];
    const bool top_left = dy < 0 || (dy == 0 && dx > 0);
    const long long E0 = (long long)dx * (py0 - ys[e]) - (long long)dy * (px0 - xs[e]) + (top_left ? 0 : -1);
    const long long ax = -256ll * dy * (bw - 1), ay = 256ll * dx * (bh - 1);
    const long long lo = E0 + min(ax, 0ll) + min(ay, 0ll), hi = E0 + max(ax, 0ll) + max(ay, 0ll);
    if (hi < 0) return 0;              // no pixel of the rectangle is on the inner side
    if (lo >= 0) {                     // the whole rectangle is on the inner side
      e0[e] = 0; sx[e] = 0; sy[e] = 0;
    } else if (abs(dx) + abs(dy) <= kEdgeMax) {
      e0[e] = (int)E0; sx[e] = -256 * dy; sy[e] = 256 * dx;
    } else {
      fallback = true;
      e0[e] = 0; sx[e] = 0; sy[e] = 0;
    }
  }
  const int qw = (bw + 1) >> 1, qh = (bh + 1) >> 1;  // 2x2 pixel quads over the rectangle
  // quad row of quad index l: __umulhi(2 l, m) = floor(l / qw) exactly for l < 2^10 with
  // m = ceil(2^31 / qw) (the error 2 l / 2^32 stays below 1 / qw)
  hdr[k] = make_int4(e0[0], e0[1], e0[2], (int)((2147483647u + (unsigned)qw) / (unsigned)qw));
  if (!fallback) {
    r.x0 = sx[0]; r.y0 = sy[0]; r.x1 = sx[1]; r.y1 = sy[1]; r.x2 = sx[2]; r.y2 = sy[2];
  }
  r.pad = (i0 - ox) | ((j0 - oy) << 8) | ((bw - 1) << 16) | ((bh - 1) << 22) | (fallback ? kRecFallback : 0);
  return qw * qh;
}

// Coverage of pixel (i, j) from a record's vertices with exact int64 edge functions.
__device__ __forceinline__ bool covers_exact(const TriRec &q, int i, int j) {
  const int px = 256 * i + 128, py = 256 * j + 128;
  return edge_ok(q.x1 - q.x0, q.y1 - q.y0, q.x0, q.y0, px, py) &&
         edge_ok(q.x2 - q.x1, q.y2 - q.y1, q.x1, q.y1, px, py) &&
         edge_ok(q.x0 - q.x2, q.y0 - q.y2, q.x2, q.y2, px, py);
}

// Inner-side test of one pixel from the three int32 edge values (wrapping adds: a value is
// only used when its pixel lies inside the record's rectangle, where it cannot wrap).
__device__ __forceinline__ bool inner3(int a, int b, int c) { return (a | b | c) >= 0; }

__device__ __forceinline__ int wadd(int a, int b) { return (int)((unsigned)a + (unsigned)b); }

// (float)i + 0.5f for 0 <= i < 2^23 without the conversion pipe: 2^23 + i is exact in the
// mantissa, and subtracting 2^23 - 0.5 (representable) leaves i + 0.5 exactly.
__device__ __forceinline__ float px_centre(int i) {
  return __fsub_rn(__int_as_float(0x4B000000 | i), 8388607.5f);
}


// Rasterise every record of one (pose, tile) bin into the shared z-buffer. Records are staged
// with one bulk copy per round; a block-wide scan of their per-tile rectangle sizes lays all
// candidate fragments out in one index space, which is split evenly over the warps. Each lane
// walks its fragments in record order (two-pointer over the scan), so no lane idles on small
// triangles and no warp waits on large ones.
template <int TW, int TH>
__device__ __forceinline__ bool raster_tile(unsigned long long *zk, TriRec *stage, int4 *hdr,
                                            int *S, int *wtot, unsigned long long *bar,
                                            const TriRec *recs, int n, int ox, int oy, int xe,
                                            int ye, const DevCam &cam, long long budget) {
  constexpr int kRecMax = kRecMaxPinhole;
  static_assert(kRecMax <= kThreads, "one record per thread");
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = kThreads / 32;
  // kept iff 0 < w, w_far <= w <= w_near: w_far >= 0, so the first two tests are one
  // comparison with the larger of w_far and the smallest positive (subnormal) float
  const float w_lo = fmaxf(cam.w_far, __int_as_float(1)), w_hi = cam.w_near;
  unsigned phase = 0;
  for (int r0 = 0; r0 < n; r0 += kRecMax) {
    const int cnt = min(kRecMax, n - r0);
    if (tid == 0) {
      fence_async_smem();
      bulk_g2s(stage, recs + r0, (unsigned)(cnt * sizeof(TriRec)), bar);
    }
    bool ok = mbar_wait(bar, phase, budget);
    ok = __syncthreads_and(ok);
    if (!ok) {
      // the copy may still be in flight: drain it (default budget) before the CTA leaves
      if (tid == 0) mbar_wait(bar, phase, kWaitCycles);
      return false;
    }
    phase ^= 1u;
    // quad count of record t, block-wide exclusive scan in record order
    const int n0 = derive_rect<TW, TH>(stage, hdr, tid, cnt, ox, oy, xe, ye);
    int incl = n0;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += v;
    }
    if (lane == 31) wtot[warp] = incl;
    __syncthreads();
    int before = 0, F = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      before += w < warp ? wtot[w] : 0;
      F += wtot[w];
    }
    if (tid < cnt) S[tid] = before + incl - n0;
    if (tid == 0) S[cnt] = F;
    __syncthreads();
    const int lo = (int)(((long long)F * warp) / NW), hi = (int)(((long long)F * (warp + 1)) / NW);
    int f = lo + lane;
    if (f < hi) {
      int a = 0, b = cnt - 1;  // last record with S[r] <= f
      while (a < b) {
        const int m = (a + b + 1) >> 1;
        if (S[m] <= f) a = m;
        else b = m - 1;
      }
      int r = a, sr = S[a], snext = S[a + 1];
      for (; f < hi; f += 32) {
        while (snext <= f) {
          ++r;
          sr = snext;
          snext = S[r + 1];
        }
        const TriRec &q = stage[r];
        const int4 h = hdr[r];
        const int l = f - sr;
        const int pad = q.pad;
        const int bw = ((pad >> 16) & 0x3f) + 1, bh = ((pad >> 22) & 0x3f) + 1;
        const int qw = (bw + 1) >> 1;
        const int qj = (int)__umulhi(2u * (unsigned)l, (unsigned)h.w);
        const int di = 2 * (l - qj * qw), dj = 2 * qj;
        const int li = (pad & 0xff) + di, lj = ((pad >> 8) & 0xff) + dj;
        const int i = ox + li, j = oy + lj;
        const bool has_r = di + 1 < bw, has_d = dj + 1 < bh;
        bool in00, in10, in01, in11;
        if (!(pad & kRecFallback)) {
          const int a = h.x + di * q.x0 + dj * q.y0;
          const int b = h.y + di * q.x1 + dj * q.y1;
          const int c = h.z + di * q.x2 + dj * q.y2;
          in00 = inner3(a, b, c);
          in10 = has_r && inner3(wadd(a, q.x0), wadd(b, q.x1), wadd(c, q.x2));
          in01 = has_d && inner3(wadd(a, q.y0), wadd(b, q.y1), wadd(c, q.y2));
          in11 = has_r && has_d &&
                 inner3(wadd(wadd(a, q.x0), q.y0), wadd(wadd(b, q.x1), q.y1), wadd(wadd(c, q.x2), q.y2));
        } else {
          in00 = covers_exact(q, i, j);
          in10 = has_r && covers_exact(q, i + 1, j);
          in01 = has_d && covers_exact(q, i, j + 1);
          in11 = has_r && has_d && covers_exact(q, i + 1, j + 1);
        }
        // inverse depth at the four samples, each exactly inv_depth_pinhole's expression
        // (i + 1.5 = (i + .5) + 1 and j + 1.5 are exact in FP32)
        const float fi = px_centre(i), fj = px_centre(j);
        const float fi1 = __fadd_rn(fi, 1.0f), fj1 = __fadd_rn(fj, 1.0f);
        const float row0 = __fmaf_rn(q.Bi, fj, q.Ci), row1 = __fmaf_rn(q.Bi, fj1, q.Ci);
        const float w00 = __fmaf_rn(q.Ai, fi, row0), w10 = __fmaf_rn(q.Ai, fi1, row0);
        const float w01 = __fmaf_rn(q.Ai, fi, row1), w11 = __fmaf_rn(q.Ai, fi1, row1);
        const unsigned id = q.id;
        const int zi = lj * TW + li;
        if (in00 && w00 >= w_lo && w00 <= w_hi) atomicMin(&zk[zi], make_key(w00, id));
        if (in10 && w10 >= w_lo && w10 <= w_hi) atomicMin(&zk[zi + 1], make_key(w10, id));
        if (in01 && w01 >= w_lo && w01 <= w_hi) atomicMin(&zk[zi + TW], make_key(w01, id));
        if (in11 && w11 >= w_lo && w11 <= w_hi) atomicMin(&zk[zi + TW + 1], make_key(w11, id));
      }
    }
    __syncthreads();
  }
  return true;
}


// Ray-table counterpart of derive_rect: clip the record's pixel rectangle to the tile and keep
// its tile-relative origin and width in rect0.
__device__ __forceinline__ int derive_ray_rect(RayRec *rec, int k, int cnt, int ox, int oy,
                                               int xe, int ye) {
  if (k >= cnt) return 0;
  RayRec &r = rec[k];
  const int i0 = max(r.rect0 & 0xffff, ox), i1 = min(r.rect0 >> 16, xe);
  const int j0 = max(r.rect1 & 0xffff, oy), j1 = min(r.rect1 >> 16, ye);
  if (i0 > i1 || j0 > j1) return 0;
  const int bw = i1 - i0 + 1;
  r.rect0 = (i0 - ox) | ((j0 - oy) << 8) | (bw << 16);
  return bw * (j1 - j0 + 1);
}

// Ray-table tile raster: the tile's rays are staged in shared memory; each fragment is a cone
// test of its ray against the three edge normals and an inverse-depth dot product.
template <int TW, int TH>
__device__ __forceinline__ bool raster_tile_ray(unsigned long long *zk, RayRec *stage,
                                                const float *rx, const float *ry, const float *rz,
                                                int *S, int *wtot, unsigned long long *bar,
                                                const RayRec *recs, int n, int ox, int oy,
                                                int xe, int ye, const DevCam &cam,
                                                long long budget) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = kThreads / 32;
  constexpr int kRecMax = kRecMaxRay;
  static_assert(kRecMax <= kThreads, "one record per thread");
  const float w_near = cam.w_near, w_far = cam.w_far;
  unsigned phase = 0;
  for (int r0 = 0; r0 < n; r0 += kRecMax) {
    const int cnt = min(kRecMax, n - r0);
    if (tid == 0) {
      fence_async_smem();
      bulk_g2s(stage, recs + r0, (unsigned)(cnt * sizeof(RayRec)), bar);
    }
    bool ok = mbar_wait(bar, phase, budget);
    ok = __syncthreads_and(ok);
    if (!ok) {
      // the copy may still be in flight: drain it (default budget) before the CTA leaves
      if (tid == 0) mbar_wait(bar, phase, kWaitCycles);
      return false;
    }
    phase ^= 1u;
    // pixel count of record t, block-wide exclusive scan in record order
    const int n0 = derive_ray_rect(stage, tid, cnt, ox, oy, xe, ye);
    int incl = n0;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += v;
    }
    if (lane == 31) wtot[warp] = incl;
    __syncthreads();
    int before = 0, F = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      before += w < warp ? wtot[w] : 0;
      F += wtot[w];
    }
    if (tid < cnt) S[tid] = before + incl - n0;
    if (tid == 0) S[cnt] = F;
    __syncthreads();
    const int lo = (int)(((long long)F * warp) / NW), hi = (int)(((long long)F * (warp + 1)) / NW);
    int f = lo + lane;
    if (f < hi) {
      int a = 0, b = cnt - 1;
      while (a < b) {
        const int m = (a + b + 1) >> 1;
        if (S[m] <= f) a = m;
        else b = m - 1;
      }
      int r = a, sr = S[a], snext = S[a + 1];
      for (; f < hi; f += 32) {
        while (snext <= f) {
          ++r;
          sr = snext;
          snext = S[r + 1];
        }
        const RayRec &q = stage[r];
        const int l = f - sr;
        const int bw = q.rect0 >> 16;
        const int dj = __float2int_rz(__fmul_rn(__int2float_rn(l) + 0.5f, __frcp_rn(__int2float_rn(bw))));
        const int li = (q.rect0 & 0xff) + (l - dj * bw), lj = ((q.rect0 >> 8) & 0xff) + dj;
        const int p = lj * TW + li;
        const float x = rx[p], y = ry[p], z = rz[p];
        const float s0 = dot_c(x, y, z, q.c0x, q.c0y, q.c0z);
        const float s1 = dot_c(x, y, z, q.c1x, q.c1y, q.c1z);
        const float s2 = dot_c(x, y, z, q.c2x, q.c2y, q.c2z);
        const bool in = ((q.sig & 1) ? s0 >= 0.0f : s0 < 0.0f) && ((q.sig & 2) ? s1 >= 0.0f : s1 < 0.0f) &&
                        ((q.sig & 4) ? s2 >= 0.0f : s2 < 0.0f);
        if (in) {
          const float w = dot_c(q.nix, q.niy, q.niz, x, y, z);
          if (w > 0.0f && w >= w_far && w <= w_near) atomicMin(&zk[p], make_key(w, q.id));
        }
      }
    }
    __syncthreads();
  }
  return true;
}

#ifndef RM_PERSIST_MIN_BLOCKS
#define RM_PERSIST_MIN_BLOCKS 4
#endif

#ifndef RM_RASTER_MIN_BLOCKS
#define RM_RASTER_MIN_BLOCKS 5  // resident CTAs per SM the register budget is sized for (48 registers)
#endif

template <int NP, int MODEL>
struct RasterSmem {
  static constexpr int NW = kThreads / 32;
  // pinhole: staged records + their int4 edge headers; ray table: records + the tile's rays
  static constexpr int kBuf = MODEL == 0 ? kRecMaxPinhole * (48 + 16) : kRecMaxRay * 64 + 12 * NP;
  unsigned long long zk[NP];
  float M[12];
  int n;
  alignas(128) unsigned char sbuf[kBuf];
  int S[(MODEL == 0 ? kRecMaxPinhole : kRecMaxRay) + 1];
  int wtot[NW];
  unsigned long long bar[1];
  float red[NW][28];
  int redc[NW][6];
};

// Camera-frame normal at a pixel of triangle `id` from the map's vertex normals (Sec. V,
// sequential alignment: the map's points rendered coloured by their normals): the hit t r on
// the triangle's camera-frame plane, its barycentrics (as the visibility buffer's), the three
// world-frame vertex normals blended by them as a rasteriser interpolates a vertex attribute,
// and the blend rotated into the camera frame (unnormalised). False when the blend is not
// finite: a vertex without a normal (NaN) leaves the pixel unassociated.
__device__ __forceinline__ bool vertex_normal(const WaveArgs &a, const float *M, unsigned id, float t,
                                           float rx, float ry, float rz, float &nx, float &ny,
                                           float &nz) {
  const int4 f = a.faces[id];
  const float4 p0 = a.v[f.x], p1 = a.v[f.y], p2 = a.v[f.z];
  float Mr[12];
  for (int k = 0; k < 12; ++k) Mr[k] = M[k];
  const float3 v0 = xform(Mr, p0.x, p0.y, p0.z), v1 = xform(Mr, p1.x, p1.y, p1.z),
               v2 = xform(Mr, p2.x, p2.y, p2.z);
  const float hx = t * rx - v0.x, hy = t * ry - v0.y, hz = t * rz - v0.z;
  const float e1x = v1.x - v0.x, e1y = v1.y - v0.y, e1z = v1.z - v0.z;
  const float e2x = v2.x - v0.x, e2y = v2.y - v0.y, e2z = v2.z - v0.z;
  const float cx = e1y * e2z - e1z * e2y, cy = e1z * e2x - e1x * e2z, cz = e1x * e2y - e1y * e2x;
  const float inn = 1.0f / (cx * cx + cy * cy + cz * cz);
  const float b1 = ((hy * e2z - hz * e2y) * cx + (hz * e2x - hx * e2z) * cy + (hx * e2y - hy * e2x) * cz) * inn;
  const float b2 = ((e1y * hz - e1z * hy) * cx + (e1z * hx - e1x * hz) * cy + (e1x * hy - e1y * hx) * cz) * inn;
  const float b0 = 1.0f - b1 - b2;
  const float4 N0 = a.vnormals[f.x], N1 = a.vnormals[f.y], N2 = a.vnormals[f.z];
  const float wx = b0 * N0.x + b1 * N1.x + b2 * N2.x;
  const float wy = b0 * N0.y + b1 * N1.y + b2 * N2.y;
  const float wz = b0 * N0.z + b1 * N1.z + b2 * N2.z;
  if (!(isfinite(wx) && isfinite(wy) && isfinite(wz))) return false;
  nx = M[0] * wx + M[1] * wy + M[2] * wz;
  ny = M[4] * wx + M[5] * wy + M[6] * wz;
  nz = M[8] * wx + M[9] * wy + M[10] * wz;
  return true;
}

__global__ void k_rotate_normals(const float *n, int V, const float *R, float4 *out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= V) return;
  const float x = n[3 * (long long)k], y = n[3 * (long long)k + 1], z = n[3 * (long long)k + 2];
  out[k] = make_float4(R[0] * x + R[1] * y + R[2] * z, R[3] * x + R[4] * y + R[5] * z,
                       R[6] * x + R[7] * y + R[8] * z, 0.0f);
}

cudaError_t launch_rotate_normals(const float *n, int V, const float *R, float4 *out, cudaStream_t s) {
  if (V <= 0) return cudaSuccess;
  k_rotate_normals<<<(V + 255) / 256, 256, 0, s>>>(n, V, R, out);
  return cudaGetLastError();
}

// One (pose q, tile) of the z-buffer and its fused epilogue. Returns false on a timed-out wait.
template <int TW, int TH, int MODE, int MODEL>
__device__ __forceinline__ void raster_block(const WaveArgs &a, int tile, int q,
                                             RasterSmem<TW * TH, MODEL> &sm) {
  constexpr int NP = TW * TH;
  unsigned long long *zk = sm.zk;
  unsigned char *sbuf = sm.sbuf;
  int *S = sm.S;
  int *wtot = sm.wtot;
  unsigned long long *bar = sm.bar;
  float(*red)[28] = sm.red;
  int(*redc)[6] = sm.redc;
  const int tid = threadIdx.x;
  const int g = a.wave_base + q;
  const int ox = (tile % a.tg.ntx) * TW, oy = (tile / a.tg.ntx) * TH;
  const int W = a.cam.W, H = a.cam.H;
  const int xe = min(ox + TW, W) - 1, ye = min(oy + TH, H) - 1;

  for (int p = tid; p < NP; p += kThreads) zk[p] = kKeyEmpty;
  const long long bin = (long long)q * a.tg.ntiles + tile;
  if (tid < 12) sm.M[tid] = __ldcg(a.Ms + 12 * (long long)g + tid);
  if (tid == 0) sm.n = min(ld_cg(&a.counts[bin]), a.tg.cap);
  float *rx = nullptr, *ry = nullptr, *rz = nullptr;
  if (MODEL != 0) {
    rx = reinterpret_cast<float *>(sbuf + kRecMaxRay * 64);
    ry = rx + NP;
    rz = ry + NP;
    for (int p = tid; p < NP; p += kThreads) {
      const int i = ox + p % TW, j = oy + p / TW;
      float x = 0.0f, y = 0.0f, z = 0.0f;
      if (i <= xe && j <= ye) {
        const float *rr = a.cam.rays + 3 * ((long long)j * W + i);
        x = rr[0];
        y = rr[1];
        z = rr[2];
      }
      rx[p] = x;
      ry[p] = y;
      rz[p] = z;
    }
  }
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    fence_mbar_init();
  }
  __syncthreads();
  const int n = sm.n;
  bool ok;
  if (MODEL == 0)
    ok = raster_tile<TW, TH>(zk, reinterpret_cast<TriRec *>(sbuf),
                             reinterpret_cast<int4 *>(sbuf + kRecMaxPinhole * 48), S, wtot, bar,
                             reinterpret_cast<const TriRec *>(a.bins) + bin * a.tg.cap, n, ox, oy,
                             xe, ye, a.cam, a.wait_cycles);
  else
    ok = raster_tile_ray<TW, TH>(zk, reinterpret_cast<RayRec *>(sbuf), rx, ry, rz, S, wtot, bar,
                                 reinterpret_cast<const RayRec *>(a.bins) + bin * a.tg.cap, n, ox,
                                 oy, xe, ye, a.cam, a.wait_cycles);
  if (!ok) {
    if (tid == 0) atomicOr(a.status, kStatusTimeout);
    return;
  }
  __syncthreads();

  const long long P = (long long)W * H;
  if (MODE == kRender) {
    for (int p = tid; p < NP; p += kThreads) {
      const int i = ox + p % TW, j = oy + p / TW;
      if (i > xe || j > ye) continue;
      const long long pix = (long long)g * P + (long long)j * W + i;
      const unsigned long long key = zk[p];
      if (key == kKeyEmpty) {
        a.depth[pix] = __int_as_float(0x7fc00000);
        if (a.tri_id) a.tri_id[pix] = -1;
        if (a.bary) {
          a.bary[2 * pix] = __int_as_float(0x7fc00000);
          a.bary[2 * pix + 1] = __int_as_float(0x7fc00000);
        }
        continue;
      }
      const unsigned id = (unsigned)key;
      const float t = key_depth(key);
      a.depth[pix] = t;
      if (a.tri_id) a.tri_id[pix] = (int)id;
      if (a.bary) {
        const int4 f = a.faces[id];
        float M[12];
        for (int k = 0; k < 12; ++k) M[k] = sm.M[k];
        const float4 w0 = a.v[f.x], w1 = a.v[f.y], w2 = a.v[f.z];
        const float3 v0 = xform(M, w0.x, w0.y, w0.z), v1 = xform(M, w1.x, w1.y, w1.z),
                     v2 = xform(M, w2.x, w2.y, w2.z);
        float rx, ry, rz;
        if (MODEL == 0) {
          rx = (i + 0.5f - a.cam.cx) / a.cam.fx;
          ry = (j + 0.5f - a.cam.cy) / a.cam.fy;
          rz = 1.0f;
        } else {
          const float *rr = a.cam.rays + 3 * ((long long)j * W + i);
          rx = rr[0];
          ry = rr[1];
          rz = rr[2];
        }
        const float hx = t * rx - v0.x, hy = t * ry - v0.y, hz = t * rz - v0.z;
        const float e1x = v1.x - v0.x, e1y = v1.y - v0.y, e1z = v1.z - v0.z;
        const float e2x = v2.x - v0.x, e2y = v2.y - v0.y, e2z = v2.z - v0.z;
        const float nx = e1y * e2z - e1z * e2y, ny = e1z * e2x - e1x * e2z, nz = e1x * e2y - e1y * e2x;
        const float nn = nx * nx + ny * ny + nz * nz;
        const float c1x = hy * e2z - hz * e2y, c1y = hz * e2x - hx * e2z, c1z = hx * e2y - hy * e2x;
        const float c2x = e1y * hz - e1z * hy, c2y = e1z * hx - e1x * hz, c2z = e1x * hy - e1y * hx;
        a.bary[2 * pix] = (c1x * nx + c1y * ny + c1z * nz) / nn;
        a.bary[2 * pix + 1] = (c2x * nx + c2y * ny + c2z * nz) / nn;
      }
    }
    return;
  }

  // ---- fused Table I + least-squares residual (+ adjoint) epilogue
  // per-thread outcome counts, 5 bits each (a thread sees at most NP / kThreads pixels)
  static_assert(NP / kThreads < 32, "count fields");
  unsigned cnt6 = 0;
  float acc[28];
#pragma unroll
  for (int k = 0; k < 28; ++k) acc[k] = 0.0f;
  float R[9];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    R[3 * k] = sm.M[4 * k];
    R[3 * k + 1] = sm.M[4 * k + 1];
    R[3 * k + 2] = sm.M[4 * k + 2];
  }
  const float eps = a.prm.eps;
  const float ifx = 1.0f / a.cam.fx, ify = 1.0f / a.cam.fy;
  float l1 = 0.0f;  // ICP: sum |Z_M - Z_1| over the associated pixels
  if (is_icp(MODE)) {
    // ---- point-to-plane ICP epilogue (Sec. V): projective association of the pixel's map
    // surface with its scan return, residual e = (d - t)(n . r), J = (n, p x n), p = d r.
    // Counts field 0 holds the associations; eps is the association tolerance.
#pragma unroll 1
    for (int p = tid; p < NP; p += kThreads) {
      const int i = ox + p % TW, j = oy + p / TW;
      if (i > xe || j > ye) continue;
      const unsigned long long key = zk[p];
      if (key == kKeyEmpty) continue;
      const long long pix = (long long)j * W + i;
      const float sd = a.scan_depth[pix];
      if (a.scan_cls[pix] != 0 || !(fabsf(sd) <= FLT_MAX)) continue;  // FO returns only
      const float4 pl = a.planes[(unsigned)key];
      if (__float_as_int(pl.w) != 0) continue;                         // FO surfaces only
      const float t = key_depth(key);
      const float dz = __fsub_rn(t, sd);
      if (!(fabsf(dz) < eps)) continue;
      float rx, ry, rz;
      if (MODEL == 0) {
        rx = (i + 0.5f - a.cam.cx) * ifx;
        ry = (j + 0.5f - a.cam.cy) * ify;
        rz = 1.0f;
      } else {
        const float *rr = a.cam.rays + 3 * pix;
        rx = rr[0];
        ry = rr[1];
        rz = rr[2];
      }
      float nx, ny, nz;
      if (MODE == kIcpVn) {
        if (!vertex_normal(a, sm.M, (unsigned)key, t, rx, ry, rz, nx, ny, nz)) continue;
      } else {
        nx = R[0] * pl.x + R[1] * pl.y + R[2] * pl.z;
        ny = R[3] * pl.x + R[4] * pl.y + R[5] * pl.z;
        nz = R[6] * pl.x + R[7] * pl.y + R[8] * pl.z;
      }
      const float nn = nx * nx + ny * ny + nz * nz;
      if (!(nn > 0.0f)) continue;  // degenerate face: no plane
      const float u = rsqrtf(nn);
      nx *= u;
      ny *= u;
      nz *= u;
      const float e = -dz * (nx * rx + ny * ry + nz * rz);
      const float px = sd * rx, py = sd * ry, pz = sd * rz;
      float J[6];
      J[0] = nx;
      J[1] = ny;
      J[2] = nz;
      J[3] = py * nz - pz * ny;
      J[4] = pz * nx - px * nz;
      J[5] = px * ny - py * nx;
      cnt6 += 1u;
      l1 += fabsf(dz);
      acc[0] += e * e;
#pragma unroll
      for (int k = 0; k < 6; ++k) acc[1 + k] += J[k] * e;
      int qk = 7;
#pragma unroll
      for (int u2 = 0; u2 < 6; ++u2)
#pragma unroll
        for (int v2 = u2; v2 < 6; ++v2) acc[qk++] += J[u2] * J[v2];
    }
  } else {
#pragma unroll 1
  for (int p = tid; p < NP; p += kThreads) {
    const int i = ox + p % TW, j = oy + p / TW;
    if (i > xe || j > ye) continue;
    const unsigned long long key = zk[p];
    if (key == kKeyEmpty) continue;  // map NaN row: ignore
    const long long pix = (long long)j * W + i;
    const float sd = a.scan_depth[pix];
    const int sc = a.scan_cls[pix];
    if (sc > 1 || !(fabsf(sd) <= FLT_MAX)) continue;  // scan NaN column: ignore
    const unsigned id = (unsigned)key;
    const float t = key_depth(key);
    const float4 pl = a.planes[id];
    const int mc = __float_as_int(pl.w);
    if (mc > 1) continue;  // unknown-occupied row: ignore
    const float dz = __fsub_rn(t, sd);
    int oc;
    if (mc == 0) oc = sc == 0 ? (fabsf(dz) <= eps ? 0 : 1) : (dz > 0.0f ? 2 : 3);
    else if (sc == 0) oc = dz <= 0.0f ? 4 : 5;
    else continue;  // FU / FU: ignore
    cnt6 += 1u << (5 * oc);
    float r, w, sgn = 0.0f;
    switch (oc) {
      case 0: w = a.prm.w_fofo; r = dz; sgn = 1.0f; break;
      case 1: w = a.prm.w_fofo; r = eps; break;
      case 2: w = a.prm.w_fofu; r = 0.0f; break;
      case 3:
        w = a.prm.w_fofu;
        if (-dz < eps) { r = -dz; sgn = -1.0f; } else { r = eps; }
        break;
      case 4: w = a.prm.w_fufo; r = 0.0f; break;
      default:
        w = a.prm.w_fufo;
        if (dz < eps) { r = dz; sgn = 1.0f; } else { r = eps; }
        break;
    }
    acc[0] += 0.5f * w * r * r;
    if (MODE == kCostGrad && sgn != 0.0f) {
      float rx, ry, rz;
      if (MODEL == 0) {
        rx = (i + 0.5f - a.cam.cx) * ifx;
        ry = (j + 0.5f - a.cam.cy) * ify;
        rz = 1.0f;
      } else {
        const float *rr = a.cam.rays + 3 * pix;
        rx = rr[0];
        ry = rr[1];
        rz = rr[2];
      }
      const float nx = R[0] * pl.x + R[1] * pl.y + R[2] * pl.z;
      const float ny = R[3] * pl.x + R[4] * pl.y + R[5] * pl.z;
      const float nz = R[6] * pl.x + R[7] * pl.y + R[8] * pl.z;
      const float inv = __fdividef(1.0f, nx * rx + ny * ry + nz * rz);  // Jacobian only
      const float s = sgn * inv;
      float J[6];
      J[0] = -nx * s;
      J[1] = -ny * s;
      J[2] = -nz * s;
      J[3] = -t * (ry * nz - rz * ny) * s;
      J[4] = -t * (rz * nx - rx * nz) * s;
      J[5] = -t * (rx * ny - ry * nx) * s;
      const float wr = w * r;
#pragma unroll
      for (int k = 0; k < 6; ++k) acc[1 + k] += wr * J[k];
      int qk = 7;
#pragma unroll
      for (int u = 0; u < 6; ++u)
#pragma unroll
        for (int v = u; v < 6; ++v) acc[qk++] += w * J[u] * J[v];
    }
  }
  }
  // fixed-order reduction: a reduce-scatter butterfly over the warp (lane L ends with the
  // warp's sum of value L), integer counts by warp reduction, then over the warps in order
  // (FP32, then one conversion to the FP64 tile partial)
  float v[32];
#pragma unroll
  for (int k = 0; k < 28; ++k) v[k] = acc[k];
#pragma unroll
  for (int k = 28; k < 32; ++k) v[k] = 0.0f;
  const int warp = tid >> 5, lane = tid & 31;
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    const bool hi = (lane & off) != 0;
#pragma unroll
    for (int m = 0; m < off; ++m) {
      const float keep = hi ? v[m + off] : v[m];
      const float send = hi ? v[m] : v[m + off];
      v[m] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
  // after the butterfly, lane L holds the warp's sum of value L
  if (lane < 28) red[warp][lane] = v[0];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const unsigned c = __reduce_add_sync(0xffffffffu, (cnt6 >> (5 * k)) & 31u);
    if (lane == 0) redc[warp][k] = (int)c;
  }
  if (is_icp(MODE)) {
    // the warp's C in counts field 1 (unused by ICP), as FP32 bits
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) l1 += __shfl_xor_sync(0xffffffffu, l1, off);
    if (lane == 0) redc[warp][1] = __float_as_int(l1);
  }
  __syncthreads();
  if (is_icp(MODE) && tid == 1) {
    float f = 0.0f;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) f = __fadd_rn(f, __int_as_float(redc[w][1]));
    a.partial[bin * kNumVals + 1] = (double)f;
  } else if (tid < 6) {
    int c = 0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) c += redc[w][tid];
    a.partial[bin * kNumVals + tid] = (double)c;
  } else if (tid < kNumVals) {
    float f = 0.0f;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) f = __fadd_rn(f, red[w][tid - 6]);
    a.partial[bin * kNumVals + tid] = (double)f;
  }
}

template <int TW, int TH, int MODE, int MODEL>
__global__ void __launch_bounds__(kThreads, RM_RASTER_MIN_BLOCKS) k_raster(WaveArgs a) {
  __shared__ RasterSmem<TW * TH, MODEL> sm;
  if (skipped(a)) return;
  raster_block<TW, TH, MODE, MODEL>(a, blockIdx.x, blockIdx.y, sm);
}

// Per pose: sum the per-tile partials. Warp w reduces values w, w+8, ...; lane l sums tiles
// l, l+32, ... and a butterfly combines the lanes, so the order is fixed run to run.
__device__ __forceinline__ void reduce_block(const WaveArgs &a, int q, double *vals) {
  const int g = a.wave_base + q;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double *base = a.partial + (long long)q * a.tg.ntiles * kNumVals;
  for (int k = warp; k < kNumVals; k += 8) {
    double s = 0.0;
    for (int t = lane; t < a.tg.ntiles; t += 32) s += __ldcg(base + (long long)t * kNumVals + k);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) vals[k] = s;
  }
  __syncthreads();
  const int k = threadIdx.x;
  if (k < 6 && a.res_counts) a.res_counts[6 * (long long)g + k] = (long long)vals[k];
  if (k == 6 && a.res_els) a.res_els[g] = vals[6];
  if (k >= 7 && k < 13 && a.res_grad) a.res_grad[6 * (long long)g + (k - 7)] = vals[k];
  if (k >= 13 && k < kNumVals && a.res_jtj) a.res_jtj[21 * (long long)g + (k - 13)] = vals[k];
  if (k == 0 && a.res_n) a.res_n[g] = (long long)vals[0];
  if (k == 1 && a.res_l1) a.res_l1[g] = vals[1];
  if (k == 0 && a.res_etable)
    a.res_etable[g] = (long long)(vals[1] + vals[3] + vals[5]) - (long long)(vals[0] + vals[2] + vals[4]);
}

__global__ void __launch_bounds__(256) k_reduce(WaveArgs a) {
  __shared__ double vals[kNumVals];
  if (skipped(a)) return;
  reduce_block(a, blockIdx.x, vals);
}

// ------------------------------------------------------------------ launch

template <int TW, int TH, int MODEL>
static cudaError_t launch_raster_m(const WaveArgs &a, int mode, cudaStream_t s) {
  dim3 grid(a.tg.ntiles, a.n_poses);
  if (mode == kRender) k_raster<TW, TH, kRender, MODEL><<<grid, kThreads, 0, s>>>(a);
  else if (mode == kCost) k_raster<TW, TH, kCost, MODEL><<<grid, kThreads, 0, s>>>(a);
  else if (mode == kIcp && a.vnormals) k_raster<TW, TH, kIcpVn, MODEL><<<grid, kThreads, 0, s>>>(a);
  else if (mode == kIcp) k_raster<TW, TH, kIcp, MODEL><<<grid, kThreads, 0, s>>>(a);
  else k_raster<TW, TH, kCostGrad, MODEL><<<grid, kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

template <int TW, int TH>
static cudaError_t launch_raster(const WaveArgs &a, int mode, cudaStream_t s) {
  return a.cam.model == 0 ? launch_raster_m<TW, TH, 0>(a, mode, s) : launch_raster_m<TW, TH, 1>(a, mode, s);
}

cudaError_t launch_wave(const WaveArgs &a, int mode, cudaStream_t s, cudaEvent_t *ev,
                        bool zero_counters) {
  cudaError_t e;
  if (zero_counters) {
    e = cudaMemsetAsync(a.counts, 0, sizeof(int) * (size_t)a.tg.ntiles * a.n_poses, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(a.vis_count, 0, sizeof(int) * (size_t)a.n_poses, s);
    if (e != cudaSuccess) return e;
  }
  if (ev && (e = cudaEventRecord(ev[0], s)) != cudaSuccess) return e;
  if (a.n_clusters > 0) {
    dim3 gc((a.n_clusters + 255) / 256, a.n_poses);
    k_cull<<<gc, 256, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (ev && (e = cudaEventRecord(ev[1], s)) != cudaSuccess) return e;
  if (a.n_clusters > 0) {
    // 16 CTAs per pose in a large wave: each warp then sets up several clusters, and the next
    // wave's setup (on the other stream) takes few enough SMs to run beside this wave's
    // raster; waves of few poses (single-pose alignment) get up to about six CTAs per SM in
    // total so that their setup spreads over the GPU
    const int per_pose = max(16, (kSetupCtasPerGpu + a.n_poses - 1) / a.n_poses);
    const int blocks = min(max(a.n_clusters / 64, 1), per_pose);
    dim3 gs(blocks, a.n_poses);
    if (a.cam.model == 0) k_setup<0><<<gs, 256, 0, s>>>(a);
    else k_setup<1><<<gs, 256, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (ev && (e = cudaEventRecord(ev[2], s)) != cudaSuccess) return e;
  if (a.tg.tw == 64 && a.tg.th == 32) e = launch_raster<64, 32>(a, mode, s);
  else if (a.tg.tw == 32 && a.tg.th == 32) e = launch_raster<32, 32>(a, mode, s);
  else if (a.tg.tw == 32 && a.tg.th == 16) e = launch_raster<32, 16>(a, mode, s);
  else e = launch_raster<16, 16>(a, mode, s);
  if (e != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[3], s)) != cudaSuccess) return e;
  if (mode != kRender) {
    k_reduce<<<a.n_poses, 256, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (ev && (e = cudaEventRecord(ev[4], s)) != cudaSuccess) return e;
  return cudaSuccess;
}

int wave_kernel_launches(const WaveArgs &a, int mode) {
  return 2 * (a.n_clusters > 0) + 1 + (mode != kRender);
}

// ------------------------------------------------------------------ Levenberg-Marquardt

__device__ __noinline__ void se3_right_dev(const double *T, const double *xi, double *out) {
  const double *rho = xi, *phi = xi + 3;
  const double th2 = phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2], th = sqrt(th2);
  double A, B, C;
  if (th < 1e-4) {
    A = 1.0 - th2 / 6.0 + th2 * th2 / 120.0;
    B = 0.5 - th2 / 24.0 + th2 * th2 / 720.0;
    C = 1.0 / 6.0 - th2 / 120.0 + th2 * th2 / 5040.0;
  } else {
    double sn, cs;
    sincos(th, &sn, &cs);
    A = sn / th;
    B = (1.0 - cs) / th2;
    C = (th - sn) / (th2 * th);
  }
  const double K[9] = {0, -phi[2], phi[1], phi[2], 0, -phi[0], -phi[1], phi[0], 0};
  double K2[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0;
      for (int k = 0; k < 3; ++k) s += K[3 * i + k] * K[3 * k + j];
      K2[3 * i + j] = s;
    }
  double E[16];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const double I = i == j ? 1.0 : 0.0;
      E[4 * i + j] = I + A * K[3 * i + j] + B * K2[3 * i + j];
    }
  for (int i = 0; i < 3; ++i) {
    double t = 0;
    for (int j = 0; j < 3; ++j) {
      const double I = i == j ? 1.0 : 0.0;
      t += (I + B * K[3 * i + j] + C * K2[3 * i + j]) * rho[j];
    }
    E[4 * i + 3] = t;
  }
  E[12] = E[13] = E[14] = 0.0;
  E[15] = 1.0;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double s = 0;
      for (int k = 0; k < 4; ++k) s += T[4 * i + k] * E[4 * k + j];
      out[4 * i + j] = s;
    }
}

// hat(v) into a row-major 3x3
__device__ __forceinline__ void hat3(const double *v, double *K) {
  K[0] = 0; K[1] = -v[2]; K[2] = v[1];
  K[3] = v[2]; K[4] = 0; K[5] = -v[0];
  K[6] = -v[1]; K[7] = v[0]; K[8] = 0;
}

__device__ __forceinline__ void mm3(const double *A, const double *B, double *C) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0;
      for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
      C[3 * i + j] = s;
    }
}

// SE(3) left Jacobian for xi = (rho, phi) (translation first), 6x6 row major:
// [[J(phi), Q(rho, phi)], [0, J(phi)]] with
// J = I + (1 - cos t)/t^2 P + (t - sin t)/t^3 P^2 and
// Q = 1/2 R + (t - sin t)/t^3 (PR + RP + PRP)
//     + (t^2 + 2 cos t - 2)/(2 t^4) (PPR + RPP - 3 PRP)
//     + (2t - 3 sin t + t cos t)/(2 t^5) (PRPP + PPRP),   P = phi^, R = rho^.
__device__ void se3_left_jacobian(const double *xi, double *J6) {
  const double *rho = xi, *phi = xi + 3;
  const double t2 = phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2], t = sqrt(t2);
  double a, b, c, d;
  if (t < 1e-3) {
    a = 0.5 - t2 / 24.0 + t2 * t2 / 720.0;
    b = 1.0 / 6.0 - t2 / 120.0 + t2 * t2 / 5040.0;
    c = 1.0 / 24.0 - t2 / 720.0 + t2 * t2 / 40320.0;
    d = 1.0 / 120.0 - t2 / 2520.0;
  } else {
    double sn, cs;
    sincos(t, &sn, &cs);
    a = (1.0 - cs) / t2;
    b = (t - sn) / (t2 * t);
    c = (t2 + 2.0 * cs - 2.0) / (2.0 * t2 * t2);
    d = (2.0 * t - 3.0 * sn + t * cs) / (2.0 * t2 * t2 * t);
  }
  double P[9], R[9], PP[9], PR[9], RP[9], PRP[9], PPR[9], RPP[9], PRPP[9], PPRP[9];
  hat3(phi, P);
  hat3(rho, R);
  mm3(P, P, PP);
  mm3(P, R, PR);
  mm3(R, P, RP);
  mm3(PR, P, PRP);
  mm3(PP, R, PPR);
  mm3(R, PP, RPP);
  mm3(PRP, P, PRPP);
  mm3(PP, RP, PPRP);
  for (int i = 0; i < 36; ++i) J6[i] = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const int k = 3 * i + j;
      const double I = i == j ? 1.0 : 0.0;
      const double Jr = I + a * P[k] + b * PP[k];
      const double Q = 0.5 * R[k] + b * (PR[k] + RP[k] + PRP[k]) +
                       c * (PPR[k] + RPP[k] - 3.0 * PRP[k]) + d * (PRPP[k] + PPRP[k]);
      J6[6 * i + j] = Jr;
      J6[6 * (i + 3) + (j + 3)] = Jr;
      J6[6 * i + (j + 3)] = Q;
    }
}

// out_k = T_k exp(xi_k^); jr_k (optional) = right Jacobian J_r(xi) = J_l(-xi).
__global__ void k_retract(const double *T, const double *xi, int n, double *out, double *jr) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  se3_right_dev(T + 16 * (long long)k, xi + 6 * (long long)k, out + 16 * (long long)k);
  if (jr) {
    double m[6];
    for (int u = 0; u < 6; ++u) m[u] = -xi[6 * (long long)k + u];
    se3_left_jacobian(m, jr + 36 * (long long)k);
  }
}

cudaError_t launch_retract(const double *T, const double *xi, int n, double *out, double *jr,
                           cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_retract<<<(n + 63) / 64, 64, 0, s>>>(T, xi, n, out, jr);
  return cudaGetLastError();
}

// out_k = scale_k J_r(xi_k)^T g_k: the chain rule from a gradient at T exp(xi^) to xi.
__global__ void k_twist_grad(const double *xi, const double *g, const double *scale, int n,
                             double *out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double m[6], J[36];
  for (int u = 0; u < 6; ++u) m[u] = -xi[6 * (long long)k + u];
  se3_left_jacobian(m, J);
  const double sc = scale ? scale[k] : 1.0;
  for (int c = 0; c < 6; ++c) {
    double acc = 0.0;
    for (int r = 0; r < 6; ++r) acc += J[6 * r + c] * g[6 * (long long)k + r];
    out[6 * (long long)k + c] = sc * acc;
  }
}

cudaError_t launch_twist_grad(const double *xi, const double *g, const double *scale, int n,
                              double *out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_twist_grad<<<(n + 63) / 64, 64, 0, s>>>(xi, g, scale, n, out);
  return cudaGetLastError();
}

// (H + lambda diag H) x = -g by Cholesky in FP64; false if not positive definite.
__device__ __noinline__ bool lm_solve_dev(const double *jtj, const double *g, double lambda, double *x) {
  double A[36], L[36];
  int q = 0;
  for (int u = 0; u < 6; ++u)
    for (int v = u; v < 6; ++v) {
      A[6 * u + v] = jtj[q];
      A[6 * v + u] = jtj[q];
      ++q;
    }
  for (int u = 0; u < 36; ++u) L[u] = 0.0;
  for (int u = 0; u < 6; ++u) A[7 * u] += lambda * A[7 * u];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j <= i; ++j) {
      double s = A[6 * i + j];
      for (int k = 0; k < j; ++k) s -= L[6 * i + k] * L[6 * j + k];
      if (i == j) {
        if (!(s > 0.0)) return false;
        L[7 * i] = sqrt(s);
      } else {
        L[6 * i + j] = s / L[7 * j];
      }
    }
  double y[6];
  for (int i = 0; i < 6; ++i) {
    double s = -g[i];
    for (int k = 0; k < i; ++k) s -= L[6 * i + k] * y[k];
    y[i] = s / L[7 * i];
  }
  for (int i = 5; i >= 0; --i) {
    double s = y[i];
    for (int k = i + 1; k < 6; ++k) s -= L[6 * k + i] * x[k];
    x[i] = s / L[7 * i];
  }
  return true;
}

__device__ __noinline__ void lm_take_initial_dev(LMState &st, const long long *counts, const double *els,
                                    const double *grad, const double *jtj) {
  st.e = els[0];
  st.e_ls0 = els[0];
  for (int k = 0; k < 6; ++k) st.g[k] = grad[k];
  for (int k = 0; k < 21; ++k) st.H[k] = jtj[k];
  st.e_table = (counts[1] + counts[3] + counts[5]) - (counts[0] + counts[2] + counts[4]);
  st.e_table0 = st.e_table;
}

// Solve for the next step; writes the candidate's matrix and clears *skip, or sets *skip when
// there is nothing to evaluate (converged, or a damped system that is not positive definite).
__device__ __noinline__ void lm_propose_dev(LMState &st, const LMArgs &a, float *M, int *skip) {
  if (st.done) {
    *skip = 1;
    return;
  }
  double dx[6];
  if (!lm_solve_dev(st.H, st.g, st.lambda, dx)) {
    st.lambda *= a.lambda_up;
    st.iters += 1;
    *skip = 1;
    return;
  }
  double nrm = 0.0;
  for (int k = 0; k < 6; ++k) nrm += dx[k] * dx[k];
  if (sqrt(nrm) < a.step_tol) {
    st.done = 1;
    st.converged = 1;
    *skip = 1;
    return;
  }
  se3_right_dev(st.T, dx, st.Tc);
  pose_to_m(st.Tc, a.cx, a.cy, a.cz, M);
  *skip = 0;
}

// Accept the evaluated candidate if it lowered the surrogate (nothing when it was skipped).
__device__ __noinline__ void lm_accept_dev(LMState &st, const LMArgs &a, const long long *counts,
                              const double *els, const double *grad, const double *jtj,
                              bool was_skipped) {
  if (was_skipped) return;
  st.iters += 1;
  if (els[0] < st.e) {
    for (int k = 0; k < 16; ++k) st.T[k] = st.Tc[k];
    st.e = els[0];
    for (int k = 0; k < 6; ++k) st.g[k] = grad[k];
    for (int k = 0; k < 21; ++k) st.H[k] = jtj[k];
    st.e_table = (counts[1] + counts[3] + counts[5]) - (counts[0] + counts[2] + counts[4]);
    st.lambda /= a.lambda_down;
    st.accepted += 1;
  } else {
    st.lambda *= a.lambda_up;
  }
}

__device__ void lm_init_dev(LMState &st, const double *T0, const LMArgs &a, float *M, int *skip) {
  for (int k = 0; k < 16; ++k) st.T[k] = st.Tc[k] = T0[k];
  st.lambda = a.lambda0;
  st.iters = st.accepted = st.converged = st.done = 0;
  st.have_candidate = 1;
  pose_to_m(T0, a.cx, a.cy, a.cz, M);
  *skip = 0;
}

__global__ void k_lm_init(LMState *st, const double *T0, LMArgs a, float *M, int *skip) {
  lm_init_dev(*st, T0, a, M, skip);
}

__global__ void k_lm_take_initial(LMState *st, const long long *counts, const double *els,
                                  const double *grad, const double *jtj) {
  lm_take_initial_dev(*st, counts, els, grad, jtj);
}

__global__ void k_lm_propose(LMState *st, LMArgs a, float *M, int *skip) {
  lm_propose_dev(*st, a, M, skip);
}

__global__ void k_lm_accept(LMState *st, LMArgs a, const long long *counts, const double *els,
                            const double *grad, const double *jtj, int *skip) {
  lm_accept_dev(*st, a, counts, els, grad, jtj, *skip != 0);
}

// ------------------------------------------------------------------ point-to-plane ICP

__device__ void icp_init_dev(IcpState &st, const double *T0, const IcpArgs &a, float *M, int *skip) {
  for (int k = 0; k < 16; ++k) st.T[k] = T0[k];
  st.l1_0 = st.l1 = 0.0;
  st.n_assoc = 0;
  st.iters = st.converged = st.done = st.evals = 0;
  pose_to_m(T0, a.cx, a.cy, a.cz, M);
  *skip = 0;
}

__global__ void k_icp_init(IcpState *st, const double *T0, IcpArgs a, float *M, int *skip) {
  icp_init_dev(*st, T0, a, M, skip);
}

// Gauss-Newton step of point-to-plane ICP: J^T J dx = -J^T e (Cholesky, no damping), then
// T <- T exp(dx^). A system that is not positive definite ends the iterations unconverged.
__device__ __noinline__ void icp_step_dev(IcpState &s, const IcpArgs &a, const long long *n,
                                          const double *l1, const double *g, const double *H,
                                          float *M, int *skip) {
  if (s.done) {
    *skip = 1;
    return;
  }
  s.n_assoc = n[0];
  s.l1 = l1[0];
  if (s.evals == 0) s.l1_0 = l1[0];
  s.evals += 1;
  double dx[6];
  if (!lm_solve_dev(H, g, 0.0, dx)) {
    s.done = 1;
    *skip = 1;
    return;
  }
  double Tn[16];
  se3_right_dev(s.T, dx, Tn);
  for (int k = 0; k < 16; ++k) s.T[k] = Tn[k];
  s.iters += 1;
  double nrm = 0.0;
  for (int k = 0; k < 6; ++k) nrm += dx[k] * dx[k];
  if (sqrt(nrm) < a.step_tol) {
    s.converged = 1;
    s.done = 1;
    *skip = 1;
    return;
  }
  pose_to_m(s.T, a.cx, a.cy, a.cz, M);
  *skip = 0;
}

__global__ void k_icp_step(IcpState *st, IcpArgs a, const long long *n, const double *l1,
                           const double *g, const double *H, float *M, int *skip) {
  icp_step_dev(*st, a, n, l1, g, H, M, skip);
}

__global__ void k_icp_init_batch(IcpState *st, const double *T0, int n, IcpArgs a, float *Ms,
                                 int *skip) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) icp_init_dev(st[k], T0 + 16 * (long long)k, a, Ms + 12 * (long long)k, skip + k);
}

cudaError_t launch_icp_init_batch(IcpState *st, const double *T0, int n, const IcpArgs &a,
                                  float *Ms, int *skip, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_icp_init_batch<<<(n + 63) / 64, 64, 0, s>>>(st, T0, n, a, Ms, skip);
  return cudaGetLastError();
}

cudaError_t launch_icp_init(IcpState *st, const double *T0, const IcpArgs &a, float *M,
                            int *skip, cudaStream_t s) {
  k_icp_init<<<1, 1, 0, s>>>(st, T0, a, M, skip);
  return cudaGetLastError();
}

cudaError_t launch_icp_step(IcpState *st, const IcpArgs &a, const long long *n,
                            const double *l1, const double *g, const double *H, float *M,
                            int *skip, cudaStream_t s) {
  k_icp_step<<<1, 1, 0, s>>>(st, a, n, l1, g, H, M, skip);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ derivative-free search

// Vertex order by value, ties by slot (stable insertion sort).
__device__ void dfo_order(const double *f, int *o) {
  for (int i = 0; i < 7; ++i) o[i] = i;
  for (int i = 1; i < 7; ++i)
    for (int j = i; j > 0 && f[o[j]] < f[o[j - 1]]; --j) {
      const int t = o[j];
      o[j] = o[j - 1];
      o[j - 1] = t;
    }
}

// Coordinate descent: converged, out of iterations, or the 12 moves +-step per axis.
__device__ void dfo_next_cd(DfoState &s, const DfoArgs &a) {
  if (s.cd_iters >= a.cd_iters) {
    s.phase = 4;
    return;
  }
  double smax = 0.0;
  for (int k = 0; k < 6; ++k) smax = fmax(smax, s.st[k] / a.scale[k]);
  if (smax < a.cd_tol) {
    s.converged = 1;
    s.phase = 4;
    return;
  }
  for (int m = 0; m < 12; ++m)
    for (int k = 0; k < 6; ++k)
      s.cand[m][k] = s.xc[k] + (k == m / 2 ? (m % 2 ? -s.st[k] : s.st[k]) : 0.0);
  s.n_cand = 12;
  s.phase = 3;
}

// Next Nelder-Mead iteration (the four candidates), or the switch to coordinate descent.
__device__ void dfo_next_nm(DfoState &s, const DfoArgs &a) {
  int o[7];
  dfo_order(s.f, o);
  double diam = 0.0;
  for (int i = 1; i < 7; ++i)
    for (int k = 0; k < 6; ++k) diam = fmax(diam, fabs(s.x[o[i]][k] - s.x[o[0]][k]) / a.scale[k]);
  if (s.nm_iters >= a.nm_iters || diam < a.nm_tol) {
    for (int k = 0; k < 6; ++k) {
      s.xc[k] = s.x[o[0]][k];
      s.st[k] = a.cd_step * a.scale[k];
    }
    s.fcur = s.f[o[0]];
    dfo_next_cd(s, a);
    return;
  }
  const int h = o[6];
  for (int k = 0; k < 6; ++k) {
    double sum = 0.0;
    for (int i = 0; i < 6; ++i) sum += s.x[o[i]][k];
    const double c = sum / 6.0, d = c - s.x[h][k];
    s.cand[0][k] = c + d;
    s.cand[1][k] = c + 2.0 * d;
    s.cand[2][k] = c + 0.5 * d;
    s.cand[3][k] = c - 0.5 * d;
  }
  s.n_cand = 4;
  s.phase = 1;
}

// Powell's line search from xc along d: the 12 points xc + (a step) d, products and sums
// rounded separately (no contraction), so the candidates equal the oracle's bit for bit.
__constant__ double kPowellA[12] = {0.25, -0.25, 0.5, -0.5, 1.0, -1.0, 2.0, -2.0, 4.0, -4.0, 8.0, -8.0};

__device__ void powell_line(DfoState &s, const double *d, double step) {
  for (int m = 0; m < 12; ++m) {
    const double am = __dmul_rn(kPowellA[m], step);
    for (int k = 0; k < 6; ++k) s.cand[m][k] = __dadd_rn(s.xc[k], __dmul_rn(am, d[k]));
  }
  s.n_cand = 12;
  s.phase = 6;
}

// The next Powell iteration (its first axis search), or the switch to coordinate descent from
// Powell's end point once out of iterations or below the step tolerance.
__device__ void powell_next(DfoState &s, const DfoArgs &a) {
  if (s.powell_iters >= a.powell_iters || !(s.ps >= a.powell_tol)) {
    for (int k = 0; k < 6; ++k) s.st[k] = a.cd_step * a.scale[k];
    dfo_next_cd(s, a);
    return;
  }
  for (int k = 0; k < 6; ++k) s.x0[k] = s.xc[k];
  s.best_drop = 0.0;
  s.best_dir = 0;
  s.pdir = 0;
  powell_line(s, s.D[0], s.ps);
}

// One finished Powell line search: take its lowest point if it lowers the value, then the
// next direction, the displacement search, or the next iteration.
__device__ void powell_step(DfoState &s, const DfoArgs &a, const double *fc) {
  int best = 0;
  for (int m = 1; m < 12; ++m)
    if (fc[m] < fc[best]) best = m;
  double drop = 0.0;
  if (fc[best] < s.fcur) {
    drop = s.fcur - fc[best];
    for (int k = 0; k < 6; ++k) s.xc[k] = s.cand[best][k];
    s.fcur = fc[best];
  }
  if (s.pdir == 6) {  // the displacement search: replace the direction of largest decrease
    const double n = __dsqrt_rn(s.n2);
    for (int k = 0; k < 6; ++k) s.D[s.best_dir][k] = __ddiv_rn(s.disp[k], n);
    powell_next(s, a);
    return;
  }
  if (drop > s.best_drop) {
    s.best_drop = drop;
    s.best_dir = s.pdir;
  }
  s.pdir += 1;
  if (s.pdir < 6) {
    powell_line(s, s.D[s.pdir], s.ps);
    return;
  }
  s.powell_iters += 1;
  double n2 = 0.0;
  for (int k = 0; k < 6; ++k) {
    s.disp[k] = __dsub_rn(s.xc[k], s.x0[k]);
    const double u = __ddiv_rn(s.disp[k], a.scale[k]);
    n2 = __dadd_rn(n2, __dmul_rn(u, u));
  }
  if (n2 == 0.0) {
    s.ps = 0.5 * s.ps;
    powell_next(s, a);
    return;
  }
  s.n2 = n2;
  s.pdir = 6;
  powell_line(s, s.disp, 1.0);
}

__device__ void dfo_write_candidates(DfoState &s, const DfoArgs &a, float *Ms) {
  for (int m = 0; m < kDfoSlots; ++m) {
    double T[16];
    se3_right_dev(s.T0, s.cand[m < s.n_cand ? m : 0], T);
    pose_to_m(T, a.cx, a.cy, a.cz, Ms + 12 * m);
  }
}

__global__ void k_dfo_init(DfoState *st, const double *T0, DfoArgs a, float *Ms, int *skip) {
  DfoState &s = *st;
  for (int k = 0; k < 16; ++k) s.T0[k] = T0[k];
  s.evals = s.nm_iters = s.nm_shrinks = s.cd_iters = s.converged = s.shrink_best = 0;
  s.powell_iters = 0;
  if (a.method == 1) {  // Powell: the origin first; directions are the scaled axes
    for (int i = 0; i < 6; ++i)
      for (int k = 0; k < 6; ++k) s.D[i][k] = i == k ? a.scale[k] : 0.0;
    for (int k = 0; k < 6; ++k) s.cand[0][k] = s.xc[k] = 0.0;
    s.ps = a.powell_step;
    s.n_cand = 1;
    s.phase = 5;
    dfo_write_candidates(s, a, Ms);
    *skip = 0;
    return;
  }
  for (int i = 0; i < 7; ++i)
    for (int k = 0; k < 6; ++k) s.cand[i][k] = (i >= 1 && k == i - 1) ? a.nm_step * a.scale[k] : 0.0;
  s.n_cand = 7;
  s.phase = 0;
  dfo_write_candidates(s, a, Ms);
  *skip = 0;
}

__global__ void k_dfo_step(DfoState *st, DfoArgs a, const long long *et, float *Ms, int *skip) {
  DfoState &s = *st;
  if (s.phase == 4) {
    *skip = 1;
    return;
  }
  double fc[kDfoSlots];
  for (int m = 0; m < s.n_cand; ++m) fc[m] = (double)et[m];
  s.evals += s.n_cand;
  if (s.phase == 0) {
    s.f_init = fc[0];
    for (int i = 0; i < 7; ++i) {
      for (int k = 0; k < 6; ++k) s.x[i][k] = s.cand[i][k];
      s.f[i] = fc[i];
    }
    dfo_next_nm(s, a);
  } else if (s.phase == 1) {
    s.nm_iters += 1;
    int o[7];
    dfo_order(s.f, o);
    const int h = o[6];
    const double fb = s.f[o[0]], fs = s.f[o[5]], fh = s.f[h];
    int take;
    if (fc[0] < fb) take = fc[1] < fc[0] ? 1 : 0;
    else if (fc[0] < fs) take = 0;
    else if (fc[0] < fh) take = fc[2] <= fc[0] ? 2 : -1;
    else take = fc[3] < fh ? 3 : -1;
    if (take >= 0) {
      for (int k = 0; k < 6; ++k) s.x[h][k] = s.cand[take][k];
      s.f[h] = fc[take];
      dfo_next_nm(s, a);
    } else {
      const int b = o[0];
      int m = 0;
      for (int i = 0; i < 7; ++i) {
        if (i == b) continue;
        for (int k = 0; k < 6; ++k) s.cand[m][k] = s.x[b][k] + 0.5 * (s.x[i][k] - s.x[b][k]);
        ++m;
      }
      s.shrink_best = b;
      s.n_cand = 6;
      s.phase = 2;
    }
  } else if (s.phase == 2) {
    s.nm_shrinks += 1;
    int m = 0;
    for (int i = 0; i < 7; ++i) {
      if (i == s.shrink_best) continue;
      for (int k = 0; k < 6; ++k) s.x[i][k] = s.cand[m][k];
      s.f[i] = fc[m];
      ++m;
    }
    dfo_next_nm(s, a);
  } else if (s.phase == 5) {
    s.f_init = s.fcur = fc[0];
    powell_next(s, a);
  } else if (s.phase == 6) {
    powell_step(s, a, fc);
  } else {
    s.cd_iters += 1;
    int best = 0;
    for (int m = 1; m < 12; ++m)
      if (fc[m] < fc[best]) best = m;
    if (fc[best] < s.fcur) {
      for (int k = 0; k < 6; ++k) s.xc[k] = s.cand[best][k];
      s.fcur = fc[best];
    } else {
      for (int k = 0; k < 6; ++k) s.st[k] *= 0.5;
    }
    dfo_next_cd(s, a);
  }
  if (s.phase == 4) {
    *skip = 1;
    return;
  }
  dfo_write_candidates(s, a, Ms);
  *skip = 0;
}

cudaError_t launch_dfo_init(DfoState *st, const double *T0, const DfoArgs &a, float *Ms,
                            int *skip, cudaStream_t s) {
  k_dfo_init<<<1, 1, 0, s>>>(st, T0, a, Ms, skip);
  return cudaGetLastError();
}

cudaError_t launch_dfo_step(DfoState *st, const DfoArgs &a, const long long *e_table, float *Ms,
                            int *skip, cudaStream_t s) {
  k_dfo_step<<<1, 1, 0, s>>>(st, a, e_table, Ms, skip);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ persistent batch kernel

__global__ void k_lm_init_batch(LMState *st, const double *T0, int n, LMArgs a, float *Ms,
                                int *skip) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) lm_init_dev(st[k], T0 + 16 * (long long)k, a, Ms + 12 * (long long)k, skip + k);
}

// Phase bodies of the persistent kernel, each compiled out of line so that its register
// allocation is its own (as in the per-phase kernels) rather than the union of all phases.
__device__ __noinline__ void persist_cull(const WaveArgs *__restrict__ pa, int item, float *sM) {
  const WaveArgs &a = *pa;
  const int c1 = min((item + 1) * kPersistCull, (a.n_clusters + 255) / 256);
  for (int c = item * kPersistCull; c < c1; ++c) {
    cull_block(a, 0, c, sM);
    __syncthreads();
  }
}

template <int MODEL>
__device__ __noinline__ void persist_setup(const WaveArgs *__restrict__ pa, int worker, int nworkers,
                                           SetupSmem &sm) {
  const WaveArgs &a = *pa;
  setup_block<MODEL>(a, 0, worker, nworkers, sm);
}

template <int MODEL>
__device__ __noinline__ void persist_raster(
    const WaveArgs *__restrict__ pa, int item, RasterSmem<kPersistTileW[MODEL] * kPersistTileH[MODEL], MODEL> &sm) {
  const WaveArgs &a = *pa;
  const int t1 = min((item + 1) * kPersistTiles[MODEL], a.tg.ntiles);
  for (int t = item * kPersistTiles[MODEL]; t < t1; ++t) {
    raster_block<kPersistTileW[MODEL], kPersistTileH[MODEL], kCostGrad, MODEL>(a, t, 0, sm);
    __syncthreads();
  }
}

template <int MODEL>
__device__ __noinline__ void persist_raster_icp(
    const WaveArgs *__restrict__ pa, int item, RasterSmem<kPersistTileW[MODEL] * kPersistTileH[MODEL], MODEL> &sm) {
  const WaveArgs &a = *pa;
  const int t1 = min((item + 1) * kPersistTiles[MODEL], a.tg.ntiles);
  for (int t = item * kPersistTiles[MODEL]; t < t1; ++t) {
    if (a.vnormals) raster_block<kPersistTileW[MODEL], kPersistTileH[MODEL], kIcpVn, MODEL>(a, t, 0, sm);
    else raster_block<kPersistTileW[MODEL], kPersistTileH[MODEL], kIcp, MODEL>(a, t, 0, sm);
    __syncthreads();
  }
}

__device__ __noinline__ void persist_reduce(const WaveArgs *__restrict__ pa, double *vals) {
  const WaveArgs &a = *pa;
  reduce_block(a, 0, vals);
}

// Copies an LM state with L2 loads (another SM may have written it during this kernel).
__device__ __noinline__ void lm_load_cg(const LMState *src, LMState &dst) {
  const long long *s = reinterpret_cast<const long long *>(src);
  long long *d = reinterpret_cast<long long *>(&dst);
  for (int k = 0; k < (int)(sizeof(LMState) / 8); ++k) d[k] = __ldcg(s + k);
}

// A load with acquire semantics at GPU scope: later loads see what the writer released.
__device__ __forceinline__ long long ld_acquire_gpu(const long long *p) {
  long long v;
  asm volatile("ld.acquire.gpu.global.s64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Orders this thread's earlier memory operations before its later ones at GPU scope (with a
// relaxed write after it: a release; with a relaxed read before it: an acquire).
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

__device__ __forceinline__ int4 unpack_item(long long v) {
  return make_int4((int)(v >> 40), (int)(v >> 21) & 3, (int)v & ((1 << kItemIndexBits) - 1),
                   (int)(v >> 23) & ((1 << kItemEvalBits) - 1));
}

// Claims the next slot of a queue that looks non-empty (one atomic add), or returns -1. Two
// CTAs racing for its last item can both claim; the later one then waits for the queue's next
// publication, or for the end of the batch.
__device__ __forceinline__ int claim_slot(int *head, const int *tail) {
  if (*(volatile const int *)head >= *(volatile const int *)tail) return -1;
  return atomicAdd(head, 1);
}

// One launch runs every phase of every problem of a batch (and, with LM, every iteration).
// Items enter a ready queue only once they can run: the launch starts with the evaluation-0
// cull items of every problem, and the CTA that completes the last item of a problem's phase
// appends the next phase (cull -> setup -> raster -> reduce and LM step -> the next
// evaluation's cull). The number of setup items follows the visible-cluster count of that
// evaluation. Raster and reduce items go to a queue that is served first, so problems that
// have reached their raster finish their evaluation before new ones start theirs. A CTA takes
// only slots that have been reserved by a publisher (whose write is then at most a few
// instructions away) and exits once every problem has finished; with nothing to take it
// sleeps and retries (bounded).
// Thread 0 of a CTA: claims the next ready item of the batch's queues into *s_item (x < 0:
// every problem has finished) and sets *s_abort when a wait ran out of its budget.
__device__ __forceinline__ void persist_claim(const BatchArgs &b, int4 *s_item, int *s_abort) {
  int4 item = make_int4(-1, 0, 0, 0);
  int abort = 0;
  const long long t0 = clock64();
  unsigned ns = 32;
  for (;;) {
    // a claim past a queue's capacity (racing claims at its very end) holds no slot
    int slot = claim_slot(b.qctl + 0, b.qctl + 1);
    if (slot >= b.cap[0]) slot = -1;
    if (slot < 0) {
      slot = claim_slot(b.qctl + 2, b.qctl + 3);
      slot = slot >= b.cap[1] ? -1 : (slot >= 0 ? slot + b.cap[0] : -1);
    }
    if (slot >= 0) {
      long long x;
      bool finished = false;
      while ((x = ld_acquire_gpu(b.items + slot)) < 0) {
        if (*(volatile const int *)(b.qctl + 4) >= b.n_problems) {  // nothing more will come
          finished = true;
          break;
        }
        if (clock64() - t0 > b.spin_limit) break;
        __nanosleep(64);
      }
      if (finished) break;
      if (x < 0) {
        atomicOr(b.status, kStatusTimeout);
        abort = 1;
        break;
      }
      item = unpack_item(x);
      break;
    }
    if (*(volatile const int *)(b.qctl + 4) >= b.n_problems) break;  // all finished
    if (clock64() - t0 > b.spin_limit) {
      atomicOr(b.status, kStatusTimeout);
      abort = 1;
      break;
    }
    __nanosleep(ns);
    if (ns < 1024) ns *= 2;
  }
  *s_item = item;
  *s_abort = abort;
}

// Thread 0 of a CTA, after `item` is done: counts it, and when it was its problem's last item
// of a phase, reserves the next phase's slots (the setup phase sized by *vis_count, the
// problem's visible clusters, clusters_per_item to an item). Returns (phase, count, first
// slot, evaluation); count 0: none.
__device__ __forceinline__ int4 persist_complete(const BatchArgs &b, int4 item, const int *vis_count,
                                                 int clusters_per_item) {
  fence_acq_rel_gpu();  // the CTA's results (after its barrier) before the count
  const int p = item.x, ph = item.y, it = item.w;
  int4 eq = make_int4(0, 0, -1, it);  // phase, count, queue, evaluation
  if (ph < 3) {
    const int c = atomicAdd(b.done + 4 * p + ph, 1) + 1;
    if (c == __ldcg(b.need + 3 * p + ph)) {
      if (ph == 0) {
        // all cull items are in: size the setup phase by the visible clusters
        const int nv = __ldcg(vis_count);
        const int nsetup = max(1, (nv + clusters_per_item - 1) / clusters_per_item);
        b.need[3 * p + 1] = nsetup;
        eq = make_int4(1, nsetup, 1, it);
      } else if (ph == 1) {
        eq = make_int4(2, b.need[3 * p + 2], 0, it);
      } else {
        eq = make_int4(3, 1, 0, it);
      }
    }
  } else if ((b.lm || b.icp) && it < b.lm_iters) {
    b.done[4 * p + 0] = 0;
    b.done[4 * p + 1] = 0;
    b.done[4 * p + 2] = 0;
    eq = make_int4(0, b.need[3 * p], 1, it + 1);
  } else {
    atomicAdd(b.qctl + 4, 1);  // the problem is finished
  }
  if (eq.y > 0) {
    const int q = eq.z;
    const int first = atomicAdd(b.qctl + 2 * q + 1, eq.y);
    if (first + eq.y > b.cap[q]) atomicOr(b.status, kStatusQueue);  // cannot happen
    eq.z = (q == 0 ? 0 : b.cap[0]) + first;
    eq.y = max(0, min(eq.y, b.cap[q] - first));
  }
  return eq;
}

// All threads of a CTA: publish the reserved successor slots, each with one 64-bit write after
// a fence (which also orders what thread 0 observed of the completion counts).
__device__ __forceinline__ void persist_publish(const BatchArgs &b, int4 eq, int problem) {
  if (eq.y > 0) {
    fence_acq_rel_gpu();
    __syncthreads();
    for (int k = threadIdx.x; k < eq.y; k += blockDim.x)
      atomicExch(reinterpret_cast<unsigned long long *>(b.items + eq.z + k),
                 (unsigned long long)pack_item(problem, eq.x, k, eq.w));
  }
}

__global__ void __launch_bounds__(kThreads, RM_PERSIST_MIN_BLOCKS) k_persist(BatchArgs b) {
  union PersistSmem {
    RasterSmem<kPersistTileW[0] * kPersistTileH[0], 0> r0;
    RasterSmem<kPersistTileW[1] * kPersistTileH[1], 1> r1;
    SetupSmem su;
    double vals[kNumVals];
  };
  __shared__ PersistSmem u;
  __shared__ float s_M[12];
  __shared__ int4 s_item;
  __shared__ int4 s_enq;       // successors to publish: phase, count, first slot, evaluation
  __shared__ int s_abort;
  for (;;) {
    if (threadIdx.x == 0) persist_claim(b, &s_item, &s_abort);
    __syncthreads();
    const int4 item = s_item;
    if (item.x < 0 || s_abort) break;
    // the problem's argument block: written before the launch and read-only during it, so
    // the phases read it in place through the read-only data path
    const WaveArgs *__restrict__ pa = b.probs + item.x;
    const WaveArgs &a = *pa;
    const bool skip = skipped(a);
    if (!skip) {
      switch (item.y) {
        case 0: persist_cull(pa, item.z, s_M); break;
        case 1:
          if (a.cam.model == 0) persist_setup<0>(pa, item.z, __ldcg(b.need + 3 * item.x + 1), u.su);
          else persist_setup<1>(pa, item.z, __ldcg(b.need + 3 * item.x + 1), u.su);
          break;
        case 2:
          if (b.icp) {
            if (a.cam.model == 0) persist_raster_icp<0>(pa, item.z, u.r0);
            else persist_raster_icp<1>(pa, item.z, u.r1);
          } else {
            if (a.cam.model == 0) persist_raster<0>(pa, item.z, u.r0);
            else persist_raster<1>(pa, item.z, u.r1);
          }
          break;
        default: persist_reduce(pa, u.vals); break;
      }
    }
    if (item.y == 3 && b.icp) {
      // ICP: every evaluation is followed by a Gauss-Newton step (a no-op once done)
      __syncthreads();
      const int p = item.x, it = item.w;
      if (threadIdx.x == 0) {
        IcpState st = b.icp[p];
        icp_step_dev(st, b.icpargs, a.res_n, a.res_l1, a.res_grad, a.res_jtj, b.Ms + 12 * (long long)p,
                     b.skip + p);
        b.icp[p] = st;
      }
      if (it < b.lm_iters) {
        for (int t = threadIdx.x; t < a.tg.ntiles; t += blockDim.x) a.counts[t] = 0;
        if (threadIdx.x == 0) a.vis_count[0] = 0;
      }
    }
    if (item.y == 3 && b.lm) {
      __syncthreads();
      const int p = item.x, it = item.w;
      if (threadIdx.x == 0) {
        LMState st;
        lm_load_cg(b.lm + p, st);
        if (it == 0) lm_take_initial_dev(st, a.res_counts, a.res_els, a.res_grad, a.res_jtj);
        else lm_accept_dev(st, b.lmargs, a.res_counts, a.res_els, a.res_grad, a.res_jtj, skip);
        if (it < b.lm_iters) lm_propose_dev(st, b.lmargs, b.Ms + 12 * (long long)p, b.skip + p);
        b.lm[p] = st;
      }
      if (it < b.lm_iters) {  // the next evaluation starts from empty lists and bins
        for (int t = threadIdx.x; t < a.tg.ntiles; t += blockDim.x) a.counts[t] = 0;
        if (threadIdx.x == 0) a.vis_count[0] = 0;
      }
    }
    __syncthreads();
    // completion; the last item of the problem's phase publishes the successors
    if (threadIdx.x == 0) s_enq = persist_complete(b, item, a.vis_count, setup_clusters(a.cam.model));
    __syncthreads();
    persist_publish(b, s_enq, item.x);
  }
}

// The persistent kernel for a homogeneous batch (every problem the same camera, scan and
// parameters, a plain evaluation): the problems are the poses of one wave, whose arguments
// are a kernel parameter, so the phases (inlined) read them as the per-wave kernels do and the
// kernel fits the per-wave raster's register budget. Same queue, items and results as
// k_persist.
#ifndef RM_PERSIST_WAVE_MIN_BLOCKS
#define RM_PERSIST_WAVE_MIN_BLOCKS 5
#endif

template <int MODEL>
__global__ void __launch_bounds__(kThreads, MODEL == 0 ? RM_PERSIST_WAVE_MIN_BLOCKS : 4)
    k_persist_wave(BatchArgs b, WaveArgs w) {
  constexpr int TW = kPersistTileW[MODEL], TH = kPersistTileH[MODEL];
  union PersistWaveSmem {
    RasterSmem<TW * TH, MODEL> r;
    SetupSmem su;
    double vals[kNumVals];
  };
  __shared__ PersistWaveSmem u;
  __shared__ float s_M[12];
  __shared__ int4 s_item;
  __shared__ int4 s_enq;
  __shared__ int s_abort;
  for (;;) {
    if (threadIdx.x == 0) persist_claim(b, &s_item, &s_abort);
    __syncthreads();
    const int4 item = s_item;
    if (item.x < 0 || s_abort) break;
    const int q = item.x;  // the problem is pose q of the wave
    switch (item.y) {
      case 0: {
        const int c1 = min((item.z + 1) * kPersistCull, (w.n_clusters + 255) / 256);
        for (int c = item.z * kPersistCull; c < c1; ++c) {
          cull_block(w, q, c, s_M);
          __syncthreads();
        }
        break;
      }
      case 1: setup_block<MODEL>(w, q, item.z, __ldcg(b.need + 3 * q + 1), u.su); break;
      case 2: {
        const int t1 = min((item.z + 1) * kPersistTiles[MODEL], w.tg.ntiles);
        for (int t = item.z * kPersistTiles[MODEL]; t < t1; ++t) {
          raster_block<TW, TH, kCostGrad, MODEL>(w, t, q, u.r);
          __syncthreads();
        }
        break;
      }
      default: reduce_block(w, q, u.vals); break;
    }
    __syncthreads();
    if (threadIdx.x == 0) s_enq = persist_complete(b, item, w.vis_count + q, setup_clusters(MODEL));
    __syncthreads();
    persist_publish(b, s_enq, item.x);
  }
}

__global__ void k_queue_init(long long *items, int n_slots, int first_low, int n_problems,
                             int cull_items, int *qctl) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int n0 = n_problems * cull_items;
  if (k < n_slots) {
    const int c = k - first_low;
    items[k] = c >= 0 && c < n0 ? pack_item(c / cull_items, 0, c % cull_items, 0) : -1ll;
  }
  if (k == 0) qctl[3] = n0;
}

cudaError_t launch_queue_init(long long *items, int n_slots, int first_low, int n_problems,
                              int cull_items, int *qctl, cudaStream_t s) {
  k_queue_init<<<(n_slots + 255) / 256, 256, 0, s>>>(items, n_slots, first_low, n_problems,
                                                     cull_items, qctl);
  return cudaGetLastError();
}

cudaError_t launch_lm_init_batch(LMState *st, const double *T0, int n, const LMArgs &a,
                                 float *Ms, int *skip, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_lm_init_batch<<<(n + 63) / 64, 64, 0, s>>>(st, T0, n, a, Ms, skip);
  return cudaGetLastError();
}

cudaError_t launch_persist(const BatchArgs &b, int grid, cudaStream_t s) {
  k_persist<<<grid, kThreads, 0, s>>>(b);
  return cudaGetLastError();
}

cudaError_t launch_persist_wave(const BatchArgs &b, const WaveArgs &w, int grid, cudaStream_t s) {
  if (w.cam.model == 0) k_persist_wave<0><<<grid, kThreads, 0, s>>>(b, w);
  else k_persist_wave<1><<<grid, kThreads, 0, s>>>(b, w);
  return cudaGetLastError();
}

int persist_wave_grid(int device, int model) {
  int sms = 0, per = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
  const cudaError_t e = model == 0 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_persist_wave<0>, kThreads, 0)
                                   : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_persist_wave<1>, kThreads, 0);
  if (e != cudaSuccess) return 0;
  return sms * (per > 0 ? per : 1);
}

int persist_grid(int device) {
  int sms = 0, per = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_persist, kThreads, 0) != cudaSuccess) return 0;
  return sms * (per > 0 ? per : 1);
}

cudaError_t launch_lm_init(LMState *st, const double *T0, const LMArgs &a, float *M, int *skip,
                           cudaStream_t s) {
  k_lm_init<<<1, 1, 0, s>>>(st, T0, a, M, skip);
  return cudaGetLastError();
}
cudaError_t launch_lm_take_initial(LMState *st, const long long *counts, const double *els,
                                   const double *grad, const double *jtj, cudaStream_t s) {
  k_lm_take_initial<<<1, 1, 0, s>>>(st, counts, els, grad, jtj);
  return cudaGetLastError();
}
cudaError_t launch_lm_propose(LMState *st, const LMArgs &a, float *M, int *skip, cudaStream_t s) {
  k_lm_propose<<<1, 1, 0, s>>>(st, a, M, skip);
  return cudaGetLastError();
}
cudaError_t launch_lm_accept(LMState *st, const LMArgs &a, const long long *counts,
                             const double *els, const double *grad, const double *jtj, int *skip,
                             cudaStream_t s) {
  k_lm_accept<<<1, 1, 0, s>>>(st, a, counts, els, grad, jtj, skip);
  return cudaGetLastError();
}

}  // namespace rmk
