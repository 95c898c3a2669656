// rm_internal.cuh -- device-side data layout and the FP32 rasterisation contract.
//
// The z-buffer of Sec. IV (R(Y) in Eq. 1) must pick, for every pixel, exactly the triangle
// the CPU reference picks. Every step that feeds coverage or the depth key therefore uses
// IEEE round-to-nearest intrinsics in a fixed order (no contraction left to the compiler):
//   vertex:   X = fma(M00, x, fma(M01, y, fma(M02, z, M03)))        (rows 1, 2 alike)
//   project:  xs = fma(fx, X / Z, cx); xi = rint(xs * 256)           (8 sub-pixel bits)
//   near cut: s = (near - a.z) / (b.z - a.z), a = lower vertex index; P = a + s (b - a)
//   plane:    n = (v1 - v0) x (v2 - v0), d = n . v0 (camera frame, stored vertex order)
//   inverse depth (affine in the image, like a GPU z-buffer value, Sec. V):
//             pinhole  w = fma(Ai, i + .5, fma(Bi, j + .5, Ci)), Ai = A / d, Bi = B / d,
//                      Ci = C / d with A = nx/fx, B = ny/fy, C = fma(-A, cx, fma(-B, cy, nz));
//             ray table w = fma(nx/d, rx, fma(ny/d, ry, (nz/d) rz))
//   key:      (~bits(w) << 32) | triangle id, kept iff 0 < w, 1/far <= w <= 1/near (FP32
//             bounds), minimum key wins (nearest, then lowest id); depth t = 1 / w.
// Coverage is decided on the snapped integer coordinates with int64 edge functions and
// the top-left rule, so it is exact.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rmk {

constexpr float kGuardPx = 2097152.0f;           // 2^21 px: snapped |x| < 2^29
constexpr unsigned long long kKeyEmpty = ~0ull;
constexpr int kSentinel = (int)0x80000000;       // vs.x of a vertex that cannot be snapped
constexpr int kNumVals = 34;                      // counts 6 | e_ls | grad 6 | jtj 21
constexpr unsigned kStatusOverflow = 1u;     // a pinhole bin overflowed
constexpr unsigned kStatusTimeout = 2u;
constexpr unsigned kStatusOverflowRay = 4u;  // a ray-table bin overflowed
constexpr unsigned kStatusQueue = 8u;        // the persistent queue ran out of slots (a bug)
constexpr float kRayMarginPx = 0.25f;        // ray-table rectangles: margin in pixels
constexpr int kThreads = 256;                     // raster CTA

struct DevCam {
  int model, W, H, pad;
  float fx, fy, cx, cy;
  float az0, az_step, el0, el_step;
  float near_m, far_m;
  float w_near, w_far;  // 1/near_m and 1/far_m rounded to FP32
  const float *rays;  // ray-table model: device H*W*3
};

struct TileGeom {
  int tw, th;          // tile size in pixels
  int ntx, nty;        // tiles per row / column
  int ntiles;
  int cap;             // records per bin
  int rec_bytes;       // bytes per bin record: sizeof(TriRec) or sizeof(RayRec)
};

// One snapped triangle (or near-clipped piece) in a screen-tile bin, 48 bytes.
struct __align__(16) TriRec {
  int x0, y0, x1, y1, x2, y2;  // 1/256 px, winding normalised so the doubled area is > 0
  float Ai, Bi, Ci;            // inverse-depth plane, see the contract above
  unsigned id;                 // parent triangle id
  int spare, pad;
};
static_assert(sizeof(TriRec) == 48, "record layout");

// One triangle of the ray-table (panoramic) model in a screen-tile bin, 64 bytes. Coverage of
// a pixel ray r: for each edge k, s = r . c_k with c_k the cross product of the edge's two
// camera-frame vertices taken in increasing vertex-index order (so neighbours share the bits);
// covered iff sigma_k s > 0 for every k, or s == 0 where sigma_k > 0.
struct __align__(16) RayRec {
  float c0x, c0y, c0z, c1x, c1y, c1z, c2x, c2y, c2z;  // edge normals c_k
  float nix, niy, niz;         // inverse-depth normal n / d: w = ni . r
  unsigned id;                 // triangle id
  int sig;                     // bit k set: sigma_k = +1
  int rect0;                   // columns i0 | i1 << 16 (no wrap); tile-relative after setup
  int rect1;                   // rows    j0 | j1 << 16
};
static_assert(sizeof(RayRec) == 64, "record layout");

// ---------------------------------------------------------------- contract helpers

__device__ __forceinline__ float3 xform(const float *M, float x, float y, float z) {
  float X = __fmaf_rn(M[0], x, __fmaf_rn(M[1], y, __fmaf_rn(M[2], z, M[3])));
  float Y = __fmaf_rn(M[4], x, __fmaf_rn(M[5], y, __fmaf_rn(M[6], z, M[7])));
  float Z = __fmaf_rn(M[8], x, __fmaf_rn(M[9], y, __fmaf_rn(M[10], z, M[11])));
  return make_float3(X, Y, Z);
}

__device__ __forceinline__ bool snap(const DevCam &c, float X, float Y, float Z, int &xi,
                                     int &yi) {
  float xs = __fmaf_rn(c.fx, __fdiv_rn(X, Z), c.cx);
  float ys = __fmaf_rn(c.fy, __fdiv_rn(Y, Z), c.cy);
  if (!(fabsf(xs) <= kGuardPx && fabsf(ys) <= kGuardPx)) return false;
  xi = __float2int_rn(__fmul_rn(xs, 256.0f));
  yi = __float2int_rn(__fmul_rn(ys, 256.0f));
  return true;
}

struct PlaneN {
  float nx, ny, nz, d;
};

__device__ __forceinline__ PlaneN plane_n(float3 a, float3 b, float3 c) {
  float e1x = __fsub_rn(b.x, a.x), e1y = __fsub_rn(b.y, a.y), e1z = __fsub_rn(b.z, a.z);
  float e2x = __fsub_rn(c.x, a.x), e2y = __fsub_rn(c.y, a.y), e2z = __fsub_rn(c.z, a.z);
  PlaneN p;
  p.nx = __fmaf_rn(e1y, e2z, -__fmul_rn(e1z, e2y));
  p.ny = __fmaf_rn(e1z, e2x, -__fmul_rn(e1x, e2z));
  p.nz = __fmaf_rn(e1x, e2y, -__fmul_rn(e1y, e2x));
  p.d = __fmaf_rn(p.nx, a.x, __fmaf_rn(p.ny, a.y, __fmul_rn(p.nz, a.z)));
  return p;
}

// Pinhole inverse-depth plane folded into pixel coordinates.
__device__ __forceinline__ void fold_pinhole(const DevCam &c, const PlaneN &p, float &Ai,
                                             float &Bi, float &Ci) {
  const float A = __fdiv_rn(p.nx, c.fx);
  const float B = __fdiv_rn(p.ny, c.fy);
  const float C = __fmaf_rn(-A, c.cx, __fmaf_rn(-B, c.cy, p.nz));
  Ai = __fdiv_rn(A, p.d);
  Bi = __fdiv_rn(B, p.d);
  Ci = __fdiv_rn(C, p.d);
}

__device__ __forceinline__ float inv_depth_pinhole(float Ai, float Bi, float Ci, int i, int j) {
  const float px = __fadd_rn(__int2float_rn(i), 0.5f);
  const float py = __fadd_rn(__int2float_rn(j), 0.5f);
  return __fmaf_rn(Ai, px, __fmaf_rn(Bi, py, Ci));
}

__device__ __forceinline__ bool keep_w(const DevCam &c, float w) {
  return w > 0.0f && w >= c.w_far && w <= c.w_near;
}

// Ray-table contract helpers: cross and dot products in a fixed FMA order.
__device__ __forceinline__ float3 cross_c(float3 p, float3 q) {
  return make_float3(__fmaf_rn(p.y, q.z, -__fmul_rn(p.z, q.y)), __fmaf_rn(p.z, q.x, -__fmul_rn(p.x, q.z)),
                     __fmaf_rn(p.x, q.y, -__fmul_rn(p.y, q.x)));
}

__device__ __forceinline__ float dot_c(float px, float py, float pz, float qx, float qy, float qz) {
  return __fmaf_rn(px, qx, __fmaf_rn(py, qy, __fmul_rn(pz, qz)));
}

__device__ __forceinline__ float3 near_cut(float3 a, float3 b, float near_m) {
  float s = __fdiv_rn(__fsub_rn(near_m, a.z), __fsub_rn(b.z, a.z));
  return make_float3(__fmaf_rn(s, __fsub_rn(b.x, a.x), a.x), __fmaf_rn(s, __fsub_rn(b.y, a.y), a.y),
                     near_m);
}

__device__ __forceinline__ unsigned long long make_key(float w, unsigned id) {
  return ((unsigned long long)(~__float_as_uint(w)) << 32) | (unsigned long long)id;
}

// Depth of a z-buffer key: t = 1 / w rounded to FP32.
__device__ __forceinline__ float key_depth(unsigned long long key) {
  return __frcp_rn(__uint_as_float(~(unsigned)(key >> 32)));
}

}  // namespace rmk
