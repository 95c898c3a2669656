// rm_normals.cu -- rm_depth_normals: surface normals of depth images (Eq. 2, Sec. V).
//
// One CTA per (64x16 output tile, image), fused: the tile's depths with a halo of r + 1
// pixels are staged in shared memory as depths and validity weights (invalid pixels
// contribute neither), smoothed with the separable Gaussian as a normalised convolution (a
// horizontal pass of weighted sums and weight sums, four outputs per thread sliding along a
// row, then a vertical pass, six per thread down a column; one instantiation per radius, so
// the taps unroll with their weights in registers), and the smoothed depth S over the tile
// plus a one-pixel ring feeds the central differences and the normal N = a x b with
// a = (0, s_y, dz/dy) and b = (s_x, 0, dz/dx). Each depth and class byte is read once from HBM
// and each normal written once (17 bytes per pixel); the convolution's instructions and
// shared-memory traffic, not HBM, set the kernel's time.
#include <cfloat>
#include <cmath>
#include <string>

#include "rendermap.h"
#include "rm_kernels.cuh"

namespace {

constexpr int kTW = 64, kTH = 16;      // output tile
constexpr int kMaxR = 16;              // Gaussian radius ceil(3 sigma) for sigma <= 5
constexpr int kSW = kTW + 2;           // smoothed region (tile plus a one-pixel ring)
constexpr int kSH = kTH + 2;
constexpr int kThreadsN = 256;
constexpr int kHG = 4;                 // horizontal pass: outputs per thread along a row
constexpr int kVG = 6;                 // vertical pass: outputs per thread down a column

struct NormalArgs {
  const float *depth;
  const uint8_t *cls;
  float *normals;
  float *smoothed;   // optional
  float *blur;       // optional: S where valid, else the input depth
  int W, H, r, metric;
  float ifx, ify;    // 1 / fx, 1 / fy
  float inv_g2;      // 1 / (sum of the taps)^2: the weight sum when every staged pixel is valid
  float g[kMaxR + 1];
};

// Dynamic shared memory, all FP32 tables: the staged depths (0 where invalid) and validity
// weights (1 or 0) of the tile plus its halo, the horizontal sums of each staged row over the
// smoothed columns (weighted depths, weights), and the smoothed depth S of the tile plus a
// one-pixel ring. The horizontal pass reads and writes the tables down their columns with
// consecutive threads on consecutive rows, so every row stride is odd: 32 consecutive rows
// then fall in 32 distinct banks and a warp's 4-byte access takes one wavefront.
__host__ __device__ constexpr int odd_stride(int n) { return n | 1; }
__host__ __device__ inline int staged_w(int r) { return kSW + 2 * r; }
__host__ __device__ inline int staged_h(int r) { return kSH + 2 * r; }
__host__ __device__ inline int staged_stride(int r) { return odd_stride(staged_w(r)); }
constexpr int kSWP = odd_stride(kSW);  // row stride of the horizontal sums
inline size_t normals_smem(int r) {
  return sizeof(float) * (2 * (size_t)staged_h(r) * staged_stride(r) + 2 * (size_t)staged_h(r) * kSWP +
                          (size_t)kSH * kSW);
}

template <int R>
__global__ void __launch_bounds__(kThreadsN) k_depth_normals(NormalArgs a) {
  extern __shared__ float4 smem_raw[];
  constexpr int dw = kSW + 2 * R, dh = kSH + 2 * R, dws = odd_stride(dw);
  float *zv = reinterpret_cast<float *>(smem_raw);  // [dh][dws]: valid ? z : 0
  float *zw = zv + dh * dws;                          // [dh][dws]: valid ? 1 : 0
  float *hn = zw + dh * dws;                          // [dh][kSWP]: horizontal sums of zv
  float *hd = hn + dh * kSWP;                         // [dh][kSWP]: horizontal sums of zw
  float *sS = hd + dh * kSWP;                         // [kSH][kSW]
  const int tid = threadIdx.x;
  float g[R + 1];
#pragma unroll
  for (int k = 0; k <= R; ++k) g[k] = a.g[k];
  const int img = blockIdx.y;
  const int ntx = (a.W + kTW - 1) / kTW;
  const int ox = (blockIdx.x % ntx) * kTW, oy = (blockIdx.x / ntx) * kTH;
  const int x0 = ox - 1 - R, y0 = oy - 1 - R;  // image coordinates of zv[0][0]
  const long long P = (long long)a.W * a.H;
  const float *dimg = a.depth + img * P;
  const uint8_t *cimg = a.cls + img * P;
  // stage: independent loads, four per thread in flight; note whether every staged pixel is
  // valid, the common case away from holes and the image border
  constexpr int n_st = dw * dh;
  bool mine_valid = true;
  for (int k0 = tid; k0 < n_st; k0 += 4 * kThreadsN) {
    float dv[4];
    int cv[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int k = k0 + m * kThreadsN;
      dv[m] = 0.0f;
      cv[m] = 1;
      if (k < n_st) {
        const int x = x0 + k % dw, y = y0 + k / dw;
        if (x >= 0 && x < a.W && y >= 0 && y < a.H) {
          const long long p = (long long)y * a.W + x;
          dv[m] = __ldg(dimg + p);
          cv[m] = __ldg(cimg + p);
        }
      }
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int k = k0 + m * kThreadsN;
      if (k < n_st) {
        const bool ok = cv[m] == 0 && fabsf(dv[m]) <= FLT_MAX;
        mine_valid = mine_valid && ok;
        const int at = (k / dw) * dws + k % dw;
        zv[at] = ok ? dv[m] : 0.0f;
        zw[at] = ok ? 1.0f : 0.0f;
      }
    }
  }
  const bool all_valid = __syncthreads_and(mine_valid);
  // horizontal pass: weighted sums of the valid depths (and of their weights, unless every
  // staged pixel is valid), kHG adjacent outputs per thread: each staged value is loaded once
  // and added to every output whose window holds it (the taps unroll: R is a template
  // parameter); consecutive threads take consecutive rows
  {
    constexpr int groups = (kSW + kHG - 1) / kHG;
    for (int it = tid; it < dh * groups; it += kThreadsN) {
      const int v = it % dh, u0 = (it / dh) * kHG;
      float num[kHG], den[kHG];
#pragma unroll
      for (int j = 0; j < kHG; ++j) num[j] = den[j] = 0.0f;
      const float *row = zv + v * dws + u0;  // output u0 + j: staged columns u0 + j .. + 2R
      const float *roww = zw + v * dws + u0;
      if (all_valid) {
#pragma unroll
        for (int t = 0; t < 2 * R + kHG; ++t) {
          const float z = (u0 + t < dw) ? row[t] : 0.0f;
#pragma unroll
          for (int j = 0; j < kHG; ++j) {
            const int d = t - j;
            if (d >= 0 && d <= 2 * R) num[j] = fmaf(g[d < R ? R - d : d - R], z, num[j]);
          }
        }
      } else {
#pragma unroll
        for (int t = 0; t < 2 * R + kHG; ++t) {
          const bool in = u0 + t < dw;
          const float z = in ? row[t] : 0.0f, zok = in ? roww[t] : 0.0f;
#pragma unroll
          for (int j = 0; j < kHG; ++j) {
            const int d = t - j;
            if (d >= 0 && d <= 2 * R) {
              const float w = g[d < R ? R - d : d - R];
              num[j] = fmaf(w, z, num[j]);
              den[j] = fmaf(w, zok, den[j]);
            }
          }
        }
      }
#pragma unroll
      for (int j = 0; j < kHG; ++j)
        if (u0 + j < kSW) {
          hn[v * kSWP + u0 + j] = num[j];
          hd[v * kSWP + u0 + j] = den[j];
        }
    }
  }
  __syncthreads();
  // vertical pass: kVG outputs per thread down a column; S where the centre pixel is valid
  {
    constexpr int groups = (kSH + kVG - 1) / kVG;
    for (int it = tid; it < kSW * groups; it += kThreadsN) {
      const int u = it % kSW, v0 = (it / kSW) * kVG;
      float num[kVG], den[kVG];
#pragma unroll
      for (int j = 0; j < kVG; ++j) num[j] = den[j] = 0.0f;
      if (all_valid) {
#pragma unroll
        for (int t = 0; t < 2 * R + kVG; ++t) {
          const float h = (v0 + t < dh) ? hn[(v0 + t) * kSWP + u] : 0.0f;
#pragma unroll
          for (int j = 0; j < kVG; ++j) {
            const int d = t - j;
            if (d >= 0 && d <= 2 * R) num[j] = fmaf(g[d < R ? R - d : d - R], h, num[j]);
          }
        }
#pragma unroll
        for (int j = 0; j < kVG; ++j)
          if (v0 + j < kSH) sS[(v0 + j) * kSW + u] = num[j] * a.inv_g2;
      } else {
#pragma unroll
        for (int t = 0; t < 2 * R + kVG; ++t) {
          const bool in = v0 + t < dh;
          const float hz = in ? hn[(v0 + t) * kSWP + u] : 0.0f, hw = in ? hd[(v0 + t) * kSWP + u] : 0.0f;
#pragma unroll
          for (int j = 0; j < kVG; ++j) {
            const int d = t - j;
            if (d >= 0 && d <= 2 * R) {
              const float w = g[d < R ? R - d : d - R];
              num[j] = fmaf(w, hz, num[j]);
              den[j] = fmaf(w, hw, den[j]);
            }
          }
        }
#pragma unroll
        for (int j = 0; j < kVG; ++j) {
          const int v = v0 + j;
          if (v < kSH) {
            const bool centre = zw[(v + R) * dws + (u + R)] != 0.0f;
            sS[v * kSW + u] = centre ? num[j] / den[j] : __int_as_float(0x7fc00000);
          }
        }
      }
    }
  }
  __syncthreads();
  for (int k = tid; k < kTW * kTH; k += kThreadsN) {
    const int u = k % kTW + 1, v = k / kTW + 1;
    const int x = ox + u - 1, y = oy + v - 1;
    if (x >= a.W || y >= a.H) continue;
    const long long p = img * P + (long long)y * a.W + x;
    const float s = sS[v * kSW + u];
    if (a.smoothed) a.smoothed[p] = s;
    if (a.blur) a.blur[p] = isnan(s) ? a.depth[p] : s;
    if (!a.normals) continue;
    float n0 = __int_as_float(0x7fc00000), n1 = n0, n2 = n0;
    const float sl = sS[v * kSW + u - 1], sr = sS[v * kSW + u + 1];
    const float su = sS[(v - 1) * kSW + u], sd = sS[(v + 1) * kSW + u];
    if (x >= 1 && x + 1 < a.W && y >= 1 && y + 1 < a.H && !isnan(s) && !isnan(sl) && !isnan(sr) &&
        !isnan(su) && !isnan(sd)) {
      const float zx = 0.5f * (sr - sl), zy = 0.5f * (sd - su);
      const float sx = a.metric ? s * a.ifx : 1.0f, sy = a.metric ? s * a.ify : 1.0f;
      // a = (0, sy, zy), b = (sx, 0, zx), N = a x b
      const float c0 = sy * zx, c1 = zy * sx, c2 = -sy * sx;
      const float inv = rsqrtf(c0 * c0 + c1 * c1 + c2 * c2);
      n0 = c0 * inv;
      n1 = c1 * inv;
      n2 = c2 * inv;
    }
    a.normals[3 * p] = n0;
    a.normals[3 * p + 1] = n1;
    a.normals[3 * p + 2] = n2;
  }
}

template <int R>
cudaError_t launch_normals_r(const NormalArgs &a, int tiles, int n, cudaStream_t s) {
  const size_t sm = normals_smem(R);
  // radii above about 7 need more than the default 48 KB (set on the current device)
  cudaError_t e = cudaFuncSetAttribute(k_depth_normals<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_depth_normals<R><<<dim3(tiles, n), kThreadsN, sm, s>>>(a);
  return cudaGetLastError();
}

template <int R>
cudaError_t launch_normals(const NormalArgs &a, int tiles, int n, cudaStream_t s) {
  if (a.r == R) return launch_normals_r<R>(a, tiles, n, s);
  if constexpr (R < kMaxR) return launch_normals<R + 1>(a, tiles, n, s);
  return cudaErrorInvalidValue;
}

bool dn_on_device(const void *p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

rm_status dn_fail(rm_status s, const std::string &m) {
  rmapi::set_error(m);
  return s;
}

// Shared driver of rm_depth_normals and rm_depth_blur; any of the three outputs may be NULL.
rm_status run_normals(const rm_intrinsics *intr, int32_t n, const float *depth, const uint8_t *cls,
                      float sigma, int32_t metric, float *normals, float *smoothed, float *blur,
                      void *stream) {
  if (!intr) return dn_fail(RM_EINVAL, "intrinsics are NULL");
  if (n < 0 || intr->width < 0 || intr->height < 0) return dn_fail(RM_EINVAL, "negative size");
  if (n > 65535) return dn_fail(RM_EINVAL, "at most 65535 images per call");
  if (!(sigma >= 0.0f) || sigma > 5.0f) return dn_fail(RM_EINVAL, "sigma must be in [0, 5]");
  if (metric != 0 && metric != 1) return dn_fail(RM_EINVAL, "metric must be 0 or 1");
  if (metric && (intr->model != RM_PINHOLE || !(intr->fx > 0.0f) || !(intr->fy > 0.0f) ||
                 !(intr->fx <= FLT_MAX) || !(intr->fy <= FLT_MAX)))
    return dn_fail(RM_EINVAL, "metric normals need a pinhole camera with finite fx, fy > 0");
  const long long P = (long long)intr->width * intr->height;
  if (n == 0 || P == 0) return RM_OK;
  if (!depth || !cls) return dn_fail(RM_EINVAL, "NULL array");
  if ((long long)n * P > (1LL << 40)) return dn_fail(RM_EINVAL, "too many pixels");
  cudaStream_t s = (cudaStream_t)stream;
  const bool host_d = !dn_on_device(depth), host_c = !dn_on_device(cls);
  const bool host_n = normals && !dn_on_device(normals), host_s = smoothed && !dn_on_device(smoothed);
  const bool host_b = blur && !dn_on_device(blur);
  const size_t np = (size_t)n * P;
  // host arrays are staged through stream-ordered device allocations
  float *d_d = host_d ? nullptr : const_cast<float *>(depth);
  float *d_n = host_n ? nullptr : normals;
  float *d_s = host_s ? nullptr : smoothed;
  float *d_b = host_b ? nullptr : blur;
  uint8_t *d_c = host_c ? nullptr : const_cast<uint8_t *>(cls);
  cudaError_t e = cudaSuccess;
  auto ck = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  if (host_d) ck(cudaMallocAsync((void **)&d_d, sizeof(float) * np, s));
  if (host_c) ck(cudaMallocAsync((void **)&d_c, np, s));
  if (host_n) ck(cudaMallocAsync((void **)&d_n, sizeof(float) * 3 * np, s));
  if (host_s) ck(cudaMallocAsync((void **)&d_s, sizeof(float) * np, s));
  if (host_b) ck(cudaMallocAsync((void **)&d_b, sizeof(float) * np, s));
  if (e == cudaSuccess && host_d) ck(cudaMemcpyAsync(d_d, depth, sizeof(float) * np, cudaMemcpyHostToDevice, s));
  if (e == cudaSuccess && host_c) ck(cudaMemcpyAsync(d_c, cls, np, cudaMemcpyHostToDevice, s));
  if (e == cudaSuccess) {
    NormalArgs a{};
    a.depth = d_d;
    a.cls = d_c;
    a.normals = d_n;
    a.smoothed = d_s;
    a.blur = d_b;
    a.W = intr->width;
    a.H = intr->height;
    a.r = sigma > 0.0f ? (int)std::ceil(3.0 * (double)sigma) : 0;
    a.metric = metric;
    a.ifx = metric ? 1.0f / intr->fx : 1.0f;
    a.ify = metric ? 1.0f / intr->fy : 1.0f;
    for (int k = 0; k <= kMaxR; ++k)
      a.g[k] = sigma > 0.0f ? (float)std::exp(-(double)(k * k) / (2.0 * (double)sigma * sigma)) : 1.0f;
    double gs = a.g[0];
    for (int k = 1; k <= a.r; ++k) gs += 2.0 * a.g[k];
    a.inv_g2 = (float)(1.0 / (gs * gs));
    const int tiles = ((a.W + kTW - 1) / kTW) * ((a.H + kTH - 1) / kTH);
    ck(launch_normals<0>(a, tiles, n, s));
  }
  if (e == cudaSuccess && host_n) ck(cudaMemcpyAsync(normals, d_n, sizeof(float) * 3 * np, cudaMemcpyDeviceToHost, s));
  if (e == cudaSuccess && host_s) ck(cudaMemcpyAsync(smoothed, d_s, sizeof(float) * np, cudaMemcpyDeviceToHost, s));
  if (e == cudaSuccess && host_b) ck(cudaMemcpyAsync(blur, d_b, sizeof(float) * np, cudaMemcpyDeviceToHost, s));
  if (host_d && d_d) cudaFreeAsync(d_d, s);
  if (host_c && d_c) cudaFreeAsync(d_c, s);
  if (host_n && d_n) cudaFreeAsync(d_n, s);
  if (host_s && d_s) cudaFreeAsync(d_s, s);
  if (host_b && d_b) cudaFreeAsync(d_b, s);
  if (e == cudaSuccess && (host_n || host_s || host_b)) ck(cudaStreamSynchronize(s));
  if (e != cudaSuccess) return dn_fail(RM_ECUDA, std::string("rm_depth_normals: ") + cudaGetErrorString(e));
  return RM_OK;
}

// True when the byte ranges [a, a + na) and [b, b + nb) share a byte (NULL overlaps nothing).
bool overlaps(const void *a, size_t na, const void *b, size_t nb) {
  if (!a || !b) return false;
  const char *a0 = static_cast<const char *>(a), *b0 = static_cast<const char *>(b);
  return a0 < b0 + nb && b0 < a0 + na;
}

}  // namespace

extern "C" rm_status rm_depth_normals(const rm_intrinsics *intr, int32_t n, const float *depth,
                                      const uint8_t *cls, float sigma, int32_t metric,
                                      float *normals, float *smoothed, void *stream) {
  if (!normals && n > 0) return dn_fail(RM_EINVAL, "normals is NULL");
  // neighbouring tiles read the inputs' halos while a tile writes its outputs, so no output
  // may share memory with an input or with the other output
  if (intr && n > 0 && intr->width > 0 && intr->height > 0) {
    const size_t np = (size_t)n * intr->width * intr->height;
    const size_t bd = sizeof(float) * np, bc = np, bn = 3 * sizeof(float) * np, bs = sizeof(float) * np;
    if (overlaps(normals, bn, depth, bd) || overlaps(normals, bn, cls, bc))
      return dn_fail(RM_EINVAL, "normals overlaps an input");
    if (overlaps(smoothed, bs, depth, bd) || overlaps(smoothed, bs, cls, bc))
      return dn_fail(RM_EINVAL, "smoothed overlaps an input");
    if (overlaps(normals, bn, smoothed, bs)) return dn_fail(RM_EINVAL, "normals overlaps smoothed");
  }
  return run_normals(intr, n, depth, cls, sigma, metric, normals, smoothed, nullptr, stream);
}

extern "C" rm_status rm_depth_blur(const rm_intrinsics *intr, int32_t n, const float *depth,
                                   const uint8_t *cls, float sigma, float *out, void *stream) {
  if (!out && n > 0) return dn_fail(RM_EINVAL, "out is NULL");
  if (intr && n > 0 && intr->width > 0 && intr->height > 0) {
    const size_t np = (size_t)n * intr->width * intr->height;
    if (overlaps(out, sizeof(float) * np, depth, sizeof(float) * np)) return dn_fail(RM_EINVAL, "out overlaps depth");
    if (overlaps(out, sizeof(float) * np, cls, np)) return dn_fail(RM_EINVAL, "out overlaps cls");
  }
  return run_normals(intr, n, depth, cls, sigma, 0, nullptr, nullptr, out, stream);
}
