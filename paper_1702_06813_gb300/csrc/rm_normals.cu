// rm_normals.cu -- rm_depth_normals: surface normals of depth images (Eq. 2, Sec. IV).
//
// One CTA per (32x16 output tile, image), fused: the tile's depths with a halo of r + 1
// pixels are staged in shared memory (invalid pixels as NaN), smoothed with the separable
// Gaussian as a normalised convolution (a horizontal pass of weighted sums and weight sums,
// then a vertical pass), and the smoothed depth S over the tile plus a one-pixel ring feeds
// the central differences and the normal N = a x b with a = (0, s_y, dz/dy) and
// b = (s_x, 0, dz/dx). Each depth and class byte is read once from HBM and each normal
// written once (17 bytes per pixel); the kernel is bound by HBM bandwidth.
#include <cfloat>
#include <cmath>
#include <string>

#include "rendermap.h"
#include "rm_kernels.cuh"

namespace {

constexpr int kTW = 32, kTH = 16;      // output tile
constexpr int kMaxR = 16;              // Gaussian radius ceil(3 sigma) for sigma <= 5
constexpr int kSW = kTW + 2;           // smoothed region (tile plus a one-pixel ring)
constexpr int kSH = kTH + 2;
constexpr int kDW = kSW + 2 * kMaxR;   // staged depth region
constexpr int kDH = kSH + 2 * kMaxR;

struct NormalArgs {
  const float *depth;
  const uint8_t *cls;
  float *normals;
  float *smoothed;   // optional
  int W, H, r, metric;
  float fx, fy;
  float g[kMaxR + 1];
};

__global__ void __launch_bounds__(256) k_depth_normals(NormalArgs a) {
  __shared__ float sz[kDH][kDW + 1];
  __shared__ float snum[kDH][kSW];
  __shared__ float sden[kDH][kSW];
  __shared__ float sS[kSH][kSW];
  __shared__ float sg[kMaxR + 1];
  const int tid = threadIdx.x;
  if (tid <= kMaxR) sg[tid] = a.g[tid];
  const int img = blockIdx.y;
  const int ntx = (a.W + kTW - 1) / kTW;
  const int ox = (blockIdx.x % ntx) * kTW, oy = (blockIdx.x / ntx) * kTH;
  const int r = a.r;
  const int dw = kSW + 2 * r, dh = kSH + 2 * r;  // staged region actually used
  const int x0 = ox - 1 - r, y0 = oy - 1 - r;    // image coordinates of sz[0][0]
  const long long P = (long long)a.W * a.H;
  const float *dimg = a.depth + img * P;
  const uint8_t *cimg = a.cls + img * P;
  for (int k = tid; k < dw * dh; k += blockDim.x) {
    const int u = k % dw, v = k / dw;
    const int x = x0 + u, y = y0 + v;
    float z = __int_as_float(0x7fc00000);
    if (x >= 0 && x < a.W && y >= 0 && y < a.H) {
      const long long p = (long long)y * a.W + x;
      const float d = dimg[p];
      if (cimg[p] == 0 && fabsf(d) <= FLT_MAX) z = d;
    }
    sz[v][u] = z;
  }
  __syncthreads();
  // horizontal pass: weighted sums of the valid depths and of their weights
  for (int k = tid; k < dh * kSW; k += blockDim.x) {
    const int u = k % kSW, v = k / kSW;
    float num = 0.0f, den = 0.0f;
    for (int dx = -r; dx <= r; ++dx) {
      const float z = sz[v][u + r + dx];
      if (!isnan(z)) {
        const float w = sg[abs(dx)];
        num = fmaf(w, z, num);
        den += w;
      }
    }
    snum[v][u] = num;
    sden[v][u] = den;
  }
  __syncthreads();
  // vertical pass: the smoothed depth where the centre pixel is valid
  for (int k = tid; k < kSH * kSW; k += blockDim.x) {
    const int u = k % kSW, v = k / kSW;
    float s = __int_as_float(0x7fc00000);
    if (!isnan(sz[v + r][u + r])) {
      float num = 0.0f, den = 0.0f;
      for (int dy = -r; dy <= r; ++dy) {
        const float w = sg[abs(dy)];
        num = fmaf(w, snum[v + r + dy][u], num);
        den = fmaf(w, sden[v + r + dy][u], den);
      }
      s = num / den;
    }
    sS[v][u] = s;
  }
  __syncthreads();
  for (int k = tid; k < kTW * kTH; k += blockDim.x) {
    const int u = k % kTW + 1, v = k / kTW + 1;
    const int x = ox + u - 1, y = oy + v - 1;
    if (x >= a.W || y >= a.H) continue;
    const long long p = img * P + (long long)y * a.W + x;
    const float s = sS[v][u];
    if (a.smoothed) a.smoothed[p] = s;
    float n0 = __int_as_float(0x7fc00000), n1 = n0, n2 = n0;
    const float sl = sS[v][u - 1], sr = sS[v][u + 1], su = sS[v - 1][u], sd = sS[v + 1][u];
    if (x >= 1 && x + 1 < a.W && y >= 1 && y + 1 < a.H && !isnan(s) && !isnan(sl) && !isnan(sr) &&
        !isnan(su) && !isnan(sd)) {
      const float zx = 0.5f * (sr - sl), zy = 0.5f * (sd - su);
      const float sx = a.metric ? s / a.fx : 1.0f, sy = a.metric ? s / a.fy : 1.0f;
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

}  // namespace

extern "C" rm_status rm_depth_normals(const rm_intrinsics *intr, int32_t n, const float *depth,
                                      const uint8_t *cls, float sigma, int32_t metric,
                                      float *normals, float *smoothed, void *stream) {
  if (!intr) return dn_fail(RM_EINVAL, "intrinsics are NULL");
  if (n < 0 || intr->width < 0 || intr->height < 0) return dn_fail(RM_EINVAL, "negative size");
  if (!(sigma >= 0.0f) || sigma > 5.0f) return dn_fail(RM_EINVAL, "sigma must be in [0, 5]");
  if (metric != 0 && metric != 1) return dn_fail(RM_EINVAL, "metric must be 0 or 1");
  if (metric && (intr->model != RM_PINHOLE || !(intr->fx > 0.0f) || !(intr->fy > 0.0f) ||
                 !(intr->fx <= FLT_MAX) || !(intr->fy <= FLT_MAX)))
    return dn_fail(RM_EINVAL, "metric normals need a pinhole camera with finite fx, fy > 0");
  const long long P = (long long)intr->width * intr->height;
  if (n == 0 || P == 0) return RM_OK;
  if (!depth || !cls || !normals) return dn_fail(RM_EINVAL, "NULL array");
  if ((long long)n * P > (1LL << 40)) return dn_fail(RM_EINVAL, "too many pixels");
  cudaStream_t s = (cudaStream_t)stream;
  const bool host_d = !dn_on_device(depth), host_c = !dn_on_device(cls);
  const bool host_n = !dn_on_device(normals), host_s = smoothed && !dn_on_device(smoothed);
  const size_t np = (size_t)n * P;
  // host arrays are staged through stream-ordered device allocations
  float *d_d = host_d ? nullptr : const_cast<float *>(depth);
  float *d_n = host_n ? nullptr : normals;
  float *d_s = host_s ? nullptr : smoothed;
  uint8_t *d_c = host_c ? nullptr : const_cast<uint8_t *>(cls);
  cudaError_t e = cudaSuccess;
  auto ck = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  if (host_d) ck(cudaMallocAsync((void **)&d_d, sizeof(float) * np, s));
  if (host_c) ck(cudaMallocAsync((void **)&d_c, np, s));
  if (host_n) ck(cudaMallocAsync((void **)&d_n, sizeof(float) * 3 * np, s));
  if (host_s) ck(cudaMallocAsync((void **)&d_s, sizeof(float) * np, s));
  if (e == cudaSuccess && host_d) ck(cudaMemcpyAsync(d_d, depth, sizeof(float) * np, cudaMemcpyHostToDevice, s));
  if (e == cudaSuccess && host_c) ck(cudaMemcpyAsync(d_c, cls, np, cudaMemcpyHostToDevice, s));
  if (e == cudaSuccess) {
    NormalArgs a{};
    a.depth = d_d;
    a.cls = d_c;
    a.normals = d_n;
    a.smoothed = d_s;
    a.W = intr->width;
    a.H = intr->height;
    a.r = sigma > 0.0f ? (int)std::ceil(3.0 * (double)sigma) : 0;
    a.metric = metric;
    a.fx = intr->fx;
    a.fy = intr->fy;
    for (int k = 0; k <= kMaxR; ++k)
      a.g[k] = sigma > 0.0f ? (float)std::exp(-(double)(k * k) / (2.0 * (double)sigma * sigma)) : 1.0f;
    const int tiles = ((a.W + kTW - 1) / kTW) * ((a.H + kTH - 1) / kTH);
    k_depth_normals<<<dim3(tiles, n), 256, 0, s>>>(a);
    ck(cudaGetLastError());
  }
  if (e == cudaSuccess && host_n) ck(cudaMemcpyAsync(normals, d_n, sizeof(float) * 3 * np, cudaMemcpyDeviceToHost, s));
  if (e == cudaSuccess && host_s) ck(cudaMemcpyAsync(smoothed, d_s, sizeof(float) * np, cudaMemcpyDeviceToHost, s));
  if (host_d && d_d) cudaFreeAsync(d_d, s);
  if (host_c && d_c) cudaFreeAsync(d_c, s);
  if (host_n && d_n) cudaFreeAsync(d_n, s);
  if (host_s && d_s) cudaFreeAsync(d_s, s);
  if (e == cudaSuccess && (host_n || host_s)) ck(cudaStreamSynchronize(s));
  if (e != cudaSuccess) return dn_fail(RM_ECUDA, std::string("rm_depth_normals: ") + cudaGetErrorString(e));
  return RM_OK;
}
