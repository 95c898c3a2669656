// rm_vgrad.cu -- the per-pixel kernel of rm_cost_grad_vertices: the gradient of the
// least-squares surrogate with respect to the map's vertex positions (map refinement).
//
// It runs on a rendered visibility buffer (triangle id, FP32 depth and barycentrics per pixel,
// from the raster's render epilogue). For every pixel whose Table I cell carries an active
// residual r (the same cells, thresholds and weights as the cost epilogue), the depth along
// the pixel's ray moves with vertex m of its triangle as d t / d v_m = b_m n_w / (n_c . r);
// each pixel adds w r sgn of that to its three vertices with FP64 atomics.
#include <cfloat>
#include <cmath>

#include "rm_kernels.cuh"

namespace rmk {

__global__ void __launch_bounds__(256) k_vertex_grad(VGradArgs a) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (long long)a.n_poses * a.P) return;
  const int q = (int)(k / a.P);
  const long long pix = k % a.P;
  const int id = a.tri_id[k];
  if (id < 0) return;
  const float sd = a.scan_depth[pix];
  const int sc = a.scan_cls[pix];
  if (sc > 1 || !(fabsf(sd) <= FLT_MAX)) return;
  const float4 pl = a.planes[id];
  const int mc = __float_as_int(pl.w);
  if (mc > 1) return;
  const float t = a.depth[k];
  const float dz = __fsub_rn(t, sd);
  const float eps = a.prm.eps;
  float r, w, sgn = 0.0f;
  if (mc == 0) {
    if (sc == 0) {
      if (!(fabsf(dz) <= eps)) return;  // truncated: no slope
      w = a.prm.w_fofo;
      r = dz;
      sgn = 1.0f;
    } else {
      if (dz > 0.0f || !(-dz < eps)) return;
      w = a.prm.w_fofu;
      r = -dz;
      sgn = -1.0f;
    }
  } else {
    if (sc != 0 || dz <= 0.0f || !(dz < eps)) return;
    w = a.prm.w_fufo;
    r = dz;
    sgn = 1.0f;
  }
  const int i = (int)(pix % a.W), j = (int)(pix / a.W);
  float rx, ry, rz;
  if (a.cam.model == 0) {
    rx = (i + 0.5f - a.cam.cx) / a.cam.fx;
    ry = (j + 0.5f - a.cam.cy) / a.cam.fy;
    rz = 1.0f;
  } else {
    const float *rr = a.cam.rays + 3 * pix;
    rx = rr[0];
    ry = rr[1];
    rz = rr[2];
  }
  const float *M = a.Ms + 12 * q;
  const float ncx = M[0] * pl.x + M[1] * pl.y + M[2] * pl.z;
  const float ncy = M[4] * pl.x + M[5] * pl.y + M[6] * pl.z;
  const float ncz = M[8] * pl.x + M[9] * pl.y + M[10] * pl.z;
  const float nr = ncx * rx + ncy * ry + ncz * rz;
  const double coef = (double)(w * r * sgn) / (double)nr;
  const float b1 = a.bary[2 * k], b2 = a.bary[2 * k + 1];
  const float b[3] = {1.0f - b1 - b2, b1, b2};
  const int4 f = a.faces[id];
  const int vid[3] = {f.x, f.y, f.z};
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    const double s = coef * (double)b[m];
    double *g = a.grad + 3 * (long long)vid[m];
    atomicAdd(g, s * (double)pl.x);
    atomicAdd(g + 1, s * (double)pl.y);
    atomicAdd(g + 2, s * (double)pl.z);
  }
}

cudaError_t launch_vertex_grad(const VGradArgs &a, cudaStream_t s) {
  const long long n = (long long)a.n_poses * a.P;
  if (n == 0) return cudaSuccess;
  k_vertex_grad<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace rmk
