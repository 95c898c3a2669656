// rm_vgrad.cu -- the per-pixel kernel of rm_cost_grad_vertices: the gradient of the
// least-squares surrogate with respect to the map's vertex positions (map refinement).
//
// It runs on a rendered visibility buffer (triangle id, FP32 depth and barycentrics per pixel,
// from the raster's render epilogue). For every pixel whose Table I cell carries an active
// residual r (the same cells, thresholds and weights as the cost epilogue), the depth along
// the pixel's ray moves with vertex m of its triangle as d t / d v_m = b_m n_w / (n_c . r);
// each pixel's w r sgn of that goes to its three vertices: runs of adjacent pixels on one
// triangle are summed in the warp first, then added with FP64 atomics.
#include <cfloat>
#include <cmath>

#include "rm_kernels.cuh"

namespace rmk {

// Per pixel: 0 and no contribution, or the triangle id and coef b_m for its three vertices
// (coef = w r sgn / (n_c . r)).
__device__ __forceinline__ bool vgrad_pixel(const VGradArgs &a, long long k, int &id, float c[3]) {
  if (k >= (long long)a.n_poses * a.P) return false;
  const int q = (int)(k / a.P);
  const long long pix = k % a.P;
  id = a.tri_id[k];
  if (id < 0) return false;
  const float sd = a.scan_depth[pix];
  const int sc = a.scan_cls[pix];
  if (sc > 1 || !(fabsf(sd) <= FLT_MAX)) return false;
  const float4 pl = a.planes[id];
  const int mc = __float_as_int(pl.w);
  if (mc > 1) return false;
  const float t = a.depth[k];
  const float dz = __fsub_rn(t, sd);
  const float eps = a.prm.eps;
  float r, w, sgn;
  if (mc == 0) {
    if (sc == 0) {
      if (!(fabsf(dz) <= eps)) return false;  // truncated: no slope
      w = a.prm.w_fofo;
      r = dz;
      sgn = 1.0f;
    } else {
      if (dz > 0.0f || !(-dz < eps)) return false;
      w = a.prm.w_fofu;
      r = -dz;
      sgn = -1.0f;
    }
  } else {
    if (sc != 0 || dz <= 0.0f || !(dz < eps)) return false;
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
  const float coef = (w * r * sgn) / nr;
  const float b1 = a.bary[2 * k], b2 = a.bary[2 * k + 1];
  c[0] = coef * (1.0f - b1 - b2);
  c[1] = coef * b1;
  c[2] = coef * b2;
  return true;
}

// One thread per (pose, pixel). Every pixel of a triangle moves its vertices along the same
// world normal, so adjacent lanes that see the same triangle (a run along the image row) sum
// their coef b_m by a segmented scan over the warp, and the run's last lane adds the three
// vertices' gradient with FP64 atomics: nine atomics per run instead of per pixel.
__global__ void __launch_bounds__(256) k_vertex_grad(VGradArgs a) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  float c[3] = {0.0f, 0.0f, 0.0f};
  int id = -1;
  const bool act = vgrad_pixel(a, k, id, c);
  const int key = act ? id : -1 - lane;  // inactive lanes form runs of their own
  const int prev = __shfl_up_sync(0xffffffffu, key, 1);
  unsigned head = (lane == 0 || prev != key) ? 1u : 0u;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const float u0 = __shfl_up_sync(0xffffffffu, c[0], off);
    const float u1 = __shfl_up_sync(0xffffffffu, c[1], off);
    const float u2 = __shfl_up_sync(0xffffffffu, c[2], off);
    const unsigned hf = __shfl_up_sync(0xffffffffu, head, off);
    if (lane >= off && !head) {
      c[0] += u0;
      c[1] += u1;
      c[2] += u2;
      head |= hf;
    }
  }
  const int next = __shfl_down_sync(0xffffffffu, key, 1);
  if (!act || (lane < 31 && next == key)) return;  // not the last lane of its run
  const float4 pl = a.planes[id];
  const int4 f = a.faces[id];
  const int vid[3] = {f.x, f.y, f.z};
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    const double s = (double)c[m];
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
