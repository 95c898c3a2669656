// rm_mesh.cu -- rm_meshify: the labelled interface mesh of one range image (Sec. IV.A, Fig. 5).
//
// Four kernels, all elementwise or per-block, in a fixed order so that the output is the same
// run to run (row-major block order, no atomics):
//   k_mesh_points  per grid pixel: class (return / no-return / dead), its FP32 camera-frame
//                  point (returns at their depth, no-returns at the maximal range), and the
//                  world vertex through the pose in FP64 (rounded once to FP32)
//   k_mesh_quads   per 2x2 block of grid pixels: dropped when a pixel is dead, else FU when a
//                  pixel is a no-return or a side or the diagonal is longer than the limit
//                  (squared lengths in FP32), else FO; plus the kept count of each CTA
//   k_mesh_scan    one CTA: exclusive scan of the per-CTA counts (the face offsets)
//   k_mesh_emit    per block: two triangles (v00, v10, v11), (v00, v11, v01) at the block's
//                  rank among the kept blocks
// The arithmetic that decides a label uses explicitly rounded operations (no contraction), so
// the decision is the same as any IEEE FP32 evaluation in the same order.
#include <cfloat>
#include <cmath>
#include <string>

#include "rendermap.h"
#include "rm_kernels.cuh"

namespace {

constexpr int kQuadThreads = 256;

struct MeshArgs {
  int model, W, H, step, Ws, Hs;
  float fx, fy, cx, cy;
  const float *rays;
  const float *depth;
  const uint8_t *cls;
  double T[12];         // camera-to-world rows (R | t) of a host pose
  const double *Tdev;   // or the pose in device memory (16 doubles)
  float max_range, lim;  // lim = max_edge^2 (FP32)
  float *vertices;
  float4 *pc;           // camera-frame points
  uint8_t *kind;        // 0 return, 1 no-return, 2 dead
  uint8_t *qcode;       // per block: 0 dropped, 1 FO, 2 FU
  int *cta_count;
  long long *cta_off;   // exclusive offsets (in blocks), then the total
  int n_cta;
  int32_t *faces;
  uint8_t *labels;
  long long *n_faces;
};

__global__ void __launch_bounds__(256) k_mesh_points(MeshArgs a) {
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= (long long)a.Ws * a.Hs) return;
  const int i = (int)(v % a.Ws), j = (int)(v / a.Ws);
  const int x = i * a.step, y = j * a.step;
  const long long p = (long long)y * a.W + x;
  const float d = a.depth[p];
  const int c = a.cls[p];
  const int k = (c > 1 || !(fabsf(d) <= FLT_MAX)) ? 2 : c;
  const float r = k == 0 ? d : (k == 1 ? a.max_range : 0.0f);
  float rx, ry, rz;
  if (a.model == RM_PINHOLE) {
    rx = __fdiv_rn(__fsub_rn(__fadd_rn((float)x, 0.5f), a.cx), a.fx);
    ry = __fdiv_rn(__fsub_rn(__fadd_rn((float)y, 0.5f), a.cy), a.fy);
    rz = 1.0f;
  } else {
    const float *q = a.rays + 3 * p;
    rx = q[0];
    ry = q[1];
    rz = q[2];
  }
  const float px = __fmul_rn(r, rx), py = __fmul_rn(r, ry), pz = __fmul_rn(r, rz);
  a.pc[v] = make_float4(px, py, pz, 0.0f);
  a.kind[v] = (uint8_t)k;
  for (int q = 0; q < 3; ++q) {
    const double *m = (a.Tdev ? a.Tdev : a.T) + 4 * q;
    double w = m[3];  // dead pixels stay at the sensor origin (unreferenced)
    if (k != 2)
      w = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(m[0], (double)px), __dmul_rn(m[1], (double)py)),
                              __dmul_rn(m[2], (double)pz)),
                    m[3]);
    a.vertices[3 * v + q] = (float)w;
  }
}

__device__ __forceinline__ float edge2(const float4 &a, const float4 &b) {
  const float dx = __fsub_rn(a.x, b.x), dy = __fsub_rn(a.y, b.y), dz = __fsub_rn(a.z, b.z);
  return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

__global__ void __launch_bounds__(kQuadThreads) k_mesh_quads(MeshArgs a) {
  const int qw = a.Ws - 1;
  const long long nq = (long long)qw * (a.Hs - 1);
  const long long q = (long long)blockIdx.x * kQuadThreads + threadIdx.x;
  int code = 0;
  if (q < nq) {
    const int i = (int)(q % qw), j = (int)(q / qw);
    const long long v00 = (long long)j * a.Ws + i, v10 = v00 + 1, v01 = v00 + a.Ws, v11 = v01 + 1;
    const int k00 = a.kind[v00], k10 = a.kind[v10], k01 = a.kind[v01], k11 = a.kind[v11];
    if (k00 != 2 && k10 != 2 && k01 != 2 && k11 != 2) {
      bool fu = k00 == 1 || k10 == 1 || k01 == 1 || k11 == 1;
      const float4 A = a.pc[v00], B = a.pc[v10], C = a.pc[v11], D = a.pc[v01];
      if (edge2(A, B) > a.lim || edge2(B, C) > a.lim || edge2(C, D) > a.lim || edge2(D, A) > a.lim ||
          edge2(A, C) > a.lim)
        fu = true;
      code = fu ? 2 : 1;
    }
    a.qcode[q] = (uint8_t)code;
  }
  const int kept = __syncthreads_count(code != 0);
  if (threadIdx.x == 0) a.cta_count[blockIdx.x] = kept;
}

__global__ void __launch_bounds__(1024) k_mesh_scan(MeshArgs a) {
  __shared__ long long carry;
  __shared__ long long wsum[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < a.n_cta; base += 1024) {
    const int idx = base + threadIdx.x;
    const long long c = idx < a.n_cta ? a.cta_count[idx] : 0;
    long long s = c;  // inclusive scan within the warp
    for (int off = 1; off < 32; off <<= 1) {
      const long long t = __shfl_up_sync(0xffffffffu, s, off);
      if (lane >= off) s += t;
    }
    if (lane == 31) wsum[warp] = s;
    __syncthreads();
    if (warp == 0) {
      long long w = wsum[lane];
      for (int off = 1; off < 32; off <<= 1) {
        const long long t = __shfl_up_sync(0xffffffffu, w, off);
        if (lane >= off) w += t;
      }
      wsum[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    const long long before = carry + (warp > 0 ? wsum[warp - 1] : 0) + s - c;
    if (idx < a.n_cta) a.cta_off[idx] = before;
    __syncthreads();
    if (threadIdx.x == 1023) carry = before + c;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    a.cta_off[a.n_cta] = carry;
    *a.n_faces = 2 * carry;
  }
}

__global__ void __launch_bounds__(kQuadThreads) k_mesh_emit(MeshArgs a) {
  __shared__ int wcount[kQuadThreads / 32];
  const int qw = a.Ws - 1;
  const long long nq = (long long)qw * (a.Hs - 1);
  const long long q = (long long)blockIdx.x * kQuadThreads + threadIdx.x;
  const int code = q < nq ? a.qcode[q] : 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned m = __ballot_sync(0xffffffffu, code != 0);
  if (lane == 0) wcount[warp] = __popc(m);
  __syncthreads();
  int rank = __popc(m & ((1u << lane) - 1));
  for (int w = 0; w < warp; ++w) rank += wcount[w];
  if (code == 0) return;
  const int i = (int)(q % qw), j = (int)(q / qw);
  const int v00 = j * a.Ws + i, v10 = v00 + 1, v01 = v00 + a.Ws, v11 = v01 + 1;
  const long long f = 2 * (a.cta_off[blockIdx.x] + rank);
  int32_t *o = a.faces + 3 * f;
  o[0] = v00;
  o[1] = v10;
  o[2] = v11;
  o[3] = v00;
  o[4] = v11;
  o[5] = v01;
  const uint8_t lab = code == 2 ? 1 : 0;
  a.labels[f] = lab;
  a.labels[f + 1] = lab;
}

rm_status mf_fail(rm_status s, const std::string &m) {
  rmapi::set_error(m);
  return s;
}

}  // namespace

extern "C" rm_status rm_meshify(const rm_scan *scan, const double *pose,
                                const rm_meshify_params *prm, float *vertices, int32_t *faces,
                                uint8_t *labels, int64_t *n_faces, void *stream) {
  if (!scan || !pose || !prm || !n_faces) return mf_fail(RM_EINVAL, "NULL argument");
  if (!scan->depth || !scan->cls) return mf_fail(RM_EINVAL, "scan arrays are NULL");
  rm_status st = rmapi::check_intrinsics(&scan->intr);
  if (st != RM_OK) return st;
  if (prm->step < 1 || prm->step > 64) return mf_fail(RM_EINVAL, "step must be 1..64");
  if (!(prm->max_range > 0.0f) || !(prm->max_range <= FLT_MAX))
    return mf_fail(RM_EINVAL, "max_range must be finite and > 0");
  if (!(prm->max_edge >= 0.0f) || !(prm->max_edge <= FLT_MAX))
    return mf_fail(RM_EINVAL, "max_edge must be finite and >= 0");
  cudaStream_t s = (cudaStream_t)stream;
  // a host pose is checked here and passed by value; a device pose is read by the kernel in
  // place (no host round trip; a non-finite one gives non-finite vertices)
  const bool dev_pose = rmapi::is_device_pointer(pose);
  if (!dev_pose)
    for (int k = 0; k < 12; ++k)
      if (!std::isfinite(pose[k])) return mf_fail(RM_EINVAL, "pose must be finite");
  const rm_intrinsics &in = scan->intr;
  const int Ws = (in.width - 1) / prm->step + 1, Hs = (in.height - 1) / prm->step + 1;
  const long long NV = (long long)Ws * Hs, NQ = (long long)(Ws - 1) * (Hs - 1);
  if (!vertices || (NQ > 0 && (!faces || !labels))) return mf_fail(RM_EINVAL, "NULL output array");
  const long long P = (long long)in.width * in.height;
  const bool host_d = !rmapi::is_device_pointer(scan->depth), host_c = !rmapi::is_device_pointer(scan->cls);
  const bool host_r = in.model == RM_RAYTABLE && !rmapi::is_device_pointer(in.rays);
  const bool host_v = !rmapi::is_device_pointer(vertices);
  const bool host_f = NQ > 0 && !rmapi::is_device_pointer(faces);
  const bool host_l = NQ > 0 && !rmapi::is_device_pointer(labels);
  const bool host_n = !rmapi::is_device_pointer(n_faces);
  const int n_cta = (int)std::max<long long>(1, (NQ + kQuadThreads - 1) / kQuadThreads);
  // one stream-ordered scratch block: staged inputs and outputs, then the work arrays
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off += (bytes + 255) / 256 * 256;
    return at;
  };
  const size_t o_d = host_d ? take(sizeof(float) * P) : 0, o_c = host_c ? take(P) : 0;
  const size_t o_r = host_r ? take(sizeof(float) * 3 * P) : 0;
  const size_t o_v = host_v ? take(sizeof(float) * 3 * NV) : 0;
  const size_t o_f = host_f ? take(sizeof(int32_t) * 6 * NQ) : 0;
  const size_t o_l = host_l ? take(2 * NQ) : 0;
  const size_t o_pc = take(sizeof(float4) * NV), o_k = take(NV), o_q = take(std::max<long long>(NQ, 1));
  const size_t o_cc = take(sizeof(int) * n_cta), o_co = take(sizeof(long long) * (n_cta + 1));
  const size_t o_n = take(sizeof(long long));
  unsigned char *buf = nullptr;
  cudaError_t e = cudaMallocAsync((void **)&buf, off, s);
  if (e != cudaSuccess) return mf_fail(RM_ENOMEM, std::string("rm_meshify: ") + cudaGetErrorString(e));
  auto ck = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  MeshArgs a{};
  a.model = in.model;
  a.W = in.width;
  a.H = in.height;
  a.step = prm->step;
  a.Ws = Ws;
  a.Hs = Hs;
  a.fx = in.fx;
  a.fy = in.fy;
  a.cx = in.cx;
  a.cy = in.cy;
  a.depth = host_d ? reinterpret_cast<float *>(buf + o_d) : scan->depth;
  a.cls = host_c ? buf + o_c : scan->cls;
  a.rays = host_r ? reinterpret_cast<float *>(buf + o_r) : in.rays;
  for (int k = 0; k < 12; ++k) a.T[k] = dev_pose ? 0.0 : pose[k];
  a.Tdev = dev_pose ? pose : nullptr;
  a.max_range = prm->max_range;
  a.lim = prm->max_edge * prm->max_edge;
  a.vertices = host_v ? reinterpret_cast<float *>(buf + o_v) : vertices;
  a.pc = reinterpret_cast<float4 *>(buf + o_pc);
  a.kind = buf + o_k;
  a.qcode = buf + o_q;
  a.cta_count = reinterpret_cast<int *>(buf + o_cc);
  a.cta_off = reinterpret_cast<long long *>(buf + o_co);
  a.n_cta = n_cta;
  a.faces = host_f ? reinterpret_cast<int32_t *>(buf + o_f) : faces;
  a.labels = host_l ? buf + o_l : labels;
  a.n_faces = host_n ? reinterpret_cast<long long *>(buf + o_n) : reinterpret_cast<long long *>(n_faces);
  if (host_d) ck(cudaMemcpyAsync((void *)a.depth, scan->depth, sizeof(float) * P, cudaMemcpyHostToDevice, s));
  if (host_c) ck(cudaMemcpyAsync((void *)a.cls, scan->cls, P, cudaMemcpyHostToDevice, s));
  if (host_r) ck(cudaMemcpyAsync((void *)a.rays, in.rays, sizeof(float) * 3 * P, cudaMemcpyHostToDevice, s));
  if (e == cudaSuccess) {
    k_mesh_points<<<(unsigned)((NV + 255) / 256), 256, 0, s>>>(a);
    ck(cudaGetLastError());
  }
  if (e == cudaSuccess) {
    k_mesh_quads<<<n_cta, kQuadThreads, 0, s>>>(a);
    ck(cudaGetLastError());
  }
  if (e == cudaSuccess) {
    k_mesh_scan<<<1, 1024, 0, s>>>(a);
    ck(cudaGetLastError());
  }
  if (e == cudaSuccess && NQ > 0) {
    k_mesh_emit<<<n_cta, kQuadThreads, 0, s>>>(a);
    ck(cudaGetLastError());
  }
  long long nf = 0;
  if (e == cudaSuccess && (host_n || host_f || host_l)) {
    ck(cudaMemcpyAsync(&nf, a.n_faces, sizeof(long long), cudaMemcpyDeviceToHost, s));
    ck(cudaStreamSynchronize(s));
  }
  if (e == cudaSuccess && host_v) ck(cudaMemcpyAsync(vertices, a.vertices, sizeof(float) * 3 * NV, cudaMemcpyDeviceToHost, s));
  if (e == cudaSuccess && host_f && nf > 0)
    ck(cudaMemcpyAsync(faces, a.faces, sizeof(int32_t) * 3 * nf, cudaMemcpyDeviceToHost, s));
  if (e == cudaSuccess && host_l && nf > 0) ck(cudaMemcpyAsync(labels, a.labels, nf, cudaMemcpyDeviceToHost, s));
  cudaFreeAsync(buf, s);
  if (e == cudaSuccess && (host_v || host_f || host_l || host_n)) ck(cudaStreamSynchronize(s));
  if (e != cudaSuccess) return mf_fail(RM_ECUDA, std::string("rm_meshify: ") + cudaGetErrorString(e));
  if (host_n) *n_faces = nf;
  return RM_OK;
}
