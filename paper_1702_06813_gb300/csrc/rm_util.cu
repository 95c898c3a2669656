// rm_util.cu -- input helpers: scan classes of raw range images (Sec. IV.A, IV.B) and poses
// from the paper's X = (x, y, z, theta_x, theta_y, theta_z) (Eq. 1). Elementwise kernels.
#include <cfloat>
#include <cmath>
#include <string>

#include "rendermap.h"
#include "rm_kernels.cuh"

namespace {

__global__ void __launch_bounds__(256) k_scan_from_range(const float *range, long long n, float rmin,
                                                         float rmax, float *depth, uint8_t *cls) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float r = range[i];
  float d;
  uint8_t c;
  if (isnan(r) || (r > 0.0f && r < rmin)) {  // dead, or closer than the sensor measures
    d = __int_as_float(0x7fc00000);
    c = RM_SCAN_NAN;
  } else if (r <= 0.0f || r > rmax) {  // no reading: free space up to the maximal range
    d = rmax;
    c = RM_SCAN_FU;
  } else {
    d = r;
    c = RM_SCAN_FO;
  }
  depth[i] = d;
  cls[i] = c;
}

// R = Rz(theta_z) Ry(theta_y) Rx(theta_x), translation (x, y, z).
__global__ void k_pose_from_x(const double *X, int n, double *T) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double *x = X + 6 * (long long)k;
  double sx, cx, sy, cy, sz, cz;
  sincos(x[3], &sx, &cx);
  sincos(x[4], &sy, &cy);
  sincos(x[5], &sz, &cz);
  const double R[9] = {cz * cy, cz * sy * sx - sz * cx, cz * sy * cx + sz * sx,
                       sz * cy, sz * sy * sx + cz * cx, sz * sy * cx - cz * sx,
                       -sy,     cy * sx,                cy * cx};
  double *t = T + 16 * (long long)k;
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) t[4 * i + j] = R[3 * i + j];
    t[4 * i + 3] = x[i];
  }
  t[12] = t[13] = t[14] = 0.0;
  t[15] = 1.0;
}

// Inputs of a cost sweep along one twist axis: n copies of the base pose and the twists
// t_i e_axis with t_i = -span + 2 span i / (n - 1) (t = 0 when n = 1).
__global__ void k_sweep_inputs(const double *pose, int axis, double span, int n, double *poses,
                               double *twists) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int k = 0; k < 16; ++k) poses[16 * (long long)i + k] = pose[k];
  const double t = n > 1 ? -span + 2.0 * span * (double)i / (double)(n - 1) : 0.0;
  for (int k = 0; k < 6; ++k) twists[6 * (long long)i + k] = k == axis ? t : 0.0;
}

rm_status ut_fail(rm_status s, const std::string &m) {
  rmapi::set_error(m);
  return s;
}

}  // namespace

namespace rmk {
cudaError_t launch_sweep_inputs(const double *pose, int axis, double span, int n, double *poses,
                                double *twists, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_sweep_inputs<<<(n + 63) / 64, 64, 0, s>>>(pose, axis, span, n, poses, twists);
  return cudaGetLastError();
}
}  // namespace rmk

extern "C" rm_status rm_scan_from_range(const float *range, int64_t n, float range_min,
                                        float range_max, float *depth, uint8_t *cls, void *stream) {
  if (n < 0) return ut_fail(RM_EINVAL, "n < 0");
  if (!(range_min >= 0.0f) || !(range_max > range_min) || !(range_max <= FLT_MAX))
    return ut_fail(RM_EINVAL, "need 0 <= range_min < range_max < inf");
  if (n == 0) return RM_OK;
  if (!range || !depth || !cls) return ut_fail(RM_EINVAL, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  const bool hr = !rmapi::is_device_pointer(range), hd = !rmapi::is_device_pointer(depth);
  const bool hc = !rmapi::is_device_pointer(cls);
  unsigned char *buf = nullptr;
  const size_t nb = (size_t)n;
  const size_t bytes = (hr ? 4 * nb : 0) + (hd ? 4 * nb : 0) + (hc ? nb : 0);
  cudaError_t e = cudaSuccess;
  if (bytes) e = cudaMallocAsync((void **)&buf, bytes, s);
  if (e != cudaSuccess) return ut_fail(RM_ENOMEM, std::string("rm_scan_from_range: ") + cudaGetErrorString(e));
  unsigned char *p = buf;
  const float *d_r = range;
  float *d_d = depth;
  uint8_t *d_c = cls;
  if (hr) { d_r = reinterpret_cast<float *>(p); p += 4 * nb; }
  if (hd) { d_d = reinterpret_cast<float *>(p); p += 4 * nb; }
  if (hc) d_c = p;
  auto ck = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  if (hr) ck(cudaMemcpyAsync((void *)d_r, range, 4 * nb, cudaMemcpyHostToDevice, s));
  if (e == cudaSuccess) {
    k_scan_from_range<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(d_r, n, range_min, range_max, d_d, d_c);
    ck(cudaGetLastError());
  }
  if (hd) ck(cudaMemcpyAsync(depth, d_d, 4 * nb, cudaMemcpyDeviceToHost, s));
  if (hc) ck(cudaMemcpyAsync(cls, d_c, nb, cudaMemcpyDeviceToHost, s));
  if (buf) cudaFreeAsync(buf, s);
  if (hd || hc) ck(cudaStreamSynchronize(s));
  if (e != cudaSuccess) return ut_fail(RM_ECUDA, std::string("rm_scan_from_range: ") + cudaGetErrorString(e));
  return RM_OK;
}

extern "C" rm_status rm_pose_from_x(const double *X, int32_t n, double *poses, void *stream) {
  if (n < 0) return ut_fail(RM_EINVAL, "n < 0");
  if (n == 0) return RM_OK;
  if (!X || !poses) return ut_fail(RM_EINVAL, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  const bool hx = !rmapi::is_device_pointer(X), ht = !rmapi::is_device_pointer(poses);
  double *buf = nullptr;
  cudaError_t e = cudaSuccess;
  if (hx || ht) e = cudaMallocAsync((void **)&buf, sizeof(double) * 22 * (size_t)n, s);
  if (e != cudaSuccess) return ut_fail(RM_ENOMEM, std::string("rm_pose_from_x: ") + cudaGetErrorString(e));
  const double *d_x = hx ? buf : X;
  double *d_t = ht ? buf + 6 * (size_t)n : poses;
  auto ck = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  if (hx) ck(cudaMemcpyAsync((void *)d_x, X, sizeof(double) * 6 * n, cudaMemcpyHostToDevice, s));
  if (e == cudaSuccess) {
    k_pose_from_x<<<(n + 63) / 64, 64, 0, s>>>(d_x, n, d_t);
    ck(cudaGetLastError());
  }
  if (ht) ck(cudaMemcpyAsync(poses, d_t, sizeof(double) * 16 * n, cudaMemcpyDeviceToHost, s));
  if (buf) cudaFreeAsync(buf, s);
  if (ht) ck(cudaStreamSynchronize(s));
  if (e != cudaSuccess) return ut_fail(RM_ECUDA, std::string("rm_pose_from_x: ") + cudaGetErrorString(e));
  return RM_OK;
}
