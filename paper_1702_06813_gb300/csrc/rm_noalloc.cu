// rm_noalloc.cu -- rm_cost_grad_noalloc: one pose's cost and gradient without allocating.
//
// Some callers cannot allocate device memory when they evaluate a pose: a real-time loop
// that must not call into the allocator after start-up (cudaMalloc may synchronise the
// device and has unbounded latency), code running under a memory manager that owns every
// byte of the device, or a process with a fixed memory budget. For them this entry point
// takes all of its scratch (the pose matrix, the visible-cluster list, the screen-tile bins,
// the per-tile partial sums and a status word) from one fixed-size array in device global
// memory that is part of the library itself, and calls no allocating routine.
//
// The array lives on every GPU that loads the library until the process exits. All calls
// share it, so calls whose work overlaps on the GPU (different streams, or different host
// threads without ordering) race on it and give wrong results; callers must order them.
#include <cstring>
#include <mutex>
#include <string>

#include "rendermap.h"
#include "rm_kernels.cuh"

namespace {

constexpr size_t kScratchBytes = size_t(48) << 20;  // RM_NOALLOC_SCRATCH_BYTES in rendermap.h
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch per device, looked up once with that device current.
unsigned char *g_scratch_ptr[kMaxDevices];
std::mutex g_scratch_mu;

rm_status na_fail(rm_status s, const std::string &m) {
  rmapi::set_error(m);
  return s;
}

// True when p is device (or managed) memory; *dev receives its device.
bool na_on_device(const void *p, int *dev = nullptr) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (dev) *dev = at.device;
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

extern "C" rm_status rm_cost_grad_noalloc(const rm_map *map, const rm_scan *scan,
                                          const double *pose, const rm_cost_params *params,
                                          const rm_cost_out *out, void *stream) {
  if (!map || !scan || !pose || !params || !out) return na_fail(RM_EINVAL, "NULL argument");
  if (!scan->depth || !scan->cls) return na_fail(RM_EINVAL, "scan arrays are NULL");
  // The kernels run on the current device and read the map's arrays there, so the map, the
  // scan and the outputs must all live on the current device (the call never switches).
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return na_fail(RM_ECUDA, "no usable current device");
  if (rmapi::map_device(map) != dev)
    return na_fail(RM_EINVAL, "rm_cost_grad_noalloc: the map lives on device " +
                                  std::to_string(rmapi::map_device(map)) + ", the current device is " +
                                  std::to_string(dev));
  int pd = -1;
  if (!na_on_device(scan->depth, &pd) || pd != dev || !na_on_device(scan->cls, &pd) || pd != dev)
    return na_fail(RM_EINVAL, "rm_cost_grad_noalloc needs the scan in device memory of the current device");
  const void *outs[5] = {out->counts, out->e_table, out->e_ls, out->grad, out->jtj};
  for (const void *p : outs)
    if (p && (!na_on_device(p, &pd) || pd != dev))
      return na_fail(RM_EINVAL, "rm_cost_grad_noalloc writes device outputs of the current device only");
  if (!(params->eps >= 0.0f)) return na_fail(RM_EINVAL, "eps must be >= 0");
  cudaStream_t s = (cudaStream_t)stream;

  unsigned char *base;
  {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
      void *p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
      if (e != cudaSuccess)
        return na_fail(RM_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_scratch_ptr[dev] = static_cast<unsigned char *>(p);
    }
    base = g_scratch_ptr[dev];
  }

  rmk::WaveArgs a{};
  double centre[3];
  const rm_status st = rmapi::wave_inputs(map, &scan->intr, &a, centre);
  if (st != RM_OK) return st;

  // carve the static array: status | pose | M | vis count | vis | bin counts | partials | bins
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char *p = base + off;
    off += up256(bytes);
    return p;
  };
  unsigned *d_status = reinterpret_cast<unsigned *>(take(sizeof(unsigned)));
  double *d_pose = reinterpret_cast<double *>(take(16 * sizeof(double)));
  float *d_M = reinterpret_cast<float *>(take(12 * sizeof(float)));
  int *d_vcount = reinterpret_cast<int *>(take(sizeof(int)));
  int4 *d_vis = reinterpret_cast<int4 *>(take(sizeof(int4) * (size_t)(a.n_clusters > 0 ? a.n_clusters : 1)));
  int *d_bcount = reinterpret_cast<int *>(take(sizeof(int) * (size_t)a.tg.ntiles));
  double *d_partial = reinterpret_cast<double *>(take(sizeof(double) * rmk::kNumVals * (size_t)a.tg.ntiles));
  if (off >= kScratchBytes)
    return na_fail(RM_EINVAL, "map or image too large for the static scratch (cluster list and tiles)");
  const size_t left = kScratchBytes - off;
  long long cap = (long long)(left / ((size_t)a.tg.ntiles * a.tg.rec_bytes));
  if (cap > 4096) cap = 4096;
  if (cap < 256)
    return na_fail(RM_EINVAL, "image too large for the static scratch: fewer than 256 triangle "
                              "records per screen tile would fit");
  a.tg.cap = (int)cap;
  unsigned char *d_bins = take((size_t)a.tg.rec_bytes * (size_t)cap * a.tg.ntiles);

  // everything that must start at zero is cleared by this call (counters are cleared by
  // the kernel launcher); the rest is written before it is read
  cudaError_t e;
  if ((e = cudaMemsetAsync(d_status, 0, sizeof(unsigned), s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(d_pose, pose, 16 * sizeof(double),
                           na_on_device(pose) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                           s)) != cudaSuccess ||
      (e = rmk::launch_pose_to_m(d_pose, 1, centre[0], centre[1], centre[2], d_M, s)) != cudaSuccess)
    return na_fail(RM_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
  a.n_poses = 1;
  a.wave_base = 0;
  a.Ms = d_M;
  a.vis = d_vis;
  a.vis_count = d_vcount;
  a.counts = d_bcount;
  a.bins = d_bins;
  a.partial = d_partial;
  a.status = d_status;
  a.skip = nullptr;
  a.scan_depth = scan->depth;
  a.scan_cls = scan->cls;
  a.prm = {params->eps, params->w_fofo, params->w_fofu, params->w_fufo};
  a.res_counts = reinterpret_cast<long long *>(out->counts);
  a.res_etable = reinterpret_cast<long long *>(out->e_table);
  a.res_els = out->e_ls;
  a.res_grad = out->grad;
  a.res_jtj = out->jtj;
  if ((e = rmk::launch_wave(a, rmk::kCostGrad, s)) != cudaSuccess)
    return na_fail(RM_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
  unsigned h_status = 0;
  if ((e = cudaMemcpyAsync(&h_status, d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return na_fail(RM_ECUDA, std::string("status read: ") + cudaGetErrorString(e));
  if (h_status & rmk::kStatusTimeout) return na_fail(RM_ETIMEOUT, "a device-side wait ran out of time");
  if (h_status & (rmk::kStatusOverflow | rmk::kStatusOverflowRay))
    return na_fail(RM_EOVERFLOW, "a screen-tile bin overflowed the static scratch (capacity " +
                                     std::to_string(cap) + " records per tile)");
  return RM_OK;
}
