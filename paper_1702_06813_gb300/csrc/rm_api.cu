// rm_api.cu -- the C ABI declared in include/rendermap.h.
//
// Host-side runtime: map upload (FP64 re-centring, face normals), a per-map scratch arena
// carved per call, host/device pointer handling, wave scheduling of poses, bin-capacity
// growth on overflow, the device status word and the Levenberg-Marquardt driver.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "rendermap.h"
#include "rm_kernels.cuh"

using rmk::DevCam;
using rmk::TileGeom;
using rmk::TriRec;
using rmk::WaveArgs;

namespace {

thread_local std::string g_err;

rm_status fail(rm_status s, const std::string &msg) {
  g_err = msg;
  return s;
}

#define RM_CK(call)                                                                       \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(e_ == cudaErrorMemoryAllocation ? RM_ENOMEM : RM_ECUDA,                 \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                   \
  } while (0)

#define RM_TRY(expr)               \
  do {                             \
    rm_status s_ = (expr);         \
    if (s_ != RM_OK) return s_;    \
  } while (0)

bool on_device(const void *p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Sequential carving of one allocation.
struct Carver {
  char *base;
  size_t off = 0;
  template <class T>
  T *take(size_t n) {
    off = align_up(off, 256);
    T *p = reinterpret_cast<T *>(base ? base + off : nullptr);
    off += sizeof(T) * std::max<size_t>(n, 1);
    return p;
  }
};

}  // namespace

struct rm_map {
  int device = 0;
  size_t wave_budget = size_t(4) << 30;  // per-wave scratch bytes that decide the poses per wave
  int64_t V = 0, T = 0;
  double centre[3] = {0, 0, 0};
  float4 *d_v = nullptr;
  int4 *d_faces = nullptr;
  float4 *d_planes = nullptr;
  float4 *d_vn = nullptr;  // optional world-frame vertex normals for the ICP
  int n_clusters = 0;
  int4 *d_cl_info = nullptr;
  float4 *d_cl_sphere = nullptr;
  float4 *d_cl_pos = nullptr;
  uchar4 *d_cl_tris = nullptr;
  int *d_cl_ids = nullptr;
  char *arena = nullptr;
  size_t arena_bytes = 0;
  unsigned *d_status = nullptr;
  unsigned *h_status = nullptr;
  rm_tuning tuning{};
  int cap = 512;      // records per pinhole tile bin; doubled whenever one overflows
  int cap_ray = 512;  // likewise for ray-table bins
  std::mutex mu;
  // profiling: events recorded around each kernel of each wave while enabled
  bool prof = false;
  std::vector<cudaEvent_t> ev_free;
  std::vector<std::array<cudaEvent_t, 5>> ev_pending;
  double prof_ms[4] = {0, 0, 0, 0};
  long long prof_n[4] = {0, 0, 0, 0};
  long long launches = 0;  // kernels launched since the last rm_profile(map, 1)
  // persistent batch: its launches captured once per batch shape and replayed as a graph
  cudaStream_t cap_stream = nullptr;
  // per-call waves alternate between the caller's stream and this one, so that one wave's
  // culling and setup overlap the previous wave's raster
  cudaStream_t aux_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaGraphExec_t batch_exec = nullptr;
  std::string batch_sig;
  // host copies of the batch queue, dependency counts and per-problem arguments last
  // uploaded into the arena; valid until another call carves the arena
  bool batch_inputs_valid = false;
  std::vector<int> batch_shape;
  std::vector<WaveArgs> batch_args;
};

namespace {

// 21-bit spread for a 63-bit Morton key.
uint64_t spread21(uint64_t x) {
  x &= 0x1fffff;
  x = (x | x << 32) & 0x1f00000000ffffull;
  x = (x | x << 16) & 0x1f0000ff0000ffull;
  x = (x | x << 8) & 0x100f00f00f00f00full;
  x = (x | x << 4) & 0x10c30c30c30c30c3ull;
  x = (x | x << 2) & 0x1249249249249249ull;
  return x;
}

struct Clusters {
  std::vector<int4> info;
  std::vector<float4> sphere;
  std::vector<float4> pos;  // vertex position with its global index's bits in w
  std::vector<uchar4> tris;
  std::vector<int> ids;
};

// Clusters of at most 64 triangles over at most 64 distinct vertices, grown greedily along
// the Morton order of the face centroids, each with an FP64 bounding sphere rounded outward.
void build_clusters(const std::vector<float4> &hv, const int32_t *faces, int64_t T, Clusters &cl) {
  if (T == 0) return;
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  std::vector<double> cen(3 * (size_t)T);
  for (int64_t k = 0; k < T; ++k)
    for (int a = 0; a < 3; ++a) {
      double c = 0.0;
      for (int m = 0; m < 3; ++m) {
        const float4 &v = hv[faces[3 * k + m]];
        c += a == 0 ? v.x : (a == 1 ? v.y : v.z);
      }
      c /= 3.0;
      cen[3 * k + a] = c;
      lo[a] = std::min(lo[a], c);
      hi[a] = std::max(hi[a], c);
    }
  std::vector<std::pair<uint64_t, int>> order((size_t)T);
  for (int64_t k = 0; k < T; ++k) {
    uint64_t key = 0;
    for (int a = 0; a < 3; ++a) {
      double ext = hi[a] - lo[a];
      double u = ext > 0 ? (cen[3 * k + a] - lo[a]) / ext : 0.0;
      key |= spread21((uint64_t)std::min(2097151.0, std::max(0.0, u * 2097151.0))) << a;
    }
    order[k] = {key, (int)k};
  }
  std::sort(order.begin(), order.end());
  int loc[64];
  int nv = 0, nt = 0, voff = 0, toff = 0;
  auto flush = [&]() {
    if (nt == 0) return;
    double bl[3] = {INFINITY, INFINITY, INFINITY}, bh[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int k = 0; k < nv; ++k) {
      const float4 &v = hv[loc[k]];
      const double p[3] = {v.x, v.y, v.z};
      for (int a = 0; a < 3; ++a) {
        bl[a] = std::min(bl[a], p[a]);
        bh[a] = std::max(bh[a], p[a]);
      }
    }
    const float c32[3] = {(float)(0.5 * (bl[0] + bh[0])), (float)(0.5 * (bl[1] + bh[1])),
                          (float)(0.5 * (bl[2] + bh[2]))};
    double r = 0.0;
    for (int k = 0; k < nv; ++k) {
      const float4 &v = hv[loc[k]];
      const double d[3] = {(double)v.x - c32[0], (double)v.y - c32[1], (double)v.z - c32[2]};
      r = std::max(r, std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]));
    }
    float r32 = (float)(r * (1.0 + 1e-6) + 1e-7);
    while ((double)r32 < r) r32 = std::nextafter(r32, INFINITY);
    cl.info.push_back(make_int4(voff, toff, nv, nt));
    cl.sphere.push_back(make_float4(c32[0], c32[1], c32[2], r32));
    for (int k = 0; k < nv; ++k) {
      float4 p = hv[loc[k]];
      std::memcpy(&p.w, &loc[k], sizeof(float));
      cl.pos.push_back(p);
    }
    voff += nv;
    toff += nt;
    nv = nt = 0;
  };
  for (const auto &o : order) {
    const int32_t *f = faces + 3 * (int64_t)o.second;
    int li[3], fresh = 0;
    for (int m = 0; m < 3; ++m) {
      li[m] = -1;
      for (int k = 0; k < nv; ++k)
        if (loc[k] == f[m]) li[m] = k;
      for (int q = 0; q < m; ++q)
        if (li[m] < 0 && f[q] == f[m]) li[m] = -2 - q;  // repeated index within the face
      fresh += li[m] == -1;
    }
    if (nt + 1 > 64 || nv + fresh > 64) {
      flush();
      for (int m = 0; m < 3; ++m) {
        li[m] = -1;
        for (int q = 0; q < m; ++q)
          if (f[q] == f[m]) li[m] = -2 - q;
      }
    }
    for (int m = 0; m < 3; ++m) {
      if (li[m] == -1) {
        loc[nv] = f[m];
        li[m] = nv++;
      } else if (li[m] <= -2) {
        li[m] = li[-2 - li[m]];
      }
    }
    cl.tris.push_back(make_uchar4((unsigned char)li[0], (unsigned char)li[1], (unsigned char)li[2], 0));
    cl.ids.push_back(o.second);
    ++nt;
  }
  flush();
}

rm_status ensure_arena(rm_map *m, size_t bytes, cudaStream_t s) {
  if (bytes <= m->arena_bytes) return RM_OK;
  RM_CK(cudaStreamSynchronize(s));
  if (m->batch_exec) {  // the captured batch graph points into the old arena
    cudaGraphExecDestroy(m->batch_exec);
    m->batch_exec = nullptr;
    m->batch_sig.clear();
  }
  m->batch_inputs_valid = false;
  if (m->arena) RM_CK(cudaFree(m->arena));
  m->arena = nullptr;
  m->arena_bytes = 0;
  size_t want = align_up(bytes + bytes / 8, 1 << 20);
  RM_CK(cudaMalloc(&m->arena, want));
  m->arena_bytes = want;
  return RM_OK;
}

rm_status check_intr(const rm_intrinsics *in) {
  if (!in) return fail(RM_EINVAL, "intrinsics is NULL");
  if (in->width < 1 || in->height < 1 || in->width > 16384 || in->height > 16384)
    return fail(RM_EINVAL, "image size must be 1..16384");
  if (!(in->near_m > 0.0f) || !(in->far_m >= in->near_m))
    return fail(RM_EINVAL, "need 0 < near_m <= far_m");
  if (in->model == RM_PINHOLE) {
    if (!(std::isfinite(in->fx) && std::isfinite(in->fy) && in->fx != 0.0f && in->fy != 0.0f &&
          std::isfinite(in->cx) && std::isfinite(in->cy)))
      return fail(RM_EINVAL, "pinhole fx, fy must be finite and non-zero, cx, cy finite");
    return RM_OK;
  }
  if (in->model == RM_RAYTABLE) {
    if (!in->rays) return fail(RM_EINVAL, "ray-table camera needs its rays");
    if (!(in->az_step > 0.0f && in->el_step > 0.0f && std::isfinite(in->az0) && std::isfinite(in->el0)))
      return fail(RM_EINVAL, "ray-table layout needs az_step > 0, el_step > 0 and finite az0, el0");
    return RM_OK;
  }
  return fail(RM_EINVAL, "unknown camera model");
}

TileGeom make_tiles(const rm_map *m, const rm_intrinsics *in) {
  TileGeom tg;
  // default: the persistent kernel's tile for the camera model (64x32 pinhole, 16x16 ray table)
  const int md = in->model == RM_RAYTABLE ? 1 : 0;
  tg.tw = m->tuning.tile_w > 0 ? m->tuning.tile_w : rmk::kPersistTileW[md];
  tg.th = m->tuning.tile_h > 0 ? m->tuning.tile_h : rmk::kPersistTileH[md];
  tg.ntx = (in->width + tg.tw - 1) / tg.tw;
  tg.nty = (in->height + tg.th - 1) / tg.th;
  tg.ntiles = tg.ntx * tg.nty;
  tg.cap = in->model == RM_RAYTABLE ? m->cap_ray : m->cap;
  tg.rec_bytes = in->model == RM_RAYTABLE ? (int)sizeof(rmk::RayRec) : (int)sizeof(TriRec);
  return tg;
}

DevCam make_cam(const rm_intrinsics *in, const float *d_rays) {
  DevCam c;
  c.model = in->model;
  c.W = in->width;
  c.H = in->height;
  c.pad = 0;
  c.fx = in->fx;
  c.fy = in->fy;
  c.cx = in->cx;
  c.cy = in->cy;
  c.az0 = in->az0;
  c.az_step = in->az_step;
  c.el0 = in->el0;
  c.el_step = in->el_step;
  c.near_m = in->near_m;
  c.far_m = in->far_m;
  c.w_near = 1.0f / in->near_m;  // FP32 division, round to nearest (host and oracle alike)
  c.w_far = 1.0f / in->far_m;
  c.rays = d_rays;
  return c;
}

int wave_size(const rm_map *m, int n, const TileGeom &tg) {
  if (m->tuning.wave_poses > 0) return std::min(n, m->tuning.wave_poses);
  // up to 128 poses per wave, keeping the per-wave scratch within the map's wave budget
  size_t per = (size_t)m->n_clusters * sizeof(int4) + (size_t)tg.ntiles * ((size_t)tg.cap * tg.rec_bytes + 8 * 40);
  size_t w = std::max<size_t>(1, m->wave_budget / std::max<size_t>(per, 1));
  return (int)std::min<size_t>(std::min<size_t>(w, 128), (size_t)n);
}

// Budget of the map's bounded device waits in cycles (dflt unless the tuning sets wait_log2).
long long wait_budget(const rm_map *m, long long dflt) {
  return m->tuning.wait_log2 > 0 ? (1ll << m->tuning.wait_log2) : dflt;
}

// The map's clusters and its wait budget in a wave's arguments.
void set_map_fields(const rm_map *m, WaveArgs &a) {
  a.wait_cycles = wait_budget(m, 0);
  a.vnormals = m->d_vn;
  a.n_clusters = m->n_clusters;
  a.cl_info = m->d_cl_info;
  a.cl_sphere = m->d_cl_sphere;
  a.cl_pos = m->d_cl_pos;
  a.cl_tris = m->d_cl_tris;
  a.cl_ids = m->d_cl_ids;
}

rm_status take_events(rm_map *m, cudaEvent_t *ev) {
  for (int k = 0; k < 5; ++k) {
    if (m->ev_free.empty()) {
      cudaEvent_t e;
      RM_CK(cudaEventCreate(&e));
      m->ev_free.push_back(e);
    }
    ev[k] = m->ev_free.back();
    m->ev_free.pop_back();
  }
  return RM_OK;
}

rm_status drain_events(rm_map *m) {
  for (auto &ev : m->ev_pending) {
    RM_CK(cudaEventSynchronize(ev[4]));
    for (int k = 0; k < 4; ++k) {
      float ms = 0.0f;
      RM_CK(cudaEventElapsedTime(&ms, ev[k], ev[k + 1]));
      m->prof_ms[k] += ms;
      m->prof_n[k] += 1;
    }
    for (auto e : ev) m->ev_free.push_back(e);
  }
  m->ev_pending.clear();
  return RM_OK;
}

// One wave, with events around its kernels when profiling.
rm_status wave(rm_map *m, const WaveArgs &a, int mode, cudaStream_t s, bool zero_counters = true) {
  cudaEvent_t ev[5];
  if (m->prof) RM_TRY(take_events(m, ev));
  RM_CK(rmk::launch_wave(a, mode, s, m->prof ? ev : nullptr, zero_counters));
  m->launches += rmk::wave_kernel_launches(a, mode);
  if (m->prof) m->ev_pending.push_back({ev[0], ev[1], ev[2], ev[3], ev[4]});
  return RM_OK;
}

// Doubles the capacity of the bins that overflowed (pinhole and ray-table tracked apart).
rm_status grow_bins(rm_map *m, unsigned st, int attempt) {
  const bool pin = st & rmk::kStatusOverflow, ray = st & rmk::kStatusOverflowRay;
  if (attempt > 16 || (pin && m->cap >= (1 << 22)) || (ray && m->cap_ray >= (1 << 22)))
    return fail(RM_EOVERFLOW, "screen-tile bin overflow at the largest capacity");
  if (pin) m->cap *= 2;
  if (ray) m->cap_ray *= 2;
  return RM_OK;
}

// Read back and clear the device status word.
rm_status read_status(rm_map *m, cudaStream_t s, unsigned *out) {
  RM_CK(cudaMemcpyAsync(m->h_status, m->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  RM_CK(cudaMemsetAsync(m->d_status, 0, sizeof(unsigned), s));
  RM_CK(cudaStreamSynchronize(s));
  *out = *m->h_status;
  return RM_OK;
}

rm_status copy_out(void *dst, const void *src, size_t bytes, cudaStream_t s, bool *host_out) {
  if (!dst || bytes == 0) return RM_OK;
  bool dev = on_device(dst);
  if (!dev) *host_out = true;
  RM_CK(cudaMemcpyAsync(dst, src, bytes, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  return RM_OK;
}

// Shared driver of rm_render_depth / rm_cost / rm_cost_grad.
struct EvalReq {
  const rm_intrinsics *intr;
  const rm_scan *scan;
  const double *poses;
  int n;
  const rm_cost_params *prm;
  int mode;
  const rm_cost_out *out;
  const rm_icp_out *icp;  // kIcp: outputs (the tolerance is prm->eps)
  float *depth;
  int32_t *tri_id;
  float *bary;
};

rm_status run_eval(rm_map *m, const EvalReq &r, cudaStream_t s) {
  const rm_intrinsics *in = r.intr;
  RM_TRY(check_intr(in));
  if (r.n < 0) return fail(RM_EINVAL, "n_poses < 0");
  if (!r.poses && r.n > 0) return fail(RM_EINVAL, "poses is NULL");
  if (r.mode == rmk::kRender && !r.depth && r.n > 0) return fail(RM_EINVAL, "depth is NULL");
  if (r.mode != rmk::kRender) {
    if (!r.scan || !r.scan->depth || !r.scan->cls) return fail(RM_EINVAL, "scan or its arrays NULL");
    if (!r.prm) return fail(RM_EINVAL, "params is NULL");
    if (!(r.prm->eps >= 0.0f)) return fail(RM_EINVAL, "eps must be >= 0");
  }
  if (r.n == 0) return RM_OK;
  RM_CK(cudaSetDevice(m->device));
  const long long P = (long long)in->width * in->height;
  const bool host_poses = !on_device(r.poses);
  const bool host_rays = in->model == RM_RAYTABLE && !on_device(in->rays);
  const bool host_scan = r.mode != rmk::kRender && !on_device(r.scan->depth);
  const bool host_cls = r.mode != rmk::kRender && !on_device(r.scan->cls);
  const bool dev_depth = r.mode == rmk::kRender && on_device(r.depth);
  const bool dev_id = r.tri_id && on_device(r.tri_id);
  const bool dev_bary = r.bary && on_device(r.bary);
  // cost outputs in device memory are written by the kernels in place; host ones are staged
  const bool cost_mode = r.mode != rmk::kRender && r.out;
  const bool grad_mode = cost_mode && r.mode == rmk::kCostGrad;
  const bool dev_counts = cost_mode && r.out->counts && on_device(r.out->counts);
  const bool dev_etable = cost_mode && r.out->e_table && on_device(r.out->e_table);
  const bool dev_els = cost_mode && r.out->e_ls && on_device(r.out->e_ls);
  const bool dev_grad = grad_mode && r.out->grad && on_device(r.out->grad);
  const bool dev_jtj = grad_mode && r.out->jtj && on_device(r.out->jtj);
  const bool icp_mode = r.mode == rmk::kIcp && r.icp;
  const bool dev_n = icp_mode && r.icp->n_assoc && on_device(r.icp->n_assoc);
  const bool dev_l1 = icp_mode && r.icp->cost_l1 && on_device(r.icp->cost_l1);
  const bool dev_e2 = icp_mode && r.icp->e2 && on_device(r.icp->e2);
  const bool dev_jte = icp_mode && r.icp->jte && on_device(r.icp->jte);
  const bool dev_ijtj = icp_mode && r.icp->jtj && on_device(r.icp->jtj);

  for (int attempt = 0;; ++attempt) {
    TileGeom tg = make_tiles(m, in);
    const int nw = wave_size(m, r.n, tg);
    // ---- plan the arena
    Carver plan{nullptr};
    if (host_poses) plan.take<double>(16 * (size_t)r.n);
    plan.take<float>(12 * (size_t)r.n);
    if (host_rays) plan.take<float>(3 * P);
    if (host_scan) plan.take<float>(P);
    if (host_cls) plan.take<uint8_t>(P);
    plan.take<long long>(6 * (size_t)r.n);
    plan.take<long long>(r.n);
    plan.take<double>(r.n);
    plan.take<double>(6 * (size_t)r.n);
    plan.take<double>(21 * (size_t)r.n);
    plan.take<double>(r.n);
    if (r.mode == rmk::kRender) {
      if (!dev_depth) plan.take<float>(P * r.n);
      if (r.tri_id && !dev_id) plan.take<int>(P * r.n);
      if (r.bary && !dev_bary) plan.take<float>(2 * P * r.n);
    }
    // two sets of per-wave buffers when there are several waves: consecutive waves run on
    // two streams and overlap (not while profiling, whose per-kernel intervals would then
    // include the other stream's kernels)
    const int nbuf = r.n > nw && !m->prof ? 2 : 1;
    plan.take<int4>((size_t)m->n_clusters * nw * nbuf);
    plan.take<int>((size_t)(tg.ntiles + 1) * r.n);
    plan.take<unsigned char>((size_t)tg.ntiles * tg.cap * nw * tg.rec_bytes * nbuf);
    plan.take<double>((size_t)tg.ntiles * rmk::kNumVals * nw * nbuf);
    RM_TRY(ensure_arena(m, plan.off, s));
    m->batch_inputs_valid = false;
    // ---- carve it
    Carver cv{m->arena};
    const double *d_poses = host_poses ? cv.take<double>(16 * (size_t)r.n) : r.poses;
    float *d_M = cv.take<float>(12 * (size_t)r.n);
    const float *d_rays = in->rays;
    if (host_rays) d_rays = cv.take<float>(3 * P);
    const float *d_sd = nullptr;
    const uint8_t *d_sc = nullptr;
    if (r.mode != rmk::kRender) {
      d_sd = host_scan ? cv.take<float>(P) : r.scan->depth;
      d_sc = host_cls ? cv.take<uint8_t>(P) : r.scan->cls;
    }
    long long *d_counts = cv.take<long long>(6 * (size_t)r.n);
    long long *d_etable = cv.take<long long>(r.n);
    double *d_els = cv.take<double>(r.n);
    double *d_grad = cv.take<double>(6 * (size_t)r.n);
    double *d_jtj = cv.take<double>(21 * (size_t)r.n);
    double *d_l1 = cv.take<double>(r.n);
    float *d_depth = nullptr;
    int *d_id = nullptr;
    float *d_bary = nullptr;
    if (r.mode == rmk::kRender) {
      d_depth = dev_depth ? r.depth : cv.take<float>(P * r.n);
      if (r.tri_id) d_id = dev_id ? r.tri_id : cv.take<int>(P * r.n);
      if (r.bary) d_bary = dev_bary ? r.bary : cv.take<float>(2 * P * r.n);
    }
    int4 *d_vis = cv.take<int4>((size_t)m->n_clusters * nw * nbuf);
    // every pose's bin counts and visible-cluster count, zeroed together once per call
    int *d_bcount = cv.take<int>((size_t)(tg.ntiles + 1) * r.n);
    int *d_vcount = d_bcount + (size_t)tg.ntiles * r.n;
    unsigned char *d_bins = cv.take<unsigned char>((size_t)tg.ntiles * tg.cap * nw * tg.rec_bytes * nbuf);
    double *d_partial = cv.take<double>((size_t)tg.ntiles * rmk::kNumVals * nw * nbuf);
    // ---- inputs
    if (host_poses)
      RM_CK(cudaMemcpyAsync((void *)d_poses, r.poses, sizeof(double) * 16 * r.n, cudaMemcpyHostToDevice, s));
    if (host_rays) RM_CK(cudaMemcpyAsync((void *)d_rays, in->rays, sizeof(float) * 3 * P, cudaMemcpyHostToDevice, s));
    if (host_scan) RM_CK(cudaMemcpyAsync((void *)d_sd, r.scan->depth, sizeof(float) * P, cudaMemcpyHostToDevice, s));
    if (host_cls) RM_CK(cudaMemcpyAsync((void *)d_sc, r.scan->cls, P, cudaMemcpyHostToDevice, s));
    RM_CK(rmk::launch_pose_to_m(d_poses, r.n, m->centre[0], m->centre[1], m->centre[2], d_M, s));
    RM_CK(cudaMemsetAsync(d_bcount, 0, sizeof(int) * (size_t)(tg.ntiles + 1) * r.n, s));
    m->launches += 1;
    // ---- waves
    WaveArgs a{};
    a.cam = make_cam(in, d_rays);
    a.tg = tg;
    a.V = (int)m->V;
    a.T = m->T;
    a.v = m->d_v;
    a.faces = m->d_faces;
    a.planes = m->d_planes;
    a.Ms = d_M;
    set_map_fields(m, a);
    a.vis = d_vis;
    a.vis_count = d_vcount;
    a.counts = d_bcount;
    a.bins = d_bins;
    a.partial = d_partial;
    a.status = m->d_status;
    a.skip = nullptr;
    a.scan_depth = d_sd;
    a.scan_cls = d_sc;
    if (r.prm) a.prm = {r.prm->eps, r.prm->w_fofo, r.prm->w_fofu, r.prm->w_fufo};
    a.res_counts = dev_counts ? reinterpret_cast<long long *>(r.out->counts) : d_counts;
    a.res_etable = dev_etable ? reinterpret_cast<long long *>(r.out->e_table) : d_etable;
    a.res_els = dev_els ? r.out->e_ls : d_els;
    a.res_grad = dev_grad ? r.out->grad : d_grad;
    a.res_jtj = dev_jtj ? r.out->jtj : d_jtj;
    if (r.mode == rmk::kIcp) {
      a.res_counts = nullptr;
      a.res_etable = nullptr;
      a.res_n = dev_n ? reinterpret_cast<long long *>(r.icp->n_assoc) : d_counts;
      a.res_l1 = dev_l1 ? r.icp->cost_l1 : d_l1;
      a.res_els = dev_e2 ? r.icp->e2 : d_els;
      a.res_grad = dev_jte ? r.icp->jte : d_grad;
      a.res_jtj = dev_ijtj ? r.icp->jtj : d_jtj;
    }
    a.depth = d_depth;
    a.tri_id = d_id;
    a.bary = d_bary;
    if (nbuf == 2) {
      if (!m->aux_stream) RM_CK(cudaStreamCreateWithFlags(&m->aux_stream, cudaStreamNonBlocking));
      if (!m->ev_fork) RM_CK(cudaEventCreateWithFlags(&m->ev_fork, cudaEventDisableTiming));
      if (!m->ev_join) RM_CK(cudaEventCreateWithFlags(&m->ev_join, cudaEventDisableTiming));
      RM_CK(cudaEventRecord(m->ev_fork, s));
      RM_CK(cudaStreamWaitEvent(m->aux_stream, m->ev_fork, 0));
    }
    for (int w0 = 0, k = 0; w0 < r.n; w0 += nw, ++k) {
      const int b = k % nbuf;  // buffer set and stream of this wave
      a.wave_base = w0;
      a.n_poses = std::min(nw, r.n - w0);
      a.counts = d_bcount + (size_t)w0 * tg.ntiles;
      a.vis_count = d_vcount + w0;
      a.vis = d_vis + (size_t)m->n_clusters * nw * b;
      a.bins = d_bins + (size_t)tg.ntiles * tg.cap * nw * tg.rec_bytes * b;
      a.partial = d_partial + (size_t)tg.ntiles * rmk::kNumVals * nw * b;
      RM_TRY(wave(m, a, r.mode, b == 0 ? s : m->aux_stream, false));
    }
    if (nbuf == 2) {
      RM_CK(cudaEventRecord(m->ev_join, m->aux_stream));
      RM_CK(cudaStreamWaitEvent(s, m->ev_join, 0));
    }
    // ---- outputs
    bool host_out = false;
    if (r.mode == rmk::kRender) {
      if (!dev_depth) RM_TRY(copy_out(r.depth, d_depth, sizeof(float) * P * r.n, s, &host_out));
      if (r.tri_id && !dev_id) RM_TRY(copy_out(r.tri_id, d_id, sizeof(int) * P * r.n, s, &host_out));
      if (r.bary && !dev_bary) RM_TRY(copy_out(r.bary, d_bary, sizeof(float) * 2 * P * r.n, s, &host_out));
    } else if (icp_mode) {
      if (!dev_n) RM_TRY(copy_out(r.icp->n_assoc, d_counts, sizeof(long long) * r.n, s, &host_out));
      if (!dev_l1) RM_TRY(copy_out(r.icp->cost_l1, d_l1, sizeof(double) * r.n, s, &host_out));
      if (!dev_e2) RM_TRY(copy_out(r.icp->e2, d_els, sizeof(double) * r.n, s, &host_out));
      if (!dev_jte) RM_TRY(copy_out(r.icp->jte, d_grad, sizeof(double) * 6 * r.n, s, &host_out));
      if (!dev_ijtj) RM_TRY(copy_out(r.icp->jtj, d_jtj, sizeof(double) * 21 * r.n, s, &host_out));
    } else if (r.mode != rmk::kIcp && r.out) {
      if (!dev_counts) RM_TRY(copy_out(r.out->counts, d_counts, sizeof(long long) * 6 * r.n, s, &host_out));
      if (!dev_etable) RM_TRY(copy_out(r.out->e_table, d_etable, sizeof(long long) * r.n, s, &host_out));
      if (!dev_els) RM_TRY(copy_out(r.out->e_ls, d_els, sizeof(double) * r.n, s, &host_out));
      if (r.mode == rmk::kCostGrad) {
        if (!dev_grad) RM_TRY(copy_out(r.out->grad, d_grad, sizeof(double) * 6 * r.n, s, &host_out));
        if (!dev_jtj) RM_TRY(copy_out(r.out->jtj, d_jtj, sizeof(double) * 21 * r.n, s, &host_out));
      }
    }
    if (m->tuning.async_status) {
      if (host_out) RM_CK(cudaStreamSynchronize(s));
      return RM_OK;
    }
    unsigned st = 0;
    RM_TRY(read_status(m, s, &st));
    if (st & rmk::kStatusTimeout) return fail(RM_ETIMEOUT, "a device-side wait ran out of time");
    if (st & (rmk::kStatusOverflow | rmk::kStatusOverflowRay)) {
      RM_TRY(grow_bins(m, st, attempt));
      continue;
    }
    return RM_OK;
  }
}

}  // namespace

namespace {

// Raster items of one problem in the persistent queue.
int raster_items(const TileGeom &tg, int model) {
  const int per = rmk::kPersistTiles[model == RM_RAYTABLE ? 1 : 0];
  return (tg.ntiles + per - 1) / per;
}

// Shared driver of rm_cost_grad_batch (lm == icp == nullptr), rm_align_batch (lm) and
// rm_icp_align_batch (icp; prm->eps then carries the association tolerance).
rm_status run_batch(rm_map *m, const rm_problem *probs, int n, const rm_cost_params *prm,
                    const rm_align_params *lm, const rm_cost_out *out, double *poses_out,
                    rm_align_report *reps, cudaStream_t s, const rm_icp_params *icp = nullptr,
                    rm_icp_report *ireps = nullptr) {
  if (n < 0) return fail(RM_EINVAL, "n < 0");
  if (n == 0) return RM_OK;
  if (n >= (1 << rmk::kItemProblemBits)) return fail(RM_EINVAL, "too many problems in one batch");
  if (!probs || !prm) return fail(RM_EINVAL, "NULL argument");
  if (!(prm->eps >= 0.0f)) return fail(RM_EINVAL, "eps must be >= 0");
  if (lm && (lm->max_iters < 0 || lm->max_iters > 100000)) return fail(RM_EINVAL, "max_iters out of range");
  if (icp && (icp->max_iters < 1 || icp->max_iters > 100000)) return fail(RM_EINVAL, "max_iters out of range (1..100000)");
  if ((lm || icp) && !poses_out) return fail(RM_EINVAL, "poses_out is NULL");
  for (int p = 0; p < n; ++p) {
    RM_TRY(check_intr(&probs[p].scan.intr));
    if (!probs[p].scan.depth || !probs[p].scan.cls || !probs[p].pose)
      return fail(RM_EINVAL, "problem " + std::to_string(p) + ": NULL scan array or pose");
  }
  RM_CK(cudaSetDevice(m->device));
  const int K = lm ? lm->max_iters : (icp ? icp->max_iters - 1 : 0);
  const int nc = m->n_clusters;
  // at least one item per phase, so that every phase completes and publishes the next
  const int ncull = std::max(1, ((nc + 255) / 256 + rmk::kPersistCull - 1) / rmk::kPersistCull);
  // setup items per evaluation are set on the device from the visible clusters; at most
  const int max_setup = std::max(1, (nc + rmk::kSetupClusters - 1) / rmk::kSetupClusters);
  if (max_setup >= (1 << rmk::kItemIndexBits)) return fail(RM_EINVAL, "map has too many clusters for a batch");
  for (int attempt = 0;; ++attempt) {
    std::vector<TileGeom> tg(n);
    std::vector<long long> P(n);
    size_t tiles_total = 0, bins_bytes = 0, px_total = 0, rays_total = 0;
    // problems that share a scan (same arrays) share one staged copy; likewise ray tables
    std::vector<int> scan_of(n), rays_of(n, -1);
    {
      using Key = std::tuple<const void *, const void *, int, int>;
      std::map<Key, int> scans, rays;
      for (int p = 0; p < n; ++p) {
        const rm_scan &sc = probs[p].scan;
        scan_of[p] = scans.emplace(Key(sc.depth, sc.cls, sc.intr.width, sc.intr.height), p).first->second;
        if (sc.intr.model == RM_RAYTABLE)
          rays_of[p] = rays.emplace(Key(sc.intr.rays, nullptr, sc.intr.width, sc.intr.height), p).first->second;
      }
    }
    for (int p = 0; p < n; ++p) {
      const rm_intrinsics *in = &probs[p].scan.intr;
      const int md = in->model == RM_RAYTABLE ? 1 : 0;
      tg[p].tw = rmk::kPersistTileW[md];
      tg[p].th = rmk::kPersistTileH[md];
      tg[p].ntx = (in->width + tg[p].tw - 1) / tg[p].tw;
      tg[p].nty = (in->height + tg[p].th - 1) / tg[p].th;
      tg[p].ntiles = tg[p].ntx * tg[p].nty;
      tg[p].cap = in->model == RM_RAYTABLE ? m->cap_ray : m->cap;
      tg[p].rec_bytes = in->model == RM_RAYTABLE ? (int)sizeof(rmk::RayRec) : (int)sizeof(TriRec);
      P[p] = (long long)in->width * in->height;
      tiles_total += tg[p].ntiles;
      bins_bytes += align_up((size_t)tg[p].ntiles * tg[p].cap * tg[p].rec_bytes, 256);
      if (scan_of[p] == p) px_total += align_up((size_t)P[p], 64);
      if (rays_of[p] == p) rays_total += 3 * (size_t)P[p];
    }
    // the ready queue: one slot per item of every evaluation of every problem; the kernel
    // publishes a problem's items phase by phase. The dependency counts are a function of
    // `shape` alone and are re-sent only when it changes or the arena was reused.
    std::vector<int> shape = {n, K, ncull};
    size_t cap_hi = 0, cap_lo = 0;  // raster + reduce slots, cull + setup slots
    for (int p = 0; p < n; ++p) {
      const int nr = raster_items(tg[p], probs[p].scan.intr.model);
      shape.push_back(nr);
      cap_hi += (size_t)(K + 1) * (nr + 1);
      cap_lo += (size_t)(K + 1) * (ncull + max_setup);
    }
    const bool same_shape = shape == m->batch_shape;
    std::vector<int> need(3 * (size_t)n);
    for (int p = 0; p < n; ++p) {
      need[3 * p] = ncull;
      need[3 * p + 1] = 0;  // set by the kernel
      need[3 * p + 2] = raster_items(tg[p], probs[p].scan.intr.model);
    }
    // ---- plan and carve the arena
    auto layout = [&](Carver &cv, bool carve, WaveArgs **d_args, long long **d_items, int **d_next,
                      int **d_done, int **d_need, float **d_M, int **d_skip, double **d_poses,
                      rmk::LMState **d_lm, int **d_vcount, int4 **d_vis, int **d_counts,
                      double **d_partial, unsigned char **d_bins, float **d_sd, uint8_t **d_sc,
                      float **d_rays, long long **r_counts, long long **r_et, double **r_els,
                      double **r_grad, double **r_jtj, rmk::IcpState **d_icp, double **r_l1) {
      (void)carve;
      *d_args = cv.take<WaveArgs>(n);
      *d_items = cv.take<long long>(cap_hi + cap_lo);
      *d_next = cv.take<int>(8);  // queue heads and tails, finished problems
      *d_done = cv.take<int>(4 * (size_t)n);
      *d_need = cv.take<int>(3 * (size_t)n);
      *d_M = cv.take<float>(12 * (size_t)n);
      *d_skip = cv.take<int>(n);
      *d_poses = cv.take<double>(16 * (size_t)n);
      *d_lm = cv.take<rmk::LMState>(n);
      *d_vcount = cv.take<int>(n);
      *d_vis = cv.take<int4>((size_t)n * std::max(nc, 1));
      *d_counts = cv.take<int>(tiles_total);
      *d_partial = cv.take<double>(tiles_total * rmk::kNumVals);
      *d_bins = cv.take<unsigned char>(bins_bytes);
      *d_sd = cv.take<float>(px_total);
      *d_sc = cv.take<uint8_t>(px_total);
      *d_rays = cv.take<float>(std::max<size_t>(rays_total, 1));
      *r_counts = cv.take<long long>(6 * (size_t)n);
      *r_et = cv.take<long long>(n);
      *r_els = cv.take<double>(n);
      *r_grad = cv.take<double>(6 * (size_t)n);
      *r_jtj = cv.take<double>(21 * (size_t)n);
      *d_icp = cv.take<rmk::IcpState>(n);
      *r_l1 = cv.take<double>(n);
    };
    WaveArgs *d_args; long long *d_items; int4 *d_vis; int *d_next, *d_done, *d_need, *d_skip, *d_vcount, *d_counts;
    float *d_M, *d_sd, *d_rays; double *d_poses, *d_partial, *r_els, *r_grad, *r_jtj; rmk::LMState *d_lm;
    unsigned char *d_bins; uint8_t *d_sc; long long *r_counts, *r_et;
    rmk::IcpState *d_icp; double *r_l1;
    Carver plan{nullptr};
    layout(plan, false, &d_args, &d_items, &d_next, &d_done, &d_need, &d_M, &d_skip, &d_poses, &d_lm,
           &d_vcount, &d_vis, &d_counts, &d_partial, &d_bins, &d_sd, &d_sc, &d_rays, &r_counts, &r_et,
           &r_els, &r_grad, &r_jtj, &d_icp, &r_l1);
    RM_TRY(ensure_arena(m, plan.off, s));
    Carver cv{m->arena};
    layout(cv, true, &d_args, &d_items, &d_next, &d_done, &d_need, &d_M, &d_skip, &d_poses, &d_lm,
           &d_vcount, &d_vis, &d_counts, &d_partial, &d_bins, &d_sd, &d_sc, &d_rays, &r_counts, &r_et,
           &r_els, &r_grad, &r_jtj, &d_icp, &r_l1);
    // ---- per-problem arguments and inputs
    // poses laid out back to back (one n x 16 array) are copied in one call
    bool poses_contiguous = true;
    for (int p = 1; p < n && poses_contiguous; ++p) poses_contiguous = probs[p].pose == probs[0].pose + 16 * (size_t)p;
    if (poses_contiguous)
      RM_CK(cudaMemcpyAsync(d_poses, probs[0].pose, sizeof(double) * 16 * n,
                            on_device(probs[0].pose) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    std::vector<WaveArgs> args(n);
    std::vector<size_t> px_at(n), rays_at(n);
    size_t t_off = 0, b_off = 0, px_off = 0, r_off = 0;
    for (int p = 0; p < n; ++p) {
      const rm_scan &sc = probs[p].scan;
      const rm_intrinsics *in = &sc.intr;
      float *rays = nullptr;
      if (in->model == RM_RAYTABLE) {
        if (rays_of[p] == p) {
          rays_at[p] = r_off;
          r_off += 3 * (size_t)P[p];
          RM_CK(cudaMemcpyAsync(d_rays + rays_at[p], in->rays, sizeof(float) * 3 * P[p],
                                on_device(in->rays) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
        } else {
          rays_at[p] = rays_at[rays_of[p]];
        }
        rays = d_rays + rays_at[p];
      }
      if (scan_of[p] == p) {
        px_at[p] = px_off;
        px_off += align_up((size_t)P[p], 64);
        RM_CK(cudaMemcpyAsync(d_sd + px_at[p], sc.depth, sizeof(float) * P[p],
                              on_device(sc.depth) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
        RM_CK(cudaMemcpyAsync(d_sc + px_at[p], sc.cls, (size_t)P[p],
                              on_device(sc.cls) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
      } else {
        px_at[p] = px_at[scan_of[p]];
      }
      if (!poses_contiguous)
        RM_CK(cudaMemcpyAsync(d_poses + 16 * (size_t)p, probs[p].pose, sizeof(double) * 16,
                              on_device(probs[p].pose) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
      WaveArgs &a = args[p];
      std::memset(&a, 0, sizeof(WaveArgs));  // padding too: the argument block is compared bytewise
      a.cam = make_cam(in, rays);
      a.tg = tg[p];
      a.V = (int)m->V;
      a.T = m->T;
      a.n_poses = 1;
      a.wave_base = 0;
      a.v = m->d_v;
      a.faces = m->d_faces;
      a.planes = m->d_planes;
      set_map_fields(m, a);
      a.Ms = d_M + 12 * (size_t)p;
      a.vis = d_vis + (size_t)p * std::max(nc, 1);
      a.vis_count = d_vcount + p;
      a.counts = d_counts + t_off;
      a.bins = d_bins + b_off;
      a.partial = d_partial + t_off * rmk::kNumVals;
      a.status = m->d_status;
      a.skip = d_skip + p;
      a.scan_depth = d_sd + px_at[p];
      a.scan_cls = d_sc + px_at[p];
      a.prm = {prm->eps, prm->w_fofo, prm->w_fofu, prm->w_fufo};
      a.res_counts = r_counts + 6 * (size_t)p;
      a.res_etable = r_et + p;
      a.res_els = r_els + p;
      a.res_grad = r_grad + 6 * (size_t)p;
      a.res_jtj = r_jtj + 21 * (size_t)p;
      if (icp) {  // ICP terms: associations, C, e^2, J^T e, J^T J
        a.res_counts = nullptr;
        a.res_etable = nullptr;
        a.res_n = r_counts + p;
        a.res_l1 = r_l1 + p;
      }
      t_off += tg[p].ntiles;
      b_off += align_up((size_t)tg[p].ntiles * tg[p].cap * tg[p].rec_bytes, 256);
    }
    // the queue, dependency counts and argument blocks are re-sent only when they changed
    // since the last batch call on this arena (same shape and buffers: nothing to send)
    // (batch_inputs_valid is read here, after ensure_arena: a reallocated arena holds nothing)
    const bool dev_shape = m->batch_inputs_valid && same_shape;
    const bool same_args = dev_shape && m->batch_args.size() == args.size() &&
                           std::memcmp(m->batch_args.data(), args.data(), sizeof(WaveArgs) * n) == 0;
    m->batch_inputs_valid = false;
    if (!dev_shape)
      RM_CK(cudaMemcpyAsync(d_need, need.data(), sizeof(int) * need.size(), cudaMemcpyHostToDevice, s));
    m->batch_shape = shape;
    if (!same_args) {
      RM_CK(cudaMemcpyAsync(d_args, args.data(), sizeof(WaveArgs) * n, cudaMemcpyHostToDevice, s));
      m->batch_args = args;
    }
    m->batch_inputs_valid = true;
    rmk::LMArgs la{};
    la.cx = m->centre[0];
    la.cy = m->centre[1];
    la.cz = m->centre[2];
    if (lm) {
      la.lambda0 = lm->lambda0;
      la.lambda_up = lm->lambda_up;
      la.lambda_down = lm->lambda_down;
      la.step_tol = lm->step_tol;
    }
    rmk::BatchArgs b{};
    b.probs = d_args;
    if (cap_hi + cap_lo > (size_t)INT32_MAX) return fail(RM_EINVAL, "batch too large for the work queue");
    b.n_problems = n;
    b.items = d_items;
    b.cap[0] = (int)cap_hi;
    b.cap[1] = (int)cap_lo;
    b.qctl = d_next;
    b.done = d_done;
    b.need = d_need;
    b.lm = lm ? d_lm : nullptr;
    b.icp = icp ? d_icp : nullptr;
    rmk::IcpArgs ia{icp ? icp->step_tol : 0.0, m->centre[0], m->centre[1], m->centre[2]};
    b.icpargs = ia;
    b.Ms = d_M;
    b.skip = d_skip;
    b.lmargs = la;
    b.lm_iters = K;
    b.status = m->d_status;
    b.spin_limit = wait_budget(m, 1ll << 32);
    // A homogeneous plain batch (one scan, camera and parameters for every problem, no LM or
    // ICP) runs as the poses of one wave: its argument block is a kernel parameter. The
    // problems' arrays are already laid out at the wave's per-pose offsets, provided each
    // problem's bins end on the 256-byte boundary where the next one's start.
    bool wave_form = !lm && !icp && nc >= 1 &&
                     ((size_t)tg[0].ntiles * tg[0].cap * tg[0].rec_bytes) % 256 == 0;
    for (int p = 1; p < n && wave_form; ++p)
      wave_form = scan_of[p] == 0 && std::memcmp(&probs[p].scan.intr, &probs[0].scan.intr, sizeof(rm_intrinsics)) == 0;
    WaveArgs w;
    std::memset(&w, 0, sizeof(w));
    if (wave_form) {
      w = args[0];
      w.n_poses = n;
      w.wave_base = 0;
      w.skip = nullptr;
    }
    const int grid = wave_form ? rmk::persist_wave_grid(m->device, w.cam.model) : rmk::persist_grid(m->device);
    if (grid <= 0) return fail(RM_ECUDA, "could not size the persistent grid");
    // counters to zero, LM state / pose matrices, the persistent kernel: one captured graph
    // per batch shape (the arena layout is a function of the shape), replayed every call
    char sig[512];
    std::snprintf(sig, sizeof(sig), "%p|%d|%d|%zu|%d|%d|%a|%a|%a|%a|%zu|%zu|%zu|%d|%a|%lld", (void *)m->arena, n,
                  K, cap_hi + cap_lo, grid, lm ? 1 : (icp ? 2 : 0), la.lambda0, la.lambda_up, la.lambda_down,
                  la.step_tol, tiles_total, px_total, rays_total, m->cap * 4096 + m->cap_ray, ia.step_tol,
                  b.spin_limit);
    std::string key(sig);
    if (wave_form) {  // the graph holds w by value: a different w needs a new capture
      key += "|wave:";
      const unsigned char *wb = reinterpret_cast<const unsigned char *>(&w);
      for (size_t k = 0; k < sizeof(w); ++k) {
        static const char hex[] = "0123456789abcdef";
        key += hex[wb[k] >> 4];
        key += hex[wb[k] & 15];
      }
    }
    for (int p = 0; p < n; ++p) key += "|" + std::to_string(probs[p].scan.intr.model) + "x" +
                                        std::to_string(probs[p].scan.intr.width) + "x" +
                                        std::to_string(probs[p].scan.intr.height);
    if (!m->batch_exec || key != m->batch_sig) {
      if (m->batch_exec) {
        RM_CK(cudaGraphExecDestroy(m->batch_exec));
        m->batch_exec = nullptr;
        m->batch_sig.clear();
      }
      if (!m->cap_stream) RM_CK(cudaStreamCreateWithFlags(&m->cap_stream, cudaStreamNonBlocking));
      cudaStream_t c = m->cap_stream;
      RM_CK(cudaStreamBeginCapture(c, cudaStreamCaptureModeThreadLocal));
      cudaError_t e = cudaSuccess;
      auto rec = [&](cudaError_t x) {
        if (e == cudaSuccess) e = x;
      };
      rec(cudaMemsetAsync(d_next, 0, 8 * sizeof(int), c));
      rec(rmk::launch_queue_init(d_items, (int)(cap_hi + cap_lo), (int)cap_hi, n, ncull, d_next, c));
      rec(cudaMemsetAsync(d_done, 0, sizeof(int) * 4 * n, c));
      rec(cudaMemsetAsync(d_skip, 0, sizeof(int) * n, c));
      rec(cudaMemsetAsync(d_vcount, 0, sizeof(int) * n, c));
      rec(cudaMemsetAsync(d_counts, 0, sizeof(int) * tiles_total, c));
      if (lm) rec(rmk::launch_lm_init_batch(d_lm, d_poses, n, la, d_M, d_skip, c));
      else if (icp) rec(rmk::launch_icp_init_batch(d_icp, d_poses, n, ia, d_M, d_skip, c));
      else rec(rmk::launch_pose_to_m(d_poses, n, m->centre[0], m->centre[1], m->centre[2], d_M, c));
      rec(wave_form ? rmk::launch_persist_wave(b, w, grid, c) : rmk::launch_persist(b, grid, c));
      cudaGraph_t graph = nullptr;
      const cudaError_t ec = cudaStreamEndCapture(c, &graph);
      if (e == cudaSuccess) e = ec;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&m->batch_exec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        m->batch_exec = nullptr;
        return fail(RM_ECUDA, std::string("batch graph capture: ") + cudaGetErrorString(e));
      }
      m->batch_sig = key;
    }
    RM_CK(cudaGraphLaunch(m->batch_exec, s));
    m->launches += 2;
    bool host_out = false;
    std::vector<rmk::LMState> hs;
    std::vector<rmk::IcpState> his;
    if (lm) {
      hs.resize(n);
      RM_CK(cudaMemcpyAsync(hs.data(), d_lm, sizeof(rmk::LMState) * n, cudaMemcpyDeviceToHost, s));
    } else if (icp) {
      his.resize(n);
      RM_CK(cudaMemcpyAsync(his.data(), d_icp, sizeof(rmk::IcpState) * n, cudaMemcpyDeviceToHost, s));
    } else if (out) {
      RM_TRY(copy_out(out->counts, r_counts, sizeof(long long) * 6 * n, s, &host_out));
      RM_TRY(copy_out(out->e_table, r_et, sizeof(long long) * n, s, &host_out));
      RM_TRY(copy_out(out->e_ls, r_els, sizeof(double) * n, s, &host_out));
      RM_TRY(copy_out(out->grad, r_grad, sizeof(double) * 6 * n, s, &host_out));
      RM_TRY(copy_out(out->jtj, r_jtj, sizeof(double) * 21 * n, s, &host_out));
    }
    unsigned st = 0;
    RM_TRY(read_status(m, s, &st));  // synchronises the stream
    if (st & rmk::kStatusQueue) return fail(RM_ECUDA, "the persistent queue ran out of slots");
    if (st & rmk::kStatusTimeout) return fail(RM_ETIMEOUT, "a device-side wait ran out of time");
    if (st & (rmk::kStatusOverflow | rmk::kStatusOverflowRay)) {
      RM_TRY(grow_bins(m, st, attempt));
      continue;
    }
    if (icp) {
      bool all_conv = true;
      std::vector<double> pout(16 * (size_t)n);
      for (int p = 0; p < n; ++p) {
        std::memcpy(&pout[16 * (size_t)p], his[p].T, sizeof(double) * 16);
        all_conv = all_conv && his[p].converged;
        if (ireps) {
          ireps[p].iters = his[p].iters;
          ireps[p].converged = his[p].converged;
          ireps[p].n_assoc = his[p].n_assoc;
          ireps[p].cost_l1_initial = his[p].l1_0;
          ireps[p].cost_l1_final = his[p].l1;
        }
      }
      if (on_device(poses_out))
        RM_CK(cudaMemcpy(poses_out, pout.data(), sizeof(double) * 16 * n, cudaMemcpyHostToDevice));
      else
        std::memcpy(poses_out, pout.data(), sizeof(double) * 16 * n);
      return all_conv ? RM_OK : fail(RM_ENOTCONV, "a problem's ICP steps did not fall below step_tol");
    }
    if (!lm) return RM_OK;
    bool all_conv = true;
    std::vector<double> pout(16 * (size_t)n);
    for (int p = 0; p < n; ++p) {
      std::memcpy(&pout[16 * (size_t)p], hs[p].T, sizeof(double) * 16);
      all_conv = all_conv && hs[p].converged;
      if (reps) {
        reps[p].iters = hs[p].iters;
        reps[p].accepted = hs[p].accepted;
        reps[p].converged = hs[p].converged;
        reps[p].reserved = 0;
        reps[p].e_ls_initial = hs[p].e_ls0;
        reps[p].e_ls_final = hs[p].e;
        reps[p].e_table_initial = hs[p].e_table0;
        reps[p].e_table_final = hs[p].e_table;
      }
    }
    if (on_device(poses_out))
      RM_CK(cudaMemcpy(poses_out, pout.data(), sizeof(double) * 16 * n, cudaMemcpyHostToDevice));
    else
      std::memcpy(poses_out, pout.data(), sizeof(double) * 16 * n);
    return all_conv ? RM_OK : fail(RM_ENOTCONV, "a problem reached max_iters before step_tol");
  }
}

// ---- single-pose device loops (rm_align, rm_icp_align, rm_dfo_align)

// The arrays every such loop carves after its own state and results: the start pose, the
// matrices of its S poses per evaluation, a skip flag, the staged scan and rays (host inputs
// only) and the wave scratch for S poses. Planned and carved by the same function, so the
// two passes agree.
struct LoopBufs {
  double *T0;
  float *M;
  int *skip;
  const float *sd, *rays;
  const uint8_t *sc;
  int4 *vis;
  int *vis_count, *counts;
  unsigned char *bins;
  double *partial;
};

void loop_arrays(Carver &cv, const rm_map *m, const rm_scan *scan, const TileGeom &tg, int S,
                 LoopBufs *b) {
  const rm_intrinsics *in = &scan->intr;
  const long long P = (long long)in->width * in->height;
  b->T0 = cv.take<double>(16);
  b->M = cv.take<float>(12 * (size_t)S);
  b->skip = cv.take<int>(1);
  b->sd = on_device(scan->depth) ? scan->depth : cv.take<float>(P);
  b->sc = on_device(scan->cls) ? scan->cls : cv.take<uint8_t>(P);
  b->rays = (in->model != RM_RAYTABLE || on_device(in->rays)) ? in->rays : cv.take<float>(3 * P);
  b->vis = cv.take<int4>((size_t)m->n_clusters * S);
  b->vis_count = cv.take<int>(S);
  b->counts = cv.take<int>((size_t)tg.ntiles * S);
  b->bins = cv.take<unsigned char>((size_t)tg.ntiles * tg.cap * tg.rec_bytes * S);
  b->partial = cv.take<double>((size_t)tg.ntiles * rmk::kNumVals * S);
}

// The loop's wave over its S poses (result pointers are the caller's), and the copies of its
// host inputs (start pose, scan, rays) into the staged arrays.
WaveArgs loop_wave(const rm_map *m, const rm_scan *scan, const TileGeom &tg, int S, const LoopBufs &b,
                   const rm_cost_params &prm) {
  WaveArgs a{};
  a.cam = make_cam(&scan->intr, b.rays);
  a.tg = tg;
  a.V = (int)m->V;
  a.T = m->T;
  a.n_poses = S;
  a.wave_base = 0;
  a.v = m->d_v;
  a.faces = m->d_faces;
  a.planes = m->d_planes;
  a.Ms = b.M;
  set_map_fields(m, a);
  a.vis = b.vis;
  a.vis_count = b.vis_count;
  a.counts = b.counts;
  a.bins = b.bins;
  a.partial = b.partial;
  a.status = m->d_status;
  a.skip = b.skip;
  a.scan_depth = b.sd;
  a.scan_cls = b.sc;
  a.prm = {prm.eps, prm.w_fofo, prm.w_fofu, prm.w_fufo};
  return a;
}

rm_status loop_inputs(const rm_scan *scan, const double *init_pose, const LoopBufs &b, cudaStream_t s) {
  const rm_intrinsics *in = &scan->intr;
  const long long P = (long long)in->width * in->height;
  RM_CK(cudaMemcpyAsync(b.T0, init_pose, sizeof(double) * 16,
                        on_device(init_pose) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  if (b.rays != in->rays)
    RM_CK(cudaMemcpyAsync((void *)b.rays, in->rays, sizeof(float) * 3 * P, cudaMemcpyHostToDevice, s));
  if (b.sd != scan->depth)
    RM_CK(cudaMemcpyAsync((void *)b.sd, scan->depth, sizeof(float) * P, cudaMemcpyHostToDevice, s));
  if (b.sc != scan->cls) RM_CK(cudaMemcpyAsync((void *)b.sc, scan->cls, P, cudaMemcpyHostToDevice, s));
  return RM_OK;
}

// After a loop: read its state back (synchronising), and map the status word to the call's
// result: RM_OK, an error, or "grow the bins and run again" (*retry).
rm_status loop_finish(rm_map *m, cudaStream_t s, void *host_state, const void *dev_state, size_t bytes,
                      int attempt, bool *retry) {
  *retry = false;
  RM_CK(cudaMemcpyAsync(host_state, dev_state, bytes, cudaMemcpyDeviceToHost, s));
  unsigned st = 0;
  RM_TRY(read_status(m, s, &st));  // synchronises the stream
  if (st & rmk::kStatusTimeout) return fail(RM_ETIMEOUT, "a device-side wait ran out of time");
  if (st & (rmk::kStatusOverflow | rmk::kStatusOverflowRay)) {
    RM_TRY(grow_bins(m, st, attempt));
    *retry = true;
  }
  return RM_OK;
}

rm_status write_pose(double *pose_out, const double *T) {
  if (on_device(pose_out)) RM_CK(cudaMemcpy(pose_out, T, sizeof(double) * 16, cudaMemcpyHostToDevice));
  else std::memcpy(pose_out, T, sizeof(double) * 16);
  return RM_OK;
}

}  // namespace

namespace rmapi {

int map_device(const rm_map *m) { return m->device; }

rm_status wave_inputs(const rm_map *m, const rm_intrinsics *in, WaveArgs *a, double centre[3]) {
  if (!m) return fail(RM_EINVAL, "map is NULL");
  RM_TRY(check_intr(in));
  if (in->model == RM_RAYTABLE && !on_device(in->rays))
    return fail(RM_EINVAL, "this entry point needs the ray table in device memory");
  a->cam = make_cam(in, in->rays);
  a->tg = make_tiles(m, in);
  a->V = (int)m->V;
  a->T = m->T;
  a->v = m->d_v;
  a->faces = m->d_faces;
  a->planes = m->d_planes;
  set_map_fields(m, *a);
  for (int k = 0; k < 3; ++k) centre[k] = m->centre[k];
  return RM_OK;
}

void set_error(const std::string &msg) { g_err = msg; }

rm_status check_intrinsics(const rm_intrinsics *in) { return check_intr(in); }

bool is_device_pointer(const void *p) { return on_device(p); }

}  // namespace rmapi

extern "C" {

const char *rm_last_error(void) { return g_err.c_str(); }

rm_status rm_map_create(const float *vertices, int64_t n_vertices, const int32_t *faces,
                        const uint8_t *labels, int64_t n_faces, rm_map **out) {
  if (!out) return fail(RM_EINVAL, "out is NULL");
  *out = nullptr;
  if (n_vertices < 0 || n_faces < 0) return fail(RM_EINVAL, "negative size");
  if (n_vertices >= (1ll << 31) || n_faces >= (1ll << 31)) return fail(RM_EINVAL, "too many vertices or faces (>= 2^31)");
  if ((n_vertices > 0 && !vertices) || (n_faces > 0 && (!faces || !labels)))
    return fail(RM_EINVAL, "null array");
  if (on_device(vertices) || on_device(faces) || on_device(labels))
    return fail(RM_EINVAL, "rm_map_create takes host arrays");
  for (int64_t k = 0; k < 3 * n_vertices; ++k)
    if (!std::isfinite(vertices[k])) return fail(RM_EINVAL, "non-finite vertex coordinate");
  for (int64_t k = 0; k < 3 * n_faces; ++k)
    if (faces[k] < 0 || faces[k] >= n_vertices) return fail(RM_EINVAL, "face index out of range");
  for (int64_t k = 0; k < n_faces; ++k)
    if (labels[k] > 2) return fail(RM_EINVAL, "label above 2");

  rm_map *m = new rm_map();
  cudaGetDevice(&m->device);
  {
    // a sixteenth of the device's memory (at least 4 GiB) for one wave's scratch: panoramic
    // views need large bins, and every extra wave repeats the slowest tile's serial work
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess)
      m->wave_budget = std::max(m->wave_budget, total_b / 16);
    else
      cudaGetLastError();
  }
  m->V = n_vertices;
  m->T = n_faces;
  // re-centre on the FP64 bounding-box centre
  for (int a = 0; a < 3; ++a) {
    double lo = INFINITY, hi = -INFINITY;
    for (int64_t k = 0; k < n_vertices; ++k) {
      double x = vertices[3 * k + a];
      lo = std::min(lo, x);
      hi = std::max(hi, x);
    }
    m->centre[a] = n_vertices > 0 ? 0.5 * (lo + hi) : 0.0;
  }
  std::vector<float4> hv(std::max<int64_t>(n_vertices, 1));
  for (int64_t k = 0; k < n_vertices; ++k)
    hv[k] = make_float4((float)((double)vertices[3 * k] - m->centre[0]),
                        (float)((double)vertices[3 * k + 1] - m->centre[1]),
                        (float)((double)vertices[3 * k + 2] - m->centre[2]), 0.0f);
  std::vector<int4> hf(std::max<int64_t>(n_faces, 1));
  std::vector<float4> hp(std::max<int64_t>(n_faces, 1));
  for (int64_t k = 0; k < n_faces; ++k) {
    int i0 = faces[3 * k], i1 = faces[3 * k + 1], i2 = faces[3 * k + 2];
    hf[k] = make_int4(i0, i1, i2, labels[k]);
    // the unit normal in FP64 from the caller's FP32 vertices (not the re-centred copies,
    // whose rounding far from the centre would tilt small triangles)
    const float *a = vertices + 3 * (int64_t)i0, *b = vertices + 3 * (int64_t)i1,
                *c = vertices + 3 * (int64_t)i2;
    double e1[3] = {(double)b[0] - a[0], (double)b[1] - a[1], (double)b[2] - a[2]};
    double e2[3] = {(double)c[0] - a[0], (double)c[1] - a[1], (double)c[2] - a[2]};
    double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    double nn = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    if (nn > 0) for (double &x : n) x /= nn;
    float lab;
    int li = labels[k];
    std::memcpy(&lab, &li, 4);
    hp[k] = make_float4((float)n[0], (float)n[1], (float)n[2], lab);
  }
  Clusters cl;
  build_clusters(hv, faces, n_faces, cl);
  m->n_clusters = (int)cl.info.size();
  auto up = [&](void **dst, const void *src, size_t bytes) -> cudaError_t {
    cudaError_t e = cudaMalloc(dst, std::max<size_t>(bytes, 16));
    if (e != cudaSuccess || bytes == 0) return e;
    return cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
  };
  auto cleanup = [&](rm_status s) {
    rm_map_destroy(m);
    return s;
  };
  cudaError_t e;
  if ((e = cudaMalloc(&m->d_v, sizeof(float4) * hv.size())) != cudaSuccess ||
      (e = cudaMalloc(&m->d_faces, sizeof(int4) * hf.size())) != cudaSuccess ||
      (e = cudaMalloc(&m->d_planes, sizeof(float4) * hp.size())) != cudaSuccess ||
      (e = cudaMalloc(&m->d_status, sizeof(unsigned))) != cudaSuccess ||
      (e = cudaMallocHost(&m->h_status, sizeof(unsigned))) != cudaSuccess ||
      (e = cudaMemcpy(m->d_v, hv.data(), sizeof(float4) * hv.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(m->d_faces, hf.data(), sizeof(int4) * hf.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(m->d_planes, hp.data(), sizeof(float4) * hp.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemset(m->d_status, 0, sizeof(unsigned))) != cudaSuccess ||
      (e = up((void **)&m->d_cl_info, cl.info.data(), sizeof(int4) * cl.info.size())) != cudaSuccess ||
      (e = up((void **)&m->d_cl_sphere, cl.sphere.data(), sizeof(float4) * cl.sphere.size())) != cudaSuccess ||
      (e = up((void **)&m->d_cl_pos, cl.pos.data(), sizeof(float4) * cl.pos.size())) != cudaSuccess ||
      (e = up((void **)&m->d_cl_tris, cl.tris.data(), sizeof(uchar4) * cl.tris.size())) != cudaSuccess ||
      (e = up((void **)&m->d_cl_ids, cl.ids.data(), sizeof(int) * cl.ids.size())) != cudaSuccess)
    return cleanup(fail(e == cudaErrorMemoryAllocation ? RM_ENOMEM : RM_ECUDA,
                        std::string("map upload: ") + cudaGetErrorString(e)));
  *out = m;
  return RM_OK;
}

void rm_map_destroy(rm_map *m) {
  if (!m) return;
  cudaSetDevice(m->device);
  cudaDeviceSynchronize();
  cudaFree(m->d_v);
  cudaFree(m->d_faces);
  cudaFree(m->d_planes);
  cudaFree(m->d_vn);
  cudaFree(m->d_cl_info);
  cudaFree(m->d_cl_sphere);
  cudaFree(m->d_cl_pos);
  cudaFree(m->d_cl_tris);
  cudaFree(m->d_cl_ids);
  cudaFree(m->arena);
  if (m->aux_stream) cudaStreamDestroy(m->aux_stream);
  if (m->ev_fork) cudaEventDestroy(m->ev_fork);
  if (m->ev_join) cudaEventDestroy(m->ev_join);
  cudaFree(m->d_status);
  if (m->h_status) cudaFreeHost(m->h_status);
  for (auto &ev : m->ev_pending)
    for (auto e : ev) cudaEventDestroy(e);
  for (auto e : m->ev_free) cudaEventDestroy(e);
  if (m->batch_exec) cudaGraphExecDestroy(m->batch_exec);
  if (m->cap_stream) cudaStreamDestroy(m->cap_stream);
  delete m;
}

rm_status rm_map_info(const rm_map *m, int64_t *nv, int64_t *nf, double centre[3]) {
  if (!m) return fail(RM_EINVAL, "map is NULL");
  if (nv) *nv = m->V;
  if (nf) *nf = m->T;
  if (centre) for (int a = 0; a < 3; ++a) centre[a] = m->centre[a];
  return RM_OK;
}

rm_status rm_map_set_tuning(rm_map *m, const rm_tuning *t) {
  if (!m) return fail(RM_EINVAL, "map is NULL");
  std::lock_guard<std::mutex> lk(m->mu);
  rm_tuning z{};
  const rm_tuning &u = t ? *t : z;
  bool ok_tile = (u.tile_w == 0 && u.tile_h == 0) || (u.tile_w == 64 && u.tile_h == 32) ||
                 (u.tile_w == 32 && u.tile_h == 32) || (u.tile_w == 32 && u.tile_h == 16) ||
                 (u.tile_w == 16 && u.tile_h == 16);
  if (!ok_tile) return fail(RM_EINVAL, "tile must be 16x16, 32x16, 32x32 or 64x32");
  if (u.bin_capacity < 0 || u.wave_poses < 0) return fail(RM_EINVAL, "negative tuning value");
  if (u.wait_log2 < 0 || u.wait_log2 > 40) return fail(RM_EINVAL, "wait_log2 must be 0..40");
  m->tuning = u;
  if (u.bin_capacity > 0) m->cap = m->cap_ray = u.bin_capacity;
  return RM_OK;
}

rm_status rm_map_set_vertex_normals(rm_map *m, const float *normals, const double *pose, void *stream) {
  if (!m) return fail(RM_EINVAL, "map is NULL");
  std::lock_guard<std::mutex> lk(m->mu);
  RM_CK(cudaSetDevice(m->device));
  cudaStream_t s = (cudaStream_t)stream;
  if (!normals) {
    if (m->d_vn) {
      RM_CK(cudaStreamSynchronize(s));
      RM_CK(cudaFree(m->d_vn));
      m->d_vn = nullptr;
    }
    return RM_OK;
  }
  if (pose && on_device(pose)) return fail(RM_EINVAL, "pose must be a host array");
  float R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
  if (pose)
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) R[3 * r + c] = (float)pose[4 * r + c];
  const int V = (int)m->V;
  if (V == 0) return RM_OK;
  if (!m->d_vn) RM_CK(cudaMalloc((void **)&m->d_vn, sizeof(float4) * (size_t)V));
  float *buf = nullptr;
  const size_t nb = sizeof(float) * 3 * (size_t)V;
  RM_CK(cudaMallocAsync((void **)&buf, nb + sizeof(R), s));
  rm_status st = RM_OK;
  auto run = [&]() -> rm_status {
    RM_CK(cudaMemcpyAsync(buf, normals, nb, on_device(normals) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    RM_CK(cudaMemcpyAsync(buf + 3 * (size_t)V, R, sizeof(R), cudaMemcpyHostToDevice, s));
    RM_CK(rmk::launch_rotate_normals(buf, V, buf + 3 * (size_t)V, m->d_vn, s));
    RM_CK(cudaStreamSynchronize(s));
    return RM_OK;
  };
  st = run();
  cudaFreeAsync(buf, s);
  return st;
}

rm_status rm_map_get_tuning(const rm_map *m, rm_tuning *t) {
  if (!m || !t) return fail(RM_EINVAL, "NULL argument");
  *t = m->tuning;
  t->bin_capacity = m->cap;
  return RM_OK;
}

rm_status rm_render_depth(rm_map *m, const double *poses, int32_t n, const rm_intrinsics *intr,
                          float *depth, int32_t *tri_id, float *bary, void *stream) {
  if (!m) return fail(RM_EINVAL, "map is NULL");
  std::lock_guard<std::mutex> lk(m->mu);
  EvalReq r{intr, nullptr, poses, n, nullptr, rmk::kRender, nullptr, nullptr, depth, tri_id, bary};
  return run_eval(m, r, (cudaStream_t)stream);
}

rm_status rm_cost(rm_map *m, const rm_scan *scan, const double *poses, int32_t n,
                  const rm_cost_params *prm, const rm_cost_out *out, void *stream) {
  if (!m) return fail(RM_EINVAL, "map is NULL");
  if (!scan) return fail(RM_EINVAL, "scan is NULL");
  std::lock_guard<std::mutex> lk(m->mu);
  EvalReq r{&scan->intr, scan, poses, n, prm, rmk::kCost, out, nullptr, nullptr, nullptr, nullptr};
  return run_eval(m, r, (cudaStream_t)stream);
}

rm_status rm_cost_grad(rm_map *m, const rm_scan *scan, const double *poses, int32_t n,
                       const rm_cost_params *prm, const rm_cost_out *out, void *stream) {
  if (!m) return fail(RM_EINVAL, "map is NULL");
  if (!scan) return fail(RM_EINVAL, "scan is NULL");
  std::lock_guard<std::mutex> lk(m->mu);
  EvalReq r{&scan->intr, scan, poses, n, prm, rmk::kCostGrad, out, nullptr, nullptr, nullptr, nullptr};
  return run_eval(m, r, (cudaStream_t)stream);
}

rm_status rm_icp_terms(rm_map *m, const rm_scan *scan, const double *poses, int32_t n, float tol,
                       const rm_icp_out *out, void *stream) {
  if (!m) return fail(RM_EINVAL, "map is NULL");
  if (!scan) return fail(RM_EINVAL, "scan is NULL");
  if (!(tol >= 0.0f)) return fail(RM_EINVAL, "tol must be >= 0");
  std::lock_guard<std::mutex> lk(m->mu);
  const rm_cost_params prm{tol, 0.0f, 0.0f, 0.0f};
  EvalReq r{&scan->intr, scan, poses, n, &prm, rmk::kIcp, nullptr, out, nullptr, nullptr, nullptr};
  return run_eval(m, r, (cudaStream_t)stream);
}

rm_status rm_cost_grad_vertices(rm_map *m, const rm_scan *scan, const double *poses, int32_t n,
                                const rm_cost_params *prm, double *grad_v, void *stream) {
  if (!m) return fail(RM_EINVAL, "map is NULL");
  if (!scan || !scan->depth || !scan->cls) return fail(RM_EINVAL, "scan or its arrays NULL");
  if (!prm || !grad_v) return fail(RM_EINVAL, "NULL argument");
  if (!(prm->eps >= 0.0f)) return fail(RM_EINVAL, "eps must be >= 0");
  if (n < 0) return fail(RM_EINVAL, "n_poses < 0");
  if (n > 0 && !poses) return fail(RM_EINVAL, "poses is NULL");
  std::lock_guard<std::mutex> lk(m->mu);
  const rm_intrinsics *in = &scan->intr;
  RM_TRY(check_intr(in));
  RM_CK(cudaSetDevice(m->device));
  cudaStream_t s = (cudaStream_t)stream;
  const long long P = (long long)in->width * in->height;
  const int chunk = (int)std::max<long long>(1, std::min<long long>(16, (1LL << 28) / std::max<long long>(P, 1)));
  const bool host_g = !on_device(grad_v), host_p = n > 0 && !on_device(poses);
  const bool host_sd = !on_device(scan->depth), host_sc = !on_device(scan->cls);
  const bool host_rays = in->model == RM_RAYTABLE && !on_device(in->rays);
  // stream-ordered scratch (the map's arena is reused by the render calls below)
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off += (bytes + 255) / 256 * 256;
    return at;
  };
  const size_t o_g = host_g ? take(sizeof(double) * 3 * (size_t)m->V) : 0;
  const size_t o_p = take(sizeof(double) * 16 * (size_t)std::max(n, 1));
  const size_t o_sd = host_sd ? take(sizeof(float) * P) : 0, o_sc = host_sc ? take(P) : 0;
  const size_t o_r = host_rays ? take(sizeof(float) * 3 * P) : 0;
  const size_t o_m = take(sizeof(float) * 12 * chunk);
  const size_t o_id = take(sizeof(int) * P * chunk), o_d = take(sizeof(float) * P * chunk);
  const size_t o_b = take(sizeof(float) * 2 * P * chunk);
  unsigned char *buf = nullptr;
  RM_CK(cudaMallocAsync((void **)&buf, off, s));
  double *d_g = host_g ? reinterpret_cast<double *>(buf + o_g) : grad_v;
  double *d_p = reinterpret_cast<double *>(buf + o_p);
  const float *d_sd = host_sd ? reinterpret_cast<float *>(buf + o_sd) : scan->depth;
  const uint8_t *d_sc = host_sc ? buf + o_sc : scan->cls;
  const float *d_rays = host_rays ? reinterpret_cast<float *>(buf + o_r) : in->rays;
  float *d_M = reinterpret_cast<float *>(buf + o_m);
  int *d_id = reinterpret_cast<int *>(buf + o_id);
  float *d_d = reinterpret_cast<float *>(buf + o_d);
  float *d_b = reinterpret_cast<float *>(buf + o_b);
  auto body = [&]() -> rm_status {
    RM_CK(cudaMemsetAsync(d_g, 0, sizeof(double) * 3 * (size_t)m->V, s));
    if (n > 0)
      RM_CK(cudaMemcpyAsync(d_p, poses, sizeof(double) * 16 * n,
                            host_p ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
    if (host_sd) RM_CK(cudaMemcpyAsync((void *)d_sd, scan->depth, sizeof(float) * P, cudaMemcpyHostToDevice, s));
    if (host_sc) RM_CK(cudaMemcpyAsync((void *)d_sc, scan->cls, P, cudaMemcpyHostToDevice, s));
    if (host_rays) RM_CK(cudaMemcpyAsync((void *)d_rays, in->rays, sizeof(float) * 3 * P, cudaMemcpyHostToDevice, s));
    rm_intrinsics ind = *in;
    ind.rays = d_rays;
    for (int p0 = 0; p0 < n; p0 += chunk) {
      const int c = std::min(chunk, n - p0);
      EvalReq r{&ind, nullptr, d_p + 16 * (size_t)p0, c, nullptr, rmk::kRender, nullptr, nullptr, d_d, d_id, d_b};
      RM_TRY(run_eval(m, r, s));
      RM_CK(rmk::launch_pose_to_m(d_p + 16 * (size_t)p0, c, m->centre[0], m->centre[1], m->centre[2], d_M, s));
      rmk::VGradArgs a{};
      a.cam = make_cam(&ind, d_rays);
      a.W = in->width;
      a.n_poses = c;
      a.P = P;
      a.Ms = d_M;
      a.planes = m->d_planes;
      a.faces = m->d_faces;
      a.tri_id = d_id;
      a.depth = d_d;
      a.bary = d_b;
      a.scan_depth = d_sd;
      a.scan_cls = d_sc;
      a.prm = {prm->eps, prm->w_fofo, prm->w_fofu, prm->w_fufo};
      a.grad = d_g;
      RM_CK(rmk::launch_vertex_grad(a, s));
      m->launches += 2;
    }
    if (host_g) RM_CK(cudaMemcpyAsync(grad_v, d_g, sizeof(double) * 3 * (size_t)m->V, cudaMemcpyDeviceToHost, s));
    return RM_OK;
  };
  rm_status st = body();
  cudaFreeAsync(buf, s);
  if (st == RM_OK && host_g) RM_CK(cudaStreamSynchronize(s));
  return st;
}

rm_status rm_cost_sweep(rm_map *m, const rm_scan *scan, const double *pose, int32_t axis, double span,
                        int32_t n, const rm_cost_params *prm, const rm_cost_out *out, void *stream) {
  if (!m) return fail(RM_EINVAL, "map is NULL");
  if (!scan) return fail(RM_EINVAL, "scan is NULL");
  if (!pose) return fail(RM_EINVAL, "pose is NULL");
  if (axis < 0 || axis > 5) return fail(RM_EINVAL, "axis must be 0..5");
  if (!(span >= 0.0) || !std::isfinite(span)) return fail(RM_EINVAL, "span must be finite and >= 0");
  if (n < 0) return fail(RM_EINVAL, "n < 0");
  if (n == 0) return RM_OK;
  std::lock_guard<std::mutex> lk(m->mu);
  RM_CK(cudaSetDevice(m->device));
  cudaStream_t s = (cudaStream_t)stream;
  double *buf = nullptr;
  RM_CK(cudaMallocAsync((void **)&buf, sizeof(double) * (16 + 38 * (size_t)n), s));
  double *d_base = buf, *d_rep = buf + 16, *d_tw = d_rep + 16 * (size_t)n, *d_poses = d_tw + 6 * (size_t)n;
  auto body = [&]() -> rm_status {
    RM_CK(cudaMemcpyAsync(d_base, pose, sizeof(double) * 16,
                          on_device(pose) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    RM_CK(rmk::launch_sweep_inputs(d_base, axis, span, n, d_rep, d_tw, s));
    RM_CK(rmk::launch_retract(d_rep, d_tw, n, d_poses, nullptr, s));
    m->launches += 2;
    EvalReq r{&scan->intr, scan, d_poses, n, prm, rmk::kCost, out, nullptr, nullptr, nullptr, nullptr};
    return run_eval(m, r, s);
  };
  const rm_status st = body();
  cudaFreeAsync(buf, s);
  return st;
}

rm_status rm_pose_retract(const double *poses, const double *twists, int32_t n, double *out,
                          double *jr, void *stream) {
  if (n < 0) return fail(RM_EINVAL, "n < 0");
  if (n == 0) return RM_OK;
  if (!poses || !twists || !out) return fail(RM_EINVAL, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  const bool dp = on_device(poses), dt = on_device(twists), dout = on_device(out);
  const bool djr = jr && on_device(jr);
  if (dp && dt && dout && (!jr || djr)) {
    RM_CK(rmk::launch_retract(poses, twists, n, out, jr, s));
    return RM_OK;
  }
  double *buf = nullptr;
  size_t per = 16 + 6 + 16 + 36;
  RM_CK(cudaMallocAsync((void **)&buf, sizeof(double) * per * n, s));
  double *bp = buf, *bt = buf + 16 * (size_t)n, *bo = bt + 6 * (size_t)n, *bj = bo + 16 * (size_t)n;
  rm_status st = RM_OK;
  auto run = [&]() -> rm_status {
    RM_CK(cudaMemcpyAsync(bp, poses, sizeof(double) * 16 * n, dp ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    RM_CK(cudaMemcpyAsync(bt, twists, sizeof(double) * 6 * n, dt ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    RM_CK(rmk::launch_retract(bp, bt, n, bo, jr ? bj : nullptr, s));
    RM_CK(cudaMemcpyAsync(out, bo, sizeof(double) * 16 * n, dout ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    if (jr) RM_CK(cudaMemcpyAsync(jr, bj, sizeof(double) * 36 * n, djr ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    RM_CK(cudaStreamSynchronize(s));
    return RM_OK;
  };
  st = run();
  cudaFreeAsync(buf, s);
  return st;
}

rm_status rm_twist_grad(const double *twists, const double *grads, const double *scale, int32_t n,
                        double *out, void *stream) {
  if (n < 0) return fail(RM_EINVAL, "n < 0");
  if (n == 0) return RM_OK;
  if (!twists || !grads || !out) return fail(RM_EINVAL, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  const bool dt = on_device(twists), dg = on_device(grads), ds = !scale || on_device(scale);
  const bool dout = on_device(out);
  if (dt && dg && ds && dout) {
    RM_CK(rmk::launch_twist_grad(twists, grads, scale, n, out, s));
    return RM_OK;
  }
  double *buf = nullptr;
  RM_CK(cudaMallocAsync((void **)&buf, sizeof(double) * 19 * (size_t)n, s));
  double *bt = buf, *bg = bt + 6 * (size_t)n, *bs = bg + 6 * (size_t)n, *bo = bs + (size_t)n;
  auto run = [&]() -> rm_status {
    RM_CK(cudaMemcpyAsync(bt, twists, sizeof(double) * 6 * n, dt ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    RM_CK(cudaMemcpyAsync(bg, grads, sizeof(double) * 6 * n, dg ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    if (scale)
      RM_CK(cudaMemcpyAsync(bs, scale, sizeof(double) * n, on_device(scale) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    RM_CK(rmk::launch_twist_grad(bt, bg, scale ? bs : nullptr, n, bo, s));
    RM_CK(cudaMemcpyAsync(out, bo, sizeof(double) * 6 * n, dout ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    RM_CK(cudaStreamSynchronize(s));
    return RM_OK;
  };
  const rm_status st = run();
  cudaFreeAsync(buf, s);
  return st;
}

rm_status rm_profile(rm_map *m, int32_t enable) {
  if (!m) return fail(RM_EINVAL, "map is NULL");
  std::lock_guard<std::mutex> lk(m->mu);
  RM_TRY(drain_events(m));
  if (enable) {
    for (int k = 0; k < 4; ++k) {
      m->prof_ms[k] = 0.0;
      m->prof_n[k] = 0;
    }
    m->launches = 0;
  }
  m->prof = enable != 0;
  return RM_OK;
}

rm_status rm_profile_read(rm_map *m, rm_kernel_time *out, int32_t cap, int32_t *n,
                          int64_t *launches) {
  if (!m || (cap > 0 && !out)) return fail(RM_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(m->mu);
  RM_TRY(drain_events(m));
  static const char *names[4] = {"k_cull", "k_setup", "k_raster", "k_reduce"};
  int k = 0;
  for (int q = 0; q < 4 && k < cap; ++q) {
    if (m->prof_n[q] == 0) continue;
    std::memset(out[k].name, 0, sizeof(out[k].name));
    std::strncpy(out[k].name, names[q], sizeof(out[k].name) - 1);
    out[k].launches = m->prof_n[q];
    out[k].total_ms = m->prof_ms[q];
    ++k;
  }
  if (n) *n = k;
  if (launches) *launches = m->launches;
  return RM_OK;
}

rm_status rm_cost_grad_batch(rm_map *m, const rm_problem *probs, int32_t n,
                             const rm_cost_params *prm, const rm_cost_out *out, void *stream) {
  if (!m) return fail(RM_EINVAL, "map is NULL");
  std::lock_guard<std::mutex> lk(m->mu);
  return run_batch(m, probs, n, prm, nullptr, out, nullptr, nullptr, (cudaStream_t)stream);
}

rm_status rm_align_batch(rm_map *m, const rm_problem *probs, int32_t n, const rm_cost_params *prm,
                         const rm_align_params *lm, double *poses_out, rm_align_report *reps,
                         void *stream) {
  if (!m) return fail(RM_EINVAL, "map is NULL");
  if (!lm) return fail(RM_EINVAL, "lm is NULL");
  std::lock_guard<std::mutex> lk(m->mu);
  return run_batch(m, probs, n, prm, lm, nullptr, poses_out, reps, (cudaStream_t)stream);
}

rm_status rm_icp_align_batch(rm_map *m, const rm_problem *probs, int32_t n, const rm_icp_params *icp,
                             double *poses_out, rm_icp_report *reps, void *stream) {
  if (!m) return fail(RM_EINVAL, "map is NULL");
  if (!icp) return fail(RM_EINVAL, "params is NULL");
  if (!(icp->tol >= 0.0f)) return fail(RM_EINVAL, "tol must be >= 0");
  std::lock_guard<std::mutex> lk(m->mu);
  const rm_cost_params prm{icp->tol, 0.0f, 0.0f, 0.0f};
  return run_batch(m, probs, n, &prm, nullptr, nullptr, poses_out, nullptr, (cudaStream_t)stream, icp, reps);
}

rm_status rm_status_sync(rm_map *m, void *stream) {
  if (!m) return fail(RM_EINVAL, "map is NULL");
  std::lock_guard<std::mutex> lk(m->mu);
  unsigned st = 0;
  RM_TRY(read_status(m, (cudaStream_t)stream, &st));
  if (st & rmk::kStatusTimeout) return fail(RM_ETIMEOUT, "a device-side wait ran out of time");
  if (st & (rmk::kStatusOverflow | rmk::kStatusOverflowRay)) return fail(RM_EOVERFLOW, "screen-tile bin overflow");
  return RM_OK;
}

rm_status rm_align(rm_map *m, const rm_scan *scan, const double *init_pose,
                   const rm_cost_params *prm, const rm_align_params *lm, double *pose_out,
                   rm_align_report *rep, void *stream) {
  if (!m) return fail(RM_EINVAL, "map is NULL");
  if (!scan || !scan->depth || !scan->cls) return fail(RM_EINVAL, "scan or its arrays NULL");
  if (!init_pose || !pose_out || !prm || !lm) return fail(RM_EINVAL, "NULL argument");
  if (lm->max_iters < 0 || lm->max_iters > 100000) return fail(RM_EINVAL, "max_iters out of range");
  std::lock_guard<std::mutex> lk(m->mu);
  cudaStream_t s = (cudaStream_t)stream;
  const rm_intrinsics *in = &scan->intr;
  RM_TRY(check_intr(in));
  RM_CK(cudaSetDevice(m->device));
  for (int attempt = 0;; ++attempt) {
    TileGeom tg = make_tiles(m, in);
    LoopBufs lb;
    auto arrays = [&](Carver &cv, rmk::LMState **st, long long **counts, long long **et, double **els,
                      double **grad, double **jtj) {
      *st = cv.take<rmk::LMState>(1);
      *counts = cv.take<long long>(6);
      *et = cv.take<long long>(1);
      *els = cv.take<double>(1);
      *grad = cv.take<double>(6);
      *jtj = cv.take<double>(21);
      loop_arrays(cv, m, scan, tg, 1, &lb);
    };
    rmk::LMState *d_st;
    long long *d_counts, *d_etable;
    double *d_els, *d_grad, *d_jtj;
    Carver plan{nullptr};
    arrays(plan, &d_st, &d_counts, &d_etable, &d_els, &d_grad, &d_jtj);
    RM_TRY(ensure_arena(m, plan.off, s));
    m->batch_inputs_valid = false;
    Carver cv{m->arena};
    arrays(cv, &d_st, &d_counts, &d_etable, &d_els, &d_grad, &d_jtj);
    WaveArgs a = loop_wave(m, scan, tg, 1, lb, *prm);
    a.res_counts = d_counts;
    a.res_etable = d_etable;
    a.res_els = d_els;
    a.res_grad = d_grad;
    a.res_jtj = d_jtj;
    RM_TRY(loop_inputs(scan, init_pose, lb, s));
    rmk::LMArgs la{lm->lambda0, lm->lambda_up, lm->lambda_down, lm->step_tol,
                   m->centre[0], m->centre[1], m->centre[2]};
    RM_CK(rmk::launch_lm_init(d_st, lb.T0, la, lb.M, lb.skip, s));
    RM_TRY(wave(m, a, rmk::kCostGrad, s));
    RM_CK(rmk::launch_lm_take_initial(d_st, d_counts, d_els, d_grad, d_jtj, s));
    for (int it = 0; it < lm->max_iters; ++it) {
      RM_CK(rmk::launch_lm_propose(d_st, la, lb.M, lb.skip, s));
      RM_TRY(wave(m, a, rmk::kCostGrad, s));
      RM_CK(rmk::launch_lm_accept(d_st, la, d_counts, d_els, d_grad, d_jtj, lb.skip, s));
    }
    rmk::LMState hs;
    bool retry;
    RM_TRY(loop_finish(m, s, &hs, d_st, sizeof(hs), attempt, &retry));
    if (retry) continue;
    RM_TRY(write_pose(pose_out, hs.T));
    if (rep) {
      rep->iters = hs.iters;
      rep->accepted = hs.accepted;
      rep->converged = hs.converged;
      rep->reserved = 0;
      rep->e_ls_initial = hs.e_ls0;
      rep->e_ls_final = hs.e;
      rep->e_table_initial = hs.e_table0;
      rep->e_table_final = hs.e_table;
    }
    return hs.converged ? RM_OK : fail(RM_ENOTCONV, "max_iters reached before step_tol");
  }
}

rm_status rm_dfo_align(rm_map *m, const rm_scan *scan, const double *init_pose,
                       const rm_cost_params *prm, const rm_dfo_params *dp, double *pose_out,
                       rm_dfo_report *rep, void *stream) {
  if (!m) return fail(RM_EINVAL, "map is NULL");
  if (!scan || !scan->depth || !scan->cls) return fail(RM_EINVAL, "scan or its arrays NULL");
  if (!init_pose || !pose_out || !prm || !dp) return fail(RM_EINVAL, "NULL argument");
  if (!(prm->eps >= 0.0f)) return fail(RM_EINVAL, "eps must be >= 0");
  if (dp->nm_iters < 0 || dp->cd_iters < 0 || dp->nm_iters > 100000 || dp->cd_iters > 100000)
    return fail(RM_EINVAL, "iteration counts out of range");
  if (!(dp->scale_t > 0.0) || !(dp->scale_r > 0.0) || !(dp->nm_step > 0.0) || !(dp->cd_step > 0.0) ||
      !(dp->nm_tol >= 0.0) || !(dp->cd_tol >= 0.0) || !std::isfinite(dp->scale_t) ||
      !std::isfinite(dp->scale_r) || !std::isfinite(dp->nm_step) || !std::isfinite(dp->cd_step))
    return fail(RM_EINVAL, "scales and steps must be finite and > 0, tolerances >= 0");
  if (dp->method != 0 && dp->method != 1) return fail(RM_EINVAL, "method must be 0 or 1");
  if (dp->method == 1 && (dp->powell_iters < 0 || dp->powell_iters > 100000 || !(dp->powell_step > 0.0) ||
                          !std::isfinite(dp->powell_step) || !(dp->powell_tol >= 0.0)))
    return fail(RM_EINVAL, "Powell: iterations 0..100000, a finite step > 0, a tolerance >= 0");
  std::lock_guard<std::mutex> lk(m->mu);
  cudaStream_t s = (cudaStream_t)stream;
  const rm_intrinsics *in = &scan->intr;
  RM_TRY(check_intr(in));
  RM_CK(cudaSetDevice(m->device));
  const int S = rmk::kDfoSlots;
  for (int attempt = 0;; ++attempt) {
    TileGeom tg = make_tiles(m, in);
    LoopBufs lb;
    auto arrays = [&](Carver &cv, rmk::DfoState **st, long long **counts, long long **et, double **els) {
      *st = cv.take<rmk::DfoState>(1);
      *counts = cv.take<long long>(6 * S);
      *et = cv.take<long long>(S);
      *els = cv.take<double>(S);
      loop_arrays(cv, m, scan, tg, S, &lb);
    };
    rmk::DfoState *d_st;
    long long *d_counts, *d_et;
    double *d_els;
    Carver plan{nullptr};
    arrays(plan, &d_st, &d_counts, &d_et, &d_els);
    RM_TRY(ensure_arena(m, plan.off, s));
    m->batch_inputs_valid = false;
    Carver cv{m->arena};
    arrays(cv, &d_st, &d_counts, &d_et, &d_els);
    WaveArgs a = loop_wave(m, scan, tg, S, lb, *prm);
    a.res_counts = d_counts;
    a.res_etable = d_et;
    a.res_els = d_els;
    RM_TRY(loop_inputs(scan, init_pose, lb, s));
    rmk::DfoArgs da{};
    da.nm_iters = dp->nm_iters;
    da.cd_iters = dp->cd_iters;
    da.method = dp->method;
    da.powell_iters = dp->method == 1 ? dp->powell_iters : 0;
    da.powell_step = dp->powell_step;
    da.powell_tol = dp->powell_tol;
    da.nm_step = dp->nm_step;
    da.nm_tol = dp->nm_tol;
    da.cd_step = dp->cd_step;
    da.cd_tol = dp->cd_tol;
    for (int k = 0; k < 3; ++k) {
      da.scale[k] = dp->scale_t;
      da.scale[3 + k] = dp->scale_r;
    }
    da.cx = m->centre[0];
    da.cy = m->centre[1];
    da.cz = m->centre[2];
    RM_CK(rmk::launch_dfo_init(d_st, lb.T0, da, lb.M, lb.skip, s));
    m->launches += 1;
    // at most: the simplex, two batches per Nelder-Mead iteration, one per descent step; or
    // the origin and seven line searches per Powell iteration
    const int max_steps = dp->method == 1 ? 1 + 7 * dp->powell_iters + dp->cd_iters
                                          : 1 + 2 * dp->nm_iters + dp->cd_iters;
    for (int it = 0; it < max_steps; ++it) {
      RM_TRY(wave(m, a, rmk::kCost, s));
      RM_CK(rmk::launch_dfo_step(d_st, da, d_et, lb.M, lb.skip, s));
      m->launches += 1;
    }
    rmk::DfoState hs;
    bool retry;
    RM_TRY(loop_finish(m, s, &hs, d_st, sizeof(hs), attempt, &retry));
    if (retry) continue;
    // the final pose T0 exp(xc^) on the device, through the library's retraction
    double *d_xi = reinterpret_cast<double *>(d_counts);  // 6 doubles of scratch
    double *d_out = d_xi + 6;
    RM_CK(cudaMemcpyAsync(d_xi, hs.xc, sizeof(double) * 6, cudaMemcpyHostToDevice, s));
    RM_CK(rmk::launch_retract(lb.T0, d_xi, 1, d_out, nullptr, s));
    m->launches += 1;
    RM_CK(cudaMemcpyAsync(pose_out, d_out, sizeof(double) * 16,
                          on_device(pose_out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    RM_CK(cudaStreamSynchronize(s));
    if (rep) {
      rep->evals = hs.evals;
      rep->nm_iters = hs.nm_iters;
      rep->nm_shrinks = hs.nm_shrinks;
      rep->cd_iters = hs.cd_iters;
      rep->converged = hs.converged;
      rep->powell_iters = hs.powell_iters;
      rep->e_table_initial = (long long)hs.f_init;
      rep->e_table_final = (long long)hs.fcur;
    }
    return hs.converged ? RM_OK : fail(RM_ENOTCONV, "coordinate descent ran out of iterations");
  }
}

rm_status rm_icp_align(rm_map *m, const rm_scan *scan, const double *init_pose,
                       const rm_icp_params *prm, double *pose_out, rm_icp_report *rep,
                       void *stream) {
  if (!m) return fail(RM_EINVAL, "map is NULL");
  if (!scan || !scan->depth || !scan->cls) return fail(RM_EINVAL, "scan or its arrays NULL");
  if (!init_pose || !pose_out || !prm) return fail(RM_EINVAL, "NULL argument");
  if (prm->max_iters < 0 || prm->max_iters > 100000) return fail(RM_EINVAL, "max_iters out of range");
  if (!(prm->tol >= 0.0f)) return fail(RM_EINVAL, "tol must be >= 0");
  std::lock_guard<std::mutex> lk(m->mu);
  cudaStream_t s = (cudaStream_t)stream;
  const rm_intrinsics *in = &scan->intr;
  RM_TRY(check_intr(in));
  RM_CK(cudaSetDevice(m->device));
  for (int attempt = 0;; ++attempt) {
    TileGeom tg = make_tiles(m, in);
    LoopBufs lb;
    auto arrays = [&](Carver &cv, rmk::IcpState **st, long long **n, double **l1, double **e2,
                      double **g, double **H) {
      *st = cv.take<rmk::IcpState>(1);
      *n = cv.take<long long>(1);
      *l1 = cv.take<double>(1);
      *e2 = cv.take<double>(1);
      *g = cv.take<double>(6);
      *H = cv.take<double>(21);
      loop_arrays(cv, m, scan, tg, 1, &lb);
    };
    rmk::IcpState *d_st;
    long long *d_n;
    double *d_l1, *d_e2, *d_g, *d_H;
    Carver plan{nullptr};
    arrays(plan, &d_st, &d_n, &d_l1, &d_e2, &d_g, &d_H);
    RM_TRY(ensure_arena(m, plan.off, s));
    m->batch_inputs_valid = false;
    Carver cv{m->arena};
    arrays(cv, &d_st, &d_n, &d_l1, &d_e2, &d_g, &d_H);
    const rm_cost_params cp{prm->tol, 0.0f, 0.0f, 0.0f};
    WaveArgs a = loop_wave(m, scan, tg, 1, lb, cp);
    a.res_n = d_n;
    a.res_l1 = d_l1;
    a.res_els = d_e2;
    a.res_grad = d_g;
    a.res_jtj = d_H;
    RM_TRY(loop_inputs(scan, init_pose, lb, s));
    const rmk::IcpArgs ia{prm->step_tol, m->centre[0], m->centre[1], m->centre[2]};
    RM_CK(rmk::launch_icp_init(d_st, lb.T0, ia, lb.M, lb.skip, s));
    m->launches += 1;
    for (int it = 0; it < prm->max_iters; ++it) {
      RM_TRY(wave(m, a, rmk::kIcp, s));
      RM_CK(rmk::launch_icp_step(d_st, ia, d_n, d_l1, d_g, d_H, lb.M, lb.skip, s));
      m->launches += 1;
    }
    rmk::IcpState hs;
    bool retry;
    RM_TRY(loop_finish(m, s, &hs, d_st, sizeof(hs), attempt, &retry));
    if (retry) continue;
    RM_TRY(write_pose(pose_out, hs.T));
    if (rep) {
      rep->iters = hs.iters;
      rep->converged = hs.converged;
      rep->n_assoc = hs.n_assoc;
      rep->cost_l1_initial = hs.l1_0;
      rep->cost_l1_final = hs.l1;
    }
    return hs.converged ? RM_OK : fail(RM_ENOTCONV, "no ICP step fell below step_tol");
  }
}

}  // extern "C"
