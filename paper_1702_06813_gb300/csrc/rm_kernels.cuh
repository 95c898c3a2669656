// rm_kernels.cuh -- launch interface between the C-ABI layer and the CUDA kernels.
#pragma once

#include <cstdint>
#include <string>
#include <cuda_runtime.h>

#include "rendermap.h"
#include "rm_internal.cuh"

namespace rmk {

struct CostParams {
  float eps, w_fofo, w_fofu, w_fufo;
};

// Per-wave scratch and per-call buffers handed to the kernels.
struct WaveArgs {
  DevCam cam;
  TileGeom tg;
  int V;
  long long T;
  int n_poses;        // poses in this wave
  int wave_base;      // global index of the wave's first pose
  const float4 *v;    // map vertices (re-centred), w unused
  const int4 *faces;  // i0, i1, i2, label
  const float4 *planes;  // unit world normal, label bits in w
  const float *Ms;    // 12 floats per global pose (world -> camera, FP32)
  // clusters of <= 64 triangles over <= 64 vertices, built at map creation
  int n_clusters;
  const int4 *cl_info;     // vertex offset, triangle offset, vertex count, triangle count
  const float4 *cl_sphere; // bounding sphere (re-centred frame)
  const float4 *cl_pos;    // per cluster vertex: position (re-centred), global index bits in w
  const uchar4 *cl_tris;   // local vertex indices per cluster triangle
  const int *cl_ids;       // original face id per cluster triangle
  int4 *vis;          // wave: the visible clusters' info records per pose (n_clusters each)
  int *vis_count;     // wave: one counter per pose
  int *counts;        // wave: ntiles per pose
  unsigned char *bins;  // wave: ntiles * cap records of tg.rec_bytes per pose
  double *partial;    // wave: ntiles * kNumVals per pose
  unsigned *status;   // device status word
  const int *skip;    // optional: non-zero means "skip this evaluation" (LM control)
  long long wait_cycles;  // budget of each bounded device wait, cycles (<= 0: about 2^31)
  const float4 *vnormals;  // optional world-frame vertex normals (ICP's normal-coloured map)
  // cost inputs
  const float *scan_depth;
  const uint8_t *scan_cls;
  CostParams prm;
  // per-pose results (global pose index): counts[6] e_table e_ls grad[6] jtj[21]
  long long *res_counts;
  long long *res_etable;
  double *res_els;
  double *res_grad;
  double *res_jtj;
  // ICP mode (the tolerance travels in prm.eps; e2, J^T e and J^T J in res_els, res_grad and
  // res_jtj): associated pixels and C = sum |Z_M - Z_1|
  long long *res_n;
  double *res_l1;
  // render outputs (global pose index)
  float *depth;
  int *tri_id;
  float *bary;
};

// kIcpVn: the ICP epilogue with the map's per-vertex normals; the raster launch picks it in
// place of kIcp when the map carries vertex normals, so the face-normal form keeps its code.
enum Mode { kRender = 0, kCost = 1, kCostGrad = 2, kIcp = 3, kIcpVn = 4 };
__host__ __device__ constexpr bool is_icp(int mode) { return mode == kIcp || mode == kIcpVn; }

cudaError_t launch_pose_to_m(const double *poses, int n, double cx, double cy, double cz,
                             float *Ms, cudaStream_t s);
// ev (optional, 5 events): recorded before the cull kernel, then after the cull, setup,
// raster and reduce kernels, on stream s.
// zero_counters: clear the wave's bin counts and visible-cluster count first (callers that
// clear them for several waves at once pass false)
cudaError_t launch_wave(const WaveArgs &a, int mode, cudaStream_t s, cudaEvent_t *ev = nullptr,
                        bool zero_counters = true);
int wave_kernel_launches(const WaveArgs &a, int mode);
cudaError_t launch_retract(const double *T, const double *xi, int n, double *out, double *jr,
                           cudaStream_t s);
// out_k = R n_k for V vertex normals (n: V*3 device floats, R row major): world-frame float4.
cudaError_t launch_rotate_normals(const float *n, int V, const float *R, float4 *out, cudaStream_t s);
// out_k = scale_k J_r(xi_k)^T g_k (scale optional: 1), device arrays.
cudaError_t launch_twist_grad(const double *xi, const double *g, const double *scale, int n,
                              double *out, cudaStream_t s);
// n copies of `pose` (device, 16 doubles) and the twists t_i e_axis of a sweep (rm_util.cu).
cudaError_t launch_sweep_inputs(const double *pose, int axis, double span, int n, double *poses,
                                double *twists, cudaStream_t s);

// Levenberg-Marquardt state on the device (one pose).
struct LMState {
  double T[16];        // current pose
  double Tc[16];       // candidate pose
  double e, g[6], H[21];
  double lambda;
  long long e_table;
  double e_ls0;
  long long e_table0;
  int iters, accepted, converged, done;
  int have_candidate;
  int pad;
};

struct LMArgs {
  double lambda0, lambda_up, lambda_down, step_tol;
  double cx, cy, cz;   // map centre
};

// Point-to-plane ICP state on the device (one pose).
struct IcpState {
  double T[16];        // current pose
  double l1_0, l1;     // C at the first and at the last evaluation
  long long n_assoc;   // associated pixels at the last evaluation
  int iters, converged, done, evals;
};

struct IcpArgs {
  double step_tol;
  double cx, cy, cz;   // map centre
};

cudaError_t launch_icp_init(IcpState *st, const double *T0, const IcpArgs &a, float *M,
                            int *skip, cudaStream_t s);
cudaError_t launch_icp_init_batch(IcpState *st, const double *T0, int n, const IcpArgs &a,
                                  float *Ms, int *skip, cudaStream_t s);
// After an evaluation at the state's pose (outputs n, l1, g = J^T e, H = J^T J): record it,
// solve, move the pose and write its matrix, or set *skip when the iterations are over.
cudaError_t launch_icp_step(IcpState *st, const IcpArgs &a, const long long *n,
                            const double *l1, const double *g, const double *H, float *M,
                            int *skip, cudaStream_t s);

// Vertex-position gradient of the surrogate from a rendered visibility buffer.
struct VGradArgs {
  DevCam cam;
  int W, n_poses;
  long long P;            // pixels per pose
  const float *Ms;        // 12 floats per pose
  const float4 *planes;   // unit world normal, label bits in w
  const int4 *faces;      // i0, i1, i2, label
  const int *tri_id;      // n_poses * P
  const float *depth;     // n_poses * P (the z-buffer depth)
  const float *bary;      // n_poses * P * 2
  const float *scan_depth;
  const uint8_t *scan_cls;
  CostParams prm;
  double *grad;           // V * 3, accumulated
};
cudaError_t launch_vertex_grad(const VGradArgs &a, cudaStream_t s);

// Derivative-free search state on the device (one pose): Nelder-Mead over scaled twists,
// then coordinate descent, on the Table I cost of T0 exp(xi^); candidates are evaluated as
// one wave of kDfoSlots poses.
constexpr int kDfoSlots = 12;
struct DfoState {
  double T0[16];
  double x[7][6], f[7];       // simplex vertices and values
  double cand[kDfoSlots][6];  // candidates of the pending evaluation
  double xc[6], fcur, st[6];  // coordinate descent: point, value, steps
  double f_init;              // the cost at the start pose
  int phase;                  // 0 simplex, 1 NM step, 2 NM shrink, 3 coordinate step, 4 done,
                              // 5 Powell start, 6 Powell line search
  int n_cand;
  int evals, nm_iters, nm_shrinks, cd_iters, converged, shrink_best;
  // Powell's method: directions, the iteration's start and displacement, the line step
  double D[6][6], x0[6], disp[6], n2, ps, best_drop;
  int pdir, best_dir, powell_iters;
};

struct DfoArgs {
  int nm_iters, cd_iters;
  int method, powell_iters;   // method 1: Powell's method in place of Nelder-Mead
  double powell_step, powell_tol;
  double nm_step, nm_tol, cd_step, cd_tol;
  double scale[6];
  double cx, cy, cz;  // map centre
};

cudaError_t launch_dfo_init(DfoState *st, const double *T0, const DfoArgs &a, float *Ms,
                            int *skip, cudaStream_t s);
// Takes the Table I costs of the pending candidates (e_table per slot), advances the search
// and writes the next candidates' matrices, or sets *skip when the search is over.
cudaError_t launch_dfo_step(DfoState *st, const DfoArgs &a, const long long *e_table, float *Ms,
                            int *skip, cudaStream_t s);

// Batch of problems (each its own camera, scan and scratch) run by one persistent kernel.
constexpr int kPersistCull = 4;   // 256-cluster chunks per cull item
// Persistent kernel screen tiles, two per raster item: 64x32 for pinhole problems, 16x16 for
// ray-table problems (a panoramic tile can hold thousands of bin records, and smaller tiles
// split that serial work over more CTAs).
constexpr int kPersistTileW[2] = {64, 16};
constexpr int kPersistTileH[2] = {32, 16};
constexpr int kPersistTiles[2] = {2, 2};
struct BatchArgs {
  const WaveArgs *probs;   // one per problem (n_poses 1, wave_base 0)
  int n_problems;
  // Two ready queues in one slot array: slots [0, cap[0]) take raster and reduce items, slots
  // [cap[0], cap[0] + cap[1]) cull and setup items. An item is (problem, phase (0 cull,
  // 1 setup, 2 raster, 3 reduce+LM), index within the phase, evaluation number), packed into
  // one 64-bit word by pack_item so that a claim reads it with a single load; a slot holds -1
  // until it is published.
  long long *items;
  int cap[2];
  int *qctl;               // head (claimed) and tail (reserved) of each queue, then the number
                           // of finished problems; zero before launch except the first tail
  int *done;               // 4 counters per problem: items completed per phase this evaluation
  int *need;               // per problem: cull items, setup items (set by the kernel each
                           // evaluation from the visible-cluster count), raster items
  LMState *lm;             // per problem, or null for a plain evaluation
  IcpState *icp;           // per problem for ICP alignment (raster in ICP mode), else null
  IcpArgs icpargs;
  float *Ms;               // 12 floats per problem (the problems' a.Ms point here)
  int *skip;               // one flag per problem (the problems' a.skip point here)
  LMArgs lmargs;
  int lm_iters;            // LM (or ICP) iterations after the first evaluation (evaluations
                           // 0..lm_iters)
  unsigned *status;
  long long spin_limit;    // cycles a CTA may go without finding work before it gives up
};

// Queue item fields: index within the phase (21 bits), phase (2), evaluation (17), problem
// (23). The host checks the limits before a launch.
constexpr int kItemIndexBits = 21, kItemEvalBits = 17, kItemProblemBits = 23;
static_assert(kItemIndexBits + 2 + kItemEvalBits + kItemProblemBits == 63, "item fields fill 63 bits");
// Evaluations (at most 100001) and raster items (at most 16384^2 / 256 / 2) always fit their
// fields; the host checks the problem count and the setup items per evaluation.
__host__ __device__ constexpr long long pack_item(int problem, int phase, int index, int eval) {
  return ((long long)problem << 40) | ((long long)eval << 23) | ((long long)phase << 21) | (long long)index;
}

constexpr int kSetupClusters = 64;  // visible clusters per setup item (eight per warp), at most
// Visible clusters per persistent setup item by camera model: pinhole 64; ray-table views,
// which see many more clusters, 128.
__host__ __device__ constexpr int setup_clusters(int model) { return model != 0 ? 128 : kSetupClusters; }
constexpr int kSetupCtasPerGpu = 912;  // setup CTAs a small wave may spread over (152 SMs x 6)

// Every slot unpublished except the evaluation-0 cull items of every problem at the head of
// the cull/setup queue; sets that queue's tail.
cudaError_t launch_queue_init(long long *items, int n_slots, int first_low, int n_problems,
                              int cull_items, int *qctl, cudaStream_t s);

cudaError_t launch_lm_init_batch(LMState *st, const double *T0, int n, const LMArgs &a,
                                 float *Ms, int *skip, cudaStream_t s);
cudaError_t launch_persist(const BatchArgs &b, int grid, cudaStream_t s);
int persist_grid(int device);
// The persistent kernel for a homogeneous plain batch: the problems are the n_poses poses of
// the one argument block w (pose q's arrays at the wave's per-pose offsets).
cudaError_t launch_persist_wave(const BatchArgs &b, const WaveArgs &w, int grid, cudaStream_t s);
int persist_wave_grid(int device, int model);

cudaError_t launch_lm_init(LMState *st, const double *T0, const LMArgs &a, float *M,
                           int *skip, cudaStream_t s);
cudaError_t launch_lm_take_initial(LMState *st, const long long *counts, const double *els,
                                   const double *grad, const double *jtj, cudaStream_t s);
cudaError_t launch_lm_propose(LMState *st, const LMArgs &a, float *M, int *skip,
                              cudaStream_t s);
cudaError_t launch_lm_accept(LMState *st, const LMArgs &a, const long long *counts,
                             const double *els, const double *grad, const double *jtj,
                             int *skip, cudaStream_t s);

}  // namespace rmk

// Host-side helpers of rm_api.cu shared with the other entry-point files.
namespace rmapi {
// Fills the map- and camera-derived fields of a (camera, tiles, mesh and cluster arrays) and
// the map centre; checks the intrinsics (RM_EINVAL with a message on failure).
rm_status wave_inputs(const rm_map *map, const rm_intrinsics *intr, rmk::WaveArgs *a,
                      double centre[3]);
// Sets the calling thread's rm_last_error message.
void set_error(const std::string &msg);
// Checks the intrinsics as every evaluation entry point does (RM_EINVAL with a message).
rm_status check_intrinsics(const rm_intrinsics *in);
// True for device (or managed) memory.
bool is_device_pointer(const void *p);
// The device the map's arrays live on (the device current at rm_map_create).
int map_device(const rm_map *map);
}  // namespace rmapi
