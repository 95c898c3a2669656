/*
 * rendermap.h -- C ABI of the GB300 RenderMap pose-cost library (librendermap.so).
 *
 * The library evaluates how well a 6-DoF sensor pose aligns an observed range image with a
 * labelled triangle-mesh map, following Ryde & Ding, "RenderMap: Exploiting the Link Between
 * Perception and Rendering for Dense Mapping" (arXiv 1702.06813):
 *   - the map is the mesh of the interfaces between free, occupied and unknown space, each
 *     face labelled free-occupied (FO), free-unknown (FU) or unknown-occupied (UO) (Sec. IV.A,
 *     Fig. 3);
 *   - E(X) = C(R(T(X)), Z_s) (Eq. 1): render the map's z-buffer R from the camera pose and
 *     compare it per pixel with the scan Z_s;
 *   - the comparison is Table I (Sec. IV.B), summed over all pixels.
 * On top of the paper's cost the library computes a truncated least-squares surrogate with
 * the same cells and thresholds, its derivative with respect to a pose twist, and
 * Levenberg-Marquardt steps on it (the paper's Sec. IV.C optimiser is derivative-free).
 * Around that path: render-accelerated point-to-plane ICP (Sec. V), the derivative-free
 * search of Sec. IV.C on the exact Table I cost, Fig. 7's cost sweeps, depth-image normals
 * (Eq. 2) and blur, the meshification of range images (Sec. IV.A), the cost's gradient with
 * respect to the map's vertices, and input helpers for raw range images and the paper's pose
 * vector.
 *
 * All work runs in CUDA kernels for sm_103a on the calling thread's current device.
 *
 * Conventions
 *  - Pose: 16 doubles, row-major 4x4 camera-to-world transform T_wc (p_w = R p_c + t).
 *  - Camera frame: x right, y down, z forward. Pinhole rays of pixel (i, j) are
 *    ((i + .5 - cx)/fx, (j + .5 - cy)/fy, 1), so pinhole depth is z-depth; ray-table rays are
 *    unit vectors, so ray-table depth is range.
 *  - Images are row-major H x W (pixel (i, j) at index j*W + i), one image per pose.
 *  - Twist: xi = (rho, phi) (translation first), right perturbation T <- T exp(xi^).
 *  - Packed symmetric 6x6: the 21 entries of the upper triangle, row major
 *    ((0,0),(0,1),...,(0,5),(1,1),...,(5,5)).
 *  - Pointers marked "host or device" may point to either; the library finds out with
 *    cudaPointerGetAttributes. Host outputs make the call wait for the stream.
 *
 * Errors: every entry point returns an rm_status. Nothing crosses the ABI as an exception and
 * no kernel traps: device-side problems (a full bin, a wait that ran out) are recorded in a
 * status word that the call reads back. rm_last_error() gives a message for the calling
 * thread's last failure.
 *
 * Threading: calls on one map are serialised by the map (they share its scratch memory).
 * Different maps may be used from different threads concurrently.
 */
#ifndef RENDERMAP_H
#define RENDERMAP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RM_OK = 0,
  RM_EINVAL = 1,     /* bad argument: null pointer, size, index, label or non-finite input */
  RM_ENOMEM = 2,     /* device memory allocation failed */
  RM_ECUDA = 3,      /* a CUDA runtime call failed (message in rm_last_error) */
  RM_EOVERFLOW = 4,  /* a screen-tile bin overflowed and could not be grown */
  RM_ETIMEOUT = 5,   /* a bounded device-side wait gave up */
  RM_ENOTCONV = 6    /* rm_align / rm_icp_align stopped without meeting step_tol */
} rm_status;

/* Face labels (Sec. IV.A): the interface a map face lies on. */
enum { RM_LABEL_FO = 0, RM_LABEL_FU = 1, RM_LABEL_UO = 2 };
/* Scan pixel classes (Sec. IV.B): a return (FO), no return drawn at the sensor's maximum
 * range (FU, Sec. IV.A), or a dead pixel (NaN). A scan pixel whose depth is not finite, or
 * whose class byte is above 2, counts as NaN. */
enum { RM_SCAN_FO = 0, RM_SCAN_FU = 1, RM_SCAN_NAN = 2 };
/* Table I outcomes, the index into every counts[6] array. */
enum {
  RM_FOFO_REWARD = 0,   /* map FO, scan FO, |dz| <= eps  : -1 */
  RM_FOFO_PENALTY = 1,  /* map FO, scan FO, |dz| >  eps  : +1 */
  RM_FOFU_REWARD = 2,   /* map FO, scan FU, dz > 0       : -1 */
  RM_FOFU_PENALTY = 3,  /* map FO, scan FU, dz <= 0      : +1 */
  RM_FUFO_REWARD = 4,   /* map FU, scan FO, dz <= 0      : -1 */
  RM_FUFO_PENALTY = 5   /* map FU, scan FO, dz > 0       : +1 */
};
enum { RM_PINHOLE = 0, RM_RAYTABLE = 1 };

typedef struct {
  int32_t model;            /* RM_PINHOLE or RM_RAYTABLE */
  int32_t width, height;    /* pixels, 1..16384 */
  int32_t reserved;         /* 0 */
  float fx, fy, cx, cy;     /* pinhole focal lengths and principal point, pixels */
  /* RM_RAYTABLE layout: column i looks at azimuth az0 + az_step*(i + .5), row j at elevation
   * el0 - el_step*j (radians; azimuth from +z toward +x, elevation toward -y). The layout only
   * bounds which pixels a triangle may cover; coverage and depth use `rays`. */
  float az0, az_step, el0, el_step;
  float near_m;             /* render clip: only depths >= near_m are kept (> 0) */
  float far_m;              /* and <= far_m (INFINITY allowed) */
  const float *rays;        /* RM_RAYTABLE only: H*W*3 float32 unit rays, camera frame, host
                               or device; each ray within 0.25 px of the layout above */
} rm_intrinsics;

/* Observed scan Z_s (Eq. 1): depth and class per pixel, same layout and size as `intr`. */
typedef struct {
  rm_intrinsics intr;
  const float *depth;       /* H*W float32 metres (z-depth / range), host or device */
  const uint8_t *cls;       /* H*W uint8 RM_SCAN_*, host or device */
} rm_scan;

typedef struct {
  float eps;                /* Table I inlier threshold, metres (the paper's 0.1) */
  float w_fofo, w_fofu, w_fufo; /* weights of the least-squares surrogate per Table I row/col */
} rm_cost_params;

/* Per-pose outputs of rm_cost / rm_cost_grad; any pointer may be NULL; host or device. */
typedef struct {
  int64_t *counts;          /* N*6 pixels per Table I outcome (RM_FOFO_REWARD ...) */
  int64_t *e_table;         /* N   Table I cost: penalties minus rewards (Sec. IV.B) */
  double *e_ls;             /* N   1/2 sum w r^2 of the truncated least-squares surrogate */
  double *grad;             /* N*6 d e_ls / d xi = sum w r J (rm_cost_grad only) */
  double *jtj;              /* N*21 packed sum w J J^T (rm_cost_grad only) */
} rm_cost_out;

/* Execution knobs; a zeroed struct (or NULL) means "library defaults / autotuned". */
typedef struct {
  int32_t tile_w, tile_h;   /* screen tile, pixels: 16x16, 32x16, 32x32 or 64x32; 0 = per
                               camera model as in the batched entry points (64x32 pinhole,
                               16x16 ray table) */
  int32_t bin_capacity;     /* triangle records per tile bin (grown on overflow) */
  int32_t wave_poses;       /* poses processed together per kernel wave */
  int32_t async_status;     /* 1: do not read the device status back (graph capture);
                               check it later with rm_status_sync */
  int32_t wait_log2;        /* 0: default budgets of the bounded device waits (about 2^31
                               cycles for a bulk copy, 2^32 for the batch kernel's work
                               queue); 1..40: every such wait gives up after 2^wait_log2
                               cycles and the call returns RM_ETIMEOUT (a copy still in
                               flight is drained with the default budget first) */
  int32_t reserved[2];
} rm_tuning;

typedef struct {
  int32_t max_iters;        /* LM iterations (each one render+residual+gradient) */
  int32_t reserved;
  double lambda0;           /* initial damping (1e-3) */
  double lambda_up, lambda_down; /* damping factor on reject / accept (10, 10) */
  double step_tol;          /* stop when |delta xi| < step_tol */
} rm_align_params;

typedef struct {
  int32_t iters, accepted, converged, reserved;
  double e_ls_initial, e_ls_final;
  int64_t e_table_initial, e_table_final;
} rm_align_report;

typedef struct rm_map rm_map;

/* Build a map from host arrays: vertices V*3 float32 (world, metres), faces T*3 int32
 * (indices into vertices), labels T uint8 (RM_LABEL_*). The map copies everything to the
 * device, re-centres the vertices on their bounding-box centre (in FP64, rounded back to
 * FP32; poses are shifted to match) and precomputes unit face normals. Ownership: the
 * caller keeps its arrays; *out is released with rm_map_destroy.
 * Errors: RM_EINVAL for null pointers, negative sizes, T >= 2^31, an index outside [0, V),
 * a label above 2 or a non-finite vertex; RM_ENOMEM; RM_ECUDA. (Sec. IV.A, Fig. 3.) */
rm_status rm_map_create(const float *vertices, int64_t n_vertices, const int32_t *faces,
                        const uint8_t *labels, int64_t n_faces, rm_map **out);
void rm_map_destroy(rm_map *map);
/* Sizes and the re-centring offset of a map (any output may be NULL). */
rm_status rm_map_info(const rm_map *map, int64_t *n_vertices, int64_t *n_faces,
                      double centre[3]);
rm_status rm_map_set_tuning(rm_map *map, const rm_tuning *tuning);

/* Attaches per-vertex normals to the map for the point-to-plane ICP entry points (Sec. V,
 * sequential depth-image alignment, steps 2-3: the normals of D_i by Eq. 2, then the points of
 * D_i rendered coloured by their normals). Afterwards the normal of an associated pixel is the
 * blend of the seen triangle's three vertex normals by the hit's barycentrics (a rasteriser
 * interpolating a vertex attribute), rotated into the current camera frame and normalised;
 * a pixel whose blend is not finite (a vertex with a NaN normal) is not associated. Without
 * vertex normals the ICP uses each triangle's plane normal.
 *  - normals: V*3 floats, host or device, in the frame of `pose`; NULL detaches the normals;
 *  - pose: 16 doubles (host), the camera-to-world pose of the frame the normals are given in
 *    (e.g. the pose of the depth image whose Eq. 2 normals they are), or NULL for world-frame
 *    normals. The library stores the normals rotated into the world frame (FP32).
 * Waits for `stream`. Errors: RM_EINVAL, RM_ENOMEM/RM_ECUDA. */
rm_status rm_map_set_vertex_normals(rm_map *map, const float *normals, const double *pose,
                                    void *stream);
rm_status rm_map_get_tuning(const rm_map *map, rm_tuning *tuning);

/* R(Y) of Eq. 1: the z-buffer of the map seen from each of N poses. The z-buffer keeps, per
 * pixel, the nearest triangle under the library's FP32 rasterisation contract (8-bit
 * sub-pixel snapping, top-left fill rule, one sample at the pixel centre, no anti-aliasing
 * as in Sec. VI; ties go to the lower triangle id).
 * depth: N*H*W float32, NaN where the ray hits nothing (the paper's NaN, Sec. IV.B);
 * tri_id: optional N*H*W int32, -1 where nothing is hit;
 * bary: optional N*H*W*2 float32 barycentrics (b1, b2) of the hit on that triangle.
 * All outputs host or device; `poses` host or device. stream: a cudaStream_t or NULL. */
rm_status rm_render_depth(rm_map *map, const double *poses, int32_t n_poses,
                          const rm_intrinsics *intr, float *depth, int32_t *tri_id,
                          float *bary, void *stream);

/* E(X) of Eq. 1 with C from Table I (Sec. IV.B) for N poses against one scan, plus the
 * least-squares surrogate: counts, e_table and e_ls in `out` (grad / jtj ignored). */
rm_status rm_cost(rm_map *map, const rm_scan *scan, const double *poses, int32_t n_poses,
                  const rm_cost_params *params, const rm_cost_out *out, void *stream);

/* As rm_cost, plus the adjoint: the gradient of e_ls with respect to the pose twist and the
 * Gauss-Newton matrix sum w J J^T, from the ray-plane depth t = d_c / (n_c . r):
 * dt/drho = -n_c / (n_c . r), dt/dphi = -t (r x n_c) / (n_c . r). */
rm_status rm_cost_grad(rm_map *map, const rm_scan *scan, const double *poses,
                       int32_t n_poses, const rm_cost_params *params, const rm_cost_out *out,
                       void *stream);

/* Pose retraction used by the Levenberg-Marquardt step and by autograd bindings:
 * out_k = poses_k exp(twists_k^) in FP64 on the device (N*16 doubles out), and optionally
 * jr (N*36, row major) = the SE(3) right Jacobian J_r(twist_k), with which
 * d e(T exp(xi)) / d xi = J_r(xi)^T grad. poses N*16, twists N*6; all host or device.
 * Uses stream-ordered device scratch when any pointer is on the host, and then waits. */
rm_status rm_pose_retract(const double *poses, const double *twists, int32_t n_poses,
                          double *out, double *jr, void *stream);

/* The same chain rule applied on the device: out_k = scale_k J_r(twists_k)^T grads_k, the
 * derivative of e(T exp(xi^)) with respect to xi from the adjoint gradient at the retracted
 * pose (rm_cost_grad), scaled by an upstream derivative (autograd's grad_output). twists and
 * grads N*6, scale N (optional: 1), out N*6 doubles; all host or device. Uses stream-ordered
 * device scratch when any pointer is on the host, and then waits. */
rm_status rm_twist_grad(const double *twists, const double *grads, const double *scale,
                        int32_t n, double *out, void *stream);

/* Levenberg-Marquardt alignment of one scan from init_pose (16 doubles, host or device):
 * each iteration renders, evaluates the surrogate and its gradient, solves
 * (H + lambda diag H) delta = -g in FP64 on the device, and accepts T exp(delta^) if e_ls
 * drops. pose_out (16 doubles) and rep (optional) are host or device / host.
 * Returns RM_ENOTCONV (with pose_out valid) when max_iters is reached first. */
rm_status rm_align(rm_map *map, const rm_scan *scan, const double *init_pose,
                   const rm_cost_params *params, const rm_align_params *lm, double *pose_out,
                   rm_align_report *rep, void *stream);

/* ---- Vertex-position gradient (map refinement) ----------------------------------------
 * grad_v (V*3 doubles, host or device, overwritten) = the sum over the n poses of
 * d e_ls / d (world vertex positions) against one scan: each pixel with an active residual r
 * (the cells and thresholds of rm_cost_grad) adds w r sgn b_m n / (n_c . ray) to vertex m of
 * its winning triangle (b_m its barycentric, n the unit world normal, n_c the camera-frame
 * one). Renders each pose's visibility buffer (ids, depths, barycentrics), then scatters with
 * FP64 atomics, so the summation order (and the last bits) vary from run to run. Errors as
 * rm_cost_grad. */
rm_status rm_cost_grad_vertices(rm_map *map, const rm_scan *scan, const double *poses,
                                int32_t n_poses, const rm_cost_params *params, double *grad_v,
                                void *stream);

/* ---- Input helpers ----------------------------------------------------------------------
 * Depth and class of n pixels of raw range images (Sec. IV.A, IV.B): a NaN reading, or a
 * return closer than range_min (and above 0), is a dead pixel (RM_SCAN_NAN, depth NaN); no
 * reading (<= 0, above range_max, +inf) is free space up to the sensor's maximal range
 * (RM_SCAN_FU, depth range_max); the rest are returns (RM_SCAN_FO, their range). Arrays host
 * or device (host outputs complete on return). RM_EINVAL unless 0 <= range_min < range_max
 * < inf. */
rm_status rm_scan_from_range(const float *range, int64_t n_pixels, float range_min,
                             float range_max, float *depth, uint8_t *cls, void *stream);

/* Camera-to-world poses (n*16 doubles) from the paper's pose vectors X = (x, y, z, theta_x,
 * theta_y, theta_z) (n*6 doubles, Eq. 1), read as R = Rz(theta_z) Ry(theta_y) Rx(theta_x)
 * (the paper does not state the order) and translation (x, y, z). Host or device. */
rm_status rm_pose_from_x(const double *X, int32_t n, double *poses, void *stream);

/* ---- Render-accelerated point-to-plane ICP (Sec. V) ----------------------------------
 * Projective association: the map is rendered at the pose and each pixel's winning surface is
 * paired with the scan return of the same pixel when the surface is FO, the scan pixel is an
 * FO return, and |Z_M - Z_1| < tol (decided in FP32 on the z-buffer depth and the scan depth,
 * the z-difference test of Sec. V). For a pair, with r the pixel's ray, t the map depth, d
 * the scan depth, p = d r the scan point and n the map surface's unit normal in the camera
 * frame, the residual is the point-to-plane distance e = (d - t) (n . r) and its Jacobian
 * with respect to the right-perturbation twist (rho, phi) of the pose (T <- T exp(xi^)) is
 * J = (n, p x n). Per pose the terms are summed over the pairs in a fixed order. */

/* Per-pose outputs of rm_icp_terms; any pointer may be NULL; host or device. */
typedef struct {
  int64_t *n_assoc;         /* N   associated pixels */
  double *cost_l1;          /* N   C = sum |Z_M - Z_1| over the associated pixels (Sec. V) */
  double *e2;               /* N   sum e^2 */
  double *jte;              /* N*6 sum J e */
  double *jtj;              /* N*21 packed sum J J^T (row-major upper triangle) */
} rm_icp_out;

/* ICP terms for N poses (poses: N*16 doubles camera-to-world, host or device) against one
 * scan. tol (metres) must be >= 0 (0 associates nothing). Arguments are checked as in
 * rm_cost_grad (RM_EINVAL); the map is not modified. */
rm_status rm_icp_terms(rm_map *map, const rm_scan *scan, const double *poses, int32_t n_poses,
                       float tol, const rm_icp_out *out, void *stream);

typedef struct {
  float tol;                /* association tolerance |Z_M - Z_1|, metres */
  int32_t max_iters;        /* Gauss-Newton iterations, each one render + association + solve */
  double step_tol;          /* stop when |delta xi| < step_tol (converged) */
} rm_icp_params;

typedef struct {
  int32_t iters;            /* pose updates applied */
  int32_t converged;        /* 1 when a step below step_tol ended the iterations */
  int64_t n_assoc;          /* associated pixels at the last evaluation */
  double cost_l1_initial;   /* C at the initial pose */
  double cost_l1_final;     /* C at the last evaluation */
} rm_icp_report;

/* Point-to-plane ICP of one scan from init_pose (16 doubles, host or device), all on the
 * device: each iteration re-renders and re-associates at the current pose, solves
 * J^T J delta = -J^T e by Cholesky in FP64 and moves the pose to T exp(delta^). Stops when
 * |delta| < step_tol, when J^T J is not positive definite (too few or degenerate pairs; the
 * pose is left where it was), or after max_iters iterations (0..100000). pose_out (16
 * doubles, host or device) and rep (optional, host) are written in every case; returns
 * RM_ENOTCONV when no step fell below step_tol. */
rm_status rm_icp_align(rm_map *map, const rm_scan *scan, const double *init_pose,
                       const rm_icp_params *params, double *pose_out, rm_icp_report *rep,
                       void *stream);


/* Surface normals of depth images (Eq. 2, Sec. V), n images of one camera (intr: width,
 * height, and fx, fy for metric normals), each H*W float depth plus H*W uint8 RM_SCAN_* class,
 * host or device. A pixel is valid when its class is FO and its depth finite. The valid depths
 * are smoothed with a Gaussian of sigma pixels (0 <= sigma <= 5, radius ceil(3 sigma), weights
 * renormalised over the valid pixels of the window; invalid pixels stay invalid), then
 * differentiated by central differences across and down the image; the normal is
 * N = a x b, a = (0, s_y, dz/dy), b = (s_x, 0, dz/dx), normalised (it faces the camera: N_z < 0).
 * metric = 0: s = 1 pixel (N ~ (dz/dx, dz/dy, -1), the paper's image-space form); metric = 1:
 * s_x = S/fx, s_y = S/fy, the pixel's footprint at its smoothed depth S (pinhole only).
 * normals: n*H*W*3 float (NaN on the border and where the pixel or a 4-neighbour is invalid);
 * smoothed (optional): n*H*W float S (NaN where invalid). Host outputs are complete on return;
 * device outputs are ordered on `stream`. Host arrays are staged through stream-ordered
 * allocations. Neither output may overlap depth, cls or the other output (other tiles still
 * read the inputs' halos while one writes). Errors: RM_EINVAL (sizes, more than 65535
 * images, sigma, metric without a pinhole, overlapping outputs), RM_ECUDA. */
rm_status rm_depth_normals(const rm_intrinsics *intr, int32_t n_images, const float *depth,
                           const uint8_t *cls, float sigma, int32_t metric, float *normals,
                           float *smoothed, void *stream);

/* Gaussian blur of depth images for cost smoothing (Sec. IV.C): the smoothing above alone.
 * out (n*H*W float, host or device) holds each FO return's smoothed depth and every other
 * pixel's input depth unchanged (FU pixels stay at their maximal range, dead pixels NaN), so
 * the result pairs with the same class image as a scan. out must not overlap depth or cls
 * (other tiles still read the inputs while one writes). Errors as rm_depth_normals. */
rm_status rm_depth_blur(const rm_intrinsics *intr, int32_t n_images, const float *depth,
                        const uint8_t *cls, float sigma, float *out, void *stream);

/* ---- Derivative-free search on the Table I cost (Sec. IV.C) ---------------------------
 * The paper minimises its piecewise-constant cost with Nelder-Mead and coordinate descent.
 * Here both run on the device over twists xi of the start pose (pose = T0 exp(xi^)), scaled
 * per axis by scale_t (metres) and scale_r (radians); each step's candidates are rendered and
 * scored together as one batch of 12 poses:
 *  - Nelder-Mead: simplex = origin plus nm_step * scale on each axis; per iteration the four
 *    points c + d, c + 2d, c + d/2, c - d/2 (c the centroid of the best six, d = c - worst)
 *    are scored together and the usual reflect / expand / contract / shrink rules applied
 *    (ties in value: the lower slot ranks first); ends after nm_iters iterations or when every
 *    vertex is within nm_tol (scaled) of the best;
 *  - or, with method = 1, Powell's conjugate-direction search in place of Nelder-Mead (the
 *    paper names it too, without settings): the directions start as the scaled axes; a line
 *    search from x along d scores the 12 points x + (a s) d, a = +-1/4, +-1/2, +-1, +-2, +-4,
 *    +-8 (in that order, + first; ties: the first), and moves to the lowest if it lowers the
 *    cost. An iteration searches the six directions in turn with the step s (powell_step at
 *    first), then the iteration's displacement d with s = 1, and replaces the direction that
 *    lowered the cost most by d over its scaled length; an iteration that does not move halves
 *    s. Ends after powell_iters iterations or once s < powell_tol;
 *  - coordinate descent from the best vertex with steps cd_step * scale: the 12 moves +-step
 *    along each axis scored together; the best move is taken if it lowers the cost, else all
 *    steps halve; converged when the largest scaled step is below cd_tol. */
typedef struct {
  int32_t nm_iters, cd_iters;
  double nm_step, nm_tol, cd_step, cd_tol;
  double scale_t, scale_r;
  int32_t method;           /* 0: Nelder-Mead, 1: Powell's method; then coordinate descent */
  int32_t powell_iters;
  double powell_step, powell_tol;
} rm_dfo_params;

typedef struct {
  int32_t evals;            /* poses scored (candidates only) */
  int32_t nm_iters, nm_shrinks, cd_iters, converged, powell_iters;
  int64_t e_table_initial, e_table_final;
} rm_dfo_report;

/* Derivative-free alignment of one scan from init_pose (16 doubles, host or device) on the
 * Table I cost with parameters `params` (the cost's eps and weights; the weights do not enter
 * E_table). pose_out (host or device) and rep (optional, host) are written in every case;
 * returns RM_ENOTCONV when coordinate descent ran out of iterations. */
rm_status rm_dfo_align(rm_map *map, const rm_scan *scan, const double *init_pose,
                       const rm_cost_params *params, const rm_dfo_params *dfo, double *pose_out,
                       rm_dfo_report *rep, void *stream);

/* Fig. 7's cost landscape: the Table I cost and surrogate at the n poses pose exp(t_i e_axis^)
 * with t_i = -span + 2 span i / (n - 1) (t = 0 for n = 1), i.e. a sweep along one twist axis
 * of the camera frame: axis 0..2 translation (metres), 3..5 rotation (radians). Evaluated as
 * one batch; pose (16 doubles) host or device; outputs as rm_cost (n per-pose entries). */
rm_status rm_cost_sweep(rm_map *map, const rm_scan *scan, const double *pose, int32_t axis,
                        double span, int32_t n, const rm_cost_params *params,
                        const rm_cost_out *out, void *stream);

/* ---- Meshification of a range image (Sec. IV.A, Fig. 5) ------------------------------ */
typedef struct {
  float max_range;          /* no-return pixels are drawn at this range (4 m for Kinect-class) */
  float max_edge;           /* quads with a side or diagonal longer than this are FU (0.1 m) */
  int32_t step;             /* grid stride in pixels (1; 2 = the factor-2 downsampling of Sec. V) */
  int32_t reserved;
} rm_meshify_params;

/* The labelled interface mesh of one range image seen from `pose` (16 doubles camera-to-world,
 * host or device). Grid pixels (every step-th across and down: Ws = (W-1)/step + 1 by
 * Hs = (H-1)/step + 1) become vertices in the world frame (vertex j*Ws + i for grid pixel
 * (i, j)): returns (scan class FO, finite depth) at their depth along the pixel's ray,
 * no-returns (FU) at max_range; dead pixels (class NaN, or a non-finite depth) are parked at
 * the sensor origin and used by no face. Each 2x2 block of adjacent grid vertices without a
 * dead pixel gives two triangles (v00, v10, v11), (v00, v11, v01), labelled RM_LABEL FU when a
 * vertex is a no-return or when a side or the diagonal v00-v11 is longer than max_edge
 * (squared camera-frame lengths compared in FP32), else FO; faces are in row-major block
 * order. Outputs (host or device): vertices Ws*Hs*3 float; faces and labels with room for
 * 2*(Ws-1)*(Hs-1) triangles; *n_faces (host or device) the count. The result feeds
 * rm_map_create. Host outputs are complete on return; with device outputs and a device pose
 * the call does not wait for the GPU. A host pose must be finite (RM_EINVAL); a device pose
 * is not checked. Errors: RM_EINVAL (arguments, as rm_cost for the intrinsics; step
 * 1..64), RM_ENOMEM, RM_ECUDA. */
rm_status rm_meshify(const rm_scan *scan, const double *pose, const rm_meshify_params *params,
                     float *vertices, int32_t *faces, uint8_t *labels, int64_t *n_faces,
                     void *stream);

/* Per-kernel timing, recorded with CUDA events on the launch stream around every kernel
 * the map launches while enabled. rm_profile(map, 1) clears the record and starts, 0 stops.
 * rm_profile_read waits for the recorded events and fills up to `cap` entries (one per
 * kernel kind: k_cull, k_setup, k_raster, k_reduce), *n with the count, and
 * *launches (optional) with the number of kernels launched since recording started. */
typedef struct {
  char name[48];
  int64_t launches;
  double total_ms;
} rm_kernel_time;
rm_status rm_profile(rm_map *map, int32_t enable);
rm_status rm_profile_read(rm_map *map, rm_kernel_time *out, int32_t cap, int32_t *n,
                          int64_t *launches);

/* One problem of a heterogeneous batch: its own scan (camera model, size and arrays, host or
 * device) and a pose (16 doubles, host or device): the pose evaluated by rm_cost_grad_batch,
 * the start pose of rm_align_batch. */
typedef struct {
  rm_scan scan;
  const double *pose;
} rm_problem;

/* rm_cost_grad for n problems that may differ in camera model, resolution and scan, in ONE
 * persistent kernel: CTAs take (problem, phase, index) items from device ready queues; an item
 * enters a queue only when its problem's previous phase has completed (cluster culling ->
 * triangle setup -> tile raster -> reduction per problem), the number of setup items follows
 * the visible clusters, and raster/reduction items are served first. Every wait is bounded
 * (RM_ETIMEOUT). Outputs as for rm_cost_grad, per problem
 * (index k = problem). Screen tiles are 64x32 for pinhole problems and 16x16 for ray-table
 * problems, the per-call entry points' defaults, so a problem's results equal those of
 * rm_cost_grad with default tiles bit for bit. (Sec. IV.C / Sec. VI: many evaluations per
 * scan match; batching them is this library's extension.) */
rm_status rm_cost_grad_batch(rm_map *map, const rm_problem *problems, int32_t n,
                             const rm_cost_params *params, const rm_cost_out *out, void *stream);

/* rm_align for n problems at once: every LM iteration of every problem runs inside one
 * persistent-kernel launch (each problem's next evaluation waits for its own LM step), so a
 * whole tracking frame of mixed sensors is one launch. poses_out: n*16 doubles (host or
 * device); reports: n entries (optional, host). Returns RM_ENOTCONV if any problem stopped at
 * max_iters (its pose is still written). */
rm_status rm_align_batch(rm_map *map, const rm_problem *problems, int32_t n,
                         const rm_cost_params *params, const rm_align_params *lm,
                         double *poses_out, rm_align_report *reports, void *stream);

/* rm_icp_align for a batch of problems (each its own scan and start pose; pinhole and
 * ray-table problems mixed), every evaluation and step of every problem in one persistent
 * kernel (as rm_align_batch): params->max_iters evaluations per problem (1..100000), each
 * followed by its Gauss-Newton step on the device. poses_out: n*16 doubles (host or device);
 * reps: n reports (optional, host). Returns RM_ENOTCONV when a problem did not converge. */
rm_status rm_icp_align_batch(rm_map *map, const rm_problem *problems, int32_t n,
                             const rm_icp_params *params, double *poses_out, rm_icp_report *reps,
                             void *stream);

/* Cost and gradient of ONE pose without allocating (the paper has no counterpart; this is a
 * deployment variant of rm_cost_grad). For callers that must not allocate device memory
 * while they evaluate poses -- a real-time loop that may not call into the allocator after
 * start-up (an allocation can synchronise the device and has unbounded latency), code under
 * a memory manager that owns the whole device, or a fixed memory budget. All scratch (pose
 * matrix, visible-cluster list, screen-tile bins, per-tile partial sums, status word) comes
 * from one array of RM_NOALLOC_SCRATCH_BYTES in device global memory that belongs to the
 * library: every GPU that loads the library holds it until the process exits.
 *  - map: created earlier with rm_map_create (read only here) on the device that is current
 *    for this call (the call does not switch devices); its tile size is used, and the bin
 *    capacity is whatever fits in the array (at most 4096 records per tile).
 *  - scan: depth and cls in DEVICE memory of that device; pose: 16 doubles, host or device.
 *  - out: DEVICE pointers of that device (any may be NULL), one pose's values as for
 *    rm_cost_grad.
 * The call waits for `stream` to read its status. The first call on each device looks up
 * the array's device address (cudaGetSymbolAddress, with that device current). Every call
 * shares the one array and leaves its contents behind; the call clears what must start at
 * zero. Calls whose GPU work overlaps
 * (other streams, unordered threads) race on the array and give wrong results.
 * Errors: RM_EINVAL when the map, the scan or an output is not on the current device (host
 * scan/output pointers included), or when the cluster list and tile arrays
 * leave room for fewer than 256 records per tile; RM_EOVERFLOW when a tile's bin overflows
 * (no growth is possible); RM_ECUDA, RM_ETIMEOUT as elsewhere. */
#define RM_NOALLOC_SCRATCH_BYTES (48u << 20)
rm_status rm_cost_grad_noalloc(const rm_map *map, const rm_scan *scan, const double *pose,
                               const rm_cost_params *params, const rm_cost_out *out,
                               void *stream);

/* Reads and clears the map's device status word after work queued with async_status = 1;
 * returns RM_OK, RM_EOVERFLOW or RM_ETIMEOUT. */
rm_status rm_status_sync(rm_map *map, void *stream);

/* Message for the calling thread's last non-RM_OK status ("" if none). */
const char *rm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* RENDERMAP_H */
