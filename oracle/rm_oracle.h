/*
 * rm_oracle.h -- CPU oracle for the RenderMap pose-cost path (Ryde & Ding, arXiv 1702.06813).
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg may call this library. It shares no code, header, table or constant with the CUDA
 * library; both are written from the paper and from the same written arithmetic contract
 * for the z-buffer (the FP32 steps that decide which triangle a pixel sees).
 *
 * Every pointer is host memory. Layouts are dense, row major, C order.
 */
#ifndef RM_ORACLE_H
#define RM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Camera. model 0: pinhole, ray of pixel (i,j) = ((i+.5-cx)/fx, (j+.5-cy)/fy, 1), depth is z.
 * model 1: ray table, `rays` holds H*W*3 float32 unit rays (camera frame), depth is range;
 * az0/az_step/el0/el_step describe the table's layout (column i at azimuth az0+az_step*(i+.5),
 * row j at elevation el0-el_step*j) and only serve to bound the pixels a triangle can cover. */
typedef struct {
  int32_t model, width, height, pad_;
  float fx, fy, cx, cy;
  float az0, az_step, el0, el_step;
  float near_m, far_m;
  const float *rays;
} orc_cam;

typedef struct {
  float eps;                 /* Table I inlier threshold (0.1 m) */
  float w_fofo, w_fofu, w_fufo; /* per-cell weights of the least-squares surrogate */
} orc_params;

typedef struct {
  int64_t n_clipped;         /* triangles cut by the near plane */
  int64_t n_guard_culled;    /* triangles dropped: a vertex projects beyond the guard band */
  int64_t n_fragments;       /* covered (triangle, pixel) pairs before the depth test */
} orc_stats;

/* Map preparation: centre = midpoint of the FP64 bounding box of the FP32 vertices,
 * out = float(v - centre). */
void orc_recentre(const float *v, int64_t V, double centre[3], float *out);

/* World-to-camera FP32 3x4 matrix from a camera-to-world FP64 pose and the map centre. */
void orc_pose_matrix(const double Twc[16], const double centre[3], float M[12]);

/* Camera-space FP32 vertices: vc = M * [v;1] in the contract's operation order. */
void orc_transform(const float M[12], const float *v, int64_t V, float *vc);

/* Z-buffer of camera-space geometry. keys: H*W uint64 (~bits(w) << 32 | tri id) with w the
 * FP32 inverse depth (depth = 1/w), 0xFFFF..FF where nothing is hit. frags (optional): per-pixel count of covering triangles
 * before the depth test. brute != 0 tests every pixel against every triangle. */
int orc_zbuffer(const float *vc, const int32_t *faces, int64_t T, const orc_cam *cam,
                uint64_t *keys, int32_t *frags, int brute, orc_stats *st);

/* Full render from a pose: recentred vertices + centre + pose -> keys. */
int orc_render(const float *vr, int64_t V, const double centre[3], const int32_t *faces,
               int64_t T, const double Twc[16], const orc_cam *cam, uint64_t *keys,
               int32_t *frags, int brute, orc_stats *st);

/* FP64 ray-plane depth of every pixel's winner, from the ORIGINAL vertices and the FP64
 * pose; NaN where keys holds no hit. */
void orc_depth_exact(const float *v, const int32_t *faces, const double Twc[16],
                     const orc_cam *cam, const uint64_t *keys, double *depth);

/* Barycentrics (b1, b2) of the ray-plane hit on the winner, FP64; NaN where no hit. */
void orc_barycentrics(const float *v, const int32_t *faces, const double Twc[16],
                      const orc_cam *cam, const uint64_t *keys, double *bary);

/* Table I outcome of one pixel: returns -1 ignore, else 0..5 =
 * {FO/FO reward, FO/FO penalty, FO/FU reward, FO/FU penalty, FU/FO reward, FU/FO penalty}.
 * map_class 0 FO, 1 FU, 2 UO, 3 NaN; scan_class 0 FO, 1 FU, 2 NaN. */
int orc_table1(int map_class, int scan_class, float dz, float eps);

/* Cost of one pose. counts[6] per outcome; e_ls = 1/2 sum w r^2; grad[6] = sum w r J;
 * jtj[21] = upper triangle (row major) of sum w J J^T. Twist xi = (rho, phi), right
 * perturbation T <- T exp(xi^). outcome (optional, H*W int8) per-pixel outcome code;
 * resid (optional, H*W double) per-pixel residual. residual_exact != 0 takes residuals from
 * the FP64 depth instead of the z-buffer's FP32 depth. */
int orc_cost(const float *v, const float *vr, int64_t V, const double centre[3],
             const int32_t *faces, const uint8_t *labels, int64_t T, const double Twc[16],
             const orc_cam *cam, const float *scan_depth, const uint8_t *scan_class,
             const orc_params *prm, int residual_exact, int64_t counts[6], double *e_ls,
             double grad[6], double jtj[21], int8_t *outcome, double *resid);

/* Frozen-visibility cost: the z-buffer winners and residual cells of pose Twc, with every
 * winner's plane re-intersected in FP64 at pose Twc * exp(xi^). */
double orc_cost_frozen(const float *v, const float *vr, int64_t V, const double centre[3],
                       const int32_t *faces, const uint8_t *labels, int64_t T,
                       const double Twc[16], const orc_cam *cam, const float *scan_depth,
                       const uint8_t *scan_class, const orc_params *prm, const double xi[6]);

/* SE(3) exponential, out = Twc * exp(xi^). */
void orc_se3_right(const double Twc[16], const double xi[6], double out[16]);

/* Levenberg-Marquardt on the least-squares surrogate (FP64, Cholesky 6x6). */
typedef struct {
  int32_t max_iters; int32_t pad_;
  double lambda0, lambda_up, lambda_down, step_tol;
} orc_lm;
typedef struct {
  int32_t iters, accepted, converged, pad_;
  double e_ls_initial, e_ls_final;
  int64_t e_table_initial, e_table_final;
} orc_lm_report;
int orc_align(const float *v, const float *vr, int64_t V, const double centre[3],
              const int32_t *faces, const uint8_t *labels, int64_t T, const double Twc0[16],
              const orc_cam *cam, const float *scan_depth, const uint8_t *scan_class,
              const orc_params *prm, const orc_lm *lm, double Twc_out[16],
              orc_lm_report *rep);

/* Cost of N poses (OpenMP over poses when built with it): e_ls[N], counts[N*6], grad[N*6],
 * jtj[N*21]. Returns the number of threads used. */
int orc_cost_batch(const float *v, const float *vr, int64_t V, const double centre[3],
                   const int32_t *faces, const uint8_t *labels, int64_t T, const double *Twc,
                   int N, const orc_cam *cam, const float *scan_depth,
                   const uint8_t *scan_class, const orc_params *prm, int64_t *counts,
                   double *e_ls, double *grad, double *jtj);

/* Render-accelerated point-to-plane ICP (Sec. V). One iteration's terms at pose Twc: a pixel
 * is associated when the map surface it sees is FO, the scan pixel is an FO return and
 * |Z_M - Z_1| < tol (FP32 z-buffer depth, FP32 difference; Sec. V's z-difference test). With
 * the scan point p = d r, the map point q = t r on the same ray and the map surface's unit
 * camera-frame normal n, the residual is e = (p - q) . n and its Jacobian w.r.t. the right-
 * perturbation twist (rho, phi) of Twc is J = (n, p x n). n_assoc counts the associations,
 * cost_l1 = sum |Z_M - Z_1| over them (the paper's C), e2 = sum e^2, jte = sum J e,
 * jtj = upper triangle of sum J J^T.
 * vnormals (V*3 world-frame vectors, or NULL): when given, n is not the face plane's normal
 * but the map's points coloured by their normals (Sec. V, sequential alignment step 3): the
 * three vertex normals of the seen triangle blended by the hit's barycentrics, rotated into
 * the camera frame and normalised; a pixel whose blend is not finite (a vertex without a
 * normal, NaN) is not associated. */
int orc_icp_terms(const float *v, const float *vr, int64_t V, const double centre[3],
                  const int32_t *faces, const uint8_t *labels, const double *vnormals, int64_t T,
                  const double Twc[16], const orc_cam *cam, const float *scan_depth,
                  const uint8_t *scan_class, float tol, int64_t *n_assoc, double *cost_l1,
                  double *e2, double jte[6], double jtj[21]);

/* 1/2 sum e^2 with the associations, map points and normals of pose Twc frozen and the scan
 * points moved by exp(xi^) in its camera frame (for finite-difference checks of jte). */
double orc_icp_frozen(const float *v, const float *vr, int64_t V, const double centre[3],
                      const int32_t *faces, const uint8_t *labels, const double *vnormals,
                      int64_t T, const double Twc[16], const orc_cam *cam,
                      const float *scan_depth, const uint8_t *scan_class, float tol,
                      const double xi[6]);

/* ICP iterations: re-render and re-associate, solve J^T J dx = -J^T e (Cholesky), Twc <-
 * Twc exp(dx^), until |dx| < step_tol (converged = 1) or max_iters iterations. */
int orc_icp_align(const float *v, const float *vr, int64_t V, const double centre[3],
                  const int32_t *faces, const uint8_t *labels, const double *vnormals, int64_t T,
                  const double Twc0[16], const orc_cam *cam, const float *scan_depth,
                  const uint8_t *scan_class, float tol, int max_iters, double step_tol,
                  double Twc_out[16], int *iters, int *converged, int64_t *n_assoc,
                  double *cost_l1);

/* Surface normals of a depth image (Eq. 2, Sec. V). A pixel is valid when its class is FO
 * (0) and its depth finite. The valid depths are smoothed with a Gaussian of standard
 * deviation sigma pixels (0 <= sigma <= 5; radius ceil(3 sigma); weights renormalised over
 * the valid pixels in the window; invalid pixels stay invalid), then differentiated by central
 * differences across (x) and down (y): dz/dx = (S(x+1) - S(x-1)) / 2 and likewise in y. The
 * normal is N = a x b with a = (0, s_y, dz/dy) and b = (s_x, 0, dz/dx), normalised, where
 * s = 1 (pixel units, metric = 0; then N ~ (dz/dx, dz/dy, -1)) or the pixel's footprint at
 * its depth s_x = S/fx, s_y = S/fy (metric = 1). Border pixels and pixels with an invalid
 * 4-neighbour get NaN. normals: H*W*3; smoothed (optional): H*W. Returns -1 on a bad sigma. */
int orc_depth_normals(const float *depth, const uint8_t *cls, int W, int H, double sigma,
                      int metric, double fx, double fy, double *normals, double *smoothed);

/* Meshification of a range image (Sec. IV.A, Fig. 5). The grid takes every step-th pixel
 * across and down (step 2 = the factor-2 downsampling of Sec. V). Each grid pixel is a
 * vertex at its range along its ray, transformed to the world by Twc: returns (FO) at their
 * depth, no-return pixels (FU) at max_range; dead pixels (scan class NaN) are parked at the
 * sensor origin and unreferenced. Each 2x2 block of adjacent grid vertices with no dead pixel
 * gives two triangles (v00, v10, v11) and (v00, v11, v01), labelled FU when a vertex is a
 * no-return or a side or the diagonal is longer than max_edge (squared lengths compared in
 * FP32 in the camera frame), else FO. Faces come in row-major block order. vertices: Hs*Ws*3
 * with Ws = (W-1)/step + 1; faces: capacity 2*(Hs-1)*(Ws-1)*3; labels likewise. */
int orc_meshify(const orc_cam *cam, const float *depth, const uint8_t *cls, const double Twc[16],
                float max_range, float max_edge, int step, float *vertices, int32_t *faces,
                uint8_t *labels, int64_t *n_faces);

/* Derivative-free search (Sec. IV.C): Nelder-Mead iterations, then coordinate descent once
 * near the minimum. The search runs over twists xi (rho in metres, phi in radians) scaled
 * per axis by `scale`; each step evaluates its candidates as one batch.
 *  - Simplex: the origin and nm_step * scale_k along each axis k. Per iteration the vertices
 *    are ordered by value (ties by slot), c is the mean of the best six (summed in that
 *    order, divided by 6), and four candidates c + d, c + 2d, c + d/2, c - d/2 with
 *    d = c - x_worst are evaluated together; the usual rules pick one (reflect: f_r below
 *    the second worst; expand: f_e < f_r < f_best; outside contraction: f_oc <= f_r < f_worst;
 *    inside contraction: f_ic < f_worst <= f_r) or shrink every vertex halfway toward the
 *    best (a batch of six). Ends after nm_iters iterations or when every vertex lies within
 *    nm_tol (scaled, per axis) of the best.
 *  - Or, with method 1, Powell's conjugate-direction search in place of Nelder-Mead (the
 *    paper names it beside Nelder-Mead; settings are not given, these are this oracle's):
 *    directions start as scale_k e_k (unit scaled length), and the origin is evaluated
 *    alone. A line search along d from x is one batch of the 12 points x + (a s) d,
 *    a = +1/4, -1/4, +1/2, -1/2, +1, -1, +2, -2, +4, -4, +8, -8 (products and sums rounded
 *    separately); the lowest (ties: the first) is taken if it is below f(x). An iteration
 *    searches along the six directions in turn (s = the current step), then, if x moved, along
 *    the displacement d = x - x0 of the iteration with s = 1, and replaces the direction
 *    whose search lowered the value most by d divided by its scaled length
 *    sqrt(sum_k (d_k / scale_k)^2). An iteration in which x did not move halves s. Ends after
 *    powell_iters iterations or once s < powell_tol.
 *  - Coordinate descent from the best vertex with steps cd_step * scale: the 12 moves +-step
 *    along each axis as one batch; the lowest (ties: the first, +axis0, -axis0, +axis1, ...)
 *    is taken if it is below the current value, else every step is halved. Converged when the
 *    largest scaled step is below cd_tol; ends after cd_iters iterations otherwise. */
typedef int (*orc_batch_fn)(void *ctx, int n, const double *xi, double *f);

typedef struct {
  int32_t nm_iters, cd_iters;
  double nm_step, nm_tol, cd_step, cd_tol;
  double scale_t, scale_r;   /* metres and radians per unit of the scaled twist */
  int32_t method;            /* 0: Nelder-Mead, 1: Powell's method; then coordinate descent */
  int32_t powell_iters;
  double powell_step, powell_tol;
} orc_dfo_params;

typedef struct {
  int32_t evals, nm_iters, nm_shrinks, cd_iters, converged, powell_iters;
} orc_dfo_report;

int orc_dfo_core(orc_batch_fn fn, void *ctx, const double scale[6], const orc_dfo_params *p,
                 double x_out[6], double *f_out, orc_dfo_report *rep);

/* The search above on f(xi) = E_table(Twc0 exp(xi^)), the Table I cost (integer valued). */
int orc_dfo_align(const float *v, const float *vr, int64_t V, const double centre[3],
                  const int32_t *faces, const uint8_t *labels, int64_t T, const double Twc0[16],
                  const orc_cam *cam, const float *scan_depth, const uint8_t *scan_class,
                  const orc_params *prm, const orc_dfo_params *p, double Twc_out[16],
                  int64_t *e_table, orc_dfo_report *rep);

/* Depth and class of each pixel of a raw range image (Sec. IV.A, IV.B): NaN, or a return
 * closer than range_min (and above 0), is dead (NaN class, NaN depth); no reading (<= 0,
 * above range_max, +inf) is free space up to the maximal range (FU, depth range_max); the rest
 * are returns (FO, their range). */
void orc_scan_from_range(const float *range, int64_t n, float range_min, float range_max,
                         float *depth, uint8_t *cls);

/* Camera-to-world pose from the paper's X = (x, y, z, theta_x, theta_y, theta_z) (Eq. 1),
 * read as R = Rz(theta_z) Ry(theta_y) Rx(theta_x) and translation (x, y, z). */
void orc_pose_from_x(const double X[6], double T[16]);

/* Gradient of e_ls w.r.t. the world positions of the map's vertices at pose Twc (V*3, map
 * refinement): each active pixel adds w r sgn b_m n_w / (n_c . r) to the vertices m of its
 * winning triangle, with b_m the barycentrics of the FP64 hit point. The residual r is the
 * cost's (FP32 z-buffer depth), the geometry FP64. */
int orc_cost_vertex_grad(const float *v, const float *vr, int64_t V, const double centre[3],
                         const int32_t *faces, const uint8_t *labels, int64_t T,
                         const double Twc[16], const orc_cam *cam, const float *scan_depth,
                         const uint8_t *scan_class, const orc_params *prm, double *gV);

/* The frozen-cell e_ls of pose Twc (winners, cells and activity of the unmoved map) with
 * vertex vk moved by delta (world) and the depths re-intersected in FP64. */
double orc_cost_frozen_vertex(const float *v, const float *vr, int64_t V, const double centre[3],
                              const int32_t *faces, const uint8_t *labels, int64_t T,
                              const double Twc[16], const orc_cam *cam, const float *scan_depth,
                              const uint8_t *scan_class, const orc_params *prm, int64_t vk,
                              const double delta[3]);

#ifdef __cplusplus
}
#endif
#endif
