/*
 * rm_oracle.c -- CPU oracle for the RenderMap pose-cost path (Ryde & Ding, arXiv 1702.06813).
 *
 * TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU-baseline leg
 * are its only callers. It is deliberately plain and slow: one loop per step, no blocking,
 * no fusion. It shares no code with the CUDA library.
 *
 * What it computes, and where the paper defines it:
 *  - Sec. IV.A: the map is a triangle mesh of the interfaces between free, occupied and
 *    unknown space, each face labelled FO / FU / UO; it is rendered into a z-buffer image.
 *  - Eq. 1: E(X) = C(R(T(X)), Z_s), R(Y) the z-buffer rendered from camera pose Y.
 *  - Table I: the per-pixel reward / penalty from the map class, the scan class and
 *    dz = d(p_r) - d(p_s) with the inlier threshold eps = 0.1 m; the cost is the sum over
 *    all pixels (Sec. IV.B).
 *  - Sec. IV.C names derivative-based and derivative-free optimisers; this oracle adds the
 *    least-squares surrogate whose Levenberg-Marquardt step the library runs (a reading, not
 *    the paper's own optimiser), with the pose derivative of the ray-plane depth, and the
 *    paper's own derivative-free search (Nelder-Mead or Powell's method, then coordinate
 *    descent) on Table I.
 *  - Sec. V: render-accelerated point-to-plane ICP (projective association with a depth
 *    tolerance, point-to-plane residual and its 6x6 normal equations), with the map's face
 *    normals or its vertex normals blended by the hit's barycentrics, and the depth-image
 *    normals of Eq. 2.
 *  - Sec. IV.A / Fig. 5: meshification of a range image into FO / FU quads; Sec. IV.A-B:
 *    the classes of raw range readings; Eq. 1: the pose of the vector X.
 *  - Map refinement: the surrogate's gradient with respect to the vertex positions.
 * Every function is pinned by tests against closed forms, invariants, brute force or finite
 * differences (see the tests named in oracle/__init__.py); no function is unpinned.
 *
 * The z-buffer follows a written FP32 arithmetic contract so that the CPU and the GPU pick
 * the same triangle for every pixel: fixed operation order, IEEE add / mul / div / fma,
 * round-to-nearest-even. Build with -ffp-contract=off so that the compiler fuses nothing.
 */
#include "rm_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define KEY_EMPTY 0xFFFFFFFFFFFFFFFFull
#define GUARD_PX 2097152.0f /* 2^21 pixels: snapped coordinates stay below 2^29 */

/* ------------------------------------------------------------------------------------- */
/* map preparation and pose                                                              */
/* ------------------------------------------------------------------------------------- */

void orc_recentre(const float *v, int64_t V, double centre[3], float *out) {
  for (int a = 0; a < 3; ++a) {
    double lo = INFINITY, hi = -INFINITY;
    for (int64_t k = 0; k < V; ++k) {
      double x = (double)v[3 * k + a];
      if (x < lo) lo = x;
      if (x > hi) hi = x;
    }
    centre[a] = V > 0 ? 0.5 * (lo + hi) : 0.0;
  }
  for (int64_t k = 0; k < V; ++k)
    for (int a = 0; a < 3; ++a) out[3 * k + a] = (float)((double)v[3 * k + a] - centre[a]);
}

/* Eq. 1's T(X) maps the observer pose to the camera pose; here the caller passes the camera
 * pose directly. M = inverse of (R, t - centre): rotation R^T, translation -R^T (t - c). */
void orc_pose_matrix(const double T[16], const double c[3], float M[12]) {
  double t0 = T[3] - c[0], t1 = T[7] - c[1], t2 = T[11] - c[2];
  for (int i = 0; i < 3; ++i) {
    double r0 = T[0 * 4 + i], r1 = T[1 * 4 + i], r2 = T[2 * 4 + i]; /* column i of R */
    double s = r0 * t0;
    s = s + r1 * t1;
    s = s + r2 * t2;
    M[4 * i + 0] = (float)r0;
    M[4 * i + 1] = (float)r1;
    M[4 * i + 2] = (float)r2;
    M[4 * i + 3] = (float)(-s);
  }
}

void orc_transform(const float M[12], const float *v, int64_t V, float *vc) {
  for (int64_t k = 0; k < V; ++k) {
    float x = v[3 * k], y = v[3 * k + 1], z = v[3 * k + 2];
    for (int r = 0; r < 3; ++r)
      vc[3 * k + r] = fmaf(M[4 * r], x, fmaf(M[4 * r + 1], y, fmaf(M[4 * r + 2], z, M[4 * r + 3])));
  }
}

/* ------------------------------------------------------------------------------------- */
/* the z-buffer (Sec. IV.A render; depth buffer as in Sec. IV)                          */
/* ------------------------------------------------------------------------------------- */

/* Camera-space plane n . p = d of a triangle, and its inverse depth w = 1/t folded per pixel:
 * pinhole w(px, py) = Ai px + Bi py + Ci (affine in the image, as a GPU z-buffer value is, Sec.
 * IV), ray table w(r) = ni . r. */
typedef struct { float nx, ny, nz, d, Ai, Bi, Ci, nix, niy, niz; } plane32;

/* Camera-space plane of a triangle from its stored vertex order. */
static void plane_of(const float *a, const float *b, const float *c, const orc_cam *cam,
                     plane32 *p) {
  float e1x = b[0] - a[0], e1y = b[1] - a[1], e1z = b[2] - a[2];
  float e2x = c[0] - a[0], e2y = c[1] - a[1], e2z = c[2] - a[2];
  p->nx = fmaf(e1y, e2z, -(e1z * e2y));
  p->ny = fmaf(e1z, e2x, -(e1x * e2z));
  p->nz = fmaf(e1x, e2y, -(e1y * e2x));
  p->d = fmaf(p->nx, a[0], fmaf(p->ny, a[1], p->nz * a[2]));
  if (cam->model == 0) {
    float A = p->nx / cam->fx;
    float B = p->ny / cam->fy;
    float C = fmaf(-A, cam->cx, fmaf(-B, cam->cy, p->nz));
    p->Ai = A / p->d;
    p->Bi = B / p->d;
    p->Ci = C / p->d;
    p->nix = p->niy = p->niz = 0.0f;
  } else {
    p->nix = p->nx / p->d;
    p->niy = p->ny / p->d;
    p->niz = p->nz / p->d;
    p->Ai = p->Bi = p->Ci = 0.0f;
  }
}

static float inv_depth_at(const plane32 *p, const orc_cam *cam, int i, int j) {
  if (cam->model == 0) {
    float px = (float)i + 0.5f, py = (float)j + 0.5f;
    return fmaf(p->Ai, px, fmaf(p->Bi, py, p->Ci));
  }
  const float *r = cam->rays + 3 * ((int64_t)j * cam->width + i);
  return fmaf(p->nix, r[0], fmaf(p->niy, r[1], p->niz * r[2]));
}

/* Keep a fragment iff its inverse depth lies in (0, 1/near] and >= 1/far (FP32 bounds); the
 * key orders by decreasing inverse depth (nearest first), then by triangle id. */
static void deposit(const plane32 *pl, const orc_cam *cam, int i, int j, uint32_t id,
                    uint64_t *keys, int32_t *frags, orc_stats *st) {
  int64_t pix = (int64_t)j * cam->width + i;
  if (frags) frags[pix] += 1;
  st->n_fragments += 1;
  float w = inv_depth_at(pl, cam, i, j);
  float w_near = 1.0f / cam->near_m, w_far = 1.0f / cam->far_m;
  if (w > 0.0f && w >= w_far && w <= w_near) {
    uint32_t bits;
    memcpy(&bits, &w, 4);
    uint64_t key = ((uint64_t)(~bits) << 32) | (uint64_t)id;
    if (key < keys[pix]) keys[pix] = key;
  }
}

/* Depth of a z-buffer key: t = 1 / w, rounded to FP32. */
static float key_depth(uint64_t key) {
  uint32_t bits = ~(uint32_t)(key >> 32);
  float w;
  memcpy(&w, &bits, 4);
  return 1.0f / w;
}

/* Pinhole: project and snap to 1/256 pixel, round half to even. */
static int snap(const orc_cam *cam, float X, float Y, float Z, int32_t *xi, int32_t *yi) {
  float xs = fmaf(cam->fx, X / Z, cam->cx);
  float ys = fmaf(cam->fy, Y / Z, cam->cy);
  if (!(fabsf(xs) <= GUARD_PX && fabsf(ys) <= GUARD_PX)) return 0;
  *xi = (int32_t)lrintf(xs * 256.0f);
  *yi = (int32_t)lrintf(ys * 256.0f);
  return 1;
}

/* One snapped triangle: integer edge functions, top-left fill rule, sample at pixel centres
 * (256 i + 128, 256 j + 128); single sample, no anti-aliasing (Sec. VI renders with AA off). */
static void raster_snapped(int32_t x[3], int32_t y[3], const plane32 *pl, uint32_t id,
                           const orc_cam *cam, uint64_t *keys, int32_t *frags, int brute,
                           orc_stats *st) {
  int64_t area = (int64_t)(x[1] - x[0]) * (y[2] - y[0]) - (int64_t)(y[1] - y[0]) * (x[2] - x[0]);
  if (area == 0) return;
  if (area < 0) {
    int32_t tx = x[1], ty = y[1];
    x[1] = x[2]; y[1] = y[2];
    x[2] = tx; y[2] = ty;
  }
  int64_t dx[3], dy[3], bias[3];
  for (int e = 0; e < 3; ++e) {
    int b = (e + 1) % 3;
    dx[e] = (int64_t)x[b] - x[e];
    dy[e] = (int64_t)y[b] - y[e];
    bias[e] = (dy[e] < 0 || (dy[e] == 0 && dx[e] > 0)) ? 0 : -1; /* top or left edge */
  }
  int64_t i0 = 0, i1 = cam->width - 1, j0 = 0, j1 = cam->height - 1;
  if (!brute) {
    int64_t xmin = x[0], xmax = x[0], ymin = y[0], ymax = y[0];
    for (int k = 1; k < 3; ++k) {
      if (x[k] < xmin) xmin = x[k];
      if (x[k] > xmax) xmax = x[k];
      if (y[k] < ymin) ymin = y[k];
      if (y[k] > ymax) ymax = y[k];
    }
    int64_t a0 = (xmin + 127) >> 8, a1 = (xmax - 128) >> 8;
    int64_t b0 = (ymin + 127) >> 8, b1 = (ymax - 128) >> 8;
    if (a0 > i0) i0 = a0;
    if (a1 < i1) i1 = a1;
    if (b0 > j0) j0 = b0;
    if (b1 < j1) j1 = b1;
  }
  for (int64_t j = j0; j <= j1; ++j) {
    int64_t py = 256 * j + 128;
    for (int64_t i = i0; i <= i1; ++i) {
      int64_t px = 256 * i + 128;
      int in = 1;
      for (int e = 0; e < 3 && in; ++e) {
        int64_t E = dx[e] * (py - y[e]) - dy[e] * (px - x[e]);
        if (E + bias[e] < 0) in = 0;
      }
      if (in) deposit(pl, cam, (int)i, (int)j, id, keys, frags, st);
    }
  }
}

/* Near-plane cut of edge (a, b), a being the endpoint with the lower vertex index. */
static void near_cut(const float *a, const float *b, float near_m, float *out) {
  float s = (near_m - a[2]) / (b[2] - a[2]);
  out[0] = fmaf(s, b[0] - a[0], a[0]);
  out[1] = fmaf(s, b[1] - a[1], a[1]);
  out[2] = near_m;
}

static void raster_pinhole(const float *vc, const int32_t *f, uint32_t id, const orc_cam *cam,
                           uint64_t *keys, int32_t *frags, int brute, orc_stats *st) {
  const float *v[3] = {vc + 3 * (int64_t)f[0], vc + 3 * (int64_t)f[1], vc + 3 * (int64_t)f[2]};
  plane32 pl;
  plane_of(v[0], v[1], v[2], cam, &pl);
  int in[3], nin = 0;
  for (int k = 0; k < 3; ++k) {
    in[k] = v[k][2] >= cam->near_m;
    nin += in[k];
  }
  if (nin == 0) return;
  float poly[4][3];
  int n = 0;
  if (nin == 3) {
    for (int k = 0; k < 3; ++k) memcpy(poly[n++], v[k], sizeof(float) * 3);
  } else {
    st->n_clipped += 1;
    for (int k = 0; k < 3; ++k) {
      int m = (k + 1) % 3;
      if (in[k]) memcpy(poly[n++], v[k], sizeof(float) * 3);
      if (in[k] != in[m]) {
        if (f[k] < f[m]) near_cut(v[k], v[m], cam->near_m, poly[n++]);
        else near_cut(v[m], v[k], cam->near_m, poly[n++]);
      }
    }
  }
  int32_t sx[4], sy[4];
  for (int k = 0; k < n; ++k) {
    if (!snap(cam, poly[k][0], poly[k][1], poly[k][2], &sx[k], &sy[k])) {
      st->n_guard_culled += 1;
      return;
    }
  }
  int32_t x[3] = {sx[0], sx[1], sx[2]}, y[3] = {sy[0], sy[1], sy[2]};
  raster_snapped(x, y, &pl, id, cam, keys, frags, brute, st);
  if (n == 4) {
    int32_t x2[3] = {sx[0], sx[2], sx[3]}, y2[3] = {sy[0], sy[2], sy[3]};
    raster_snapped(x2, y2, &pl, id, cam, keys, frags, brute, st);
  }
}

/* ---- ray-table (panoramic) model: coverage by cone side tests ---- */

static void cross3f(const float *p, const float *q, float *c) {
  c[0] = fmaf(p[1], q[2], -(p[2] * q[1]));
  c[1] = fmaf(p[2], q[0], -(p[0] * q[2]));
  c[2] = fmaf(p[0], q[1], -(p[1] * q[0]));
}

static float dot3f(const float *p, const float *q) {
  return fmaf(p[0], q[0], fmaf(p[1], q[1], p[2] * q[2]));
}

static double clampd(double x, double lo, double hi) { return x < lo ? lo : (x > hi ? hi : x); }

/* Pixel rectangle (columns may wrap) that can hold rays inside the triangle's cone, from the
 * table's parametric layout in FP64 with a two-pixel margin. Returns 0 if empty. */
static int sph_bounds(const float *v0, const float *v1, const float *v2, const orc_cam *cam,
                      int64_t *i0, int64_t *ni, int64_t *j0, int64_t *j1) {
  double d[3][3];
  const float *vv[3] = {v0, v1, v2};
  for (int k = 0; k < 3; ++k) {
    double n = sqrt((double)vv[k][0] * vv[k][0] + (double)vv[k][1] * vv[k][1] +
                    (double)vv[k][2] * vv[k][2]);
    if (!(n > 0)) return 0;
    for (int a = 0; a < 3; ++a) d[k][a] = vv[k][a] / n;
  }
  /* normal sides of the cone (orientation-corrected) */
  double cr[3][3], det;
  for (int k = 0; k < 3; ++k) {
    const double *p = d[k], *q = d[(k + 1) % 3];
    cr[k][0] = p[1] * q[2] - p[2] * q[1];
    cr[k][1] = p[2] * q[0] - p[0] * q[2];
    cr[k][2] = p[0] * q[1] - p[1] * q[0];
  }
  det = d[0][0] * cr[1][0] + d[0][1] * cr[1][1] + d[0][2] * cr[1][2];
  if (det == 0) return 0;
  double sg = det > 0 ? 1.0 : -1.0;
  int has_up = 1, has_dn = 1; /* up = (0,-1,0), down = (0,1,0) */
  for (int k = 0; k < 3; ++k) {
    if (-sg * cr[k][1] < -1e-9) has_up = 0;
    if (sg * cr[k][1] < -1e-9) has_dn = 0;
  }
  double el_hi = -M_PI / 2, el_lo = M_PI / 2;
  for (int k = 0; k < 3; ++k) {
    double e = asin(clampd(-d[k][1], -1, 1));
    if (e > el_hi) el_hi = e;
    if (e < el_lo) el_lo = e;
  }
  for (int k = 0; k < 3; ++k) { /* extrema of elevation along each great-circle arc */
    const double *a = d[k], *b = d[(k + 1) % 3];
    double c[3] = {cr[k][0], cr[k][1], cr[k][2]};
    double cn = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    if (!(cn > 1e-15)) continue;
    for (int a2 = 0; a2 < 3; ++a2) c[a2] /= cn;
    double up[3] = {0, -1, 0};
    double s = up[1] * c[1];
    double u[3] = {up[0] - s * c[0], up[1] - s * c[1], up[2] - s * c[2]};
    double un = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    if (!(un > 1e-15)) continue;
    for (int a2 = 0; a2 < 3; ++a2) u[a2] /= un;
    for (int sgn = -1; sgn <= 1; sgn += 2) {
      double w[3] = {sgn * u[0], sgn * u[1], sgn * u[2]};
      double aw[3] = {a[1] * w[2] - a[2] * w[1], a[2] * w[0] - a[0] * w[2], a[0] * w[1] - a[1] * w[0]};
      double wb[3] = {w[1] * b[2] - w[2] * b[1], w[2] * b[0] - w[0] * b[2], w[0] * b[1] - w[1] * b[0]};
      if (aw[0] * c[0] + aw[1] * c[1] + aw[2] * c[2] >= -1e-12 &&
          wb[0] * c[0] + wb[1] * c[1] + wb[2] * c[2] >= -1e-12) {
        double e = asin(clampd(-w[1], -1, 1));
        if (e > el_hi) el_hi = e;
        if (e < el_lo) el_lo = e;
      }
    }
  }
  if (has_up) el_hi = M_PI / 2;
  if (has_dn) el_lo = -M_PI / 2;
  double m_el = 2.0 * cam->el_step, m_az = 2.0 * cam->az_step;
  double jlo = ceil((cam->el0 - el_hi - m_el) / cam->el_step);
  double jhi = floor((cam->el0 - el_lo + m_el) / cam->el_step);
  if (jlo < 0) jlo = 0;
  if (jhi > cam->height - 1) jhi = cam->height - 1;
  if (jlo > jhi) return 0;
  *j0 = (int64_t)jlo;
  *j1 = (int64_t)jhi;
  if (has_up || has_dn) {
    *i0 = 0;
    *ni = cam->width;
    return 1;
  }
  double az[3];
  for (int k = 0; k < 3; ++k) az[k] = atan2(d[k][0], d[k][2]);
  /* smallest circular arc holding the three azimuths: drop the largest gap */
  double s0 = az[0], s1 = az[1], s2 = az[2], t;
  if (s0 > s1) { t = s0; s0 = s1; s1 = t; }
  if (s1 > s2) { t = s1; s1 = s2; s2 = t; }
  if (s0 > s1) { t = s0; s0 = s1; s1 = t; }
  double g01 = s1 - s0, g12 = s2 - s1, g20 = s0 + 2 * M_PI - s2;
  double lo, hi;
  if (g20 >= g01 && g20 >= g12) { lo = s0; hi = s2; }
  else if (g01 >= g12) { lo = s1; hi = s0 + 2 * M_PI; }
  else { lo = s2; hi = s1 + 2 * M_PI; }
  double ilo = ceil((lo - m_az - cam->az0) / cam->az_step - 0.5);
  double ihi = floor((hi + m_az - cam->az0) / cam->az_step - 0.5);
  if (ihi - ilo + 1 >= cam->width) {
    *i0 = 0;
    *ni = cam->width;
  } else {
    int64_t a = (int64_t)ilo % cam->width;
    if (a < 0) a += cam->width;
    *i0 = a;
    *ni = (int64_t)(ihi - ilo) + 1;
  }
  return 1;
}

static void raster_raytable(const float *vc, const int32_t *f, uint32_t id, const orc_cam *cam,
                            uint64_t *keys, int32_t *frags, int brute, orc_stats *st) {
  const float *v[3] = {vc + 3 * (int64_t)f[0], vc + 3 * (int64_t)f[1], vc + 3 * (int64_t)f[2]};
  plane32 pl;
  plane_of(v[0], v[1], v[2], cam, &pl);
  float c12[3];
  cross3f(v[1], v[2], c12);
  float det = dot3f(v[0], c12);
  if (det == 0.0f || det != det) return;
  float side[3][3], sig[3];
  for (int k = 0; k < 3; ++k) {
    int m = (k + 1) % 3;
    int lo = f[k] < f[m] ? k : m, hi = f[k] < f[m] ? m : k;
    cross3f(v[lo], v[hi], side[k]);
    sig[k] = (det > 0.0f ? 1.0f : -1.0f) * (lo == k ? 1.0f : -1.0f);
  }
  int64_t i0 = 0, ni = cam->width, j0 = 0, j1 = cam->height - 1;
  if (!brute && !sph_bounds(v[0], v[1], v[2], cam, &i0, &ni, &j0, &j1)) return;
  for (int64_t j = j0; j <= j1; ++j) {
    for (int64_t q = 0; q < ni; ++q) {
      int64_t i = (i0 + q) % cam->width;
      const float *r = cam->rays + 3 * (j * cam->width + i);
      int in = 1;
      for (int k = 0; k < 3 && in; ++k) {
        float s = dot3f(r, side[k]);
        if (!(sig[k] * s > 0.0f || (s == 0.0f && sig[k] > 0.0f))) in = 0;
      }
      if (in) deposit(&pl, cam, (int)i, (int)j, id, keys, frags, st);
    }
  }
}

int orc_zbuffer(const float *vc, const int32_t *faces, int64_t T, const orc_cam *cam,
                uint64_t *keys, int32_t *frags, int brute, orc_stats *st) {
  int64_t P = (int64_t)cam->width * cam->height;
  orc_stats local = {0, 0, 0};
  for (int64_t p = 0; p < P; ++p) keys[p] = KEY_EMPTY;
  if (frags) memset(frags, 0, sizeof(int32_t) * P);
  for (int64_t k = 0; k < T; ++k) {
    const int32_t *f = faces + 3 * k;
    if (cam->model == 0) raster_pinhole(vc, f, (uint32_t)k, cam, keys, frags, brute, &local);
    else raster_raytable(vc, f, (uint32_t)k, cam, keys, frags, brute, &local);
  }
  if (st) *st = local;
  return 0;
}

int orc_render(const float *vr, int64_t V, const double centre[3], const int32_t *faces,
               int64_t T, const double Twc[16], const orc_cam *cam, uint64_t *keys,
               int32_t *frags, int brute, orc_stats *st) {
  float M[12];
  orc_pose_matrix(Twc, centre, M);
  float *vc = (float *)malloc(sizeof(float) * 3 * (V > 0 ? V : 1));
  if (!vc) return -1;
  orc_transform(M, vr, V, vc);
  int rc = orc_zbuffer(vc, faces, T, cam, keys, frags, brute, st);
  free(vc);
  return rc;
}

/* ------------------------------------------------------------------------------------- */
/* FP64 geometry of the winners                                                           */
/* ------------------------------------------------------------------------------------- */

static void ray64(const orc_cam *cam, int i, int j, double r[3]) {
  if (cam->model == 0) {
    r[0] = ((double)i + 0.5 - (double)cam->cx) / (double)cam->fx;
    r[1] = ((double)j + 0.5 - (double)cam->cy) / (double)cam->fy;
    r[2] = 1.0;
  } else {
    const float *q = cam->rays + 3 * ((int64_t)j * cam->width + i);
    r[0] = q[0];
    r[1] = q[1];
    r[2] = q[2];
  }
}

/* Camera-frame plane n_c . p = d_c of triangle k in FP64 at pose T. */
static void plane64(const float *v, const int32_t *faces, int64_t k, const double T[16],
                    double n[3], double *d) {
  const float *a = v + 3 * (int64_t)faces[3 * k], *b = v + 3 * (int64_t)faces[3 * k + 1],
              *c = v + 3 * (int64_t)faces[3 * k + 2];
  double e1[3] = {(double)b[0] - a[0], (double)b[1] - a[1], (double)b[2] - a[2]};
  double e2[3] = {(double)c[0] - a[0], (double)c[1] - a[1], (double)c[2] - a[2]};
  double nw[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                  e1[0] * e2[1] - e1[1] * e2[0]};
  double q[3] = {(double)a[0] - T[3], (double)a[1] - T[7], (double)a[2] - T[11]};
  *d = nw[0] * q[0] + nw[1] * q[1] + nw[2] * q[2];
  for (int i = 0; i < 3; ++i) n[i] = T[0 * 4 + i] * nw[0] + T[1 * 4 + i] * nw[1] + T[2 * 4 + i] * nw[2];
}

void orc_depth_exact(const float *v, const int32_t *faces, const double Twc[16],
                     const orc_cam *cam, const uint64_t *keys, double *depth) {
  for (int j = 0; j < cam->height; ++j)
    for (int i = 0; i < cam->width; ++i) {
      int64_t p = (int64_t)j * cam->width + i;
      if (keys[p] == KEY_EMPTY) {
        depth[p] = NAN;
        continue;
      }
      double n[3], d, r[3];
      plane64(v, faces, (int64_t)(keys[p] & 0xFFFFFFFFu), Twc, n, &d);
      ray64(cam, i, j, r);
      depth[p] = d / (n[0] * r[0] + n[1] * r[1] + n[2] * r[2]);
    }
}

/* Barycentrics (b1, b2) of pixel (i, j)'s ray-plane hit on triangle k at pose T: the hit is
 * (1 - b1 - b2) w0 + b1 w1 + b2 w2 with w the triangle's camera-frame vertices, in face
 * order (FP64 throughout). */
static void bary_px(const float *v, const int32_t *faces, const double T[16], const orc_cam *cam,
                    int64_t k, int i, int j, double *b1, double *b2) {
  double w[3][3];
  for (int m = 0; m < 3; ++m) { /* vertices in the camera frame */
    const float *a = v + 3 * (int64_t)faces[3 * k + m];
    double q[3] = {(double)a[0] - T[3], (double)a[1] - T[7], (double)a[2] - T[11]};
    for (int c = 0; c < 3; ++c) w[m][c] = T[0 * 4 + c] * q[0] + T[1 * 4 + c] * q[1] + T[2 * 4 + c] * q[2];
  }
  double r[3];
  ray64(cam, i, j, r);
  double e1[3], e2[3], n[3];
  for (int c = 0; c < 3; ++c) {
    e1[c] = w[1][c] - w[0][c];
    e2[c] = w[2][c] - w[0][c];
  }
  n[0] = e1[1] * e2[2] - e1[2] * e2[1];
  n[1] = e1[2] * e2[0] - e1[0] * e2[2];
  n[2] = e1[0] * e2[1] - e1[1] * e2[0];
  double t = (n[0] * w[0][0] + n[1] * w[0][1] + n[2] * w[0][2]) /
             (n[0] * r[0] + n[1] * r[1] + n[2] * r[2]);
  double h[3] = {t * r[0] - w[0][0], t * r[1] - w[0][1], t * r[2] - w[0][2]};
  double nn = n[0] * n[0] + n[1] * n[1] + n[2] * n[2];
  double c1[3] = {h[1] * e2[2] - h[2] * e2[1], h[2] * e2[0] - h[0] * e2[2], h[0] * e2[1] - h[1] * e2[0]};
  double c2[3] = {e1[1] * h[2] - e1[2] * h[1], e1[2] * h[0] - e1[0] * h[2], e1[0] * h[1] - e1[1] * h[0]};
  *b1 = (c1[0] * n[0] + c1[1] * n[1] + c1[2] * n[2]) / nn;
  *b2 = (c2[0] * n[0] + c2[1] * n[1] + c2[2] * n[2]) / nn;
}

void orc_barycentrics(const float *v, const int32_t *faces, const double T[16],
                      const orc_cam *cam, const uint64_t *keys, double *bary) {
  for (int j = 0; j < cam->height; ++j)
    for (int i = 0; i < cam->width; ++i) {
      int64_t p = (int64_t)j * cam->width + i;
      if (keys[p] == KEY_EMPTY) {
        bary[2 * p] = bary[2 * p + 1] = NAN;
        continue;
      }
      bary_px(v, faces, T, cam, (int64_t)(keys[p] & 0xFFFFFFFFu), i, j, &bary[2 * p], &bary[2 * p + 1]);
    }
}

/* ------------------------------------------------------------------------------------- */
/* Table I and the least-squares surrogate                                                */
/* ------------------------------------------------------------------------------------- */

int orc_table1(int mc, int sc, float dz, float eps) {
  if (mc == 0 && sc == 0) return fabsf(dz) <= eps ? 0 : 1;
  if (mc == 0 && sc == 1) return dz > 0.0f ? 2 : 3;
  if (mc == 1 && sc == 0) return dz <= 0.0f ? 4 : 5;
  return -1; /* FU/FU, UO row, NaN row, NaN column: ignore */
}

/* Truncated-L2 residual of one pixel. On return *active says whether r varies with the pose
 * (then d r / d t = *sgn), and *w is the cell weight; 0 is returned for ignored cells. */
static double ls_residual(int outcome, float dz32, double dz, float eps, const orc_params *prm,
                          int *active, double *sgn, double *w) {
  *active = 0;
  *sgn = 0.0;
  switch (outcome) {
    case 0: /* FO/FO inlier */
      *w = prm->w_fofo;
      *active = 1;
      *sgn = 1.0;
      return dz;
    case 1: /* FO/FO outlier: truncated */
      *w = prm->w_fofo;
      return (double)eps;
    case 2: /* FO map behind the FU scan interface: consistent */
      *w = prm->w_fofu;
      return 0.0;
    case 3: /* FO map inside the scan's free space */
      *w = prm->w_fofu;
      if (-dz32 < eps) {
        *active = 1;
        *sgn = -1.0;
        return -dz;
      }
      return (double)eps;
    case 4: /* scan surface beyond the map's FU interface: consistent */
      *w = prm->w_fufo;
      return 0.0;
    case 5: /* scan surface inside the map's free space */
      *w = prm->w_fufo;
      if (dz32 < eps) {
        *active = 1;
        *sgn = 1.0;
        return dz;
      }
      return (double)eps;
    default:
      *w = 0.0;
      return 0.0;
  }
}

static int scan_class_of(const float *sd, const uint8_t *sc, int64_t p) {
  float d = sd[p];
  int c = sc[p];
  if (c > 1 || !(fabsf(d) <= FLT_MAX)) return 2;
  return c;
}

/* d t / d xi for twist xi = (rho, phi) under T <- T exp(xi^): -n/(n.r) and -t (r x n)/(n.r). */
static void depth_jacobian(const double n[3], const double r[3], double t, double J[6]) {
  double nr = n[0] * r[0] + n[1] * r[1] + n[2] * r[2];
  double rxn[3] = {r[1] * n[2] - r[2] * n[1], r[2] * n[0] - r[0] * n[2], r[0] * n[1] - r[1] * n[0]};
  for (int a = 0; a < 3; ++a) {
    J[a] = -n[a] / nr;
    J[3 + a] = -t * rxn[a] / nr;
  }
}

int orc_cost(const float *v, const float *vr, int64_t V, const double centre[3],
             const int32_t *faces, const uint8_t *labels, int64_t T, const double Twc[16],
             const orc_cam *cam, const float *scan_depth, const uint8_t *scan_class,
             const orc_params *prm, int residual_exact, int64_t counts[6], double *e_ls,
             double grad[6], double jtj[21], int8_t *outcome, double *resid) {
  int64_t P = (int64_t)cam->width * cam->height;
  uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (P > 0 ? P : 1));
  if (!keys) return -1;
  orc_render(vr, V, centre, faces, T, Twc, cam, keys, NULL, 0, NULL);
  for (int k = 0; k < 6; ++k) counts[k] = 0;
  double E = 0.0, g[6] = {0}, H[36] = {0};
  for (int j = 0; j < cam->height; ++j)
    for (int i = 0; i < cam->width; ++i) {
      int64_t p = (int64_t)j * cam->width + i;
      uint64_t key = keys[p];
      int mc = key == KEY_EMPTY ? 3 : (int)labels[key & 0xFFFFFFFFu];
      int sc = scan_class_of(scan_depth, scan_class, p);
      float t32 = key != KEY_EMPTY ? key_depth(key) : 0.0f;
      float dz32 = t32 - scan_depth[p];
      int oc = (mc == 3 || sc == 2) ? -1 : orc_table1(mc, sc, dz32, prm->eps);
      if (outcome) outcome[p] = (int8_t)oc;
      if (resid) resid[p] = 0.0;
      if (oc < 0) continue;
      counts[oc] += 1;
      double n[3], d, r[3];
      plane64(v, faces, (int64_t)(key & 0xFFFFFFFFu), Twc, n, &d);
      ray64(cam, i, j, r);
      double t64 = d / (n[0] * r[0] + n[1] * r[1] + n[2] * r[2]);
      double dz = (residual_exact ? t64 : (double)t32) - (double)scan_depth[p];
      int active;
      double sgn, w;
      double res = ls_residual(oc, dz32, dz, prm->eps, prm, &active, &sgn, &w);
      if (resid) resid[p] = res;
      E += 0.5 * w * res * res;
      if (active) {
        double J[6];
        depth_jacobian(n, r, t64, J);
        for (int a = 0; a < 6; ++a) {
          J[a] *= sgn;
          g[a] += w * res * J[a];
        }
        for (int a = 0; a < 6; ++a)
          for (int b = 0; b < 6; ++b) H[6 * a + b] += w * J[a] * J[b];
      }
    }
  free(keys);
  *e_ls = E;
  for (int a = 0; a < 6; ++a) grad[a] = g[a];
  int q = 0;
  for (int a = 0; a < 6; ++a)
    for (int b = a; b < 6; ++b) jtj[q++] = H[6 * a + b];
  return 0;
}

/* ------------------------------------------------------------------------------------- */
/* SE(3)                                                                                  */
/* ------------------------------------------------------------------------------------- */

void orc_se3_right(const double T[16], const double xi[6], double out[16]) {
  const double *rho = xi, *phi = xi + 3;
  double th2 = phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2], th = sqrt(th2);
  double A, B, C; /* sin t / t, (1 - cos t)/t^2, (t - sin t)/t^3 */
  if (th < 1e-4) {
    A = 1.0 - th2 / 6.0 + th2 * th2 / 120.0;
    B = 0.5 - th2 / 24.0 + th2 * th2 / 720.0;
    C = 1.0 / 6.0 - th2 / 120.0 + th2 * th2 / 5040.0;
  } else {
    A = sin(th) / th;
    B = (1.0 - cos(th)) / th2;
    C = (th - sin(th)) / (th2 * th);
  }
  double K[9] = {0, -phi[2], phi[1], phi[2], 0, -phi[0], -phi[1], phi[0], 0};
  double K2[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0;
      for (int k = 0; k < 3; ++k) s += K[3 * i + k] * K[3 * k + j];
      K2[3 * i + j] = s;
    }
  double R[9], Vm[9];
  for (int i = 0; i < 9; ++i) {
    double I = (i % 4 == 0) ? 1.0 : 0.0;
    R[i] = I + A * K[i] + B * K2[i];
    Vm[i] = I + B * K[i] + C * K2[i];
  }
  double t[3];
  for (int i = 0; i < 3; ++i) t[i] = Vm[3 * i] * rho[0] + Vm[3 * i + 1] * rho[1] + Vm[3 * i + 2] * rho[2];
  double E[16] = {R[0], R[1], R[2], t[0], R[3], R[4], R[5], t[1], R[6], R[7], R[8], t[2], 0, 0, 0, 1};
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double s = 0;
      for (int k = 0; k < 4; ++k) s += T[4 * i + k] * E[4 * k + j];
      out[4 * i + j] = s;
    }
}

double orc_cost_frozen(const float *v, const float *vr, int64_t V, const double centre[3],
                       const int32_t *faces, const uint8_t *labels, int64_t T,
                       const double Twc[16], const orc_cam *cam, const float *scan_depth,
                       const uint8_t *scan_class, const orc_params *prm, const double xi[6]) {
  int64_t P = (int64_t)cam->width * cam->height;
  uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (P > 0 ? P : 1));
  if (!keys) return NAN;
  orc_render(vr, V, centre, faces, T, Twc, cam, keys, NULL, 0, NULL);
  double Tp[16];
  orc_se3_right(Twc, xi, Tp);
  double E = 0.0;
  for (int j = 0; j < cam->height; ++j)
    for (int i = 0; i < cam->width; ++i) {
      int64_t p = (int64_t)j * cam->width + i;
      uint64_t key = keys[p];
      if (key == KEY_EMPTY) continue;
      int mc = (int)labels[key & 0xFFFFFFFFu];
      int sc = scan_class_of(scan_depth, scan_class, p);
      if (sc == 2) continue;
      float t32 = key_depth(key);
      float dz32 = t32 - scan_depth[p];
      int oc = orc_table1(mc, sc, dz32, prm->eps);
      if (oc < 0) continue;
      double n[3], d, r[3];
      plane64(v, faces, (int64_t)(key & 0xFFFFFFFFu), Tp, n, &d);
      ray64(cam, i, j, r);
      double dz = d / (n[0] * r[0] + n[1] * r[1] + n[2] * r[2]) - (double)scan_depth[p];
      int active;
      double sgn, w;
      /* activity is decided by the FP32 dz of the unperturbed pose: cells stay frozen */
      double res = ls_residual(oc, dz32, dz, prm->eps, prm, &active, &sgn, &w);
      E += 0.5 * w * res * res;
    }
  free(keys);
  return E;
}

/* ------------------------------------------------------------------------------------- */
/* Levenberg-Marquardt                                                                    */
/* ------------------------------------------------------------------------------------- */

/* Solve (H + lambda diag H) x = -g by Cholesky; returns 0 if not positive definite. */
static int lm_solve(const double jtj[21], const double g[6], double lambda, double x[6]) {
  double A[36], L[36] = {0};
  int q = 0;
  for (int a = 0; a < 6; ++a)
    for (int b = a; b < 6; ++b) {
      A[6 * a + b] = A[6 * b + a] = jtj[q++];
    }
  for (int a = 0; a < 6; ++a) A[7 * a] += lambda * A[7 * a];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j <= i; ++j) {
      double s = A[6 * i + j];
      for (int k = 0; k < j; ++k) s -= L[6 * i + k] * L[6 * j + k];
      if (i == j) {
        if (!(s > 0)) return 0;
        L[7 * i] = sqrt(s);
      } else {
        L[6 * i + j] = s / L[7 * j];
      }
    }
  double y[6];
  for (int i = 0; i < 6; ++i) {
    double s = -g[i];
    for (int k = 0; k < i; ++k) s -= L[6 * i + k] * y[k];
    y[i] = s / L[7 * i];
  }
  for (int i = 5; i >= 0; --i) {
    double s = y[i];
    for (int k = i + 1; k < 6; ++k) s -= L[6 * k + i] * x[k];
    x[i] = s / L[7 * i];
  }
  return 1;
}

int orc_align(const float *v, const float *vr, int64_t V, const double centre[3],
              const int32_t *faces, const uint8_t *labels, int64_t T, const double Twc0[16],
              const orc_cam *cam, const float *scan_depth, const uint8_t *scan_class,
              const orc_params *prm, const orc_lm *lm, double Twc_out[16],
              orc_lm_report *rep) {
  double Tc[16], Tn[16];
  memcpy(Tc, Twc0, sizeof(Tc));
  int64_t cnt[6], cnt_n[6];
  double E, g[6], H[21], En, gn[6], Hn[21];
  orc_cost(v, vr, V, centre, faces, labels, T, Tc, cam, scan_depth, scan_class, prm, 0, cnt, &E,
           g, H, NULL, NULL);
  memset(rep, 0, sizeof(*rep));
  rep->e_ls_initial = E;
  rep->e_table_initial = cnt[1] + cnt[3] + cnt[5] - cnt[0] - cnt[2] - cnt[4];
  double lambda = lm->lambda0;
  int it;
  for (it = 0; it < lm->max_iters; ++it) {
    double dx[6];
    if (!lm_solve(H, g, lambda, dx)) {
      lambda *= lm->lambda_up;
      continue;
    }
    double nrm = 0;
    for (int a = 0; a < 6; ++a) nrm += dx[a] * dx[a];
    if (sqrt(nrm) < lm->step_tol) {
      rep->converged = 1;
      break;
    }
    orc_se3_right(Tc, dx, Tn);
    orc_cost(v, vr, V, centre, faces, labels, T, Tn, cam, scan_depth, scan_class, prm, 0, cnt_n,
             &En, gn, Hn, NULL, NULL);
    if (En < E) {
      memcpy(Tc, Tn, sizeof(Tc));
      E = En;
      memcpy(g, gn, sizeof(g));
      memcpy(H, Hn, sizeof(H));
      memcpy(cnt, cnt_n, sizeof(cnt));
      lambda /= lm->lambda_down;
      rep->accepted += 1;
    } else {
      lambda *= lm->lambda_up;
    }
  }
  rep->iters = it;
  rep->e_ls_final = E;
  rep->e_table_final = cnt[1] + cnt[3] + cnt[5] - cnt[0] - cnt[2] - cnt[4];
  memcpy(Twc_out, Tc, sizeof(Tc));
  return 0;
}

int orc_cost_batch(const float *v, const float *vr, int64_t V, const double centre[3],
                   const int32_t *faces, const uint8_t *labels, int64_t T, const double *Twc,
                   int N, const orc_cam *cam, const float *scan_depth,
                   const uint8_t *scan_class, const orc_params *prm, int64_t *counts,
                   double *e_ls, double *grad, double *jtj) {
  int threads = 1;
#ifdef _OPENMP
#pragma omp parallel
  {
#pragma omp single
    threads = omp_get_num_threads();
  }
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int k = 0; k < N; ++k)
    orc_cost(v, vr, V, centre, faces, labels, T, Twc + 16 * k, cam, scan_depth, scan_class, prm,
             0, counts + 6 * k, e_ls + k, grad + 6 * k, jtj + 21 * k, NULL, NULL);
  return threads;
}

/* ------------------------------------------------------------------------------------- */
/* Render-accelerated point-to-plane ICP (Sec. V)                                         */
/* ------------------------------------------------------------------------------------- */

/* One ICP association at pixel p of the render at Twc: the map surface seen at the pixel
 * must be occupied (FO), the scan pixel a return (FO), and |Z_M - Z_1| below the tolerance
 * (Sec. V), decided on the FP32 z-buffer depth and the FP32 difference. On success returns
 * 1 with the unit camera-frame normal of the map surface nu, the ray r, the map depth t and
 * the scan depth d (both as FP64 from the FP32 values) and the FP32 difference. */
static int icp_pair(const float *v, const int32_t *faces, const uint8_t *labels,
                    const double *vnormals, const double Twc[16], const orc_cam *cam,
                    const float *scan_depth, const uint8_t *scan_class, float tol,
                    const uint64_t *keys, int i, int j, double nu[3], double r[3], double *t,
                    double *d, float *dz_out) {
  int64_t p = (int64_t)j * cam->width + i;
  uint64_t key = keys[p];
  if (key == KEY_EMPTY) return 0;
  int64_t id = (int64_t)(key & 0xFFFFFFFFu);
  if (labels[id] != 0) return 0;
  if (scan_class_of(scan_depth, scan_class, p) != 0) return 0;
  float t32 = key_depth(key);
  float dz32 = t32 - scan_depth[p];
  if (!(fabsf(dz32) < tol)) return 0;
  double n[3], dc;
  if (vnormals) {
    /* the map's points coloured by their normals (Sec. V, step 3): the normal seen at the
     * pixel blends the triangle's three vertex normals by the hit's barycentrics, as a
     * rasteriser interpolates a vertex attribute; a vertex without a normal (NaN) leaves the
     * pixel unassociated */
    double b1, b2, nw[3];
    bary_px(v, faces, Twc, cam, id, i, j, &b1, &b2);
    const double b[3] = {1.0 - b1 - b2, b1, b2};
    for (int c = 0; c < 3; ++c) {
      nw[c] = 0.0;
      for (int m = 0; m < 3; ++m) nw[c] += b[m] * vnormals[3 * (int64_t)faces[3 * id + m] + c];
    }
    if (!(isfinite(nw[0]) && isfinite(nw[1]) && isfinite(nw[2]))) return 0;
    for (int c = 0; c < 3; ++c) n[c] = Twc[0 * 4 + c] * nw[0] + Twc[1 * 4 + c] * nw[1] + Twc[2 * 4 + c] * nw[2];
  } else {
    plane64(v, faces, id, Twc, n, &dc);
  }
  double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  if (!(nn > 0)) return 0;
  for (int a = 0; a < 3; ++a) nu[a] = n[a] / nn;
  ray64(cam, i, j, r);
  *t = (double)t32;
  *d = (double)scan_depth[p];
  *dz_out = dz32;
  return 1;
}

int orc_icp_terms(const float *v, const float *vr, int64_t V, const double centre[3],
                  const int32_t *faces, const uint8_t *labels, const double *vnormals, int64_t T,
                  const double Twc[16], const orc_cam *cam, const float *scan_depth,
                  const uint8_t *scan_class, float tol, int64_t *n_assoc, double *cost_l1,
                  double *e2, double jte[6], double jtj[21]) {
  int64_t P = (int64_t)cam->width * cam->height;
  uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (P > 0 ? P : 1));
  if (!keys) return -1;
  orc_render(vr, V, centre, faces, T, Twc, cam, keys, NULL, 0, NULL);
  int64_t na = 0;
  double C = 0.0, E2 = 0.0, g[6] = {0}, H[36] = {0};
  for (int j = 0; j < cam->height; ++j)
    for (int i = 0; i < cam->width; ++i) {
      double nu[3], r[3], t, d;
      float dz32;
      if (!icp_pair(v, faces, labels, vnormals, Twc, cam, scan_depth, scan_class, tol, keys, i, j,
                    nu, r, &t, &d, &dz32))
        continue;
      /* scan point p = d r and map point q = t r on the same ray; residual (p - q) . nu */
      double pnt[3] = {d * r[0], d * r[1], d * r[2]};
      double e = (d - t) * (r[0] * nu[0] + r[1] * nu[1] + r[2] * nu[2]);
      /* d e / d (rho, phi) for Twc <- Twc exp(xi^): the scan point moves by rho + phi x p */
      double J[6] = {nu[0], nu[1], nu[2], pnt[1] * nu[2] - pnt[2] * nu[1],
                     pnt[2] * nu[0] - pnt[0] * nu[2], pnt[0] * nu[1] - pnt[1] * nu[0]};
      na += 1;
      C += fabs((double)dz32);
      E2 += e * e;
      for (int a = 0; a < 6; ++a) {
        g[a] += J[a] * e;
        for (int b = 0; b < 6; ++b) H[6 * a + b] += J[a] * J[b];
      }
    }
  free(keys);
  *n_assoc = na;
  *cost_l1 = C;
  *e2 = E2;
  int q = 0;
  for (int a = 0; a < 6; ++a) {
    jte[a] = g[a];
    for (int b = a; b < 6; ++b) jtj[q++] = H[6 * a + b];
  }
  return 0;
}

double orc_icp_frozen(const float *v, const float *vr, int64_t V, const double centre[3],
                      const int32_t *faces, const uint8_t *labels, const double *vnormals,
                      int64_t T, const double Twc[16], const orc_cam *cam,
                      const float *scan_depth, const uint8_t *scan_class, float tol,
                      const double xi[6]) {
  int64_t P = (int64_t)cam->width * cam->height;
  uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (P > 0 ? P : 1));
  if (!keys) return NAN;
  orc_render(vr, V, centre, faces, T, Twc, cam, keys, NULL, 0, NULL);
  static const double I[16] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1};
  double X[16];
  orc_se3_right(I, xi, X); /* exp(xi^): moves the scan points in the current camera frame */
  double E = 0.0;
  for (int j = 0; j < cam->height; ++j)
    for (int i = 0; i < cam->width; ++i) {
      double nu[3], r[3], t, d;
      float dz32;
      if (!icp_pair(v, faces, labels, vnormals, Twc, cam, scan_depth, scan_class, tol, keys, i, j,
                    nu, r, &t, &d, &dz32))
        continue;
      double p[3] = {d * r[0], d * r[1], d * r[2]}, q[3] = {t * r[0], t * r[1], t * r[2]};
      double pm[3];
      for (int a = 0; a < 3; ++a) pm[a] = X[4 * a] * p[0] + X[4 * a + 1] * p[1] + X[4 * a + 2] * p[2] + X[4 * a + 3];
      double e = (pm[0] - q[0]) * nu[0] + (pm[1] - q[1]) * nu[1] + (pm[2] - q[2]) * nu[2];
      E += 0.5 * e * e;
    }
  free(keys);
  return E;
}

int orc_icp_align(const float *v, const float *vr, int64_t V, const double centre[3],
                  const int32_t *faces, const uint8_t *labels, const double *vnormals, int64_t T,
                  const double Twc0[16], const orc_cam *cam, const float *scan_depth,
                  const uint8_t *scan_class, float tol, int max_iters, double step_tol,
                  double Twc_out[16], int *iters, int *converged, int64_t *n_assoc,
                  double *cost_l1) {
  double Tc[16], Tn[16];
  memcpy(Tc, Twc0, sizeof(Tc));
  *converged = 0;
  int it;
  int64_t na = 0;
  double C = 0.0;
  for (it = 0; it < max_iters; ++it) {
    double e2, g[6], H[21], dx[6];
    orc_icp_terms(v, vr, V, centre, faces, labels, vnormals, T, Tc, cam, scan_depth, scan_class,
                  tol, &na, &C, &e2, g, H);
    if (!lm_solve(H, g, 0.0, dx)) break; /* Gauss-Newton: J^T J dx = -J^T e */
    double nrm = 0;
    for (int a = 0; a < 6; ++a) nrm += dx[a] * dx[a];
    orc_se3_right(Tc, dx, Tn);
    memcpy(Tc, Tn, sizeof(Tc));
    if (sqrt(nrm) < step_tol) {
      *converged = 1;
      ++it;
      break;
    }
  }
  *iters = it;
  if (n_assoc) *n_assoc = na;
  if (cost_l1) *cost_l1 = C;
  memcpy(Twc_out, Tc, sizeof(Tc));
  return 0;
}

/* ------------------------------------------------------------------------------------- */
/* Depth-image surface normals (Eq. 2)                                                     */
/* ------------------------------------------------------------------------------------- */

static int depth_valid(const float *depth, const uint8_t *cls, int64_t p) {
  return cls[p] == 0 && fabsf(depth[p]) <= FLT_MAX;
}

int orc_depth_normals(const float *depth, const uint8_t *cls, int W, int H, double sigma,
                      int metric, double fx, double fy, double *normals, double *smoothed) {
  if (W < 0 || H < 0 || !(sigma >= 0.0) || sigma > 5.0) return -1;
  const int r = sigma > 0.0 ? (int)ceil(3.0 * sigma) : 0;
  double g[17];
  for (int k = 0; k <= r; ++k) g[k] = sigma > 0.0 ? exp(-(double)(k * k) / (2.0 * sigma * sigma)) : 1.0;
  const int64_t P = (int64_t)W * H;
  double *S = smoothed ? smoothed : (double *)malloc(sizeof(double) * (P > 0 ? P : 1));
  if (!S) return -1;
  /* Gaussian smoothing of the valid depths (weights renormalised over the valid ones) */
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      const int64_t p = (int64_t)y * W + x;
      if (!depth_valid(depth, cls, p)) {
        S[p] = NAN;
        continue;
      }
      double num = 0.0, den = 0.0;
      for (int dy = -r; dy <= r; ++dy)
        for (int dx = -r; dx <= r; ++dx) {
          const int xx = x + dx, yy = y + dy;
          if (xx < 0 || xx >= W || yy < 0 || yy >= H) continue;
          const int64_t q = (int64_t)yy * W + xx;
          if (!depth_valid(depth, cls, q)) continue;
          const double wgt = g[abs(dx)] * g[abs(dy)];
          num += wgt * (double)depth[q];
          den += wgt;
        }
      S[p] = num / den;
    }
  /* central differences across and down, then N = a x b with a = (0, s_y, dz/dy) and
   * b = (s_x, 0, dz/dx): s = 1 pixel, or the pixel's footprint S/f at its depth (metric) */
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      const int64_t p = (int64_t)y * W + x;
      double *n = normals + 3 * p;
      n[0] = n[1] = n[2] = NAN;
      if (x < 1 || x + 1 >= W || y < 1 || y + 1 >= H) continue;
      if (isnan(S[p]) || isnan(S[p - 1]) || isnan(S[p + 1]) || isnan(S[p - W]) || isnan(S[p + W])) continue;
      const double zx = 0.5 * (S[p + 1] - S[p - 1]);
      const double zy = 0.5 * (S[p + W] - S[p - W]);
      const double sx = metric ? S[p] / fx : 1.0, sy = metric ? S[p] / fy : 1.0;
      const double a[3] = {0.0, sy, zy}, b[3] = {sx, 0.0, zx};
      const double c[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
      const double nn = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
      for (int k = 0; k < 3; ++k) n[k] = c[k] / nn;
    }
  if (!smoothed) free(S);
  return 0;
}

/* ------------------------------------------------------------------------------------- */
/* Meshification of a range image (Sec. IV.A, Fig. 5)                                     */
/* ------------------------------------------------------------------------------------- */

/* Camera-frame point of pixel (x, y) at range d along its ray, in FP32 (the label test is an
 * integer decision taken in FP32 on both sides). */
static void mesh_point32(const orc_cam *cam, int x, int y, float d, float p[3]) {
  float rx, ry, rz;
  if (cam->model == 0) {
    rx = ((float)x + 0.5f - cam->cx) / cam->fx;
    ry = ((float)y + 0.5f - cam->cy) / cam->fy;
    rz = 1.0f;
  } else {
    const float *q = cam->rays + 3 * ((int64_t)y * cam->width + x);
    rx = q[0];
    ry = q[1];
    rz = q[2];
  }
  p[0] = d * rx;
  p[1] = d * ry;
  p[2] = d * rz;
}

static float edge2_32(const float a[3], const float b[3]) {
  float dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
  float xx = dx * dx, yy = dy * dy, zz = dz * dz;
  float s = xx + yy;
  return s + zz;
}

int orc_meshify(const orc_cam *cam, const float *depth, const uint8_t *cls, const double Twc[16],
                float max_range, float max_edge, int step, float *vertices, int32_t *faces,
                uint8_t *labels, int64_t *n_faces) {
  if (step < 1 || !(max_range > 0.0f) || !(max_edge >= 0.0f)) return -1;
  const int W = cam->width, H = cam->height;
  const int Ws = W > 0 ? (W - 1) / step + 1 : 0, Hs = H > 0 ? (H - 1) / step + 1 : 0;
  const int64_t NV = (int64_t)Ws * Hs;
  /* per grid vertex: kind 0 return (FO), 1 no return (FU, drawn at max_range), 2 dead */
  uint8_t *kind = (uint8_t *)malloc(NV > 0 ? NV : 1);
  float *pc = (float *)malloc(sizeof(float) * 3 * (NV > 0 ? NV : 1));
  if (!kind || !pc) {
    free(kind);
    free(pc);
    return -1;
  }
  for (int j = 0; j < Hs; ++j)
    for (int i = 0; i < Ws; ++i) {
      const int x = i * step, y = j * step;
      const int64_t p = (int64_t)y * W + x, v = (int64_t)j * Ws + i;
      const int c = scan_class_of(depth, cls, p);
      float d = 0.0f;
      kind[v] = (uint8_t)c;
      if (c == 0) d = depth[p];
      else if (c == 1) d = max_range;
      mesh_point32(cam, x, y, d, pc + 3 * v);
      double w[3];
      for (int a = 0; a < 3; ++a) {
        if (c == 2) {
          w[a] = Twc[4 * a + 3];  /* unreferenced: parked at the sensor origin */
        } else {
          w[a] = Twc[4 * a] * (double)pc[3 * v] + Twc[4 * a + 1] * (double)pc[3 * v + 1] +
                 Twc[4 * a + 2] * (double)pc[3 * v + 2] + Twc[4 * a + 3];
        }
        vertices[3 * v + a] = (float)w[a];
      }
    }
  const float lim = max_edge * max_edge;
  int64_t nf = 0;
  for (int j = 0; j + 1 < Hs; ++j)
    for (int i = 0; i + 1 < Ws; ++i) {
      const int64_t v00 = (int64_t)j * Ws + i, v10 = v00 + 1, v01 = v00 + Ws, v11 = v01 + 1;
      if (kind[v00] == 2 || kind[v10] == 2 || kind[v01] == 2 || kind[v11] == 2) continue;
      int fu = kind[v00] == 1 || kind[v10] == 1 || kind[v01] == 1 || kind[v11] == 1;
      const float *a = pc + 3 * v00, *b = pc + 3 * v10, *c = pc + 3 * v11, *d = pc + 3 * v01;
      if (edge2_32(a, b) > lim || edge2_32(b, c) > lim || edge2_32(c, d) > lim ||
          edge2_32(d, a) > lim || edge2_32(a, c) > lim)
        fu = 1;
      const int32_t t0[3] = {(int32_t)v00, (int32_t)v10, (int32_t)v11};
      const int32_t t1[3] = {(int32_t)v00, (int32_t)v11, (int32_t)v01};
      for (int k = 0; k < 3; ++k) {
        faces[3 * nf + k] = t0[k];
        faces[3 * nf + 3 + k] = t1[k];
      }
      labels[nf] = labels[nf + 1] = (uint8_t)(fu ? 1 : 0);
      nf += 2;
    }
  *n_faces = nf;
  free(kind);
  free(pc);
  return 0;
}

/* ------------------------------------------------------------------------------------- */
/* Derivative-free search on the Table I cost (Sec. IV.C): Nelder-Mead, then coordinate  */
/* (compass) descent near the minimum                                                      */
/* ------------------------------------------------------------------------------------- */

/* The order of simplex vertices: by value, ties by slot index. */
static void nm_order(const double f[7], int ord[7]) {
  for (int i = 0; i < 7; ++i) ord[i] = i;
  for (int i = 1; i < 7; ++i) /* insertion sort, stable */
    for (int j = i; j > 0 && f[ord[j]] < f[ord[j - 1]]; --j) {
      int t = ord[j];
      ord[j] = ord[j - 1];
      ord[j - 1] = t;
    }
}

/* Powell's line search: the 12 points x + (a s) d in the order of kPowellA, one batch; x and
 * *f move to the lowest if it is below *f. *drop = how much the value fell (0: no move). */
static const double kPowellA[12] = {0.25, -0.25, 0.5, -0.5, 1.0, -1.0, 2.0, -2.0, 4.0, -4.0, 8.0, -8.0};

static int powell_line(orc_batch_fn fn, void *ctx, double x[6], double *f, const double d[6],
                       double s, int *evals, double *drop) {
  double cand[12][6], fc[12];
  for (int m = 0; m < 12; ++m) {
    const double a = kPowellA[m] * s;
    for (int k = 0; k < 6; ++k) {
      const double step = a * d[k];
      cand[m][k] = x[k] + step;
    }
  }
  if (fn(ctx, 12, &cand[0][0], fc)) return -1;
  *evals += 12;
  int best = 0;
  for (int m = 1; m < 12; ++m)
    if (fc[m] < fc[best]) best = m;
  *drop = 0.0;
  if (fc[best] < *f) {
    *drop = *f - fc[best];
    for (int k = 0; k < 6; ++k) x[k] = cand[best][k];
    *f = fc[best];
  }
  return 0;
}

/* Powell's conjugate-direction search from the origin (see the header); x, *f: its end. */
static int powell_search(orc_batch_fn fn, void *ctx, const double scale[6], const orc_dfo_params *p,
                         double x[6], double *f, int *evals, int *iters) {
  double D[6][6];
  for (int i = 0; i < 6; ++i)
    for (int k = 0; k < 6; ++k) D[i][k] = i == k ? scale[k] : 0.0;
  for (int k = 0; k < 6; ++k) x[k] = 0.0;
  if (fn(ctx, 1, x, f)) return -1;
  *evals += 1;
  double s = p->powell_step;
  *iters = 0;
  while (*iters < p->powell_iters && s >= p->powell_tol) {
    double x0[6], best_drop = 0.0, drop;
    int best_dir = 0;
    for (int k = 0; k < 6; ++k) x0[k] = x[k];
    for (int i = 0; i < 6; ++i) {
      if (powell_line(fn, ctx, x, f, D[i], s, evals, &drop)) return -1;
      if (drop > best_drop) {
        best_drop = drop;
        best_dir = i;
      }
    }
    ++*iters;
    double d[6], n2 = 0.0;
    for (int k = 0; k < 6; ++k) {
      d[k] = x[k] - x0[k];
      const double u = d[k] / scale[k];
      n2 = n2 + u * u;
    }
    if (n2 == 0.0) {
      s = 0.5 * s;
      continue;
    }
    if (powell_line(fn, ctx, x, f, d, 1.0, evals, &drop)) return -1;
    const double n = sqrt(n2);
    for (int k = 0; k < 6; ++k) D[best_dir][k] = d[k] / n;
  }
  return 0;
}

int orc_dfo_core(orc_batch_fn fn, void *ctx, const double scale[6], const orc_dfo_params *p,
                 double x_out[6], double *f_out, orc_dfo_report *rep) {
  double x[7][6], f[7], cand[12][6], fc[12];
  int evals = 0, nm_iters = 0, shrinks = 0, cd_iters = 0, powell_iters = 0;
  if (p->method == 1) {
    /* Powell's method in place of Nelder-Mead: its end point becomes the best vertex */
    double xp[6], fp;
    if (powell_search(fn, ctx, scale, p, xp, &fp, &evals, &powell_iters)) return -1;
    for (int i = 0; i < 7; ++i) {
      for (int k = 0; k < 6; ++k) x[i][k] = xp[k];
      f[i] = fp;
    }
  } else {
    /* initial simplex: the origin and one step along each axis */
    for (int i = 0; i < 7; ++i)
      for (int k = 0; k < 6; ++k) x[i][k] = (i >= 1 && k == i - 1) ? p->nm_step * scale[k] : 0.0;
    if (fn(ctx, 7, &x[0][0], f)) return -1;
    evals += 7;
    while (nm_iters < p->nm_iters) {
      int o[7];
      nm_order(f, o);
      /* stop when every vertex is within nm_tol (in units of scale) of the best */
      double diam = 0.0;
      for (int i = 1; i < 7; ++i)
        for (int k = 0; k < 6; ++k) {
          double d = fabs(x[o[i]][k] - x[o[0]][k]) / scale[k];
          if (d > diam) diam = d;
        }
      if (diam < p->nm_tol) break;
      const int h = o[6];
      double c[6];
      for (int k = 0; k < 6; ++k) {
        double s = 0.0;
        for (int i = 0; i < 6; ++i) s += x[o[i]][k];
        c[k] = s / 6.0;
      }
      /* reflection, expansion, outside and inside contraction, evaluated together */
      for (int k = 0; k < 6; ++k) {
        double dk = c[k] - x[h][k];
        cand[0][k] = c[k] + dk;
        cand[1][k] = c[k] + 2.0 * dk;
        cand[2][k] = c[k] + 0.5 * dk;
        cand[3][k] = c[k] - 0.5 * dk;
      }
      if (fn(ctx, 4, &cand[0][0], fc)) return -1;
      evals += 4;
      ++nm_iters;
      const double fb = f[o[0]], fs = f[o[5]], fh = f[h];
      int take = -1;
      if (fc[0] < fb) take = fc[1] < fc[0] ? 1 : 0;
      else if (fc[0] < fs) take = 0;
      else if (fc[0] < fh) take = fc[2] <= fc[0] ? 2 : -1;
      else take = fc[3] < fh ? 3 : -1;
      if (take >= 0) {
        for (int k = 0; k < 6; ++k) x[h][k] = cand[take][k];
        f[h] = fc[take];
      } else {
        /* shrink toward the best vertex */
        const int b = o[0];
        int m = 0;
        for (int i = 0; i < 7; ++i) {
          if (i == b) continue;
          for (int k = 0; k < 6; ++k) cand[m][k] = x[b][k] + 0.5 * (x[i][k] - x[b][k]);
          ++m;
        }
        if (fn(ctx, 6, &cand[0][0], fc)) return -1;
        evals += 6;
        ++shrinks;
        m = 0;
        for (int i = 0; i < 7; ++i) {
          if (i == b) continue;
          for (int k = 0; k < 6; ++k) x[i][k] = cand[m][k];
          f[i] = fc[m];
          ++m;
        }
      }
    }
  }
  int o[7];
  nm_order(f, o);
  double xc[6], fcur = f[o[0]], st[6];
  for (int k = 0; k < 6; ++k) {
    xc[k] = x[o[0]][k];
    st[k] = p->cd_step * scale[k];
  }
  /* coordinate descent: the best of the 12 moves +-step along each axis, else halve */
  int converged = 0;
  while (cd_iters < p->cd_iters) {
    double smax = 0.0;
    for (int k = 0; k < 6; ++k)
      if (st[k] / scale[k] > smax) smax = st[k] / scale[k];
    if (smax < p->cd_tol) {
      converged = 1;
      break;
    }
    for (int a = 0; a < 12; ++a)
      for (int k = 0; k < 6; ++k) cand[a][k] = xc[k] + (k == a / 2 ? (a % 2 ? -st[k] : st[k]) : 0.0);
    if (fn(ctx, 12, &cand[0][0], fc)) return -1;
    evals += 12;
    ++cd_iters;
    int best = 0;
    for (int a = 1; a < 12; ++a)
      if (fc[a] < fc[best]) best = a;
    if (fc[best] < fcur) {
      for (int k = 0; k < 6; ++k) xc[k] = cand[best][k];
      fcur = fc[best];
    } else {
      for (int k = 0; k < 6; ++k) st[k] *= 0.5;
    }
  }
  for (int k = 0; k < 6; ++k) x_out[k] = xc[k];
  *f_out = fcur;
  if (rep) {
    rep->evals = evals;
    rep->nm_iters = nm_iters;
    rep->nm_shrinks = shrinks;
    rep->cd_iters = cd_iters;
    rep->converged = converged;
    rep->powell_iters = powell_iters;
  }
  return 0;
}

/* The Table I cost of T0 exp(xi^) for a batch of twists. */
typedef struct {
  const float *v, *vr;
  int64_t V, T;
  const double *centre, *T0;
  const int32_t *faces;
  const uint8_t *labels;
  const orc_cam *cam;
  const float *sd;
  const uint8_t *sc;
  const orc_params *prm;
} etable_ctx;

static int etable_batch(void *vctx, int n, const double *xi, double *f) {
  etable_ctx *c = (etable_ctx *)vctx;
  for (int i = 0; i < n; ++i) {
    double T[16], g[6], h[21], e;
    int64_t counts[6];
    orc_se3_right(c->T0, xi + 6 * i, T);
    if (orc_cost(c->v, c->vr, c->V, c->centre, c->faces, c->labels, c->T, T, c->cam, c->sd, c->sc,
                 c->prm, 0, counts, &e, g, h, NULL, NULL))
      return -1;
    f[i] = (double)((counts[1] + counts[3] + counts[5]) - (counts[0] + counts[2] + counts[4]));
  }
  return 0;
}

int orc_dfo_align(const float *v, const float *vr, int64_t V, const double centre[3],
                  const int32_t *faces, const uint8_t *labels, int64_t T, const double Twc0[16],
                  const orc_cam *cam, const float *scan_depth, const uint8_t *scan_class,
                  const orc_params *prm, const orc_dfo_params *p, double Twc_out[16],
                  int64_t *e_table, orc_dfo_report *rep) {
  etable_ctx c = {v, vr, V, T, centre, Twc0, faces, labels, cam, scan_depth, scan_class, prm};
  const double scale[6] = {p->scale_t, p->scale_t, p->scale_t, p->scale_r, p->scale_r, p->scale_r};
  double xi[6], fb;
  if (orc_dfo_core(etable_batch, &c, scale, p, xi, &fb, rep)) return -1;
  orc_se3_right(Twc0, xi, Twc_out);
  *e_table = (int64_t)fb;
  return 0;
}

/* ------------------------------------------------------------------------------------- */
/* Scan classes from a raw range image (Sec. IV.A, IV.B); pose from X (Eq. 1)             */
/* ------------------------------------------------------------------------------------- */

void orc_scan_from_range(const float *range, int64_t n, float range_min, float range_max,
                         float *depth, uint8_t *cls) {
  for (int64_t i = 0; i < n; ++i) {
    const float r = range[i];
    if (isnan(r) || (r > 0.0f && r < range_min)) {
      /* dead pixel, or a return closer than the sensor can measure */
      depth[i] = NAN;
      cls[i] = 2;
    } else if (r <= 0.0f || r > range_max) {
      /* no reading: free space up to the maximal range */
      depth[i] = range_max;
      cls[i] = 1;
    } else {
      depth[i] = r;
      cls[i] = 0;
    }
  }
}

void orc_pose_from_x(const double X[6], double T[16]) {
  const double cx = cos(X[3]), sx = sin(X[3]), cy = cos(X[4]), sy = sin(X[4]);
  const double cz = cos(X[5]), sz = sin(X[5]);
  const double Rx[9] = {1, 0, 0, 0, cx, -sx, 0, sx, cx};
  const double Ry[9] = {cy, 0, sy, 0, 1, 0, -sy, 0, cy};
  const double Rz[9] = {cz, -sz, 0, sz, cz, 0, 0, 0, 1};
  double A[9], R[9];
  for (int i = 0; i < 3; ++i) /* A = Rz Ry */
    for (int j = 0; j < 3; ++j) A[3 * i + j] = Rz[3 * i] * Ry[j] + Rz[3 * i + 1] * Ry[3 + j] + Rz[3 * i + 2] * Ry[6 + j];
  for (int i = 0; i < 3; ++i) /* R = A Rx */
    for (int j = 0; j < 3; ++j) R[3 * i + j] = A[3 * i] * Rx[j] + A[3 * i + 1] * Rx[3 + j] + A[3 * i + 2] * Rx[6 + j];
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) T[4 * i + j] = R[3 * i + j];
    T[4 * i + 3] = X[i];
  }
  T[12] = T[13] = T[14] = 0.0;
  T[15] = 1.0;
}

/* ------------------------------------------------------------------------------------- */
/* Vertex-position gradient of the least-squares surrogate (map refinement)               */
/* ------------------------------------------------------------------------------------- */

/* Camera-frame plane of the triangle (a, b, c) given in FP64 world coordinates: unnormalised
 * camera-frame normal n_c, world normal n_w, offset d with n_c . (t r) = d on the plane. */
static void plane64d(const double a[3], const double b[3], const double c[3], const double T[16],
                     double nc[3], double nw[3], double *d) {
  double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
  double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
  nw[0] = e1[1] * e2[2] - e1[2] * e2[1];
  nw[1] = e1[2] * e2[0] - e1[0] * e2[2];
  nw[2] = e1[0] * e2[1] - e1[1] * e2[0];
  double q[3] = {a[0] - T[3], a[1] - T[7], a[2] - T[11]};
  *d = nw[0] * q[0] + nw[1] * q[1] + nw[2] * q[2];
  for (int i = 0; i < 3; ++i) nc[i] = T[0 * 4 + i] * nw[0] + T[1 * 4 + i] * nw[1] + T[2 * 4 + i] * nw[2];
}

static void face_vertices64(const float *v, const int32_t *faces, int64_t k, int64_t vk,
                            const double delta[3], double P[3][3]) {
  for (int m = 0; m < 3; ++m) {
    const int64_t id = faces[3 * k + m];
    for (int a = 0; a < 3; ++a) P[m][a] = (double)v[3 * id + a] + (id == vk && delta ? delta[a] : 0.0);
  }
}

int orc_cost_vertex_grad(const float *v, const float *vr, int64_t V, const double centre[3],
                         const int32_t *faces, const uint8_t *labels, int64_t T,
                         const double Twc[16], const orc_cam *cam, const float *scan_depth,
                         const uint8_t *scan_class, const orc_params *prm, double *gV) {
  int64_t P = (int64_t)cam->width * cam->height;
  uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (P > 0 ? P : 1));
  if (!keys) return -1;
  orc_render(vr, V, centre, faces, T, Twc, cam, keys, NULL, 0, NULL);
  for (int64_t i = 0; i < 3 * V; ++i) gV[i] = 0.0;
  for (int j = 0; j < cam->height; ++j)
    for (int i = 0; i < cam->width; ++i) {
      int64_t p = (int64_t)j * cam->width + i;
      uint64_t key = keys[p];
      if (key == KEY_EMPTY) continue;
      const int64_t k = (int64_t)(key & 0xFFFFFFFFu);
      int mc = (int)labels[k];
      int sc = scan_class_of(scan_depth, scan_class, p);
      if (sc == 2) continue;
      float t32 = key_depth(key);
      float dz32 = t32 - scan_depth[p];
      int oc = orc_table1(mc, sc, dz32, prm->eps);
      if (oc < 0) continue;
      int active;
      double sgn, w;
      double res = ls_residual(oc, dz32, (double)t32 - (double)scan_depth[p], prm->eps, prm, &active, &sgn, &w);
      if (!active) continue;
      double Pv[3][3], nc[3], nw[3], d, r[3];
      face_vertices64(v, faces, k, -1, NULL, Pv);
      plane64d(Pv[0], Pv[1], Pv[2], Twc, nc, nw, &d);
      ray64(cam, i, j, r);
      const double nr = nc[0] * r[0] + nc[1] * r[1] + nc[2] * r[2];
      const double t = d / nr;
      /* the hit point in the world and its barycentrics (sub-triangle areas along n_w) */
      double dir[3], h[3];
      for (int a = 0; a < 3; ++a) dir[a] = Twc[4 * a] * r[0] + Twc[4 * a + 1] * r[1] + Twc[4 * a + 2] * r[2];
      for (int a = 0; a < 3; ++a) h[a] = Twc[4 * a + 3] + t * dir[a];
      const double nn = nw[0] * nw[0] + nw[1] * nw[1] + nw[2] * nw[2];
      double b[3];
      for (int m = 0; m < 3; ++m) {
        const double *A = Pv[(m + 1) % 3], *B = Pv[(m + 2) % 3];
        double e1[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
        double e2[3] = {h[0] - A[0], h[1] - A[1], h[2] - A[2]};
        double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        b[m] = (cr[0] * nw[0] + cr[1] * nw[1] + cr[2] * nw[2]) / nn;
      }
      /* d t / d v_m = b_m n_w / (n_c . r) */
      for (int m = 0; m < 3; ++m) {
        const int64_t id = faces[3 * k + m];
        for (int a = 0; a < 3; ++a) gV[3 * id + a] += w * res * sgn * b[m] * nw[a] / nr;
      }
    }
  free(keys);
  return 0;
}

double orc_cost_frozen_vertex(const float *v, const float *vr, int64_t V, const double centre[3],
                              const int32_t *faces, const uint8_t *labels, int64_t T,
                              const double Twc[16], const orc_cam *cam, const float *scan_depth,
                              const uint8_t *scan_class, const orc_params *prm, int64_t vk,
                              const double delta[3]) {
  int64_t P = (int64_t)cam->width * cam->height;
  uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (P > 0 ? P : 1));
  if (!keys) return NAN;
  orc_render(vr, V, centre, faces, T, Twc, cam, keys, NULL, 0, NULL);
  double E = 0.0;
  for (int j = 0; j < cam->height; ++j)
    for (int i = 0; i < cam->width; ++i) {
      int64_t p = (int64_t)j * cam->width + i;
      uint64_t key = keys[p];
      if (key == KEY_EMPTY) continue;
      const int64_t k = (int64_t)(key & 0xFFFFFFFFu);
      int mc = (int)labels[k];
      int sc = scan_class_of(scan_depth, scan_class, p);
      if (sc == 2) continue;
      float t32 = key_depth(key);
      float dz32 = t32 - scan_depth[p];
      int oc = orc_table1(mc, sc, dz32, prm->eps);
      if (oc < 0) continue;
      double Pv[3][3], nc[3], nw[3], d, r[3];
      face_vertices64(v, faces, k, vk, delta, Pv);
      plane64d(Pv[0], Pv[1], Pv[2], Twc, nc, nw, &d);
      ray64(cam, i, j, r);
      double dz = d / (nc[0] * r[0] + nc[1] * r[1] + nc[2] * r[2]) - (double)scan_depth[p];
      int active;
      double sgn, w;
      /* cells and activity frozen at the unperturbed map */
      double res = ls_residual(oc, dz32, dz, prm->eps, prm, &active, &sgn, &w);
      E += 0.5 * w * res * res;
    }
  free(keys);
  return E;
}
