/*
 * em_oracle.c -- plain FP64 CPU oracle for fusing point clouds into a
 * robot-centric 2.5D elevation grid, following Miki et al., "Elevation Mapping
 * for Locomotion and Navigation using GPU" (arXiv 2204.12876).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file.  Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark use it.  It shares no code, header, table or constant with the CUDA
 * path; it is written as plain loops over points and cells in the order the
 * paper describes, in double precision, so that it can be checked against the
 * paper by eye.
 *
 * Steps of one update (Section II-A, Fig. 2 caption; Section II-C..II-E):
 *   1. snapshot the cell state (h, sigma_m^2, last-update time, normals)
 *   2. per point: finiteness / range check, transform by the sensor pose,
 *      distance d from the sensor, point variance from the noise model
 *      (Section II-C), cell indices; then, with drift compensation (Section
 *      II-D), the mean height error of the points that fall into flat cells
 *      holding an estimate is added to every estimate
 *   3. per cell, its points in input order: wall rule (Section II-C, last
 *      paragraph), Mahalanobis outlier gate against the snapshot (Section
 *      II-C), then Eq. 1 and Eq. 2 applied point after point
 *   4. ray casting against the snapshot (Section II-E, Eq. 3, Eq. 4); with the
 *      upper-bound layer (Section II-H), samples in cells that are empty in the
 *      snapshot lower the cell's bound to the sample height
 *   5. removal of penetrated cells that were not updated recently; cells that
 *      hold an estimate after the update have no upper bound
 *   6. optional per-cell filters on the updated map: normals (Section II-A),
 *      smoothing (box, median or Gaussian) and in-painting (Section II-I)
 * The map shift (robot-centric map, Section I) is a physical array copy.
 *
 * Readings of passages the paper leaves open (all listed in the design notes):
 *   - an empty cell has sigma_m^2 = infinity, so its first point sets (h,
 *     sigma_m^2) = (p_z, sigma_p^2): the limit of Eq. 1/2 as sigma_m^2 -> inf;
 *   - noise model sigma_p = a0 + a1 d + a2 d^2, sigma_p^2 floored at var_min
 *     (the paper's alpha_d d^2 is a0 = a2 = 0, a1 = sqrt(alpha_d));
 *   - the gate and the wall rule look at the snapshot (pre-update) estimate,
 *     so the result does not depend on the order of the points; the gate's
 *     distance is |p_z - h| / sqrt(sigma_m^2 + sigma_p^2), reject iff > k;
 *   - each rejected point adds outlier_variance to sigma_m^2 before the
 *     accepted points are fused;
 *   - time variance: sigma_t^2 per update, applied lazily from the cell's
 *     last-update index (a Kalman prediction step);
 *   - Eq. 3 is read with the standard deviation sqrt(sigma_m^2);
 *   - ray samples o + k*step*rhat for k = 1, 2, ... while k*step < d, the
 *     endpoint's own cell skipped; removal only for cells whose last update is
 *     at least max(1, cleanup_min_age) updates old, the normal taken from the
 *     previous normal layer ((0,0,1) where it is NaN).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_NORMALS 1u
#define ORC_SMOOTH 2u
#define ORC_INPAINT 4u
#define ORC_MEDIAN 8u
#define ORC_GAUSS 16u
#define ORC_UPPER 32u

/* per-point status codes of the trace */
enum { ST_NONFINITE = 0, ST_RANGE = 1, ST_OUTSIDE = 2, ST_ACCEPT = 3, ST_REJECT = 4, ST_WALL = 5 };
/* per-point marginal flags */
enum { PF_BIN = 1, PF_GATE = 2, PF_WALL = 4, PF_RANGE = 8 };
/* per-cell marginal flags */
enum { CF_VALUE = 1, CF_MARK = 2 };

typedef struct orc_params {
  int32_t width, height;
  double resolution;
  double noise_a0, noise_a1, noise_a2;
  double var_min;
  double min_range, max_range;
  double mahalanobis_k;
  double outlier_variance;
  int32_t wall_num_thresh;
  double time_variance;
  double ray_step;
  int32_t cleanup_min_age;
  double cleanup_normal_thresh;
  uint32_t flags;
  double drift_flatness; /* drift compensation: cells with normal n_z >= this count as flat; 0 = off */
  /* exclusion area (Section II-C, Fig. 3 not available; reading): a point whose
   * height above the sensor exceeds b for a horizontal distance r <= c, else
   * b + (r - c) tan(theta), at most d, is ignored; d <= 0 = off */
  double excl_b, excl_c, excl_theta, excl_d;
  /* overlap clearance (Section II-F; reading): after the update, estimates whose
   * cell centre lies within overlap_radius of the sensor origin (horizontally)
   * and whose height differs from the origin's by more than overlap_dz are
   * cleared; overlap_dz <= 0 = off */
  double overlap_radius, overlap_dz;
} orc_params;

typedef struct orc_cloud {
  const float* pts;
  int64_t n;
  int32_t stride;
  float pose[12]; /* sensor -> map, row-major 3x4 [R | t] */
} orc_cloud;

/* Optional per-update trace.  Every pointer may be NULL.  Per-point arrays are
 * indexed over the clouds' points concatenated in order; per-cell arrays are
 * logical row-major [iy][ix].  unit > 0 turns on the marginal bands: a
 * decision is flagged when the exact value lies within
 * abs_band + c * unit * (magnitude of the operands) of its threshold, c a small
 * constant, i.e. where arithmetic with unit roundoff `unit` could decide it
 * the other way. */
typedef struct orc_trace {
  int32_t* ix;
  int32_t* iy;
  uint8_t* status;
  uint8_t* pflags;
  uint8_t* mark;
  uint8_t* cleared;
  uint8_t* cflags;
  int64_t counts[8]; /* in, valid, in-map, accepted, rejected, wall, cells updated, cells cleared */
  double unit;
  double abs_band;
} orc_trace;

typedef struct orc_map {
  orc_params p;
  int64_t shift_x, shift_y;
  int32_t t_now;
  double* h;
  double* var;
  int32_t* t_last;
  double* nx;
  double* ny;
  double* nz;
  double* smooth;
  double* inpaint;
  double* upper; /* upper bound of the ground height (Section II-H), +inf where none */
  double last_drift;    /* mean height error added by the last update's drift compensation */
  int64_t drift_points; /* points that entered that mean */
  double drift_unc;     /* marginal band of that mean (metres), with the trace's marginal bands */
} orc_map;

static double* alloc_fill(int64_t n, double v) {
  double* a = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) a[i] = v;
  return a;
}

static void clear_cell(orc_map* m, int64_t c) {
  m->h[c] = NAN;
  m->var[c] = INFINITY;
  m->t_last[c] = 0;
  m->nx[c] = m->ny[c] = m->nz[c] = NAN;
  m->smooth[c] = NAN;
  m->inpaint[c] = NAN;
  m->upper[c] = INFINITY;
}

orc_map* orc_create(const orc_params* p) {
  if (!p || p->width <= 0 || p->height <= 0 || !(p->resolution > 0)) return NULL;
  orc_map* m = (orc_map*)calloc(1, sizeof(orc_map));
  m->p = *p;
  int64_t nc = (int64_t)p->width * p->height;
  m->h = alloc_fill(nc, NAN);
  m->var = alloc_fill(nc, INFINITY);
  m->t_last = (int32_t*)calloc((size_t)nc, sizeof(int32_t));
  m->nx = alloc_fill(nc, NAN);
  m->ny = alloc_fill(nc, NAN);
  m->nz = alloc_fill(nc, NAN);
  m->smooth = alloc_fill(nc, NAN);
  m->inpaint = alloc_fill(nc, NAN);
  m->upper = alloc_fill(nc, INFINITY);
  return m;
}

void orc_destroy(orc_map* m) {
  if (!m) return;
  free(m->h); free(m->var); free(m->t_last);
  free(m->nx); free(m->ny); free(m->nz); free(m->smooth); free(m->inpaint); free(m->upper);
  free(m);
}

/* lower-left corner of the map in the map frame: the map is centred on
 * (shift_x * r, shift_y * r) and spans width*r by height*r. */
void orc_origin(const orc_map* m, double* x0, double* y0) {
  *x0 = m->p.resolution * ((double)m->shift_x - 0.5 * m->p.width);
  *y0 = m->p.resolution * ((double)m->shift_y - 0.5 * m->p.height);
}

int32_t orc_t_now(const orc_map* m) { return m->t_now; }

void orc_last_drift(const orc_map* m, double* drift, int64_t* points, double* band) {
  *drift = m->last_drift;
  *points = m->drift_points;
  *band = m->drift_unc;
}

void orc_get_shift(const orc_map* m, int64_t* sx, int64_t* sy) {
  *sx = m->shift_x;
  *sy = m->shift_y;
}

static void copy_out(double* dst, const double* src, int64_t n) {
  if (dst) memcpy(dst, src, sizeof(double) * (size_t)n);
}

void orc_get(const orc_map* m, double* h, double* var, int32_t* t_last, double* nx, double* ny,
             double* nz, double* smooth, double* inpaint) {
  int64_t nc = (int64_t)m->p.width * m->p.height;
  copy_out(h, m->h, nc);
  copy_out(var, m->var, nc);
  if (t_last) memcpy(t_last, m->t_last, sizeof(int32_t) * (size_t)nc);
  copy_out(nx, m->nx, nc);
  copy_out(ny, m->ny, nc);
  copy_out(nz, m->nz, nc);
  copy_out(smooth, m->smooth, nc);
  copy_out(inpaint, m->inpaint, nc);
}

/* The upper-bound layer (logical row-major), read and written on its own. */
void orc_get_upper(const orc_map* m, double* upper) {
  copy_out(upper, m->upper, (int64_t)m->p.width * m->p.height);
}

void orc_set_upper(orc_map* m, const double* upper) {
  int64_t nc = (int64_t)m->p.width * m->p.height;
  for (int64_t c = 0; c < nc; ++c) m->upper[c] = upper[c];
}

/* Overwrite the state.  A cell is empty iff its variance is not finite; such a
 * cell gets h = NaN.  Any pointer may be NULL (that layer is kept). */
void orc_set(orc_map* m, const double* h, const double* var, const int32_t* t_last, const double* nx,
             const double* ny, const double* nz, int32_t t_now, int64_t shift_x, int64_t shift_y) {
  int64_t nc = (int64_t)m->p.width * m->p.height;
  for (int64_t c = 0; c < nc; ++c) {
    if (h) m->h[c] = h[c];
    if (var) m->var[c] = var[c];
    if (t_last) m->t_last[c] = t_last[c];
    if (nx) m->nx[c] = nx[c];
    if (ny) m->ny[c] = ny[c];
    if (nz) m->nz[c] = nz[c];
    if (!isfinite(m->var[c])) { m->var[c] = INFINITY; m->h[c] = NAN; }
  }
  m->t_now = t_now;
  m->shift_x = shift_x;
  m->shift_y = shift_y;
}

/* ---------------------------------------------------------------- helpers */

static int in_map(const orc_map* m, int64_t ix, int64_t iy) {
  return ix >= 0 && iy >= 0 && ix < m->p.width && iy < m->p.height;
}

/* The neighbouring cells a coordinate q (in cells) may fall into when float32
 * arithmetic computes it within `band` metres: bit 0 the cell below
 * (floor(q) - 1), bit 1 the cell above (floor(q) + 1). */
static int edge_alts(double q, double r, double band) {
  double f = q - floor(q);
  int a = 0;
  if (f * r < band) a |= 1;
  if ((1.0 - f) * r < band) a |= 2;
  return a;
}

static int64_t clamp_index(double q) {
  double f = floor(q);
  if (f < -1e9) return -1000000000LL;
  if (f > 1e9) return 1000000000LL;
  return (int64_t)f;
}

/* Cell (ix, iy) and its alternatives (ax, ay: edge_alts bits of each axis):
 * the in-map cells (ix + i, iy + j), i and j in {0} plus the alternatives.
 * Writes their flat indices to out[] (at most 9) and returns how many. */
static int candidates(const orc_map* m, int64_t ix, int64_t iy, int ax, int ay, int64_t* out) {
  int n = 0;
  for (int j = -1; j <= 1; ++j) {
    if ((j == -1 && !(ay & 1)) || (j == 1 && !(ay & 2))) continue;
    for (int i = -1; i <= 1; ++i) {
      if ((i == -1 && !(ax & 1)) || (i == 1 && !(ax & 2))) continue;
      if (in_map(m, ix + i, iy + j)) out[n++] = (iy + j) * m->p.width + (ix + i);
    }
  }
  return n;
}

/* 1 when every cell of (ix, iy) and its alternatives lies in the map */
static int all_in_map(const orc_map* m, int64_t ix, int64_t iy, int ax, int ay) {
  return in_map(m, ix - ((ax & 1) ? 1 : 0), iy - ((ay & 1) ? 1 : 0)) &&
         in_map(m, ix + ((ax & 2) ? 1 : 0), iy + ((ay & 2) ? 1 : 0));
}

/* effective variance at update t_now of a cell last written at t_last:
 * sigma_m^2 grows by sigma_t^2 per update (Section II-C, time variance) */
static double var_eff(const orc_params* p, double var, int32_t t_last, int32_t t_now) {
  if (!isfinite(var)) return INFINITY;
  return var + p->time_variance * (double)(t_now - t_last);
}

typedef struct pt_info {
  double z, var_p, d;
  double vx, vy, vz;    /* R * p_s: sensor-to-point vector in the map frame */
  double sx, sy, sz;    /* magnitudes |R_r0 px| + |R_r1 py| + |R_r2 pz| per row */
  int64_t ix, iy;
  int ax, ay;           /* edge_alts bits of the cell indices (marginal bands only) */
  int cloud;
  int status;
  int flags;
} pt_info;

/* ------------------------------------------------------------ stencils */

/* Per-cell surface normal from a least-squares plane z = a*x + b*y + c fitted
 * to the valid cells of the 3x3 neighbourhood (normal calculation, Section
 * II-A).  Needs at least 3 non-collinear valid cells, else NaN.  The normal is
 * (-a, -b, 1) normalised. */
static void compute_normals(orc_map* m) {
  const int W = m->p.width, H = m->p.height;
  const double r = m->p.resolution;
  for (int iy = 0; iy < H; ++iy)
    for (int ix = 0; ix < W; ++ix) {
      int64_t c = (int64_t)iy * W + ix;
      m->nx[c] = m->ny[c] = m->nz[c] = NAN;
      if (!isfinite(m->var[c])) continue;
      /* normal equations A^T A x = A^T b with rows [dx*r, dy*r, 1] */
      double M[3][3] = {{0}}, rhs[3] = {0};
      int n = 0;
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          int jx = ix + dx, jy = iy + dy;
          if (!in_map(m, jx, jy)) continue;
          int64_t k = (int64_t)jy * W + jx;
          if (!isfinite(m->var[k])) continue;
          double row[3] = {dx * r, dy * r, 1.0};
          for (int a = 0; a < 3; ++a) {
            for (int b = 0; b < 3; ++b) M[a][b] += row[a] * row[b];
            rhs[a] += row[a] * m->h[k];
          }
          ++n;
        }
      if (n < 3) continue;
      /* collinearity test on the integer offsets (exact) */
      double det_int;
      {
        double sxx = M[0][0] / (r * r), sxy = M[0][1] / (r * r), syy = M[1][1] / (r * r);
        double sx = M[0][2] / r, sy = M[1][2] / r, s1 = M[2][2];
        det_int = sxx * (syy * s1 - sy * sy) - sxy * (sxy * s1 - sy * sx) + sx * (sxy * sy - syy * sx);
      }
      if (fabs(det_int) < 0.5) continue; /* integer-valued: 0 iff collinear */
      /* Cramer's rule */
      double det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                   M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                   M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
      double sol[3];
      for (int col = 0; col < 3; ++col) {
        double A[3][3];
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) A[a][b] = (b == col) ? rhs[a] : M[a][b];
        double dc = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
                    A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                    A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
        sol[col] = dc / det;
      }
      double nxv = -sol[0], nyv = -sol[1], nzv = 1.0;
      double nn = sqrt(nxv * nxv + nyv * nyv + nzv * nzv);
      m->nx[c] = nxv / nn;
      m->ny[c] = nyv / nn;
      m->nz[c] = nzv / nn;
    }
}

/* 5x5 box mean over the valid cells of the window, for valid cells only
 * (smoothing filter, Section II-I). */
static void compute_smooth(orc_map* m) {
  const int W = m->p.width, H = m->p.height;
  for (int iy = 0; iy < H; ++iy)
    for (int ix = 0; ix < W; ++ix) {
      int64_t c = (int64_t)iy * W + ix;
      m->smooth[c] = NAN;
      if (!isfinite(m->var[c])) continue;
      double s = 0.0;
      int n = 0;
      for (int dy = -2; dy <= 2; ++dy)
        for (int dx = -2; dx <= 2; ++dx) {
          int jx = ix + dx, jy = iy + dy;
          if (!in_map(m, jx, jy)) continue;
          int64_t k = (int64_t)jy * W + jx;
          if (!isfinite(m->var[k])) continue;
          s += m->h[k];
          ++n;
        }
      m->smooth[c] = s / n;
    }
}

/* 5x5 median over the valid cells of the window, for valid cells only
 * (median smoothing, Section II-I): the lower median, i.e. the element of rank
 * floor((n - 1) / 2) of the n valid heights sorted ascending. */
static void compute_median(orc_map* m) {
  const int W = m->p.width, H = m->p.height;
  for (int iy = 0; iy < H; ++iy)
    for (int ix = 0; ix < W; ++ix) {
      int64_t c = (int64_t)iy * W + ix;
      m->smooth[c] = NAN;
      if (!isfinite(m->var[c])) continue;
      double v[25];
      int n = 0;
      for (int dy = -2; dy <= 2; ++dy)
        for (int dx = -2; dx <= 2; ++dx) {
          int jx = ix + dx, jy = iy + dy;
          if (!in_map(m, jx, jy)) continue;
          int64_t k = (int64_t)jy * W + jx;
          if (!isfinite(m->var[k])) continue;
          v[n++] = m->h[k];
        }
      for (int a = 1; a < n; ++a) { /* insertion sort */
        double x = v[a];
        int b = a - 1;
        while (b >= 0 && v[b] > x) {
          v[b + 1] = v[b];
          --b;
        }
        v[b + 1] = x;
      }
      m->smooth[c] = v[(n - 1) / 2];
    }
}

/* 5x5 Gaussian over the valid cells of the window, for valid cells only
 * (Gaussian smoothing, Section II-I): weights exp(-(dx^2 + dy^2) / (2 s^2))
 * with s = 1 cell, normalised over the valid cells of the window. */
static void compute_gauss(orc_map* m) {
  const int W = m->p.width, H = m->p.height;
  for (int iy = 0; iy < H; ++iy)
    for (int ix = 0; ix < W; ++ix) {
      int64_t c = (int64_t)iy * W + ix;
      m->smooth[c] = NAN;
      if (!isfinite(m->var[c])) continue;
      double s = 0.0, ws = 0.0;
      for (int dy = -2; dy <= 2; ++dy)
        for (int dx = -2; dx <= 2; ++dx) {
          int jx = ix + dx, jy = iy + dy;
          if (!in_map(m, jx, jy)) continue;
          int64_t k = (int64_t)jy * W + jx;
          if (!isfinite(m->var[k])) continue;
          double w = exp(-0.5 * (double)(dx * dx + dy * dy));
          s += w * m->h[k];
          ws += w;
        }
      m->smooth[c] = s / ws;
    }
}

/* Minimum in-painting (Section II-I): every 4-connected component of empty
 * cells that does not touch the map border and has at most 8 cells is filled
 * with the minimum height of the valid cells 8-adjacent to it.  Valid cells
 * keep their height; other empty cells stay NaN.  Plain flood fill labelling. */
static void compute_inpaint(orc_map* m) {
  const int W = m->p.width, H = m->p.height;
  const int64_t nc = (int64_t)W * H;
  int32_t* label = (int32_t*)malloc(sizeof(int32_t) * (size_t)nc);
  int64_t* queue = (int64_t*)malloc(sizeof(int64_t) * (size_t)nc);
  for (int64_t c = 0; c < nc; ++c) {
    label[c] = -1;
    m->inpaint[c] = isfinite(m->var[c]) ? m->h[c] : NAN;
  }
  int32_t next_label = 0;
  for (int64_t seed = 0; seed < nc; ++seed) {
    if (isfinite(m->var[seed]) || label[seed] >= 0) continue;
    int64_t qh = 0, qt = 0;
    queue[qt++] = seed;
    label[seed] = next_label;
    int touches_edge = 0;
    while (qh < qt) {
      int64_t c = queue[qh++];
      int cx = (int)(c % W), cy = (int)(c / W);
      if (cx == 0 || cy == 0 || cx == W - 1 || cy == H - 1) touches_edge = 1;
      const int ddx[4] = {1, -1, 0, 0}, ddy[4] = {0, 0, 1, -1};
      for (int q = 0; q < 4; ++q) {
        int jx = cx + ddx[q], jy = cy + ddy[q];
        if (!in_map(m, jx, jy)) continue;
        int64_t k = (int64_t)jy * W + jx;
        if (isfinite(m->var[k]) || label[k] >= 0) continue;
        label[k] = next_label;
        queue[qt++] = k;
      }
    }
    if (!touches_edge && qt <= 8) {
      double mn = INFINITY;
      for (int64_t q = 0; q < qt; ++q) {
        int cx = (int)(queue[q] % W), cy = (int)(queue[q] / W);
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            int jx = cx + dx, jy = cy + dy;
            if (!in_map(m, jx, jy)) continue;
            int64_t k = (int64_t)jy * W + jx;
            if (isfinite(m->var[k]) && m->h[k] < mn) mn = m->h[k];
          }
      }
      for (int64_t q = 0; q < qt; ++q) m->inpaint[queue[q]] = mn;
    }
    ++next_label;
  }
  free(label);
  free(queue);
}

/* -------------------------------------------------------------- update */

/* Ray samples whose upper-bound update float32 may place differently (a
 * candidate cell, the sample's height + band): flagged after all rays, when
 * the cells' final bounds are known. */
typedef struct upper_unsure {
  int64_t* cell;
  double* z;
  int64_t n, cap;
} upper_unsure;

static void upper_unsure_add(upper_unsure* uu, int64_t c, double z) {
  if (uu->n == uu->cap) {
    uu->cap = uu->cap ? 2 * uu->cap : 1024;
    uu->cell = (int64_t*)realloc(uu->cell, sizeof(int64_t) * (size_t)uu->cap);
    uu->z = (double*)realloc(uu->z, sizeof(double) * (size_t)uu->cap);
  }
  uu->cell[uu->n] = c;
  uu->z[uu->n] = z;
  ++uu->n;
}

/* Eq. 4 guard: |rhat . n| > alpha_n for the cell's previous normal, (0, 0, 1)
 * when that normal is not finite; *dot receives |rhat . n|. */
static int guard_pass(const orc_params* p, double rx, double ry, double rz, double n0, double n1, double n2,
                      double* dot) {
  if (!(isfinite(n0) && isfinite(n1) && isfinite(n2))) { n0 = 0; n1 = 0; n2 = 1; }
  *dot = fabs(rx * n0 + ry * n1 + rz * n2);
  return p->cleanup_normal_thresh > 0 ? *dot > p->cleanup_normal_thresh : 1;
}

/* Walk one ray against the snapshot (Section II-E).  A ray that exists marks
 * every cell one of its samples lies in below the cell's threshold h - sigma
 * (Eq. 3) when the Eq. 4 guard lets it; with the upper-bound layer its samples
 * in empty cells lower their bound (Section II-H).  With marginal bands on, it
 * also flags (CF_MARK) each cell whose mark or bound a float32 computation of
 * this ray may decide otherwise: the sample's cell or one of the cells its
 * position may round into, the endpoint's own cell (skipped) or one of its
 * alternatives, the last sample (k step ~ d), a ray whose existence is
 * marginal, a sample height within its band of the threshold, a guard value
 * within its band of alpha_n.  Such a sample, when some reading has it mark a
 * cell (below the threshold plus band, the guard passing within its band),
 * sets maybe[c]; a sample that marks c in every reading sets sure[c].  A cell
 * is flagged after all rays when maybe is set and sure is not: a mark that one
 * sample makes for certain no other sample can undo.  An uncertain sample in
 * an empty cell is collected in *uu: it is flagged later if it may be that
 * cell's minimum. */
static void walk_ray(orc_map* m, const pt_info* pi, const float* pose, const double* h0, const double* ve0,
                     const double* nx0, const double* ny0, const double* nz0, uint8_t* mark, orc_trace* tr,
                     upper_unsure* uu, uint8_t* sure, uint8_t* maybe, double x0, double y0) {
  const orc_params* p = &m->p;
  const int W = p->width;
  const double r = p->resolution, step = p->ray_step, d = pi->d;
  const double ox = pose[3], oy = pose[7], oz = pose[11];
  const double u = tr ? tr->unit : 0.0, ab = tr ? tr->abs_band : 0.0;
  uint8_t* cflags = (tr && u > 0) ? tr->cflags : NULL;
  const int ray_on = pi->status != ST_RANGE;               /* every valid point casts a ray */
  const int ray_unsure = cflags && (pi->flags & PF_RANGE); /* float32 may decide its validity otherwise */
  if (!(step > 0) || !(d > 0)) return;
  if (!ray_on && !ray_unsure) return;
  const double rx = pi->vx / d, ry = pi->vy / d, rz = pi->vz / d;
  /* the endpoint's own cell, and the cells float32 binning may give it instead */
  int64_t own[9];
  const int n_own = cflags ? candidates(m, pi->ix, pi->iy, pi->ax, pi->ay, own) : 0;
  const int own_exact = (pi->ax | pi->ay) == 0;
  /* samples k = 1, 2, ... while k*step < d; with marginal bands also the next one */
  for (int64_t k = 1;; ++k) {
    const double len = (double)k * step;
    const int last_unsure = cflags && fabs(len - d) < ab + 8.0 * u * d;
    if (!(len < d) && !last_unsure) break;
    const int exists = len < d;
    const double f = len / d;
    const double sx = ox + f * pi->vx, sy = oy + f * pi->vy, sz = oz + f * pi->vz;
    const double qx = (sx - x0) / r, qy = (sy - y0) / r;
    const int64_t cx = clamp_index(qx), cy = clamp_index(qy);
    if (ray_on && exists && in_map(m, cx, cy) && !(cx == pi->ix && cy == pi->iy)) {
      const int64_t c = cy * W + cx;
      double dot;
      if (isfinite(ve0[c])) {
        if (sz < h0[c] - sqrt(ve0[c]) && guard_pass(p, rx, ry, rz, nx0[c], ny0[c], nz0[c], &dot)) mark[c] = 1;
      } else if (p->flags & ORC_UPPER) {
        if (sz < m->upper[c]) m->upper[c] = sz; /* the ground is not above the ray here */
      }
    }
    if (cflags) {
      const double esx = ab + 8.0 * u * (fabs(ox) + f * pi->sx + fabs(x0) + fabs(sx - x0));
      const double esy = ab + 8.0 * u * (fabs(oy) + f * pi->sy + fabs(y0) + fabs(sy - y0));
      const int axs = edge_alts(qx, r, esx), ays = edge_alts(qy, r, esy);
      const int sample_unsure = ray_unsure || last_unsure || (axs | ays) != 0;
      int64_t cand[9];
      const int nc = candidates(m, cx, cy, axs, ays, cand);
      for (int q = 0; q < nc; ++q) {
        const int64_t c = cand[q];
        int own_unsure = 0;
        for (int o = 0; o < n_own; ++o)
          if (own[o] == c) own_unsure = 1;
        if (own_unsure && own_exact) continue; /* the endpoint's own cell in every reading: skipped */
        const int unsure = sample_unsure || own_unsure;
        if (isfinite(ve0[c])) {
          const double sd = sqrt(ve0[c]), thr = h0[c] - sd;
          const double bt = ab + m->drift_unc + 8.0 * u * (fabs(oz) + f * pi->sz + fabs(h0[c]) + sd);
          if (!(sz < thr + bt)) continue; /* above the threshold in every reading */
          double dot;
          guard_pass(p, rx, ry, rz, nx0[c], ny0[c], nz0[c], &dot);
          const double bg = ab + 8.0 * u;
          const int guard_on = p->cleanup_normal_thresh > 0;
          if (guard_on && !(dot > p->cleanup_normal_thresh - bg)) continue; /* the guard holds in every reading */
          const int thr_unsure = fabs(sz - thr) < bt;
          const int guard_unsure = guard_on && fabs(dot - p->cleanup_normal_thresh) < bg;
          if (unsure || thr_unsure || guard_unsure) maybe[c] = 1; /* some reading marks c, another not */
          else sure[c] = 1;                                       /* every reading marks c */
        } else if ((p->flags & ORC_UPPER) && unsure) {
          upper_unsure_add(uu, c, sz - (ab + 8.0 * u * (fabs(oz) + f * pi->sz)));
        }
      }
    }
    if (!exists) break;
  }
}

int orc_update(orc_map* m, const orc_cloud* clouds, int32_t ncloud, orc_trace* tr) {
  if (!m || ncloud < 0 || (ncloud > 0 && !clouds)) return -1;
  const orc_params* p = &m->p;
  const int W = p->width, H = p->height;
  const int64_t nc = (int64_t)W * H;
  const double r = p->resolution;
  const int32_t t_now = m->t_now + 1;
  const double u = tr ? tr->unit : 0.0, ab = tr ? tr->abs_band : 0.0;
  double x0, y0;
  orc_origin(m, &x0, &y0);

  int64_t npts = 0;
  for (int ci = 0; ci < ncloud; ++ci) npts += clouds[ci].n > 0 ? clouds[ci].n : 0;
  if (tr) {
    memset(tr->counts, 0, sizeof(tr->counts));
    if (tr->mark) memset(tr->mark, 0, (size_t)nc);
    if (tr->cleared) memset(tr->cleared, 0, (size_t)nc);
    if (tr->cflags) memset(tr->cflags, 0, (size_t)nc);
  }

  /* 1. snapshot */
  double* h0 = (double*)malloc(sizeof(double) * (size_t)nc);
  double* ve0 = (double*)malloc(sizeof(double) * (size_t)nc);
  double* nx0 = (double*)malloc(sizeof(double) * (size_t)nc);
  double* ny0 = (double*)malloc(sizeof(double) * (size_t)nc);
  double* nz0 = (double*)malloc(sizeof(double) * (size_t)nc);
  for (int64_t c = 0; c < nc; ++c) {
    h0[c] = m->h[c];
    ve0[c] = var_eff(p, m->var[c], m->t_last[c], t_now);
    nx0[c] = m->nx[c];
    ny0[c] = m->ny[c];
    nz0[c] = m->nz[c];
  }

  /* 2. per point: validity, transform, noise variance, cell */
  pt_info* pts = (pt_info*)calloc((size_t)(npts > 0 ? npts : 1), sizeof(pt_info));
  int64_t gi = 0;
  for (int ci = 0; ci < ncloud; ++ci) {
    const orc_cloud* cl = &clouds[ci];
    const float* R = cl->pose;
    for (int64_t i = 0; i < cl->n; ++i, ++gi) {
      pt_info* pi = &pts[gi];
      const float* q = cl->pts + i * cl->stride;
      double px = q[0], py = q[1], pz = q[2];
      pi->cloud = ci;
      pi->ix = pi->iy = INT32_MIN;
      if (!(isfinite(px) && isfinite(py) && isfinite(pz))) { pi->status = ST_NONFINITE; continue; }
      double d = sqrt(px * px + py * py + pz * pz);
      pi->d = d;
      int in_range = d >= p->min_range && d <= p->max_range;
      if (u > 0) {
        double bd = ab + 8.0 * u * d;
        if (fabs(d - p->min_range) < bd || fabs(d - p->max_range) < bd) pi->flags |= PF_RANGE;
      }
      /* transform to the map frame */
      pi->vx = R[0] * px + R[1] * py + R[2] * pz;
      pi->vy = R[4] * px + R[5] * py + R[6] * pz;
      pi->vz = R[8] * px + R[9] * py + R[10] * pz;
      pi->sx = fabs(R[0] * px) + fabs(R[1] * py) + fabs(R[2] * pz);
      pi->sy = fabs(R[4] * px) + fabs(R[5] * py) + fabs(R[6] * pz);
      pi->sz = fabs(R[8] * px) + fabs(R[9] * py) + fabs(R[10] * pz);
      double x = pi->vx + R[3], y = pi->vy + R[7], z = pi->vz + R[11];
      pi->z = z;
      /* noise model (Section II-C) */
      double sig = p->noise_a0 + p->noise_a1 * d + p->noise_a2 * d * d;
      double vp = sig * sig;
      pi->var_p = vp > p->var_min ? vp : p->var_min;
      /* cell indices */
      double qx = (x - x0) / r, qy = (y - y0) / r;
      pi->ix = clamp_index(qx);
      pi->iy = clamp_index(qy);
      if (u > 0) {
        /* float32 binning (a 3-term FMA chain, the translation, the subtraction
         * of x0 and the product with the rounded 1/r) stays within about 2u of
         * these magnitudes; the band takes twice that */
        double bx = ab + 4.0 * u * (pi->sx + fabs(R[3]) + fabs(x0) + fabs(x - x0));
        double by = ab + 4.0 * u * (pi->sy + fabs(R[7]) + fabs(y0) + fabs(y - y0));
        pi->ax = edge_alts(qx, r, bx);
        pi->ay = edge_alts(qy, r, by);
        if (pi->ax | pi->ay) pi->flags |= PF_BIN;
      }
      /* exclusion area (Section II-C): the point is ignored above the ramp */
      if (in_range && p->excl_d > 0) {
        const double dxs = x - R[3], dys = y - R[7], zr = z - R[11];
        const double rxy = sqrt(dxs * dxs + dys * dys);
        double lim = rxy <= p->excl_c ? p->excl_b : p->excl_b + (rxy - p->excl_c) * tan(p->excl_theta);
        if (lim > p->excl_d) lim = p->excl_d;
        if (zr > lim) in_range = 0;
        if (u > 0) {
          const double band = ab + 8.0 * u * (pi->sx + pi->sy + pi->sz + fabs(R[3]) + fabs(R[7]) + fabs(R[11]) +
                                              fabs(lim) + fabs(p->excl_b) + fabs(p->excl_d) + rxy * 4.0);
          if (fabs(zr - lim) < band || fabs(rxy - p->excl_c) < band) pi->flags |= PF_RANGE;
        }
      }
      if (!in_range) { pi->status = ST_RANGE; continue; }
      pi->status = in_map(m, pi->ix, pi->iy) ? ST_ACCEPT : ST_OUTSIDE; /* decided per cell below */
    }
  }

  /* height drift compensation (Section II-D): the error of each point against
   * the estimate of its cell, over cells that hold an estimate and are flat
   * (the previous normal has n_z >= drift_flatness; a NaN normal is not flat);
   * the mean error is added to every estimate before the update uses them */
  if (p->drift_flatness > 0) {
    double eps = 0.0;
    int64_t n_eps = 0;
    for (int64_t i = 0; i < npts; ++i) {
      const pt_info* pi = &pts[i];
      if (pi->status != ST_ACCEPT) continue;
      int64_t c = pi->iy * W + pi->ix;
      if (!isfinite(ve0[c]) || !(nz0[c] >= p->drift_flatness)) continue;
      eps += pi->z - h0[c];
      ++n_eps;
    }
    m->drift_unc = 0.0;
    if (n_eps > 0) {
      const double mean = eps / (double)n_eps;
      if (u > 0) {
        /* Marginal band of the mean.  A point whose cell or validity is
         * marginal (PF_BIN, PF_RANGE) may enter the float32 mean with the error
         * of another candidate cell, or not at all (a candidate that is not a
         * flat cell with an estimate, or outside the map), or enter it although
         * the oracle leaves it out.  Changing the contributions (e_i, n_i) to
         * (e', n') moves the mean by (dS - mean dN) / (n + dN), so the sum over
         * such points of their largest |(e' - e_i) - mean (n' - n_i)|, over n
         * minus the number of points whose count may change, bounds that move.  Added: float32
         * rounding of every error (the transform of z and the subtraction),
         * the 2^-44 truncation of the exact sum, and the rounding of the mean. */
        double dev = 0.0, rnd = 0.0;
        int64_t k_unsure = 0;
        for (int64_t i = 0; i < npts; ++i) {
          const pt_info* pi = &pts[i];
          if (pi->status == ST_NONFINITE) continue;
          const double tz = fabs((double)clouds[pi->cloud].pose[11]);
          int in_mean = 0;
          double e_i = 0.0;
          if (pi->status == ST_ACCEPT) {
            const int64_t c = pi->iy * W + pi->ix;
            if (isfinite(ve0[c]) && nz0[c] >= p->drift_flatness) {
              in_mean = 1;
              e_i = pi->z - h0[c];
              rnd += 8.0 * u * (pi->sz + tz) + u * fabs(e_i) + 0x1p-44;
            }
          }
          if (!(pi->flags & (PF_BIN | PF_RANGE))) continue;
          const int can_valid = pi->status != ST_RANGE || (pi->flags & PF_RANGE);
          int can_out = pi->status == ST_RANGE || (pi->flags & PF_RANGE) ||
                        !all_in_map(m, pi->ix, pi->iy, pi->ax, pi->ay);
          double worst = 0.0;
          int n_moves = 0;
          if (can_valid) {
            int64_t cand[9];
            const int ncand = candidates(m, pi->ix, pi->iy, pi->ax, pi->ay, cand);
            for (int q = 0; q < ncand; ++q) {
              const int64_t c = cand[q];
              if (!(isfinite(ve0[c]) && nz0[c] >= p->drift_flatness)) { can_out = 1; continue; }
              const double e = pi->z - h0[c];
              const double w = fabs(e - e_i - (in_mean ? 0.0 : mean));
              if (w > worst) worst = w;
              if (!in_mean) n_moves = 1;
              rnd += in_mean ? 0.0 : 8.0 * u * (pi->sz + tz) + u * fabs(e) + 0x1p-44;
            }
          }
          if (can_out && in_mean) {
            const double w = fabs(mean - e_i);
            if (w > worst) worst = w;
            n_moves = 1;
          }
          dev += worst;
          k_unsure += n_moves;
        }
        m->drift_unc = n_eps > k_unsure ? (dev + rnd) / (double)(n_eps - k_unsure) + 3.0 * u * fabs(mean) : 1e30;
      }
      for (int64_t c = 0; c < nc; ++c) {
        if (!isfinite(ve0[c])) continue;
        h0[c] += mean;
        m->h[c] += mean;
      }
    }
    m->last_drift = n_eps > 0 ? eps / (double)n_eps : 0.0;
    m->drift_points = n_eps;
  } else {
    m->drift_unc = 0.0;
  }
  const double du = m->drift_unc; /* widens every decision taken against the moved estimates */

  /* 3. per cell: points in input order (linked lists built back to front) */
  int64_t* head = (int64_t*)malloc(sizeof(int64_t) * (size_t)nc);
  int64_t* next = (int64_t*)malloc(sizeof(int64_t) * (size_t)(npts > 0 ? npts : 1));
  int64_t* cnt = (int64_t*)calloc((size_t)nc, sizeof(int64_t));
  for (int64_t c = 0; c < nc; ++c) head[c] = -1;
  for (int64_t i = npts - 1; i >= 0; --i) {
    if (pts[i].status != ST_ACCEPT) continue;
    int64_t c = pts[i].iy * W + pts[i].ix;
    next[i] = head[c];
    head[c] = i;
    cnt[c]++;
  }
  int64_t n_acc = 0, n_rej = 0, n_wall = 0, n_upd = 0;
  for (int64_t c = 0; c < nc; ++c) {
    if (head[c] < 0) continue;
    const int valid = isfinite(ve0[c]);
    int64_t rej = 0, acc = 0;
    /* decisions against the snapshot */
    for (int64_t i = head[c]; i >= 0; i = next[i]) {
      pt_info* pi = &pts[i];
      if (p->wall_num_thresh > 0 && valid && cnt[c] > p->wall_num_thresh) {
        if (u > 0 && fabs(pi->z - h0[c]) < ab + du + 8.0 * u * (pi->sz + fabs(clouds[pi->cloud].pose[11]) + fabs(h0[c])))
          pi->flags |= PF_WALL;
        if (pi->z < h0[c]) { pi->status = ST_WALL; continue; }
      }
      if (valid && p->mahalanobis_k > 0) {
        double s = sqrt(ve0[c] + pi->var_p);
        double md = fabs(pi->z - h0[c]) / s;
        if (u > 0) {
          double band = ab + 16.0 * u * md +
                        (8.0 * u * (pi->sz + fabs(clouds[pi->cloud].pose[11]) + fabs(h0[c])) + du) / s;
          if (fabs(md - p->mahalanobis_k) < band) pi->flags |= PF_GATE;
        }
        if (md > p->mahalanobis_k) { pi->status = ST_REJECT; ++rej; continue; }
      }
      pi->status = ST_ACCEPT;
      ++acc;
    }
    if (acc + rej == 0) continue;
    /* the variance grows with every rejected point, then Eq. 1 / Eq. 2 */
    double hm = h0[c];
    double vm = valid ? ve0[c] + (double)rej * p->outlier_variance : INFINITY;
    for (int64_t i = head[c]; i >= 0; i = next[i]) {
      const pt_info* pi = &pts[i];
      if (pi->status != ST_ACCEPT) continue;
      if (!isfinite(vm)) { /* first measurement of an empty cell */
        hm = pi->z;
        vm = pi->var_p;
      } else {
        double vp = pi->var_p;
        hm = (vp * hm + vm * pi->z) / (vm + vp); /* Eq. 1 */
        vm = (vm * vp) / (vm + vp);               /* Eq. 2 */
      }
    }
    m->h[c] = hm;
    m->var[c] = vm;
    m->t_last[c] = t_now;
    n_acc += acc;
    n_rej += rej;
    ++n_upd;
  }
  for (int64_t i = 0; i < npts; ++i) n_wall += pts[i].status == ST_WALL;

  /* 4. ray casting against the snapshot (Section II-E) */
  uint8_t* mark = (uint8_t*)calloc((size_t)nc, 1);
  uint8_t* sure = (uint8_t*)calloc((size_t)nc, 1);
  uint8_t* maybe = (uint8_t*)calloc((size_t)nc, 1);
  upper_unsure uu = {NULL, NULL, 0, 0};
  if (p->ray_step > 0) {
    for (int64_t i = 0; i < npts; ++i) {
      const pt_info* pi = &pts[i];
      if (pi->status == ST_NONFINITE) continue;
      const float* pose = clouds[pi->cloud].pose;
      walk_ray(m, pi, pose, h0, ve0, nx0, ny0, nz0, mark, tr, &uu, sure, maybe, x0, y0);
    }
  }
  if (tr && tr->cflags)
    for (int64_t c = 0; c < nc; ++c)
      if (maybe[c] && !sure[c]) tr->cflags[c] |= CF_MARK;
  free(sure);
  free(maybe);
  /* an uncertain sample may change an empty cell's bound only if it may be
   * that cell's minimum (its height less its band below the final bound) */
  for (int64_t q = 0; q < uu.n; ++q)
    if (uu.z[q] < m->upper[uu.cell[q]]) tr->cflags[uu.cell[q]] |= CF_MARK;
  free(uu.cell);
  free(uu.z);

  /* 5. removal: penetrated and not updated for max(1, cleanup_min_age) updates */
  int64_t n_clr = 0;
  const int32_t min_age = p->cleanup_min_age > 1 ? p->cleanup_min_age : 1;
  for (int64_t c = 0; c < nc; ++c) {
    if (!mark[c] || !isfinite(m->var[c])) continue;
    if (t_now - m->t_last[c] < min_age) continue;
    m->h[c] = NAN;
    m->var[c] = INFINITY;
    if (tr && tr->cleared) tr->cleared[c] = 1;
    ++n_clr;
  }
  if (p->flags & ORC_UPPER)
    for (int64_t c = 0; c < nc; ++c)
      if (isfinite(m->var[c])) m->upper[c] = INFINITY; /* observed: no bound needed */

  /* overlap clearance (Section II-F): estimates near the robot (the first
   * cloud's sensor origin) that are far from its height belong to another floor */
  if (p->overlap_dz > 0 && ncloud > 0) {
    const double ox = clouds[0].pose[3], oy = clouds[0].pose[7], oz = clouds[0].pose[11];
    for (int iy = 0; iy < H; ++iy)
      for (int ix = 0; ix < W; ++ix) {
        const int64_t c = (int64_t)iy * W + ix;
        if (!isfinite(m->var[c])) continue;
        const double cx = x0 + (ix + 0.5) * r - ox, cy = y0 + (iy + 0.5) * r - oy;
        const double dist = sqrt(cx * cx + cy * cy), dz = fabs(m->h[c] - oz);
        if (u > 0 && tr && tr->cflags) {
          const double bd = ab + 8.0 * u * (fabs(x0) + fabs(ox) + fabs(y0) + fabs(oy) + dist + W * r + H * r);
          const double bz = ab + 8.0 * u * (fabs(m->h[c]) + fabs(oz)) + 1e-5; /* the estimate's parity tolerance */
          if (fabs(dist - p->overlap_radius) < bd || fabs(dz - p->overlap_dz) < bz) tr->cflags[c] |= CF_VALUE;
        }
        if (dist <= p->overlap_radius && dz > p->overlap_dz) {
          m->h[c] = NAN;
          m->var[c] = INFINITY;
          if (tr && tr->cleared) tr->cleared[c] = 1; /* a removal (not counted as visibility) */
        }
      }
  }

  /* 6. per-cell filters on the updated map */
  if (p->flags & ORC_NORMALS) compute_normals(m);
  if (p->flags & ORC_SMOOTH) compute_smooth(m);
  if (p->flags & ORC_MEDIAN) compute_median(m);
  if (p->flags & ORC_GAUSS) compute_gauss(m);
  if (p->flags & ORC_INPAINT) compute_inpaint(m);
  m->t_now = t_now;

  if (tr) {
    int64_t n_valid = 0, n_inmap = 0;
    for (int64_t i = 0; i < npts; ++i) {
      const pt_info* pi = &pts[i];
      n_valid += pi->status != ST_NONFINITE && pi->status != ST_RANGE;
      n_inmap += pi->status >= ST_ACCEPT;
      if (tr->ix) tr->ix[i] = (int32_t)(pi->ix < INT32_MIN ? INT32_MIN : pi->ix > INT32_MAX ? INT32_MAX : pi->ix);
      if (tr->iy) tr->iy[i] = (int32_t)(pi->iy < INT32_MIN ? INT32_MIN : pi->iy > INT32_MAX ? INT32_MAX : pi->iy);
      if (tr->status) tr->status[i] = (uint8_t)pi->status;
      if (tr->pflags) tr->pflags[i] = (uint8_t)pi->flags;
      if (tr->cflags && pi->flags && pi->status != ST_NONFINITE) {
        /* the point's cell and the cells float32 binning may give it instead */
        int64_t cand[9];
        const int nc = candidates(m, pi->ix, pi->iy, pi->ax, pi->ay, cand);
        for (int q = 0; q < nc; ++q) tr->cflags[cand[q]] |= CF_VALUE;
      }
    }
    if (tr->mark) memcpy(tr->mark, mark, (size_t)nc);
    tr->counts[0] = npts;
    tr->counts[1] = n_valid;
    tr->counts[2] = n_inmap;
    tr->counts[3] = n_acc;
    tr->counts[4] = n_rej;
    tr->counts[5] = n_wall;
    tr->counts[6] = n_upd;
    tr->counts[7] = n_clr;
  }
  free(mark); free(head); free(next); free(cnt); free(pts);
  free(h0); free(ve0); free(nx0); free(ny0); free(nz0);
  return 0;
}

/* Move the map by (dx, dy) cells: new cell (ix, iy) holds old cell
 * (ix + dx, iy + dy); cells that come into view are empty. */
void orc_shift(orc_map* m, int32_t dx, int32_t dy) {
  const int W = m->p.width, H = m->p.height;
  const int64_t nc = (int64_t)W * H;
  orc_map* old = orc_create(&m->p);
  orc_get(m, old->h, old->var, old->t_last, old->nx, old->ny, old->nz, old->smooth, old->inpaint);
  orc_get_upper(m, old->upper);
  for (int iy = 0; iy < H; ++iy)
    for (int ix = 0; ix < W; ++ix) {
      int64_t c = (int64_t)iy * W + ix;
      int64_t sx = (int64_t)ix + dx, sy = (int64_t)iy + dy;
      if (!in_map(m, sx, sy)) { clear_cell(m, c); continue; }
      int64_t s = sy * W + sx;
      m->h[c] = old->h[s];
      m->var[c] = old->var[s];
      m->t_last[c] = old->t_last[s];
      m->nx[c] = old->nx[s];
      m->ny[c] = old->ny[s];
      m->nz[c] = old->nz[s];
      m->smooth[c] = old->smooth[s];
      m->inpaint[c] = old->inpaint[s];
      m->upper[c] = old->upper[s];
    }
  (void)nc;
  m->shift_x += dx;
  m->shift_y += dy;
  orc_destroy(old);
}

/* Run the filters of Section II-A / II-I on the current state (used by the
 * tests to pin them on hand-made maps). */
void orc_filters(orc_map* m, uint32_t which) {
  if (which & ORC_NORMALS) compute_normals(m);
  if (which & ORC_SMOOTH) compute_smooth(m);
  if (which & ORC_MEDIAN) compute_median(m);
  if (which & ORC_GAUSS) compute_gauss(m);
  if (which & ORC_INPAINT) compute_inpaint(m);
}
