/*
 * FP64 reference Joseph projector P and its literal transpose P^T.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is part of the oracle: the plain,
 * slow, obviously correct CPU statement of what the CUDA path computes.
 * Only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load it; the product library never links or calls it, and
 * it shares no code, header or table with the product library.
 *
 * What it computes (the paper factorises the projection as P E{f}, Sec. 3,
 * with P in R^{m x n} a discrete forward projector; the paper delegates P to
 * an external package and does not name a model, so the model here is the
 * ray-driven Joseph interpolation projector):
 *
 *   grid      N^d pixel/voxel centres c_k = -1 + (k + 1/2) * D, D = 2/N,
 *             flat index i = ((iz*N) + iy)*N + ix  (row-major, x fastest).
 *   ray       point s, unit direction e.
 *   driving   axis a = argmax_k |e_k|, ties (within a relative 1e-12) to the
 *             lowest axis (x, y, z).
 *   sum       for every slice j = 0..N-1 of axis a: intersect the ray with the
 *             plane/line x_a = c_j, convert the transverse coordinates to
 *             fractional indices u = (p + 1)/D - 1/2, interpolate linearly
 *             (2-D) or bilinearly (3-D) with zero outside the grid, add.
 *   scale     the sum times D / |e_a| (the path length per slice).
 *
 * Geometries (angles in radians, lengths in pixel units at the isocentre
 * unless stated; world units are those of the grid square [-1, 1]^d):
 *   view angle  ang_k = angle0 + span * k / V
 *   PAR2D   bin b: t_b = (b - (A-1)/2) * du * D; s = t_b (cos, sin);
 *           e = (-sin, cos).
 *   FAN2D   equiangular (curved) detector.  Source S = R (cos, sin),
 *           R = sod * D; fan angle gamma_b = (b - (A-1)/2) * du / sod;
 *           e = -(cos(ang + gamma_b), sin(ang + gamma_b)).
 *   CONE3D  flat panel.  Source S = R (cos, sin, 0); detector centre
 *           -(sdd - sod) D (cos, sin, 0); axes u = (-sin, cos, 0),
 *           v = (0, 0, 1); pitches du*D*sdd/sod and dv*D*sdd/sod; bin
 *           (row, col) centre = centre + (col-(A-1)/2) pu u + (row-(B-1)/2) pv v;
 *           e = normalise(bin - S).  Sinogram index (k*B + row)*A + col.
 *
 * Compile with -ffp-contract=off so every FP64 operation rounds once.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_PAR2D = 0, ORC_FAN2D = 1, ORC_CONE3D = 2 };

typedef struct {
  int kind;   /* ORC_PAR2D, ORC_FAN2D, ORC_CONE3D */
  int N;      /* grid side */
  int V;      /* views */
  int A;      /* detector bins along u (columns) */
  int B;      /* detector rows along v (cone only; 1 otherwise) */
  double du, dv, sod, sdd, angle0, span;
} orc_geom;

static int dim_of(const orc_geom* g) { return g->kind == ORC_CONE3D ? 3 : 2; }

int64_t orc_num_rays(const orc_geom* g) {
  return (int64_t)g->V * (g->kind == ORC_CONE3D ? g->B : 1) * g->A;
}

/* Point s on the ray and unit direction e of ray (view k, row, col). */
void orc_ray(const orc_geom* g, int k, int row, int col, double s[3], double e[3]) {
  const double D = 2.0 / g->N;
  const double ang = g->angle0 + g->span * (double)k / (double)g->V;
  const double cb = cos(ang), sb = sin(ang);
  s[0] = s[1] = s[2] = 0.0;
  e[0] = e[1] = e[2] = 0.0;
  if (g->kind == ORC_PAR2D) {
    const double t = ((double)col - 0.5 * (g->A - 1)) * g->du * D;
    s[0] = t * cb;
    s[1] = t * sb;
    e[0] = -sb;
    e[1] = cb;
  } else if (g->kind == ORC_FAN2D) {
    const double R = g->sod * D;
    const double gam = ((double)col - 0.5 * (g->A - 1)) * g->du / g->sod;
    s[0] = R * cb;
    s[1] = R * sb;
    e[0] = -cos(ang + gam);
    e[1] = -sin(ang + gam);
  } else {
    const double R = g->sod * D;
    const double pu = g->du * D * g->sdd / g->sod;
    const double pv = g->dv * D * g->sdd / g->sod;
    const double ua = ((double)col - 0.5 * (g->A - 1)) * pu;
    const double vb = ((double)row - 0.5 * (g->B - 1)) * pv;
    const double dc = -(g->sdd - g->sod) * D;
    const double bin[3] = {dc * cb - ua * sb, dc * sb + ua * cb, vb};
    s[0] = R * cb;
    s[1] = R * sb;
    s[2] = 0.0;
    double n2 = 0.0;
    for (int q = 0; q < 3; q++) {
      e[q] = bin[q] - s[q];
      n2 += e[q] * e[q];
    }
    const double nrm = sqrt(n2);
    for (int q = 0; q < 3; q++) e[q] /= nrm;
  }
}

static int64_t flat_index(int d, int N, const int idx[3]) {
  if (d == 2) return (int64_t)idx[1] * N + idx[0];
  return ((int64_t)idx[2] * N + idx[1]) * N + idx[0];
}

/*
 * Driving axis: the axis of largest |e_k|.  An axis only wins over a lower one
 * when it is larger by more than a relative 1e-12, so that rays at exactly 45
 * degrees (whose components agree up to the rounding of cos/sin) drive the
 * lowest axis whatever the platform's trigonometric rounding.
 */
static int driving_axis(int d, const double e[3]) {
  int a = 0;
  for (int q = 1; q < d; q++)
    if (fabs(e[q]) > fabs(e[a]) * (1.0 + 1e-12)) a = q;
  return a;
}

/*
 * Walk one ray.  mode 0: return P_ray . img.  mode 1: img_out += P_ray^T * val.
 */
static double walk(const orc_geom* g, const double s[3], const double e[3],
                   const double* img, double* img_out, double val, int mode) {
  const int d = dim_of(g);
  const int N = g->N;
  const double D = 2.0 / N;
  const int a = driving_axis(d, e);
  int tq[2], nt = 0;
  for (int q = 0; q < d; q++)
    if (q != a) tq[nt++] = q;
  const double scale = D / fabs(e[a]);
  double sum = 0.0;
  for (int j = 0; j < N; j++) {
    const double c = -1.0 + ((double)j + 0.5) * D;
    const double t = (c - s[a]) / e[a];
    double u[2];
    int i0[2];
    double f[2];
    for (int m = 0; m < nt; m++) {
      u[m] = (s[tq[m]] + t * e[tq[m]] + 1.0) / D - 0.5;
      i0[m] = (int)floor(u[m]);
      f[m] = u[m] - (double)i0[m];
    }
    int idx[3] = {0, 0, 0};
    idx[a] = j;
    if (nt == 1) {
      for (int m0 = 0; m0 < 2; m0++) {
        const int iq = i0[0] + m0;
        if (iq < 0 || iq >= N) continue;
        const double w = m0 ? f[0] : 1.0 - f[0];
        idx[tq[0]] = iq;
        const int64_t fi = flat_index(d, N, idx);
        if (mode == 0)
          sum += w * img[fi];
        else
          img_out[fi] += w * scale * val;
      }
    } else {
      for (int m0 = 0; m0 < 2; m0++) {
        const int iq0 = i0[0] + m0;
        if (iq0 < 0 || iq0 >= N) continue;
        const double w0 = m0 ? f[0] : 1.0 - f[0];
        for (int m1 = 0; m1 < 2; m1++) {
          const int iq1 = i0[1] + m1;
          if (iq1 < 0 || iq1 >= N) continue;
          const double w1 = m1 ? f[1] : 1.0 - f[1];
          idx[tq[0]] = iq0;
          idx[tq[1]] = iq1;
          const int64_t fi = flat_index(d, N, idx);
          if (mode == 0)
            sum += w0 * w1 * img[fi];
          else
            img_out[fi] += w0 * w1 * scale * val;
        }
      }
    }
  }
  return sum * scale;
}

static void ray_coords(const orc_geom* g, int64_t r, int* k, int* row, int* col) {
  const int rows = g->kind == ORC_CONE3D ? g->B : 1;
  *col = (int)(r % g->A);
  *row = (int)((r / g->A) % rows);
  *k = (int)(r / ((int64_t)g->A * rows));
}

/* z = P img, every ray.  Rays are independent, so they run in parallel. */
void orc_project(const orc_geom* g, const double* img, double* sino) {
  const int64_t m = orc_num_rays(g);
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t r = 0; r < m; r++) {
    int k, row, col;
    double s[3], e[3];
    ray_coords(g, r, &k, &row, &col);
    orc_ray(g, k, row, col, s, e);
    sino[r] = walk(g, s, e, img, NULL, 0.0, 0);
  }
}

/* z_r = (P img)_r for a list of ray indices. */
void orc_project_at(const orc_geom* g, const double* img, int64_t nr, const int64_t* rays,
                    double* out) {
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t q = 0; q < nr; q++) {
    int k, row, col;
    double s[3], e[3];
    ray_coords(g, rays[q], &k, &row, &col);
    orc_ray(g, k, row, col, s, e);
    out[q] = walk(g, s, e, img, NULL, 0.0, 0);
  }
}

/* img = P^T sino: the literal transpose, one ray at a time, serial. */
void orc_backproject(const orc_geom* g, const double* sino, double* img) {
  const int d = dim_of(g);
  int64_t n = 1;
  for (int q = 0; q < d; q++) n *= g->N;
  memset(img, 0, sizeof(double) * (size_t)n);
  const int64_t m = orc_num_rays(g);
  for (int64_t r = 0; r < m; r++) {
    if (sino[r] == 0.0) continue;
    int k, row, col;
    double s[3], e[3];
    ray_coords(g, r, &k, &row, &col);
    orc_ray(g, k, row, col, s, e);
    walk(g, s, e, NULL, img, sino[r], 1);
  }
}

/*
 * One matrix entry P[ray, pixel] written out directly: the ray crosses the
 * pixel's slice of the driving axis at transverse fractional index u; the
 * pixel receives the interpolation weight of that crossing.
 */
double orc_matrix_entry(const orc_geom* g, int64_t ray, int64_t pix) {
  const int d = dim_of(g);
  const int N = g->N;
  const double D = 2.0 / N;
  int k, row, col;
  double s[3], e[3];
  ray_coords(g, ray, &k, &row, &col);
  orc_ray(g, k, row, col, s, e);
  int idx[3];
  idx[0] = (int)(pix % N);
  idx[1] = (int)((pix / N) % N);
  idx[2] = d == 3 ? (int)(pix / ((int64_t)N * N)) : 0;
  const int a = driving_axis(d, e);
  const double c = -1.0 + ((double)idx[a] + 0.5) * D;
  const double t = (c - s[a]) / e[a];
  double w = D / fabs(e[a]);
  for (int q = 0; q < d; q++) {
    if (q == a) continue;
    const double u = (s[q] + t * e[q] + 1.0) / D - 0.5;
    const int i0 = (int)floor(u);
    const double f = u - (double)i0;
    if (idx[q] == i0)
      w *= 1.0 - f;
    else if (idx[q] == i0 + 1)
      w *= f;
    else
      return 0.0;
  }
  return w;
}

/* (P^T sino)_pix for a list of pixels, by summing matrix entries over every ray. */
void orc_backproject_at(const orc_geom* g, const double* sino, int64_t np, const int64_t* pix,
                        double* out) {
  const int64_t m = orc_num_rays(g);
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t q = 0; q < np; q++) {
    double acc = 0.0;
    for (int64_t r = 0; r < m; r++) {
      if (sino[r] == 0.0) continue;
      const double w = orc_matrix_entry(g, r, pix[q]);
      if (w != 0.0) acc += w * sino[r];
    }
    out[q] = acc;
  }
}
