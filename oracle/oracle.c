/* oracle.c -- plain FP64 CPU oracle of the collapse-time hot path.
 *
 * TEST INFRASTRUCTURE: slow and deliberately plain. Only tests/,
 * __graft_entry__.smoke() and bench.py's CPU-baseline / reference legs use it.
 * It shares no code with the CUDA library. Every routine cites the passage of
 * arXiv:2510.02873 it restates; the readings taken where the paper is silent
 * are listed in oracle.h.
 *
 * Build: gcc -std=c11 -O2 -ffp-contract=off -fopenmp -shared -fPIC oracle.c -lm
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* Linear growth factor D(a) (Sec. 3: "the D(a) function is first computed by
 * solving the ODE governing its evolution"; Sec. 4.2: built once, reused).
 * The ODE (standard linear growth of matter perturbations, dust + Lambda +
 * curvature background) in the variable a:
 *     D'' + (3/a + E'/E) D' - 3/2 Omega_m a^-5 E^-2 D = 0,
 *     E^2 = Omega_m a^-3 + Omega_k a^-2 + Omega_L,  Omega_k = 1 - Omega_m - Omega_L.
 * Initial conditions deep in matter domination: a = 1e-5, D = a, D' = 1.
 * Classical RK4 in a, with step sizes that are a fixed fraction of a
 * (geometric steps), normalised so that D(1) = 1.                             */

#define OR_A_START 1e-5
#define OR_DLOG_MAX 1e-4 /* largest step in ln a */

typedef struct { double om, ok, ol; } or_cosmo;

static double or_E2(const or_cosmo *c, double a) {
  return c->om / (a * a * a) + c->ok / (a * a) + c->ol;
}

static double or_dlnE_da(const or_cosmo *c, double a) {
  double dE2 = -3.0 * c->om / (a * a * a * a) - 2.0 * c->ok / (a * a * a);
  return dE2 / (2.0 * or_E2(c, a));
}

/* derivative of (D, V = dD/da) */
static void or_growth_rhs(const or_cosmo *c, double a, double D, double V, double *dD, double *dV) {
  *dD = V;
  *dV = -(3.0 / a + or_dlnE_da(c, a)) * V + 1.5 * c->om / (a * a * a * a * a * or_E2(c, a)) * D;
}

static void or_rk4_step(const or_cosmo *c, double a, double h, double *D, double *V) {
  double k1D, k1V, k2D, k2V, k3D, k3V, k4D, k4V;
  or_growth_rhs(c, a, *D, *V, &k1D, &k1V);
  or_growth_rhs(c, a + 0.5 * h, *D + 0.5 * h * k1D, *V + 0.5 * h * k1V, &k2D, &k2V);
  or_growth_rhs(c, a + 0.5 * h, *D + 0.5 * h * k2D, *V + 0.5 * h * k2V, &k3D, &k3V);
  or_growth_rhs(c, a + h, *D + h * k3D, *V + h * k3V, &k4D, &k4V);
  *D += h / 6.0 * (k1D + 2.0 * k2D + 2.0 * k3D + k4D);
  *V += h / 6.0 * (k1V + 2.0 * k2V + 2.0 * k3V + k4V);
}

/* advance (D, V) from a0 to a1 (> a0) in geometric sub-steps */
static void or_integrate(const or_cosmo *c, double a0, double a1, double *D, double *V) {
  if (!(a1 > a0)) return;
  int nsub = (int)ceil(log(a1 / a0) / OR_DLOG_MAX);
  if (nsub < 1) nsub = 1;
  double ratio = log(a1 / a0) / nsub;
  double a = a0;
  for (int j = 1; j <= nsub; ++j) {
    double an = (j == nsub) ? a1 : a0 * exp(ratio * j);
    or_rk4_step(c, a, an - a, D, V);
    a = an;
  }
}

static double or_growth_unnormalised(const or_cosmo *c, double a) {
  double D = OR_A_START, V = 1.0;
  or_integrate(c, OR_A_START, a, &D, &V);
  return D;
}

double or_growth_at(double omega_m, double omega_l, double a) {
  or_cosmo c = {omega_m, 1.0 - omega_m - omega_l, omega_l};
  return or_growth_unnormalised(&c, a) / or_growth_unnormalised(&c, 1.0);
}

int or_growth_table(double omega_m, double omega_l, int n_knots, double a_min, double a_max,
                    double *a_k, double *D_k) {
  if (n_knots < 2 || !(a_min > OR_A_START) || !(a_max > a_min)) return -1;
  or_cosmo c = {omega_m, 1.0 - omega_m - omega_l, omega_l};
  /* knots log-spaced in a (a reading: the paper gives no knot rule) */
  for (int k = 0; k < n_knots; ++k)
    a_k[k] = (k == n_knots - 1) ? a_max
                                : exp(log(a_min) + (log(a_max) - log(a_min)) * k / (n_knots - 1));
  double D = OR_A_START, V = 1.0, a = OR_A_START;
  for (int k = 0; k < n_knots; ++k) {
    or_integrate(&c, a, a_k[k], &D, &V);
    a = a_k[k];
    D_k[k] = D;
  }
  double D1 = or_growth_unnormalised(&c, 1.0);
  for (int k = 0; k < n_knots; ++k) D_k[k] /= D1;
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Cubic spline (Sec. 4.2: GSL cubic spline replaced by a GPU-native routine;
 * natural end conditions are the reading of "cubic spline"). The end second
 * derivatives M0, Mn are parameters; natural is M0 = Mn = 0.
 * Continuity of the first derivative at interior knots gives, for i = 1..n-2,
 *   h_{i-1} M_{i-1} + 2 (h_{i-1} + h_i) M_i + h_i M_{i+1}
 *       = 6 [ (y_{i+1} - y_i)/h_i - (y_i - y_{i-1})/h_{i-1} ],
 * solved here by plain tridiagonal elimination (Thomas algorithm).          */

int or_spline_build(int n, const double *x, const double *y, double M0, double Mn, double *M) {
  if (n < 2) return -1;
  for (int i = 0; i + 1 < n; ++i)
    if (!(x[i + 1] > x[i])) return -2;
  M[0] = M0;
  M[n - 1] = Mn;
  if (n == 2) return 0;
  int m = n - 2;
  double *sub = malloc(sizeof(double) * m), *dia = malloc(sizeof(double) * m);
  double *sup = malloc(sizeof(double) * m), *rhs = malloc(sizeof(double) * m);
  if (!sub || !dia || !sup || !rhs) { free(sub); free(dia); free(sup); free(rhs); return -3; }
  for (int i = 1; i <= n - 2; ++i) {
    double hl = x[i] - x[i - 1], hr = x[i + 1] - x[i];
    sub[i - 1] = hl;
    dia[i - 1] = 2.0 * (hl + hr);
    sup[i - 1] = hr;
    rhs[i - 1] = 6.0 * ((y[i + 1] - y[i]) / hr - (y[i] - y[i - 1]) / hl);
  }
  rhs[0] -= sub[0] * M0;
  rhs[m - 1] -= sup[m - 1] * Mn;
  for (int i = 1; i < m; ++i) { /* forward elimination */
    double w = sub[i] / dia[i - 1];
    dia[i] -= w * sup[i - 1];
    rhs[i] -= w * rhs[i - 1];
  }
  M[m] = rhs[m - 1] / dia[m - 1]; /* back substitution; M index = row + 1 */
  for (int i = m - 2; i >= 0; --i) M[i + 1] = (rhs[i] - sup[i] * M[i + 2]) / dia[i];
  free(sub); free(dia); free(sup); free(rhs);
  return 0;
}

/* interval k with x_k <= t < x_{k+1}; the last interval is closed; outside the
 * knots the end interval is used (extrapolation) */
static int or_find_interval(int n, const double *x, double t) {
  if (t < x[0]) return 0;
  if (t >= x[n - 1]) return n - 2;
  int lo = 0, hi = n - 1; /* x[lo] <= t < x[hi] */
  while (hi - lo > 1) {
    int mid = (lo + hi) / 2;
    if (x[mid] <= t) lo = mid; else hi = mid;
  }
  return lo;
}

double or_spline_eval(int n, const double *x, const double *y, const double *M, double t) {
  int k = or_find_interval(n, x, t);
  double h = x[k + 1] - x[k];
  double A = x[k + 1] - t, B = t - x[k];
  return M[k] * A * A * A / (6.0 * h) + M[k + 1] * B * B * B / (6.0 * h)
       + (y[k] / h - M[k] * h / 6.0) * A + (y[k + 1] / h - M[k + 1] * h / 6.0) * B;
}

/* ------------------------------------------------------------------------- */
/* Bilinear interpolation on a non-uniform grid (Sec. 3 / Sec. 4.3: bilinear
 * in x = l1 - l2 and y = l2 - l3). Cell by the same interval rule.          */
double or_bilinear(int nx, const double *xg, int ny, const double *yg, const double *z,
                   double x, double y) {
  int ix = or_find_interval(nx, xg, x), iy = or_find_interval(ny, yg, y);
  double tx = (x - xg[ix]) / (xg[ix + 1] - xg[ix]);
  double ty = (y - yg[iy]) / (yg[iy + 1] - yg[iy]);
  double z00 = z[ix * ny + iy], z10 = z[(ix + 1) * ny + iy];
  double z01 = z[ix * ny + iy + 1], z11 = z[(ix + 1) * ny + iy + 1];
  return (1.0 - tx) * (1.0 - ty) * z00 + tx * (1.0 - ty) * z10 + (1.0 - tx) * ty * z01 + tx * ty * z11;
}

/* ------------------------------------------------------------------------- */
/* Eigenvalues of the symmetric Hessian (Sec. 3: "a diagonalization of this
 * matrix to obtain the eigenvalues", sorted in descending order).
 * Brute force: cyclic Jacobi rotations applied as explicit matrix products
 * until the off-diagonal part vanishes.                                     */

static void or_sort3_desc(double l[3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = i + 1; j < 3; ++j)
      if (l[j] > l[i]) { double t = l[i]; l[i] = l[j]; l[j] = t; }
}

void or_eigen_jacobi(const double h[6], double lam[3]) {
  double A[3][3] = {{h[0], h[3], h[4]}, {h[3], h[1], h[5]}, {h[4], h[5], h[2]}};
  double norm2 = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) norm2 += A[i][j] * A[i][j];
  const int pairs[3][2] = {{0, 1}, {0, 2}, {1, 2}};
  for (int sweep = 0; sweep < 64; ++sweep) {
    double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
    if (off == 0.0 || off <= 1e-40 * norm2) break;
    for (int pp = 0; pp < 3; ++pp) {
      int p = pairs[pp][0], q = pairs[pp][1];
      if (A[p][q] == 0.0) continue;
      double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
      double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
      double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
      double P[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
      P[p][p] = c; P[q][q] = c; P[p][q] = s; P[q][p] = -s;
      double T[3][3], R[3][3];
      for (int i = 0; i < 3; ++i) /* T = A P */
        for (int j = 0; j < 3; ++j) {
          double acc = 0.0;
          for (int k = 0; k < 3; ++k) acc += A[i][k] * P[k][j];
          T[i][j] = acc;
        }
      for (int i = 0; i < 3; ++i) /* R = P^T T */
        for (int j = 0; j < 3; ++j) {
          double acc = 0.0;
          for (int k = 0; k < 3; ++k) acc += P[k][i] * T[k][j];
          R[i][j] = acc;
        }
      for (int i = 0; i < 3; ++i) /* symmetrise and zero the rotated pair */
        for (int j = 0; j < 3; ++j) A[i][j] = 0.5 * (R[i][j] + R[j][i]);
      A[p][q] = A[q][p] = 0.0;
    }
  }
  lam[0] = A[0][0]; lam[1] = A[1][1]; lam[2] = A[2][2];
  or_sort3_desc(lam);
}

/* Closed-form trigonometric eigenvalues (Smith 1961, CACM 4:168): kept only as
 * a cross-check of the Jacobi values. */
void or_eigen_trig(const double h[6], double lam[3]) {
  double q = (h[0] + h[1] + h[2]) / 3.0;
  double p1 = h[3] * h[3] + h[4] * h[4] + h[5] * h[5];
  double p2 = (h[0] - q) * (h[0] - q) + (h[1] - q) * (h[1] - q) + (h[2] - q) * (h[2] - q) + 2.0 * p1;
  if (p2 == 0.0) { lam[0] = lam[1] = lam[2] = q; return; }
  double p = sqrt(p2 / 6.0);
  double b00 = (h[0] - q) / p, b11 = (h[1] - q) / p, b22 = (h[2] - q) / p;
  double b01 = h[3] / p, b02 = h[4] / p, b12 = h[5] / p;
  double det = b00 * (b11 * b22 - b12 * b12) - b01 * (b01 * b22 - b12 * b02) + b02 * (b01 * b12 - b11 * b02);
  double r = det / 2.0;
  if (r < -1.0) r = -1.0;
  if (r > 1.0) r = 1.0;
  double phi = acos(r) / 3.0;
  lam[0] = q + 2.0 * p * cos(phi);
  lam[2] = q + 2.0 * p * cos(phi + 2.0 * M_PI / 3.0);
  lam[1] = 3.0 * q - lam[0] - lam[2];
}

/* ------------------------------------------------------------------------- */
/* Collapse condition (Sec. 3: "the evolution of the ellipsoid is approximated
 * using third-order LPT, leading to a non-linear algebraic formulation of the
 * collapse time in terms of the Hessian eigenvalues"). The formula is not
 * printed in the paper; the reading used (R-LPT) is stated in oracle.h.    */

void or_axis_coeffs(const double l[3], int axis, double c[4]) {
  int i = axis, j = (axis + 1) % 3, k = (axis + 2) % 3;
  c[0] = 1.0;
  c[1] = -l[i];
  c[2] = -3.0 / 7.0 * l[j] * l[k];
  c[3] = l[0] * l[1] * l[2] / 9.0 - 5.0 / 21.0 * l[i] * (l[j] * l[j] + l[k] * l[k]);
}

double or_axis_stretch(const double l[3], int axis, double D) {
  double c[4];
  or_axis_coeffs(l, axis, c);
  return c[0] + c[1] * D + c[2] * D * D + c[3] * D * D * D;
}

static int or_cmp_double(const void *a, const void *b) {
  double x = *(const double *)a, y = *(const double *)b;
  return (x > y) - (x < y);
}

/* interior critical points of c0 + c1 D + c2 D^2 + c3 D^3 (roots of the derivative) */
static int or_critical_points(const double c[4], double out[2]) {
  double qa = 3.0 * c[3], qb = 2.0 * c[2], qc = c[1];
  int n = 0;
  if (qa == 0.0) {
    if (qb != 0.0) out[n++] = -qc / qb;
    return n;
  }
  double disc = qb * qb - 4.0 * qa * qc;
  if (disc < 0.0) return 0;
  double sq = sqrt(disc);
  double qq = -0.5 * (qb + (qb >= 0.0 ? sq : -sq));
  if (qq != 0.0) {
    out[n++] = qq / qa;
    out[n++] = qc / qq;
  } else {
    out[n++] = 0.0;
  }
  return n;
}

#define OR_GRID 1024
#define OR_EDGE_TOL 1e-9

/* smallest D in (0, D_top] with A(D) <= 0 for the given axis, or 0 if none;
 * the scan stops past D_stop (diagnostic scans need only D < D_c) */
static double or_first_root(const double l[3], int axis, double D_top, double D_stop, int bisect) {
  double c[4], crit[2];
  or_axis_coeffs(l, axis, c);
  int nc = or_critical_points(c, crit);
  double nodes[OR_GRID + 2];
  int nn = 0;
  for (int k = 1; k <= OR_GRID; ++k) nodes[nn++] = D_top * k / OR_GRID;
  for (int m = 0; m < nc; ++m)
    if (crit[m] > 0.0 && crit[m] < D_top) nodes[nn++] = crit[m];
  qsort(nodes, nn, sizeof(double), or_cmp_double);
  double prev = 0.0;
  for (int m = 0; m < nn; ++m) {
    double D = nodes[m];
    if (D > D_stop) break;
    if (or_axis_stretch(l, axis, D) <= 0.0) {
      if (!bisect) return D;
      double lo = prev, hi = D; /* A(lo) > 0 >= A(hi) */
      for (int it = 0; it < 400; ++it) {
        double mid = lo + 0.5 * (hi - lo);
        if (mid <= lo || mid >= hi) break;
        if (or_axis_stretch(l, axis, mid) > 0.0) lo = mid; else hi = mid;
      }
      return hi;
    }
    prev = D;
  }
  return 0.0;
}

double or_collapse_D(const double l[3], double D_top, int *flags) {
  int f = 0;
  double lmax = fmax(fabs(l[0]), fmax(fabs(l[1]), fabs(l[2])));
  if (fabs(l[0]) <= 1e-9 * lmax) f |= OR_FLAG_SIGN0;
  double Dc = 0.0;
  if (l[0] > 0.0) {
    if (fabs(or_axis_stretch(l, 0, D_top)) <= OR_EDGE_TOL) f |= OR_FLAG_EDGE;
    Dc = or_first_root(l, 0, D_top, D_top, 1);
    if (Dc > 0.0) {
      f |= OR_FLAG_COLLAPSED;
      for (int ax = 1; ax < 3; ++ax) {
        double d = or_first_root(l, ax, D_top, Dc, 0);
        if (d > 0.0 && d < Dc) f |= OR_FLAG_AXIS23;
      }
    }
  }
  if (flags) *flags |= f;
  return Dc;
}

/* ------------------------------------------------------------------------- */
/* Tables: D(a_k) by the growth ODE and the natural spline of a(D) through
 * (D_k, a_k) (Sec. 3: "interpolated with a cubic spline to obtain its
 * inverse a(D)"; Sec. 4.2: built once and reused).                          */

int or_tables_init(or_tables *t, double omega_m, double omega_l, int n_knots, double a_min, double a_max) {
  memset(t, 0, sizeof(*t));
  t->n = n_knots;
  t->a = malloc(sizeof(double) * n_knots);
  t->D = malloc(sizeof(double) * n_knots);
  t->M = malloc(sizeof(double) * n_knots);
  if (!t->a || !t->D || !t->M) { or_tables_free(t); return -3; }
  int rc = or_growth_table(omega_m, omega_l, n_knots, a_min, a_max, t->a, t->D);
  if (rc) { or_tables_free(t); return rc; }
  rc = or_spline_build(n_knots, t->D, t->a, 0.0, 0.0, t->M);
  if (rc) { or_tables_free(t); return rc; }
  return 0;
}

void or_tables_free(or_tables *t) {
  free(t->a); free(t->D); free(t->M);
  t->a = t->D = t->M = NULL;
}

/* a(D): spline inside the table, EdS limit (a proportional to D) below it. */
double or_a_of_D(const or_tables *t, double D, int *flags) {
  if (D < t->D[0]) {
    if (flags) *flags |= OR_FLAG_EDS;
    return t->a[0] * D / t->D[0];
  }
  return or_spline_eval(t->n, t->D, t->a, t->M, D);
}

/* Collapse value of one point (Sec. 3: z_coll = 1/a_coll - 1; F = 1 + z). */
double or_F_point(const or_tables *t, const double h[6], int *flags) {
  double l[3];
  or_eigen_jacobi(h, l);
  double Dc = or_collapse_D(l, t->D[t->n - 1], flags);
  if (Dc <= 0.0) return 0.0;
  return 1.0 / or_a_of_D(t, Dc, flags);
}

/* ------------------------------------------------------------------------- */
/* One smoothing radius over all points (Sec. 4.1: each grid point loads the
 * six Hessian components, evaluates its collapse time, then updates the two
 * per-element maxima with a read/modify/write).                              */

static int or_threads(int nthreads) {
#ifdef _OPENMP
  return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
  (void)nthreads;
  return 1;
#endif
}

void or_collapse_scale(const or_tables *t, const double *hess, int64_t n, int64_t plane_stride,
                       double *F_max, int32_t *idx, int32_t scale_idx, int32_t *flags, int nthreads) {
  int nt = or_threads(nthreads);
  (void)nt;
#pragma omp parallel for schedule(dynamic, 256) num_threads(nt)
  for (int64_t p = 0; p < n; ++p) {
    double h[6];
    for (int c = 0; c < 6; ++c) h[c] = hess[c * plane_stride + p];
    int f = 0;
    double F = or_F_point(t, h, &f);
    if (F > F_max[p]) { F_max[p] = F; idx[p] = scale_idx; }
    if (flags) flags[p] = f;
  }
}

void or_collapse_scale_f32(const or_tables *t, const float *hess, int64_t n, int64_t plane_stride,
                           double *F_max, int32_t *idx, int32_t scale_idx, int32_t *flags, int nthreads) {
  int nt = or_threads(nthreads);
  (void)nt;
#pragma omp parallel for schedule(dynamic, 256) num_threads(nt)
  for (int64_t p = 0; p < n; ++p) {
    double h[6];
    for (int c = 0; c < 6; ++c) h[c] = (double)hess[c * plane_stride + p];
    int f = 0;
    double F = or_F_point(t, h, &f);
    if (F > F_max[p]) { F_max[p] = F; idx[p] = scale_idx; }
    if (flags) flags[p] = f;
  }
}

void or_F_points(const or_tables *t, const double *hess, int64_t n, int64_t plane_stride,
                 double *F, int32_t *flags, int nthreads) {
  int nt = or_threads(nthreads);
  (void)nt;
#pragma omp parallel for schedule(dynamic, 256) num_threads(nt)
  for (int64_t p = 0; p < n; ++p) {
    double h[6];
    for (int c = 0; c < 6; ++c) h[c] = hess[c * plane_stride + p];
    int f = 0;
    F[p] = or_F_point(t, h, &f);
    if (flags) flags[p] = f;
  }
}

/* ------------------------------------------------------------------------- */
/* Exact-background growth ratios (see oracle.h). State y = (D1, D1', D2, D2',
 * D3a, D3a', D3b, D3b') in the variable a, classical RK4 on the same
 * geometric steps as the linear growth factor.                              */

static void or_ratio_rhs(const or_cosmo *c, double a, const double y[8], double dy[8]) {
  double damp = 3.0 / a + or_dlnE_da(c, a);
  double w = 1.5 * c->om / (a * a * a * a * a * or_E2(c, a));
  double D1 = y[0], D2 = y[2];
  double s[4] = {0.0, -w * D1 * D1, -2.0 * w * D1 * D1 * D1, -2.0 * w * (D1 * D2 - D1 * D1 * D1)};
  for (int o = 0; o < 4; ++o) {
    dy[2 * o] = y[2 * o + 1];
    dy[2 * o + 1] = -damp * y[2 * o + 1] + w * y[2 * o] + s[o];
  }
}

static void or_ratio_rk4_step(const or_cosmo *c, double a, double h, double y[8]) {
  double k1[8], k2[8], k3[8], k4[8], t[8];
  or_ratio_rhs(c, a, y, k1);
  for (int i = 0; i < 8; ++i) t[i] = y[i] + 0.5 * h * k1[i];
  or_ratio_rhs(c, a + 0.5 * h, t, k2);
  for (int i = 0; i < 8; ++i) t[i] = y[i] + 0.5 * h * k2[i];
  or_ratio_rhs(c, a + 0.5 * h, t, k3);
  for (int i = 0; i < 8; ++i) t[i] = y[i] + h * k3[i];
  or_ratio_rhs(c, a + h, t, k4);
  for (int i = 0; i < 8; ++i) y[i] += h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
}

static void or_ratio_integrate(const or_cosmo *c, double a0, double a1, double y[8]) {
  if (!(a1 > a0)) return;
  int nsub = (int)ceil(log(a1 / a0) / OR_DLOG_MAX);
  if (nsub < 1) nsub = 1;
  double ratio = log(a1 / a0) / nsub;
  double a = a0;
  for (int j = 1; j <= nsub; ++j) {
    double an = (j == nsub) ? a1 : a0 * exp(ratio * j);
    or_ratio_rk4_step(c, a, an - a, y);
    a = an;
  }
}

int or_growth_ratios(double omega_m, double omega_l, int n_knots, double a_min, double a_max, double *a_k,
                     double *D_k, double *r2_k, double *r3a_k, double *r3b_k) {
  int rc = or_growth_table(omega_m, omega_l, n_knots, a_min, a_max, a_k, D_k);
  if (rc) return rc;
  or_cosmo c = {omega_m, 1.0 - omega_m - omega_l, omega_l};
  double a = OR_A_START;
  double y[8] = {a, 1.0, -3.0 / 7.0 * a * a, -6.0 / 7.0 * a, -1.0 / 3.0 * a * a * a, -a * a,
                 10.0 / 21.0 * a * a * a, 10.0 / 7.0 * a * a};
  for (int k = 0; k < n_knots; ++k) {
    or_ratio_integrate(&c, a, a_k[k], y);
    a = a_k[k];
    double D1 = y[0];
    r2_k[k] = y[2] / (D1 * D1);
    r3a_k[k] = y[4] / (D1 * D1 * D1);
    r3b_k[k] = y[6] / (D1 * D1 * D1);
  }
  return 0;
}

int or_ratio_tables_init(or_ratio_tables *t, double omega_m, double omega_l, int n_knots, double a_min,
                         double a_max) {
  memset(t, 0, sizeof(*t));
  int rc = or_tables_init(&t->base, omega_m, omega_l, n_knots, a_min, a_max);
  if (rc) return rc;
  for (int o = 0; o < 3; ++o) {
    t->r[o] = malloc(sizeof(double) * n_knots);
    t->Mr[o] = malloc(sizeof(double) * n_knots);
    if (!t->r[o] || !t->Mr[o]) { or_ratio_tables_free(t); return -3; }
  }
  double *a_k = malloc(sizeof(double) * n_knots), *D_k = malloc(sizeof(double) * n_knots);
  if (!a_k || !D_k) { free(a_k); free(D_k); or_ratio_tables_free(t); return -3; }
  rc = or_growth_ratios(omega_m, omega_l, n_knots, a_min, a_max, a_k, D_k, t->r[0], t->r[1], t->r[2]);
  free(a_k);
  free(D_k);
  for (int o = 0; o < 3 && !rc; ++o) rc = or_spline_build(n_knots, t->base.D, t->r[o], 0.0, 0.0, t->Mr[o]);
  if (rc) { or_ratio_tables_free(t); return rc; }
  return 0;
}

void or_ratio_tables_free(or_ratio_tables *t) {
  or_tables_free(&t->base);
  for (int o = 0; o < 3; ++o) {
    free(t->r[o]);
    free(t->Mr[o]);
    t->r[o] = t->Mr[o] = NULL;
  }
}

void or_ratios_at(const or_ratio_tables *t, double D, double r[3]) {
  static const double eds[3] = {-3.0 / 7.0, -1.0 / 3.0, 10.0 / 21.0};
  for (int o = 0; o < 3; ++o)
    r[o] = (D < t->base.D[0]) ? eds[o] : or_spline_eval(t->base.n, t->base.D, t->r[o], t->Mr[o], D);
}

double or_axis_stretch_exact(const or_ratio_tables *t, const double l[3], int axis, double D) {
  int i = axis, j = (axis + 1) % 3, k = (axis + 2) % 3;
  double r[3];
  or_ratios_at(t, D, r);
  double c3 = -r[1] / 3.0 * l[0] * l[1] * l[2] - r[2] / 2.0 * l[i] * (l[j] * l[j] + l[k] * l[k]);
  return 1.0 - l[i] * D + r[0] * l[j] * l[k] * D * D + c3 * D * D * D;
}

/* smallest D in (0, D_top] with A_1(D) <= 0: a grid scan, then bisection */
double or_collapse_D_exact(const or_ratio_tables *t, const double l[3], int *flags) {
  int f = 0;
  double D_top = t->base.D[t->base.n - 1];
  double lmax = fmax(fabs(l[0]), fmax(fabs(l[1]), fabs(l[2])));
  if (fabs(l[0]) <= 1e-9 * lmax) f |= OR_FLAG_SIGN0;
  double Dc = 0.0;
  if (l[0] > 0.0) {
    if (fabs(or_axis_stretch_exact(t, l, 0, D_top)) <= OR_EDGE_TOL) f |= OR_FLAG_EDGE;
    double prev = 0.0;
    for (int m = 1; m <= 4 * OR_GRID; ++m) {
      double D = D_top * m / (4 * OR_GRID);
      if (or_axis_stretch_exact(t, l, 0, D) <= 0.0) {
        double lo = prev, hi = D;
        for (int it = 0; it < 400; ++it) {
          double mid = lo + 0.5 * (hi - lo);
          if (mid <= lo || mid >= hi) break;
          if (or_axis_stretch_exact(t, l, 0, mid) > 0.0) lo = mid; else hi = mid;
        }
        Dc = hi;
        break;
      }
      prev = D;
    }
    if (Dc > 0.0) f |= OR_FLAG_COLLAPSED;
  }
  if (flags) *flags |= f;
  return Dc;
}

double or_F_point_exact(const or_ratio_tables *t, const double h[6], int *flags) {
  double l[3];
  or_eigen_jacobi(h, l);
  double Dc = or_collapse_D_exact(t, l, flags);
  if (Dc <= 0.0) return 0.0;
  return 1.0 / or_a_of_D(&t->base, Dc, flags);
}

void or_F_points_exact(const or_ratio_tables *t, const double *hess, int64_t n, int64_t plane_stride, double *F,
                       int32_t *flags, int nthreads) {
  int nt = or_threads(nthreads);
  (void)nt;
#pragma omp parallel for schedule(dynamic, 256) num_threads(nt)
  for (int64_t p = 0; p < n; ++p) {
    double h[6];
    for (int c = 0; c < 6; ++c) h[c] = hess[c * plane_stride + p];
    int f = 0;
    F[p] = or_F_point_exact(t, h, &f);
    if (flags) flags[p] = f;
  }
}

/* ------------------------------------------------------------------------- */
/* Tabulated collapse (Sec. 3: collapse times precomputed on a grid of
 * delta = sum l_i, x = l1 - l2, y = l2 - l3 with eigenvalues sorted
 * descending, a cubic spline along delta and bilinear interpolation in x and
 * y; Sec. 4.2: the mixed spline/bilinear scheme). The tabulated quantity is
 * read as u = 1/D_c (see oracle.h).                                          */

double or_cubic_largest_root(double b, double c, double d) {
  /* all real roots lie in [-B, B] (Cauchy bound); P is increasing right of its
   * last critical point and left of its first one */
  double B = 1.0 + fmax(fabs(b), fmax(fabs(c), fabs(d)));
  double lo = -B, hi = B;
  double disc = b * b - 3.0 * c; /* critical points of P: 3u^2 + 2bu + c = 0 */
  if (disc > 0.0) {
    double s = sqrt(disc);
    double e1 = (-b - s) / 3.0, e2 = (-b + s) / 3.0; /* local max, local min */
    double Pe2 = ((e2 + b) * e2 + c) * e2 + d;
    if (Pe2 <= 0.0) lo = e2; else hi = e1;
  }
  for (int it = 0; it < 400; ++it) {
    double mid = lo + 0.5 * (hi - lo);
    if (mid <= lo || mid >= hi) break;
    double P = ((mid + b) * mid + c) * mid + d;
    if (P < 0.0) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}

double or_tab_node_value(double delta, double x, double y) {
  double l2 = (delta - x + y) / 3.0;
  double l[3] = {l2 + x, l2, l2 - y};
  double c[4];
  or_axis_coeffs(l, 0, c); /* A_1 = 1 + c1 D + c2 D^2 + c3 D^3 -> u^3 + c1 u^2 + c2 u + c3 */
  return or_cubic_largest_root(c[1], c[2], c[3]);
}

void or_tab_free(or_tab *t) {
  free(t->dg); free(t->xg); free(t->yg); free(t->val); free(t->M);
  memset(t, 0, sizeof(*t));
}

int or_tab_init(or_tab *t, int nd, const double *dg, int nx, const double *xg, int ny, const double *yg,
                const double *val) {
  memset(t, 0, sizeof(*t));
  if (nd < 2 || nx < 2 || ny < 2) return -1;
  t->nd = nd; t->nx = nx; t->ny = ny;
  size_t nv = (size_t)nx * ny * nd;
  t->dg = malloc(sizeof(double) * nd);
  t->xg = malloc(sizeof(double) * nx);
  t->yg = malloc(sizeof(double) * ny);
  t->val = malloc(sizeof(double) * nv);
  t->M = malloc(sizeof(double) * nv);
  if (!t->dg || !t->xg || !t->yg || !t->val || !t->M) { or_tab_free(t); return -3; }
  memcpy(t->dg, dg, sizeof(double) * nd);
  memcpy(t->xg, xg, sizeof(double) * nx);
  memcpy(t->yg, yg, sizeof(double) * ny);
  memcpy(t->val, val, sizeof(double) * nv);
  for (int i = 0; i + 1 < nx; ++i) if (!(xg[i + 1] > xg[i])) { or_tab_free(t); return -2; }
  for (int i = 0; i + 1 < ny; ++i) if (!(yg[i + 1] > yg[i])) { or_tab_free(t); return -2; }
  for (size_t s = 0; s < (size_t)nx * ny; ++s) {
    int rc = or_spline_build(nd, dg, t->val + s * nd, 0.0, 0.0, t->M + s * nd);
    if (rc) { or_tab_free(t); return rc; }
  }
  return 0;
}

double or_tab_query(const or_tab *t, double delta, double x, double y) {
  int ix = or_find_interval(t->nx, t->xg, x), iy = or_find_interval(t->ny, t->yg, y);
  double z[4]; /* corners (ix, iy), (ix+1, iy), (ix, iy+1), (ix+1, iy+1) */
  for (int c = 0; c < 4; ++c) {
    size_t s = (size_t)(ix + (c & 1)) * t->ny + (iy + (c >> 1));
    z[c] = or_spline_eval(t->nd, t->dg, t->val + s * t->nd, t->M + s * t->nd, delta);
  }
  double xg2[2] = {t->xg[ix], t->xg[ix + 1]}, yg2[2] = {t->yg[iy], t->yg[iy + 1]};
  double zz[4] = {z[0], z[2], z[1], z[3]}; /* or_bilinear layout z[ix*ny + iy] */
  return or_bilinear(2, xg2, 2, yg2, zz, x, y);
}

void or_tab_query_many(const or_tab *t, const double *delta, const double *x, const double *y, int64_t m,
                       double *out, int nthreads) {
  int nt = or_threads(nthreads);
  (void)nt;
#pragma omp parallel for schedule(static) num_threads(nt)
  for (int64_t i = 0; i < m; ++i) out[i] = or_tab_query(t, delta[i], x[i], y[i]);
}

void or_spline_eval_many(int n, const double *x, const double *y, const double *M, const double *t, int64_t m,
                         double *out, int nthreads) {
  int nt = or_threads(nthreads);
  (void)nt;
#pragma omp parallel for schedule(static) num_threads(nt)
  for (int64_t i = 0; i < m; ++i) out[i] = or_spline_eval(n, x, y, M, t[i]);
}

static int or_near(double v, double edge) {
  return fabs(v - edge) <= 1e-12 * fmax(1.0, fabs(edge));
}

double or_F_tab_point(const or_tables *t, const or_tab *tab, const double h[6], int *flags) {
  double l[3];
  or_eigen_jacobi(h, l);
  int f = 0;
  double lmax = fmax(fabs(l[0]), fmax(fabs(l[1]), fabs(l[2])));
  if (fabs(l[0]) <= 1e-9 * lmax) f |= OR_FLAG_SIGN0;
  double F = 0.0;
  if (l[0] > 0.0) {
    double delta = l[0] + l[1] + l[2], x = l[0] - l[1], y = l[1] - l[2];
    double D_top = t->D[t->n - 1];
    int inside = delta >= tab->dg[0] && delta <= tab->dg[tab->nd - 1] && x <= tab->xg[tab->nx - 1] &&
                 y <= tab->yg[tab->ny - 1] && x >= tab->xg[0] && y >= tab->yg[0];
    /* on a face of the hull either side is a valid answer; x and y are >= 0,
     * so a face at x = 0 or y = 0 has no outside */
    if (or_near(delta, tab->dg[0]) || or_near(delta, tab->dg[tab->nd - 1]) ||
        or_near(x, tab->xg[tab->nx - 1]) || or_near(y, tab->yg[tab->ny - 1]) ||
        (tab->xg[0] > 0.0 && or_near(x, tab->xg[0])) || (tab->yg[0] > 0.0 && or_near(y, tab->yg[0])))
      f |= OR_FLAG_HULL_EDGE;
    double Dc = 0.0;
    if (inside) {
      double u = or_tab_query(tab, delta, x, y);
      if (u > 0.0) {
        Dc = 1.0 / u;
        if (fabs(Dc - D_top) <= 1e-9 * D_top) f |= OR_FLAG_EDGE;
        if (Dc > D_top) Dc = 0.0;
      }
    } else {
      f |= OR_FLAG_HULL_OUT;
      Dc = or_collapse_D(l, D_top, &f);
    }
    if (Dc > 0.0) {
      f |= OR_FLAG_COLLAPSED;
      F = 1.0 / or_a_of_D(t, Dc, &f);
    }
  }
  if (flags) *flags |= f;
  return F;
}

void or_F_tab_points(const or_tables *t, const or_tab *tab, const double *hess, int64_t n, int64_t plane_stride,
                     double *F, int32_t *flags, int nthreads) {
  int nt = or_threads(nthreads);
  (void)nt;
#pragma omp parallel for schedule(dynamic, 256) num_threads(nt)
  for (int64_t p = 0; p < n; ++p) {
    double h[6];
    for (int c = 0; c < 6; ++c) h[c] = hess[c * plane_stride + p];
    int f = 0;
    F[p] = or_F_tab_point(t, tab, h, &f);
    if (flags) flags[p] = f;
  }
}

void or_tab_node_values(int nd, const double *dg, int nx, const double *xg, int ny, const double *yg,
                        double *out) {
#pragma omp parallel for schedule(static)
  for (int ix = 0; ix < nx; ++ix)
    for (int iy = 0; iy < ny; ++iy)
      for (int k = 0; k < nd; ++k)
        out[((size_t)ix * ny + iy) * nd + k] = or_tab_node_value(dg[k], xg[ix], yg[iy]);
}

/* ------------------------------------------------------------------------- */
/* MLP surrogate reference (FP64, plain loops). No counterpart in the paper. */

static double or_silu(double v) { return v / (1.0 + exp(-v)); }
static double or_dsilu(double v) {
  double s = 1.0 / (1.0 + exp(-v));
  return s * (1.0 + v * (1.0 - s));
}

typedef struct {
  const double *W1, *b1, *W2, *b2, *W3, *b3, *W4, *b4;
} or_mlp_view;

static or_mlp_view or_mlp_split(const double *p) {
  or_mlp_view v;
  v.W1 = p; p += 3 * OR_MLP_H;
  v.b1 = p; p += OR_MLP_H;
  v.W2 = p; p += OR_MLP_H * OR_MLP_H;
  v.b2 = p; p += OR_MLP_H;
  v.W3 = p; p += OR_MLP_H * OR_MLP_H;
  v.b3 = p; p += OR_MLP_H;
  v.W4 = p; p += OR_MLP_H;
  v.b4 = p;
  return v;
}

/* forward pass keeping pre-activations u1..u3 and activations a1..a3 */
static double or_mlp_fwd(const or_mlp_view *m, const double z[3], double *u1, double *a1, double *u2, double *a2,
                         double *u3, double *a3) {
  for (int j = 0; j < OR_MLP_H; ++j) {
    double s = m->b1[j];
    for (int i = 0; i < 3; ++i) s += z[i] * m->W1[i * OR_MLP_H + j];
    u1[j] = s; a1[j] = or_silu(s);
  }
  for (int j = 0; j < OR_MLP_H; ++j) {
    double s = m->b2[j];
    for (int i = 0; i < OR_MLP_H; ++i) s += a1[i] * m->W2[i * OR_MLP_H + j];
    u2[j] = s; a2[j] = or_silu(s);
  }
  for (int j = 0; j < OR_MLP_H; ++j) {
    double s = m->b3[j];
    for (int i = 0; i < OR_MLP_H; ++i) s += a2[i] * m->W3[i * OR_MLP_H + j];
    u3[j] = s; a3[j] = or_silu(s);
  }
  double f = m->b4[0];
  for (int i = 0; i < OR_MLP_H; ++i) f += a3[i] * m->W4[i];
  return f;
}

double or_mlp_forward(const double *params, const double z[3]) {
  or_mlp_view m = or_mlp_split(params);
  double u1[OR_MLP_H], a1[OR_MLP_H], u2[OR_MLP_H], a2[OR_MLP_H], u3[OR_MLP_H], a3[OR_MLP_H];
  return or_mlp_fwd(&m, z, u1, a1, u2, a2, u3, a3);
}

double or_mlp_loss_grad(const double *params, const double *z, const double *t, int n, double *grad) {
  or_mlp_view m = or_mlp_split(params);
  memset(grad, 0, sizeof(double) * OR_MLP_NPARAM);
  double *gW1 = grad, *gb1 = gW1 + 3 * OR_MLP_H, *gW2 = gb1 + OR_MLP_H, *gb2 = gW2 + OR_MLP_H * OR_MLP_H;
  double *gW3 = gb2 + OR_MLP_H, *gb3 = gW3 + OR_MLP_H * OR_MLP_H, *gW4 = gb3 + OR_MLP_H, *gb4 = gW4 + OR_MLP_H;
  double loss = 0.0;
  for (int s = 0; s < n; ++s) {
    double u1[OR_MLP_H], a1[OR_MLP_H], u2[OR_MLP_H], a2[OR_MLP_H], u3[OR_MLP_H], a3[OR_MLP_H];
    const double *zs = z + 3 * s;
    double f = or_mlp_fwd(&m, zs, u1, a1, u2, a2, u3, a3);
    double r = f - t[s];
    loss += r * r;
    double df = 2.0 * r / n;
    double d3[OR_MLP_H], d2[OR_MLP_H], d1[OR_MLP_H];
    gb4[0] += df;
    for (int i = 0; i < OR_MLP_H; ++i) {
      gW4[i] += a3[i] * df;
      d3[i] = df * m.W4[i] * or_dsilu(u3[i]);
    }
    for (int j = 0; j < OR_MLP_H; ++j) gb3[j] += d3[j];
    for (int i = 0; i < OR_MLP_H; ++i) {
      double acc = 0.0;
      for (int j = 0; j < OR_MLP_H; ++j) {
        gW3[i * OR_MLP_H + j] += a2[i] * d3[j];
        acc += m.W3[i * OR_MLP_H + j] * d3[j];
      }
      d2[i] = acc * or_dsilu(u2[i]);
    }
    for (int j = 0; j < OR_MLP_H; ++j) gb2[j] += d2[j];
    for (int i = 0; i < OR_MLP_H; ++i) {
      double acc = 0.0;
      for (int j = 0; j < OR_MLP_H; ++j) {
        gW2[i * OR_MLP_H + j] += a1[i] * d2[j];
        acc += m.W2[i * OR_MLP_H + j] * d2[j];
      }
      d1[i] = acc * or_dsilu(u1[i]);
    }
    for (int j = 0; j < OR_MLP_H; ++j) gb1[j] += d1[j];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < OR_MLP_H; ++j) gW1[i * OR_MLP_H + j] += zs[i] * d1[j];
  }
  return loss / n;
}
