/* oracle.h -- plain FP64 CPU oracle of the collapse-time hot path.
 *
 * TEST INFRASTRUCTURE. This library is the slow, obviously correct statement
 * of what the GPU path computes. Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline / reference legs of bench.py may load or call it. It shares no
 * code with the CUDA library (paper_2510_02873_gb300/csrc), and neither
 * includes nor links the other.
 *
 * Paper: Lepinzan et al., "Accelerating cosmological simulations on GPUs: a
 * portable approach using OpenMP" (arXiv:2510.02873). Section 3 describes the
 * computation: per grid point and smoothing radius, the Hessian of the
 * smoothed potential is diagonalised, a third-order LPT ellipsoidal collapse
 * condition gives the growth factor at collapse, and the inverse growth
 * function a(D), a cubic spline through the ODE solution D(a), maps it to the
 * collapse scale factor; Sec. 4.1 adds the per-element maxima update.
 *
 * Readings of the paper (it does not print the collapse condition; see the
 * repository's design notes for the full list):
 *   - eigenvalues sorted descending, lambda1 >= lambda2 >= lambda3 (Sec. 3);
 *   - axis stretch (R-LPT: local third-order LPT with EdS growth ratios
 *     D2 = -3/7 D^2, D3a = -1/3 D^3, D3b = 10/21 D^3):
 *       A_i(D) = 1 - D l_i - 3/7 D^2 l_j l_k
 *                + D^3 [ l1 l2 l3 / 9 - 5/21 l_i (l_j^2 + l_k^2) ]
 *   - collapse growth factor D_c = smallest root of A_1 in (0, D_top];
 *     lambda1 <= 0 or no such root: no collapse, F = 0. For sorted
 *     eigenvalues with lambda1 > 0, A_1 is strictly decreasing on D > 0 (a
 *     positive D^2 coefficient needs l2 l3 < 0, and then c2^2 < 3 |c3| l1), so
 *     the root is unique and never tangent;
 *   - a_c from a natural cubic spline through (D(a_k), a_k); below the first
 *     knot a_c = a_0 D_c / D_0 (EdS limit); F = 1/a_c = 1 + z_c;
 *   - running maximum over radii with a strict '>' (ties keep the earlier
 *     radius), F_max starts at 0 and idx at -1.
 *
 * Pins (tests/test_oracle_pins.py): spherical limit against the textbook
 * Lagrangian and Eulerian 3LPT series; plane wave against Zel'dovich; the
 * 2LPT density of the product A_1 A_2 A_3; symmetry and homogeneity of the
 * stretch; uniqueness of the collapse root; Jacobi against LAPACK and known
 * spectra; spline exactness (knots, lines, cubics with true end curvature) and
 * agreement with SciPy's natural spline; bilinear exactness; the growth ODE
 * against the Heath integral and the EdS solution; brute force on 8^3 x 3.
 *
 * Third-order pins: the stretches satisfy the Einstein-de Sitter Lagrangian
 * equation of motion of a homogeneous ellipsoid to third order in D, which
 * fixes the trace of each order (at third order the textbook 3LPT divergence
 * (1/3) mu3 - (10/21) mu2(phi1, phi2)); and they equal the eigenvalues of the
 * deformation tensor built in any frame from H, its cofactor matrix and the
 * mixed cofactor of H and adj(H) (the local split, stated without eigenvalues).
 *
 * PARITY UNPINNED (partially): the choice of the local split in
 * or_axis_coeffs. The equation of motion fixes only the trace of each order;
 * which share of it each axis takes (here the cofactor rule: axis i receives
 * the principal minor of the other two axes) is the reading. Monaco et al.
 * 2002 may instead use ellipsoid shape factors; that source is not available,
 * so nothing outside the reading fixes the per-axis distribution.
 */
#ifndef COLLAPSE_ORACLE_H
#define COLLAPSE_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Per-evaluation diagnostic flags (bit mask). */
#define OR_FLAG_COLLAPSED   1  /* a root was found in (0, D_top]                    */
#define OR_FLAG_EDGE        4  /* |A_1(D_top)| <= 1e-9: collapse by a_max ambiguous    */
#define OR_FLAG_SIGN0       8  /* |lambda1| <= 1e-9 * max|lambda|: lambda1>0 test ambiguous */
#define OR_FLAG_EDS        16  /* D_c below the first knot: EdS limit used             */
#define OR_FLAG_AXIS23     32  /* A_2 or A_3 crosses zero before A_1 does (diagnostic) */
#define OR_FLAG_HULL_OUT   64  /* tabulated: outside the table, R-LPT used instead        */
#define OR_FLAG_HULL_EDGE 128  /* tabulated: within 1e-12 of the table's hull (either side valid) */

/* ---- linear growth factor (Sec. 3, Sec. 4.2) ---- */
int or_growth_table(double omega_m, double omega_l, int n_knots, double a_min, double a_max,
                    double *a_k, double *D_k);
double or_growth_at(double omega_m, double omega_l, double a); /* D(a)/D(1), same integrator */

/* ---- cubic spline with prescribed end second derivatives (natural: 0, 0) ---- */
int or_spline_build(int n, const double *x, const double *y, double M0, double Mn, double *M);
double or_spline_eval(int n, const double *x, const double *y, const double *M, double t);
/* the same at m points t (OpenMP over the points; nthreads <= 0: all) */
void or_spline_eval_many(int n, const double *x, const double *y, const double *M, const double *t, int64_t m,
                         double *out, int nthreads);

/* ---- bilinear interpolation on a non-uniform grid, z[ix*ny + iy] ---- */
double or_bilinear(int nx, const double *xg, int ny, const double *yg, const double *z,
                   double x, double y);

/* ---- symmetric 3x3 eigenvalues, h = (xx, yy, zz, xy, xz, yz), sorted descending ---- */
void or_eigen_jacobi(const double h[6], double lam[3]);
void or_eigen_trig(const double h[6], double lam[3]);

/* ---- collapse condition ---- */
double or_axis_stretch(const double l[3], int axis, double D);        /* A_axis(D), axis 0..2 */
void   or_axis_coeffs(const double l[3], int axis, double c[4]);      /* A = c0 + c1 D + c2 D^2 + c3 D^3 */
double or_collapse_D(const double l[3], double D_top, int *flags);    /* D_c or 0 when none   */

/* ---- tables and the per-point collapse value ---- */
typedef struct {
  int n;            /* knots */
  double *a;        /* a_k, increasing */
  double *D;        /* D(a_k), increasing */
  double *M;        /* second derivatives of a(D) at the knots (natural) */
} or_tables;

int  or_tables_init(or_tables *t, double omega_m, double omega_l, int n_knots, double a_min, double a_max);
void or_tables_free(or_tables *t);
double or_a_of_D(const or_tables *t, double D, int *flags);           /* spline + EdS branch */
double or_F_point(const or_tables *t, const double h[6], int *flags); /* F = 1/a_c or 0 */

/* One radius over n points: hess = 6 planes, component c of point p at hess[c*plane_stride + p].
 * Updates F_max/idx with a strict '>' and writes per-point flags (may be NULL).
 * nthreads <= 0: all OpenMP threads. */
void or_collapse_scale(const or_tables *t, const double *hess, int64_t n, int64_t plane_stride,
                       double *F_max, int32_t *idx, int32_t scale_idx, int32_t *flags, int nthreads);

/* Same, for FP32 planes (the values are widened exactly to FP64 first). */
void or_collapse_scale_f32(const or_tables *t, const float *hess, int64_t n, int64_t plane_stride,
                           double *F_max, int32_t *idx, int32_t scale_idx, int32_t *flags, int nthreads);

/* F of each point (no max), with flags. */
void or_F_points(const or_tables *t, const double *hess, int64_t n, int64_t plane_stride,
                 double *F, int32_t *flags, int nthreads);

/* ---- exact-background growth ratios (a reading beyond the paper: the
 * EdS ratios of the R-LPT condition replaced by the second- and third-order
 * growth factors of the actual background) ----
 * With D1 the linear growth factor and w(a) = 3/2 Omega_m a^-5 E^-2, every
 * order solves f'' + (3/a + E'/E) f' - w f = s(a):
 *   D2:  s = -w D1^2,  D3a: s = -2 w D1^3,  D3b: s = -2 w (D1 D2 - D1^3),
 * from EdS initial conditions at a = 1e-5 (D1 = a, D2 = -3/7 a^2,
 * D3a = -1/3 a^3, D3b = 10/21 a^3), which these sources keep exactly in EdS.
 * The ratios r2 = D2/D1^2, r3a = D3a/D1^3, r3b = D3b/D1^3 (independent of the
 * normalisation of D1) enter the stretch as
 *   A_i = 1 - D l_i + r2 D^2 l_j l_k + D^3 [-r3a/3 l1 l2 l3 - r3b/2 l_i (l_j^2 + l_k^2)],
 * which is the R-LPT A_i for the EdS values (-3/7, -1/3, 10/21). */
int or_growth_ratios(double omega_m, double omega_l, int n_knots, double a_min, double a_max, double *a_k,
                     double *D_k, double *r2_k, double *r3a_k, double *r3b_k);

typedef struct {
  or_tables base;        /* D(a) and a(D) as in the classic path */
  double *r[3];          /* r2, r3a, r3b at the knots D_k */
  double *Mr[3];         /* natural-spline second derivatives of r(D) */
} or_ratio_tables;

int  or_ratio_tables_init(or_ratio_tables *t, double omega_m, double omega_l, int n_knots, double a_min,
                          double a_max);
void or_ratio_tables_free(or_ratio_tables *t);
/* r2, r3a, r3b at D (natural splines in D over the knots; EdS values below the first knot) */
void or_ratios_at(const or_ratio_tables *t, double D, double r[3]);
double or_axis_stretch_exact(const or_ratio_tables *t, const double l[3], int axis, double D);
double or_collapse_D_exact(const or_ratio_tables *t, const double l[3], int *flags);
double or_F_point_exact(const or_ratio_tables *t, const double h[6], int *flags);
void or_F_points_exact(const or_ratio_tables *t, const double *hess, int64_t n, int64_t plane_stride, double *F,
                       int32_t *flags, int nthreads);

/* ---- tabulated collapse (Sec. 3 "Tabulated" option; Sec. 4.2 spline x bilinear) ----
 * Reading: the table holds u = 1/D_c, the largest real root of the monic
 * cubic u^3 - l1 u^2 + c2 u + c3 (finite everywhere, ~linear in (delta, x, y)),
 * on non-uniform axes delta (nd), x = l1 - l2 (nx), y = l2 - l3 (ny);
 * val[(ix * ny + iy) * nd + k]. A query splines delta (natural cubic) at the
 * four (x, y) corners of its cell and blends them bilinearly. Outside the
 * table the R-LPT root is used. */
double or_cubic_largest_root(double b, double c, double d); /* of u^3 + b u^2 + c u + d */
double or_tab_node_value(double delta, double x, double y);  /* u at a node, eigenvalues from (delta, x, y) */
void or_tab_node_values(int nd, const double *dg, int nx, const double *xg, int ny, const double *yg,
                        double *out); /* every node, layout [ix][iy][k] */

typedef struct {
  int nd, nx, ny;
  double *dg, *xg, *yg;  /* axes */
  double *val, *M;       /* values and natural-spline second derivatives along delta */
} or_tab;

int  or_tab_init(or_tab *t, int nd, const double *dg, int nx, const double *xg, int ny, const double *yg,
                 const double *val);
void or_tab_free(or_tab *t);
double or_tab_query(const or_tab *t, double delta, double x, double y);
/* the same at m points (OpenMP over the points; nthreads <= 0: all) */
void or_tab_query_many(const or_tab *t, const double *delta, const double *x, const double *y, int64_t m,
                       double *out, int nthreads);
double or_F_tab_point(const or_tables *t, const or_tab *tab, const double h[6], int *flags);
void or_F_tab_points(const or_tables *t, const or_tab *tab, const double *hess, int64_t n, int64_t plane_stride,
                     double *F, int32_t *flags, int nthreads);

/* ---- learned surrogate: MLP 3-64-64-64-1 with SiLU, FP64 (gradient reference) ----
 * f(z) = W4 . s(W3 s(W2 s(W1 z + b1) + b2) + b3) + b4, s(v) = v / (1 + exp(-v)),
 * z = (l1, l2, l3) / sigma, f ~ log(D_c sigma). Parameters flattened as
 * W1[3][64], b1[64], W2[64][64], b2[64], W3[64][64], b3[64], W4[64], b4
 * (W[in][out]). Loss = mean (f(z_i) - t_i)^2. No counterpart in the paper:
 * this checks the GPU training kernels. */
#define OR_MLP_H 64
#define OR_MLP_NPARAM (3 * 64 + 64 + 64 * 64 + 64 + 64 * 64 + 64 + 64 + 1)
double or_mlp_forward(const double *params, const double z[3]);
double or_mlp_loss_grad(const double *params, const double *z, const double *t, int n, double *grad);

#ifdef __cplusplus
}
#endif
#endif
