// cc_tables.cpp -- host-side FP64 tables of libcollapse.
//
// The linear growth factor D(a) is the solution of the growth ODE (Sec. 3:
// "the D(a) function is first computed by solving the ODE governing its
// evolution, then interpolated with a cubic spline to obtain its inverse
// a(D)"); the spline is built once on the host and copied to the device once
// (Sec. 4.2). This file solves the ODE in the variable x = ln a for the state
// (D, dD/dx):
//     D_xx + (2 + dlnE/dx) D_x - 3/2 Omega_m(a) D = 0,
//     Omega_m(a) = Omega_m a^-3 / E^2,
// with classical RK4 on a uniform grid in x, from the matter-dominated growing
// mode D = a, D_x = a at a = 1e-5, normalised so that D(1) = 1. The natural
// cubic spline of a(D) through (D_k, a_k) is stored as per-interval
// polynomials in t = D - D_k for Horner evaluation on the device.
// growth_ratios_into adds the second- and third-order growth factors of the
// same background (the collapse condition with exact growth ratios).
#include "cc_internal.h"

#include <cmath>
#include <cstring>
#include <vector>

namespace cc {

namespace {

struct Background {
  double om, ok, ol;
  double E2(double a) const { return om / (a * a * a) + ok / (a * a) + ol; }
  // d ln E / d ln a
  double dlnE(double a) const {
    return (-3.0 * om / (a * a * a) - 2.0 * ok / (a * a)) / (2.0 * E2(a));
  }
  double om_a(double a) const { return om / (a * a * a) / E2(a); }
};

constexpr double kAStart = 1e-5;
constexpr double kMaxStep = 5e-5;  // largest RK4 step in ln a

// y = (D, D_x); returns dy/dx at x = ln a
inline void rhs(const Background& bg, double x, const double y[2], double dy[2]) {
  const double a = std::exp(x);
  dy[0] = y[1];
  dy[1] = -(2.0 + bg.dlnE(a)) * y[1] + 1.5 * bg.om_a(a) * y[0];
}

// advance y from x0 to x1 with uniform RK4 steps no longer than kMaxStep
void advance(const Background& bg, double x0, double x1, double y[2]) {
  if (!(x1 > x0)) return;
  const long steps = static_cast<long>(std::ceil((x1 - x0) / kMaxStep));
  const double h = (x1 - x0) / static_cast<double>(steps);
  for (long s = 0; s < steps; ++s) {
    const double x = x0 + h * static_cast<double>(s);
    double k1[2], k2[2], k3[2], k4[2], t[2];
    rhs(bg, x, y, k1);
    for (int i = 0; i < 2; ++i) t[i] = y[i] + 0.5 * h * k1[i];
    rhs(bg, x + 0.5 * h, t, k2);
    for (int i = 0; i < 2; ++i) t[i] = y[i] + 0.5 * h * k2[i];
    rhs(bg, x + 0.5 * h, t, k3);
    for (int i = 0; i < 2; ++i) t[i] = y[i] + h * k3[i];
    rhs(bg, x + h, t, k4);
    for (int i = 0; i < 2; ++i) y[i] += h * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]) / 6.0;
  }
}

}  // namespace

int growth_table_into(const cc_cosmology& c, double* a_k, double* D_k) {
  const int n = c.n_knots;
  if (n < 2 || n > kMaxKnots || !(c.a_min > kAStart) || !(c.a_max > c.a_min) ||
      !std::isfinite(c.omega_m) || !std::isfinite(c.omega_l) || !(c.omega_m > 0.0))
    return CC_EINVAL;
  Background bg{c.omega_m, 1.0 - c.omega_m - c.omega_l, c.omega_l};
  const double xlo = std::log(c.a_min), xhi = std::log(c.a_max);
  double y[2] = {kAStart, kAStart};
  double x = std::log(kAStart);
  for (int k = 0; k < n; ++k) {
    const double xk = (k == n - 1) ? xhi : xlo + (xhi - xlo) * k / (n - 1);
    advance(bg, x, xk, y);
    x = xk;
    a_k[k] = (k == n - 1) ? c.a_max : std::exp(xk);
    D_k[k] = y[0];
  }
  // normalisation D(a = 1) = 1
  double y1[2] = {kAStart, kAStart};
  advance(bg, std::log(kAStart), 0.0, y1);
  for (int k = 0; k < n; ++k) D_k[k] /= y1[0];
  for (int k = 0; k + 1 < n; ++k)
    if (!(D_k[k + 1] > D_k[k]) || !std::isfinite(D_k[k])) return CC_ERANGE;
  return CC_OK;
}

namespace {

// Second- and third-order growth in x = ln a, state
// y = (D1, D1_x, D2, D2_x, D3a, D3a_x, D3b, D3b_x):
//   f_xx + (2 + dlnE/dx) f_x - 3/2 Omega_m(a) f = s,
//   s = 0, -3/2 Om(a) D1^2, -3 Om(a) D1^3, -3 Om(a) (D1 D2 - D1^3)
// (the equations of D1 with the second- and third-order sources; their EdS
// solutions are D2 = -3/7 D1^2, D3a = -1/3 D1^3, D3b = 10/21 D1^3).
inline void rhs8(const Background& bg, double x, const double y[8], double dy[8]) {
  const double a = std::exp(x);
  const double damp = 2.0 + bg.dlnE(a), w = 1.5 * bg.om_a(a);
  const double D1 = y[0], D2 = y[2];
  const double src[4] = {0.0, -w * D1 * D1, -2.0 * w * D1 * D1 * D1, -2.0 * w * (D1 * D2 - D1 * D1 * D1)};
  for (int o = 0; o < 4; ++o) {
    dy[2 * o] = y[2 * o + 1];
    dy[2 * o + 1] = -damp * y[2 * o + 1] + w * y[2 * o] + src[o];
  }
}

void advance8(const Background& bg, double x0, double x1, double y[8]) {
  if (!(x1 > x0)) return;
  const long steps = static_cast<long>(std::ceil((x1 - x0) / kMaxStep));
  const double h = (x1 - x0) / static_cast<double>(steps);
  for (long s = 0; s < steps; ++s) {
    const double x = x0 + h * static_cast<double>(s);
    double k1[8], k2[8], k3[8], k4[8], t[8];
    rhs8(bg, x, y, k1);
    for (int i = 0; i < 8; ++i) t[i] = y[i] + 0.5 * h * k1[i];
    rhs8(bg, x + 0.5 * h, t, k2);
    for (int i = 0; i < 8; ++i) t[i] = y[i] + 0.5 * h * k2[i];
    rhs8(bg, x + 0.5 * h, t, k3);
    for (int i = 0; i < 8; ++i) t[i] = y[i] + h * k3[i];
    rhs8(bg, x + h, t, k4);
    for (int i = 0; i < 8; ++i) y[i] += h * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]) / 6.0;
  }
}

}  // namespace

int growth_ratios_into(const cc_cosmology& c, double* r2, double* r3a, double* r3b) {
  const int n = c.n_knots;
  if (n < 2 || n > kMaxKnots || !(c.a_min > kAStart) || !(c.a_max > c.a_min) ||
      !std::isfinite(c.omega_m) || !std::isfinite(c.omega_l) || !(c.omega_m > 0.0))
    return CC_EINVAL;
  Background bg{c.omega_m, 1.0 - c.omega_m - c.omega_l, c.omega_l};
  const double xlo = std::log(c.a_min), xhi = std::log(c.a_max);
  const double a0 = kAStart;
  double y[8] = {a0, a0, -3.0 / 7.0 * a0 * a0, -6.0 / 7.0 * a0 * a0, -1.0 / 3.0 * a0 * a0 * a0, -a0 * a0 * a0,
                 10.0 / 21.0 * a0 * a0 * a0, 10.0 / 7.0 * a0 * a0 * a0};
  double x = std::log(kAStart);
  for (int k = 0; k < n; ++k) {
    const double xk = (k == n - 1) ? xhi : xlo + (xhi - xlo) * k / (n - 1);
    advance8(bg, x, xk, y);
    x = xk;
    const double D1 = y[0];
    r2[k] = y[2] / (D1 * D1);
    r3a[k] = y[4] / (D1 * D1 * D1);
    r3b[k] = y[6] / (D1 * D1 * D1);
    if (!std::isfinite(r2[k]) || !std::isfinite(r3a[k]) || !std::isfinite(r3b[k])) return CC_ERANGE;
  }
  return CC_OK;
}

int build_growth_table(const cc_cosmology& c, std::vector<double>& a_k, std::vector<double>& D_k) {
  if (c.n_knots < 2 || c.n_knots > kMaxKnots) return CC_EINVAL;
  a_k.resize(c.n_knots);
  D_k.resize(c.n_knots);
  return growth_table_into(c, a_k.data(), D_k.data());
}

// Natural cubic spline y(x) through (x_k, y_k): solve for the knot slopes'
// second derivatives s_k (s_0 = s_{n-1} = 0) of the tridiagonal system
//   (x_k - x_{k-1}) s_{k-1} + 2 (x_{k+1} - x_{k-1}) s_k + (x_{k+1} - x_k) s_{k+1}
//       = 6 (slope_k - slope_{k-1}),
// then expand interval k as y_k + b t + c t^2 + d t^3, t = x - x_k.
int natural_spline_into(int n, const double* x, const double* y, double* coef, double* work) {
  if (n < 2) return CC_EINVAL;
  // work: h, slope (n - 1 each), s (n), diag, upper, rhs (n - 2 each)
  double* h = work;
  double* slope = h + (n - 1);
  double* s = slope + (n - 1);
  double* diag = s + n;
  double* upper = diag + (n - 2 > 0 ? n - 2 : 0);
  double* rhs = upper + (n - 2 > 0 ? n - 2 : 0);
  for (int k = 0; k < n; ++k) s[k] = 0.0;
  for (int k = 0; k + 1 < n; ++k) {
    h[k] = x[k + 1] - x[k];
    if (!(h[k] > 0.0)) return CC_EINVAL;
    slope[k] = (y[k + 1] - y[k]) / h[k];
  }
  if (n > 2) {
    const int m = n - 2;  // unknowns s_1 .. s_{n-2}
    for (int i = 0; i < m; ++i) {
      diag[i] = 2.0 * (h[i] + h[i + 1]);
      upper[i] = h[i + 1];
      rhs[i] = 6.0 * (slope[i + 1] - slope[i]);
    }
    // elimination of the sub-diagonal h[i] of row i against row i-1
    for (int i = 1; i < m; ++i) {
      const double f = h[i] / diag[i - 1];
      diag[i] -= f * upper[i - 1];
      rhs[i] -= f * rhs[i - 1];
    }
    s[m] = rhs[m - 1] / diag[m - 1];
    for (int i = m - 2; i >= 0; --i) s[i + 1] = (rhs[i] - upper[i] * s[i + 2]) / diag[i];
  }
  for (int k = 0; k + 1 < n; ++k) {
    coef[4 * k + 0] = y[k];
    coef[4 * k + 1] = slope[k] - h[k] * (2.0 * s[k] + s[k + 1]) / 6.0;
    coef[4 * k + 2] = 0.5 * s[k];
    coef[4 * k + 3] = (s[k + 1] - s[k]) / (6.0 * h[k]);
  }
  return CC_OK;
}

int f32_knots_within_factor2(int n, const double* x) {
  for (int k = 0; k + 1 < n; ++k) {
    const double e0 = static_cast<double>(static_cast<float>(x[k]));
    const double e1 = static_cast<double>(static_cast<float>(x[k + 1]));
    if (!(e0 > 0.0) || !(e1 > e0) || !(e1 <= 2.0 * e0)) return CC_EINVAL;
  }
  return CC_OK;
}

void expand_about_f32_knots(int n, const double* x, double* coef) {
  for (int k = 0; k + 1 < n; ++k) {
    double* c = coef + 4 * k;
    const double d = static_cast<double>(static_cast<float>(x[k])) - x[k];
    const double c0 = c[0], c1 = c[1], c2 = c[2], c3 = c[3];
    c[0] = c0 + d * (c1 + d * (c2 + d * c3));
    c[1] = c1 + d * (2.0 * c2 + 3.0 * d * c3);
    c[2] = c2 + 3.0 * d * c3;
  }
}

int bit_buckets_into(int n, const float* xf, int max_nb, unsigned short* bucket, int* nb_out, int* shift_out,
                     unsigned* b0_out) {
  // positive FP32 numbers order like their bit patterns, so bucket
  // b = (bits(x) - bits(x_0)) >> shift is exact: pick the largest shift
  // (fewest buckets) at which no bucket holds more than two of the knots a
  // search can step to (x_1 .. x_{n-2})
  std::vector<uint32_t> kb(n);
  for (int k = 0; k < n; ++k) std::memcpy(&kb[k], &xf[k], sizeof(uint32_t));
  const uint32_t b0 = kb[0], range = kb[n - 1] - kb[0];
  for (int shift = 31; shift >= 0; --shift) {
    const int64_t nb = static_cast<int64_t>(range >> shift) + 1;
    if (nb > max_nb) break;  // finer shifts only add buckets
    int worst = 0, run = 0;
    int64_t cur = -1;
    for (int k = 1; k <= n - 2; ++k) {
      const int64_t b = static_cast<int64_t>((kb[k] - b0) >> shift);
      run = (b == cur) ? run + 1 : 1;
      cur = b;
      worst = run > worst ? run : worst;
    }
    if (worst > 2) continue;
    int k = 0;
    for (int64_t i = 0; i < nb; ++i) {
      const uint64_t edge = static_cast<uint64_t>(b0) + (static_cast<uint64_t>(i) << shift);
      while (k + 1 <= n - 2 && kb[k + 1] <= edge) ++k;
      bucket[i] = static_cast<unsigned short>(k);
    }
    *nb_out = static_cast<int>(nb);
    *shift_out = shift;
    *b0_out = b0;
    return CC_OK;
  }
  return CC_EINVAL;
}

int build_natural_spline(const std::vector<double>& x, const std::vector<double>& y,
                         std::vector<double>& coef /* 4 per interval */) {
  const int n = static_cast<int>(x.size());
  if (n < 2) return CC_EINVAL;
  std::vector<double> work(6 * static_cast<size_t>(n));
  coef.resize(4 * static_cast<size_t>(n - 1));
  return natural_spline_into(n, x.data(), y.data(), coef.data(), work.data());
}

}  // namespace cc
