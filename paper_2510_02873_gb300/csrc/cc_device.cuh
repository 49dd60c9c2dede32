// cc_device.cuh -- device arithmetic of the collapse-time path.
//
// Per point (arXiv:2510.02873, Sec. 3): eigenvalues of the symmetric 3x3
// Hessian (closed-form trigonometric solve, sorted descending), the
// third-order LPT collapse condition solved for the growth factor at
// collapse, and the natural cubic spline a(D) of the inverse growth function.
//
// GB300 executes FP64 at 1/64 of the FP32 rate (2 FP64 lanes per clock per
// SM), so a warp-wide FP64 instruction holds an SM sub-partition's FP64 unit
// for ~64 cycles while ~63 other instructions can issue. The FP64 routines
// below are therefore written to minimise FP64 instructions: every
// approximation (eigenvalue seeds, the cubic's root, interval search, the
// reciprocals of derivatives) is computed in FP32, and FP64 is spent only on
// the quantities that set the final accuracy (matrix invariants, Newton
// corrections, the cubic coefficients, the spline polynomial). Tests on signs,
// ranges and the running maximum compare FP64 bit patterns as integers
// (monotone for non-negative doubles), which costs no FP64 instruction.
// Control flow is predicated (Sec. 4.1); the only branches are the rare
// near-degenerate eigenvalue pair and the EdS range below the table.
#pragma once

#include <cstring>

#include "cc_internal.h"

namespace cc {

constexpr float kSqrt3f = 1.7320508075688772935f;
// 1 + r (FP32) below this: l1 and l2 are too close for a Newton step from the
// FP32 trigonometric seed to converge quadratically; the pair is re-solved by
// deflation in FP64 instead (about 5e-5 of the evaluations on isotropic Gaussian Hessians).
constexpr float kPairTauF = 1e-4f;

__device__ __forceinline__ long long bits(double x) { return __double_as_longlong(x); }

// FP64 <-> FP32 conversions on the integer pipes. The hardware conversions
// issue to the FP64 unit like any FP64 instruction; these rebias the exponent
// (1023 - 127 = 896) and move the mantissa with shifts instead.
// to_f32_trunc: the FP32 value with the mantissa truncated (relative error
// < 2^-23, used for seeds only); below the FP32 normal range it gives a signed
// zero, above it a signed infinity; NaN is not expected.
__device__ __forceinline__ float to_f32_trunc(double v) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v));
  const unsigned sign = static_cast<unsigned>(b >> 32) & 0x80000000u;
  const long long m = static_cast<long long>((b << 1) >> 30) - (896ll << 23);  // |v|'s exponent|mantissa, rebiased
  const unsigned mag = (m < (1ll << 23)) ? 0u : (m >= (255ll << 23)) ? (255u << 23) : static_cast<unsigned>(m);
  return __uint_as_float(sign | mag);
}
// to_f64: exact widening of an FP32 value; subnormals flush to a signed zero,
// infinities and NaNs stay what they are.
__device__ __forceinline__ double to_f64(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned sign = u & 0x80000000u, mag = u & 0x7fffffffu;
  unsigned hi = sign | ((mag >> 3) + (896u << 20));
  unsigned lo = mag << 29;
  if (mag < 0x00800000u) { hi = sign; lo = 0u; }
  if (mag >= 0x7f800000u) hi = sign | 0x7ff00000u | ((mag >> 3) & 0x000fffffu);
  return __hiloint2double(static_cast<int>(hi), static_cast<int>(lo));
}
// to_f64_normal: the same widening without the special cases, for operands
// that are normal FP32 numbers wherever the result is used (five integer
// instructions instead of ten). Zero and subnormals map to a number below
// 2^-126 in magnitude with their sign; infinities and NaNs to finite values.
__device__ __forceinline__ double to_f64_normal(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned hi = (((u & 0x7fffffffu) >> 3) + (896u << 20)) | (u & 0x80000000u);
  return __hiloint2double(static_cast<int>(hi), static_cast<int>(u << 29));
}

// to_f64_pos / to_f64_neg: the widening of an FP32 number known to be
// positive (negative) wherever the result is used, in three integer
// instructions: the logical shift moves a positive number's exponent and
// mantissa into place and the constant rebiases the exponent; for a negative
// number it also turns the shifted sign (bit 28) into bit 31. Any other input
// gives a finite number of no meaning.
__device__ __forceinline__ double to_f64_pos(float f) {
  const unsigned u = __float_as_uint(f);
  return __hiloint2double(static_cast<int>((u >> 3) + (896u << 20)), static_cast<int>(u << 29));
}
__device__ __forceinline__ double to_f64_neg(float f) {
  const unsigned u = __float_as_uint(f);
  return __hiloint2double(static_cast<int>((u >> 3) + 0xa8000000u), static_cast<int>(u << 29));
}

// tail_f32: v - hi as an FP32 value, where hi = to_f32_trunc(v): the 29
// mantissa bits of v below hi's 23, of which the top 23 are kept (relative
// error 2^-23 of the tail, 2^-46 of v), scaled by hi's exponent - 23. Built
// as the FP32 number 2^k (1 + m 2^-23) minus 2^k, both with v's sign, so the
// subtraction is exact. Zero where hi's biased exponent is 23 or less
// (|v| < 2^-103, or hi = 0).
__device__ __forceinline__ float tail_f32(double v, float hi) {
  const unsigned hb = __float_as_uint(hi);
  const unsigned base = (hb & 0xff800000u) - (23u << 23);
  const unsigned mant = (static_cast<unsigned>(__double_as_longlong(v)) >> 6) & 0x007fffffu;
  const float t = __fsub_rn(__uint_as_float(base | mant), __uint_as_float(base));
  return ((hb & 0x7f800000u) > (23u << 23)) ? t : 0.0f;
}

// Re-solve l1 >= l2 when they are nearly equal: l3 (isolated) gives an
// eigenvector v3 as the largest cross product of two rows of A - l3 I; A
// restricted to the plane orthogonal to v3 is a 2x2 symmetric matrix whose
// eigenvalues follow without cancellation (mean +- hypot(half difference, off-diagonal)).
static __device__ __noinline__ void refine_top_pair(double xx, double yy, double zz, double xy, double xz,
                                             double yz, double l3, double& l1, double& l2) {
  const double r0x = xx - l3, r0y = xy, r0z = xz;
  const double r1x = xy, r1y = yy - l3, r1z = yz;
  const double r2x = xz, r2y = yz, r2z = zz - l3;
  double ax = r0y * r1z - r0z * r1y, ay = r0z * r1x - r0x * r1z, az = r0x * r1y - r0y * r1x;
  double bx = r0y * r2z - r0z * r2y, by = r0z * r2x - r0x * r2z, bz = r0x * r2y - r0y * r2x;
  double cx = r1y * r2z - r1z * r2y, cy = r1z * r2x - r1x * r2z, cz = r1x * r2y - r1y * r2x;
  const double na = ax * ax + ay * ay + az * az;
  const double nb = bx * bx + by * by + bz * bz;
  const double nc = cx * cx + cy * cy + cz * cz;
  double vx = ax, vy = ay, vz = az, nv = na;
  if (nb > nv) { vx = bx; vy = by; vz = bz; nv = nb; }
  if (nc > nv) { vx = cx; vy = cy; vz = cz; nv = nc; }
  if (!(nv > 0.0)) return;  // l3 not isolated either: all equal, keep the incoming values
  const double iv = rsqrt(nv);
  vx *= iv; vy *= iv; vz *= iv;
  double ux, uy, uz;  // u orthogonal to v, then w = v x u
  if (fabs(vx) > fabs(vy)) {
    const double iu = rsqrt(vx * vx + vz * vz);
    ux = -vz * iu; uy = 0.0; uz = vx * iu;
  } else {
    const double iu = rsqrt(vy * vy + vz * vz);
    ux = 0.0; uy = vz * iu; uz = -vy * iu;
  }
  const double wx = vy * uz - vz * uy, wy = vz * ux - vx * uz, wz = vx * uy - vy * ux;
  const double aux = xx * ux + xy * uy + xz * uz;
  const double auy = xy * ux + yy * uy + yz * uz;
  const double auz = xz * ux + yz * uy + zz * uz;
  const double awx = xx * wx + xy * wy + xz * wz;
  const double awy = xy * wx + yy * wy + yz * wz;
  const double awz = xz * wx + yz * wy + zz * wz;
  const double m11 = ux * aux + uy * auy + uz * auz;
  const double m22 = wx * awx + wy * awy + wz * awz;
  const double m12 = wx * aux + wy * auy + wz * auz;
  const double mean = 0.5 * (m11 + m22);
  const double rad = hypot(0.5 * (m11 - m22), m12);
  l1 = mean + rad;
  l2 = mean - rad;
}

// ---- FP32 seeds. Newton corrections follow every seed (two on l1, two FP32
// and one FP64 on D_c), so a relative accuracy of 1e-4 is enough and the
// seeds use the special-function unit directly.

// square root and reciprocal of a seed: the hardware's approximate forms (one
// special-function instruction each, relative error near 2^-22) instead of
// the correctly rounded ones, which take several more instructions
__device__ __forceinline__ float sqrt_seed(float x) {
  float r;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float rcp_seed(float x) {
  float r;
  asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// cos(acos(x) / 3) for x in [-1, 1]. With s = sqrt((1 + x) / 2) = cos(acos(x) / 2)
// it is cos(2/3 acos(s)), an even function of acos(s) and so analytic on
// [0, 1]: a degree-5 polynomial in s, fitted by least squares on 4000
// Chebyshev nodes of [0, 1], is within 1.3e-6 of it (in FP32, with the
// approximate square root). One square root and five FMAs replace an
// arccos approximation and a cosine.
__device__ __forceinline__ float cos_third_acos(float x) {
  const float s = sqrt_seed(fmaf(0.5f, x, 0.5f));
  return fmaf(fmaf(fmaf(fmaf(fmaf(0.004192705f, s, -0.01930408f), s, 0.047796876f), s, -0.109943892f), s,
                   0.577258104f),
              s, 0.50000121f);
}
// the matching sine, sin(acos(x) / 3) >= 0, from the cosine c
__device__ __forceinline__ float sin_from_cos(float c) { return sqrt_seed(fmaxf(fmaf(-c, c, 1.0f), 0.0f)); }

// Largest real root of the monic cubic u^3 + b u^2 + c u + d: Cardano's
// formula when one root is real, the trigonometric form when three are.
__device__ __forceinline__ float cubic_largest_root_seed(float b, float c, float d) {
  const float b3 = b * (1.0f / 3.0f);
  const float pp = fmaf(-b, b3, c);
  const float qq = fmaf(b3, fmaf(2.0f * b3, b3, -c), d);
  const float disc = fmaf(0.25f * qq, qq, pp * pp * pp * (1.0f / 27.0f));
  float t;
  if (disc > 0.0f) {
    const float A = __powf(fmaf(0.5f, fabsf(qq), sqrt_seed(disc)), 1.0f / 3.0f);  // cube root, A >= 0
    const float C = (qq > 0.0f) ? -A : A;
    t = (C != 0.0f) ? C - __fdividef(pp, 3.0f * C) : 0.0f;
  } else {
    const float m = sqrt_seed(-pp * (1.0f / 3.0f));
    float arg = (m > 0.0f) ? __fdividef(-0.5f * qq, m * m * m) : 0.0f;
    arg = fminf(1.0f, fmaxf(-1.0f, arg));
    t = 2.0f * m * cos_third_acos(arg);
  }
  return t - b3;
}

// Interval of the a(D) spline holding D (FP32 search on FP32 knots): positive
// FP32 numbers order like their bit patterns, so the bucket (bits(D) - bits(D_0))
// >> b_shift is exact; it holds the largest k with D_k at or below its lower
// edge, and no bucket holds more than two knots, so two predicated steps end
// on the interval with D_k <= D < D_{k+1} (clamped to the first and last
// interval; D below D_0, negative or NaN lands in one of those).
__device__ __forceinline__ int spline_interval(const float* __restrict__ Dkf,
                                               const unsigned short* __restrict__ bucket,
                                               const DevTable& tab, float Df) {
  int b = static_cast<int>(__float_as_uint(Df) - tab.b0) >> tab.b_shift;
  b = min(max(b, 0), tab.n_buckets - 1);
  CC_DBG_CLAMP(b, 0, tab.n_buckets - 1, tab.dbg);
  int k = bucket[b];
  CC_DBG_CLAMP(k, 0, tab.n - 2, tab.dbg);
#pragma unroll
  for (int s = 0; s < 2; ++s) k += (k < tab.n - 2 && Dkf[k + 1] <= Df) ? 1 : 0;
  CC_DBG_CLAMP(k, 0, tab.n - 2, tab.dbg);
  return k;
}

struct PointResult {
  double F;  // 1/a_c, 0 without collapse
  double a;  // a_c, +inf without collapse (F is monotone in a: max F = 1/min a)
  bool collapsed, eds, refined;
};

struct EigenTop {
  double s, q, x, p2x3, det;  // tr, tr/3, l1 - q, 3 p^2, det(A - qI)
  float p2f;
  bool refined;               // l1 ~ l2 re-solved by deflation
};

// Largest eigenvalue l1 = q + x of the symmetric matrix in FP64 (FP32 trigonometric
// seed, two FP32 Newton steps and one FP64 Newton step on the depressed
// characteristic cubic, deflation when l1 ~ l2) together with the invariants
// the collapse condition needs.
__device__ __forceinline__ EigenTop eigen_top_fp64(double xx, double yy, double zz, double xy, double xz,
                                                   double yz) {
  EigenTop e;
  // ---- invariants (FP64)
  // M = A - qI, q = s/3 with s the trace; its diagonal a = xx - s/3, b, c each
  // in one FMA from s (a single rounding, and no separate subtraction from a
  // rounded q). |M|_F^2 / 2 = a^2 + a b + b^2 + off = a (a + b) + b^2 + off
  // with a + b = -c (no cancellation: a^2 + ab + b^2 >= 3/4 b^2); the three
  // rounded entries sum to d = O(eps |s|) instead of zero, which moves p^2 and
  // det M by O(eps |s| p), the size of the rounding of the entries themselves.
  // Only a matrix isotropic to within that rounding (|a|, |b| ~ |d|) can then
  // give 3 p^2 < 0; it is set to 0 there (its sign bit, an integer test).
  const double s = xx + yy + zz;
  const double q = s * (1.0 / 3.0);
  const double a = fma(s, -1.0 / 3.0, xx), b = fma(s, -1.0 / 3.0, yy), c = fma(s, -1.0 / 3.0, zz);
  const double yz2 = yz * yz;
  const double off = fma(xz, xz, fma(xy, xy, yz2));
  double p2x3 = fma(a, -c, fma(b, b, off));  // 3 p^2 = |M|_F^2 / 2
  p2x3 = bits(p2x3) < 0 ? 0.0 : p2x3;
  const double det = fma(xz, fma(xy, yz, -b * xz), fma(a, fma(b, c, -yz2), -xy * fma(xy, c, -yz * xz)));
  // ---- FP32 heads and tails: 3 p^2 = Ph + Pl, det = Dh + Dl, p^2 = p2f + p2l
  // (fmaf(-3, p2f, Ph) is the exact remainder of Ph / 3)
  const float Ph = to_f32_trunc(p2x3), Pl = tail_f32(p2x3, Ph);
  const float Dh = to_f32_trunc(det), Dl = tail_f32(det, Dh);
  const float p2f = Ph * (1.0f / 3.0f);
  const float p2l = __fmul_rn(__fadd_rn(fmaf(-3.0f, p2f, Ph), Pl), 1.0f / 3.0f);
  // ---- FP32 trigonometric seed
  const float pf = sqrt_seed(p2f);
  float rf = (p2f > 0.0f) ? __fdividef(Dh, 2.0f * p2f * pf) : 0.0f;
  rf = fminf(1.0f, fmaxf(-1.0f, rf));
  const float cs = cos_third_acos(rf), sn = sin_from_cos(cs);
  const float x1f = 2.0f * pf * cs;                   // l1 - q
  const float x3f = -pf * fmaf(kSqrt3f, sn, cs);      // l3 - q
  // ---- Newton on g(x) = x (x^2 - 3p^2) - det: one FP32 step on the heads, one
  // FP32 step on the float-float residual (x^2 exact as h2 + l2, x^2 - 3p^2
  // by TwoSum, x s1 exact as mh + ml; mh - Dh is exact near the root, where
  // x s1 ~ det), which lands within FP32 rounding of the root, then one FP64
  // step. Derivatives 3 (x^2 - p^2) in FP32 from p2f + p2l.
  float xf = x1f;
  {
    const float gpf = 3.0f * fmaf(xf, xf, -p2f);
    xf = (gpf != 0.0f) ? xf - __fdividef(fmaf(xf, fmaf(xf, xf, -Ph), -Dh), gpf) : xf;
  }
  {
    const float h2 = __fmul_rn(xf, xf), l2 = fmaf(xf, xf, -h2);
    const float s1 = __fsub_rn(h2, Ph), bb = __fsub_rn(s1, h2);
    const float e1 = __fadd_rn(__fsub_rn(h2, __fsub_rn(s1, bb)), __fsub_rn(-Ph, bb));
    const float ul = __fadd_rn(e1, __fsub_rn(l2, Pl));
    const float mh = __fmul_rn(xf, s1);
    const float ml = fmaf(xf, ul, fmaf(xf, s1, -mh));
    const float gf = __fadd_rn(__fsub_rn(mh, Dh), __fsub_rn(ml, Dl));
    const float gpf = 3.0f * __fsub_rn(fmaf(xf, xf, -p2f), p2l);
    xf = (gpf != 0.0f) ? __fsub_rn(xf, __fdividef(gf, gpf)) : xf;
  }
  const float gpf = 3.0f * __fsub_rn(fmaf(xf, xf, -p2f), p2l);
  const double x0 = to_f64(xf);
  const double x = fma(-fma(x0, fma(x0, x0, -p2x3), -det), to_f64((gpf != 0.0f) ? rcp_seed(gpf) : 0.0f), x0);
  double xr = x;
  e.refined = (1.0f + rf) < kPairTauF && p2f > 0.0f;
  if (e.refined) {
    // l1 ~ l2: refine the isolated l3 by Newton (FP64 derivative), then deflate
    double x3 = static_cast<double>(x3f);
#pragma unroll
    for (int it = 0; it < 3; ++it) {
      const double x32 = x3 * x3;
      x3 -= fma(x3, x32 - p2x3, -det) / fma(3.0, x32, -p2x3);
    }
    double l1r = q + x, l2r = 0.0;
    refine_top_pair(xx, yy, zz, xy, xz, yz, q + x3, l1r, l2r);
    xr = l1r - q;
  }
  e.s = s;
  e.q = q;
  e.x = xr;
  e.p2x3 = p2x3;
  e.det = det;
  e.p2f = p2f;
  return e;
}

// Growth factor at collapse from l1, l2 l3 and l2 + l3 (R-LPT): the FP64
// coefficients of A_1(D) = 1 - l1 D + c2 D^2 + c3 D^3, an FP32 seed from them
// (closed form in u = 1/D and two FP32 Newton steps) and one FP64 Newton step.
struct Root {
  double D;  // after the FP64 Newton step
  float Df;  // the FP32 root it started from
};

__device__ __forceinline__ Root rlpt_root_fp64(double lam1, double Pp, double S) {
  // c3 = l1 (l2 l3 / 9 - 5/21 (l2^2 + l3^2)) with l2^2 + l3^2 = S^2 - 2 l2 l3
  const double c2 = (-3.0 / 7.0) * Pp;
  const double c3 = lam1 * fma(-5.0 / 21.0, S * S, Pp * (37.0 / 63.0));
  // ---- FP32 root seed from the FP64 coefficients rounded to FP32: largest
  // root of u^3 - l1 u^2 + c2 u + c3 (u = 1/D), polished on A_1(D) in FP32
  const float l1f = to_f32_trunc(lam1);
  const float c2f = to_f32_trunc(c2);
  const float c3f = to_f32_trunc(c3);
  const float uf = cubic_largest_root_seed(-l1f, c2f, c3f);
  float Df = __fdividef(1.0f, uf);
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const float Af = fmaf(fmaf(fmaf(c3f, Df, c2f), Df, -l1f), Df, 1.0f);
    const float dAf = fmaf(fmaf(3.0f * c3f, Df, 2.0f * c2f), Df, -l1f);
    Df -= __fdividef(Af, dAf);
  }
  const float dAf = fmaf(fmaf(3.0f * c3f, Df, 2.0f * c2f), Df, -l1f);
  // ---- one FP64 Newton step on A_1
  Root r;
  r.Df = Df;
  const double D0 = to_f64(Df);
  const double A1 = fma(fma(fma(c3, D0, c2), D0, -lam1), D0, 1.0);
  r.D = fma(-A1, to_f64(rcp_seed(dAf)), D0);
  return r;
}

// 1/a: FP32 reciprocal and one FP64 Newton step
__device__ __forceinline__ double recip_fp64(double a) {
  const double y0 = to_f64(1.0f / to_f32_trunc(a));
  return fma(y0, fma(-a, y0, 1.0), y0);
}

constexpr double kInf = __builtin_huge_val();

// a(D_c) on spline interval k, or on the EdS segment below the first knot,
// a = (a_0 / D_0) D_c, evaluated by the same Horner scheme with that segment's
// coefficients selected in (c1 = a_0 / D_0; c0, c2, c3 and the knot 0): no
// separate multiply is issued for the rare branch, and fma(c1, D_c, 0) rounds
// the product once, as the multiply would.
__device__ __forceinline__ double spline_a(const Coef4& cf, double knot, double Dc, bool eds, const DevTable& tab) {
  const double t = Dc - (eds ? 0.0 : knot);
  return fma(fma(fma(eds ? 0.0 : cf.c3, t, eds ? 0.0 : cf.c2), t, eds ? tab.eds_slope : cf.c1), t, eds ? 0.0 : cf.c0);
}

// Running maximum of F = 1/a_c over the radii of one launch, kept as the
// running minimum of a_c (F is decreasing in a, so max F = 1/min a): the
// reciprocal is taken once per point and per launch instead of once per
// evaluation. Strict '<' keeps the earliest radius on ties (the paper's
// strict '>' on F); a_c > 0, so integer order of the bit patterns is value order.
struct MinA {
  double a = kInf;
  int r = -1;
  __device__ __forceinline__ void add(bool collapsed, double av, int radius) {
    if (collapsed && bits(av) < bits(a)) {
      a = av;
      r = radius;
    }
  }
  // the same minimum when radii arrive out of order: ties go to the smaller radius
  __device__ __forceinline__ void add_any_order(bool collapsed, double av, int radius) {
    if (collapsed && (bits(av) < bits(a) || (bits(av) == bits(a) && radius < r))) {
      a = av;
      r = radius;
    }
  }
  // the same merge against a value of F_max read earlier by this thread
  template <bool kF32Recip>
  __device__ __forceinline__ void store_vs(double F_old, double* F_max, int32_t* idx, int32_t scale_idx0) const {
    if (r < 0) return;
    const double F = kF32Recip ? to_f64(1.0f / to_f32_trunc(a)) : recip_fp64(a);
    if (bits(F) > bits(F_old)) {
      *F_max = F;
      *idx = scale_idx0 + r;
    }
  }
  // merge into the stored maximum: F = 1/a (FP64, or through the FP32
  // reciprocal for the reduced-precision modes), strict '>' against F_max
  template <bool kF32Recip>
  __device__ __forceinline__ void store(double* F_max, int32_t* idx, int32_t scale_idx0) const {
    if (r < 0) return;
    const double F = kF32Recip ? to_f64(1.0f / to_f32_trunc(a)) : recip_fp64(a);
    if (bits(F) > bits(*F_max)) {  // both >= 0
      *F_max = F;
      *idx = scale_idx0 + r;
    }
  }
};

// Finiteness of an FP64 value from its bit pattern (exponent not all ones),
// on the integer pipes: the high word comes from an opaque move, because the
// compiler recognises the masked 64-bit test as a floating-point class check
// and issues an FP64 compare, which this GPU runs on its FP64 unit.
__device__ __forceinline__ bool finite_bits(double v) {
  unsigned lo, hi;
  asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "d"(v));
  return (hi & 0x7ff00000u) != 0x7ff00000u;
}

// a on the spline interval whose polynomial is expanded about the FP32 knot
// e_k (t = D - e_k), or on the EdS segment below the first knot,
// a = (a_0 / D_0) D with t = D: the same Horner scheme with that segment's
// coefficients selected in (c1 = a_0 / D_0, c0 = c2 = c3 = 0).
__device__ __forceinline__ double spline_a_t(const Coef4& cf, double t, bool eds, const DevTable& tab) {
  return fma(fma(fma(eds ? 0.0 : cf.c3, t, eds ? 0.0 : cf.c2), t, eds ? tab.eds_slope : cf.c1), t, eds ? 0.0 : cf.c0);
}

// FP64 collapse value of one point, F = 1/a_c (0 when there is no collapse).
//   eigenvalues: invariants of M = A - qI in FP64 (s = tr, q = s/3,
//     |M|_F^2 = 6 p^2, det M); l1 = q + x with x the largest root of
//     x^3 - 3 p^2 x - det M = 0, seeded by the FP32 trigonometric solution,
//     brought to FP32 rounding of the root by two FP32 Newton steps (the second
//     on the float-float residual from FP32 heads and tails of 3 p^2 and
//     det M) and corrected by one FP64 Newton step (FP32 derivative);
//   collapse: A_1(D) = 1 - l1 D + c2 D^2 + c3 D^3 from the centred invariants
//     (w = x^2 - 3p^2 = (l2 - q)(l3 - q), l2 l3 = q (q - x) + w,
//     c2 = -3/7 l2 l3, c3 = l1 K with 63 K = -23 l2 l3 + 15 (3 w - 3p^2), which is
//     l1 (l2 l3 / 9 - 5/21 (l2^2 + l3^2)) written without l2 + l3); the root is
//     seeded in FP32 from the FP64 coefficients rounded to FP32 (closed form in
//     u = 1/D, two FP32 Newton steps) and corrected by one FP64 Newton step;
//   spline: the table's polynomials are expanded about the FP32 knots e_k, so
//     the FP32 root Df gives t0 = Df - e_k exactly in FP32 (knots within a
//     factor 2 of each other), and the FP64 Newton step lands directly on
//     t = D - e_k (on the EdS segment t = D); FP64 Horner in t;
//   collapse test: l1 > 0 and Df > 0 (FP32 and FP64 roots agree in sign and in
//     their interval to ~1e-7), and on the last interval t <= D_top - e_{n-2}
//     on the FP64 bit pattern (exact); EdS segment where Df < e_0 (the two
//     formulas meet at D_0, so taking the FP32 decision within ~1e-7 D_0 of it
//     moves a by ~1e-14 relative);
//   F by one FP64 Newton step of the reciprocal from the FP32 reciprocal.
__device__ __forceinline__ PointResult collapse_point_fp64(
    double xx, double yy, double zz, double xy, double xz, double yz, const double* __restrict__ Dk,
    const Coef4* __restrict__ coef, const float* __restrict__ Dkf,
    const unsigned short* __restrict__ bucket, const DevTable& tab) {
  (void)Dk;
  PointResult res;
  const EigenTop e = eigen_top_fp64(xx, yy, zz, xy, xz, yz);
  res.refined = e.refined;
  const double s = e.s, x = e.x, p2x3 = e.p2x3;
  // ---- collapse condition coefficients (FP64)
  const double lam1 = fma(s, 1.0 / 3.0, x);
  const double qmx = fma(s, 1.0 / 3.0, -x);
  const double w = fma(x, x, -p2x3);
  const double Pp = fma(e.q, qmx, w);                      // l2 l3
  const double v = fma(w, 3.0, -p2x3);
  const double K = fma(v, 15.0 / 63.0, Pp * (-23.0 / 63.0));
  const double c2 = Pp * (-3.0 / 7.0);
  const double c3 = lam1 * K;
  // ---- FP32 root seed from the FP64 coefficients rounded to FP32: largest
  // root of u^3 - l1 u^2 + c2 u + c3 (u = 1/D), polished on A_1(D) in FP32
  const float l1f = to_f32_trunc(lam1);
  const float c2f = to_f32_trunc(c2);
  const float c3f = to_f32_trunc(c3);
  const float uf = cubic_largest_root_seed(-l1f, c2f, c3f);
  float Df = __fdividef(1.0f, uf);
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const float Af = fmaf(fmaf(fmaf(c3f, Df, c2f), Df, -l1f), Df, 1.0f);
    const float dAf = fmaf(fmaf(3.0f * c3f, Df, 2.0f * c2f), Df, -l1f);
    Df -= __fdividef(Af, dAf);
  }
  const float dAf = fmaf(fmaf(3.0f * c3f, Df, 2.0f * c2f), Df, -l1f);
  // ---- interval, then one FP64 Newton step on A_1 that yields t = D - e_k
  const int k = spline_interval(Dkf, bucket, tab, Df);
  res.eds = Df < Dkf[0];
  const float t0 = res.eds ? Df : __fsub_rn(Df, Dkf[k]);
  const double D0 = to_f64(Df);
  const double A1 = fma(fma(fma(c3, D0, c2), D0, -lam1), D0, 1.0);
  const double t = fma(-A1, to_f64(rcp_seed(dAf)), to_f64_normal(t0));
  // ---- collapse test: l1 > 0, 0 < D <= D_top
  res.collapsed = bits(lam1) > 0 && Df > 0.0f && (k < tab.n - 2 || bits(t) <= bits(tab.Dtop_t)) && finite_bits(t);
  res.eds = res.eds && res.collapsed;
  const double av = spline_a_t(coef[k], t, res.eds, tab);
  res.a = res.collapsed ? av : kInf;
  const double F = recip_fp64(av);
  res.F = res.collapsed ? F : 0.0;
  return res;
}

// ---------------------------------------------------------------------------
// Mixed precision (CC_MODE_MIXED): FP32 bulk, FP64 only for (i) points whose
// eigenvalues are (nearly) degenerate, (ii) the collapse-condition root polish
// and (iii) the a(D) spline, as the mixed path is specified. Target: F within
// 3e-5 of the FP64 oracle.
//
// The FP32 eigenvalue l1 = q + x carries an absolute error of about
// eps32 p^3 / ((x1 - x2)(x1 - x3)) (the FP32 residual of the characteristic
// cubic over its slope), and D_c is relatively as sensitive to l1 as to the
// other coefficients (c3 is proportional to l1). Points where that estimate
// divided by |l1| exceeds kMixedEstTau get one FP64 Newton step on
// det(A - l I), evaluated from the FP32 entries widened to FP64 (products of
// two FP32 numbers are exact in FP64). Points with 1 + r < kPairTauF (l1 ~ l2)
// or l1 - l3 below 1e-4 s (all three close; s = rms of tr H at this radius)
// take the whole FP64 path.
constexpr float kMixedEstTau = 3e-6f;
constexpr float kMixedEstCoef = 2.4e-7f;  // ~4 eps32: rounding of det and of the cubic residual

struct MixedResult {
  double F, a;  // as PointResult (F = 1/a through an FP32 reciprocal)
  bool collapsed, eds, refined, fp64;
};

// FP32 eigenvalue stage of the mixed path (shared with the surrogate path).
struct MixedEigen {
  float q, x, x2, x3, p2, p2x3;  // x = l1 - q (x2, x3: FP32 seeds of l2 - q, l3 - q)
  float lam1f;                    // l1 in FP32 (truncated from lam1 after the FP64 refinement)
  double lam1;                    // l1, refined in FP64 when flagged
  bool full;                      // take the whole FP64 path instead
  bool need64;                    // l1 needs the FP64 refinement (mixed_refine64)
  bool fp64;                      // the FP64 eigenvalue refinement ran
};

// The FP32 part: invariants, trigonometric eigenvalues, one FP32 Newton
// step (the seed's error of ~3e-5 p drops to FP32 rounding of the cubic's
// coefficients; a second step measured no change), and the flags that send a point to the FP64 refinement or to the
// whole FP64 path.
__device__ __forceinline__ MixedEigen mixed_eigen_f32(float xx, float yy, float zz, float xy, float xz, float yz,
                                                      float tri_thr) {
  MixedEigen m;
  m.fp64 = false;
  const float q = (xx + yy + zz) * (1.0f / 3.0f);
  const float a = xx - q, b = yy - q, c = zz - q;
  const float s6 = fmaf(2.0f, fmaf(yz, yz, fmaf(xz, xz, xy * xy)), fmaf(c, c, fmaf(b, b, a * a)));
  const float p2 = s6 * (1.0f / 6.0f), p2x3 = 0.5f * s6;
  const float det = fmaf(xz, fmaf(xy, yz, -b * xz), fmaf(a, fmaf(b, c, -yz * yz), -xy * fmaf(xy, c, -yz * xz)));
  const float pf = sqrt_seed(p2);
  float rf = (p2 > 0.0f) ? __fdividef(det, 2.0f * p2 * pf) : 0.0f;
  rf = fminf(1.0f, fmaxf(-1.0f, rf));
  const float cs = cos_third_acos(rf), sn = sin_from_cos(cs);
  float x = 2.0f * pf * cs;
  const float x2 = pf * fmaf(kSqrt3f, sn, -cs);
  const float x3 = -pf * fmaf(kSqrt3f, sn, cs);
  // one FP32 Newton step on x (x^2 - 3p^2) - det; its derivative
  // 3 (x^2 - p^2) equals (x - x2)(x - x3) (Vieta: x + x2 + x3 = 0,
  // x x2 + x x3 + x2 x3 = -3 p^2), the product the estimate below needs
  const float gp = 3.0f * fmaf(x, x, -p2);
  x = (gp != 0.0f) ? x - __fdividef(fmaf(x, fmaf(x, x, -p2x3), -det), gp) : x;
  m.full = ((1.0f + rf) < kPairTauF && p2 > 0.0f) || (x - x3) < tri_thr;
  const float lam1f = q + x;
  // the estimate over |l1| against kMixedEstTau, compared as a product (no division)
  m.need64 = !m.full && kMixedEstCoef * p2 * pf > kMixedEstTau * fmaxf(gp * fabsf(lam1f), 1e-30f);
  m.q = q;
  m.x = x;
  m.x2 = x2;
  m.x3 = x3;
  m.p2 = p2;
  m.p2x3 = p2x3;
  m.lam1f = lam1f;
  m.lam1 = to_f64_pos(lam1f);  // exact wherever l1 > 0 can collapse (a positive normal lam1f)
  return m;
}

// One FP64 Newton step on g(l) = det(A - l I) from the FP32 l1 (g'(l) =
// -3 (x^2 - p^2) from FP32), the FP32 entries widened to FP64 (products of
// two FP32 numbers are exact in FP64).
__device__ __forceinline__ void mixed_refine64(MixedEigen& m, float xx, float yy, float zz, float xy, float xz,
                                               float yz) {
  const double lam1 = to_f64_normal(m.lam1f);
  const double dxx = to_f64(xx) - lam1, dyy = to_f64(yy) - lam1;
  const double dzz = to_f64(zz) - lam1;
  const double dxy = to_f64(xy), dxz = to_f64(xz), dyz = to_f64(yz);
  const double g = fma(dxx, fma(dyy, dzz, -dyz * dyz),
                       fma(-dxy, fma(dxy, dzz, -dyz * dxz), dxz * fma(dxy, dyz, -dyy * dxz)));
  const float gpf = 3.0f * fmaf(m.x, m.x, -m.p2);
  m.lam1 = fma(g, to_f64(__fdividef(1.0f, gpf)), lam1);
  m.x = to_f32_trunc(m.lam1 - to_f64(m.q));
  m.lam1f = to_f32_trunc(m.lam1);
  m.fp64 = true;
}

__device__ __forceinline__ MixedEigen mixed_eigen(float xx, float yy, float zz, float xy, float xz, float yz,
                                                  float tri_thr) {
  MixedEigen m = mixed_eigen_f32(xx, yy, zz, xy, xz, yz, tri_thr);
  if (m.need64) mixed_refine64(m, xx, yy, zz, xy, xz, yz);
  return m;
}

// FP32 collapse-condition coefficients of the mixed path
struct MixedCoef {
  float l1f, c2f, c3f;
};

__device__ __forceinline__ MixedCoef mixed_coef(const MixedEigen& m) {
  const float q = m.q, x = m.x;
  const float Pp = fmaf(q, q - x, fmaf(x, x, -m.p2x3));  // l2 l3
  const float S = fmaf(2.0f, q, -x);                     // l2 + l3
  const float Q2 = fmaf(-2.0f, Pp, S * S);               // l2^2 + l3^2
  MixedCoef k;
  k.l1f = m.lam1f;
  k.c2f = (-3.0f / 7.0f) * Pp;
  k.c3f = k.l1f * fmaf(-5.0f / 21.0f, Q2, Pp * (1.0f / 9.0f));
  return k;
}

// One FP32 Newton step on A_1 that also returns the reciprocal of the
// derivative it took (at the iterate before the step). The FP64 polish reuses
// it: A_1' moves by ~1e-5 relative over that step (the seed's error), which
// moves the polish's correction (~1e-7 D) by ~1e-12 D.
struct RootF32 {
  float D, rdA;
};
__device__ __forceinline__ RootF32 newton_f32_r(const MixedCoef& k, float Df) {
  const float Af = fmaf(fmaf(fmaf(k.c3f, Df, k.c2f), Df, -k.l1f), Df, 1.0f);
  const float dAf = fmaf(fmaf(3.0f * k.c3f, Df, 2.0f * k.c2f), Df, -k.l1f);
  const float r = rcp_seed(dAf);
  return RootF32{fmaf(-Af, r, Df), r};
}

// FP32 Newton steps on A_1(D) = 1 - l1 D + c2 D^2 + c3 D^3 from Df
template <int kSteps>
__device__ __forceinline__ float newton_f32(const MixedCoef& k, float Df) {
#pragma unroll
  for (int it = 0; it < kSteps; ++it) {
    const float Af = fmaf(fmaf(fmaf(k.c3f, Df, k.c2f), Df, -k.l1f), Df, 1.0f);
    const float dAf = fmaf(fmaf(3.0f * k.c3f, Df, 2.0f * k.c2f), Df, -k.l1f);
    Df -= __fdividef(Af, dAf);
  }
  return Df;
}

// From an FP32 root Df: one FP64 Newton step (the root polish), the FP64
// a(D) spline and F.
//   polish: A_1(D0) at D0 = Df in FP64 except c3 D0 + c2, which is formed in
//     FP32 (c2 and c3 are FP32 values here; that rounding is of the size of
//     theirs);
//   spline: the polished root enters only through t = D - D_k, formed in the
//     same FP64 FMA as the Newton step, t = (D0 - D_k) - A_1 / A_1', with
//     D0 - D_k = (Df - hi(D_k)) - lo(D_k) in FP32 (the first difference is
//     exact, the second rounds by ~2^-24 |t| <= 1e-9 D). Then a = c0 + t v
//     with v = c1 + t (c2 + c3 t) in FP32 and c0 + t v in FP64: c1 t is at
//     most ~1.4e-2 of a over an interval, so v's FP32 rounding (and taking
//     the unpolished t there) moves a by ~1e-9 relative. On the EdS segment
//     below the first knot, a = (a_0 / D_0) D is the same FMA with
//     v = hi(a_0 / D_0), t = D and the head lo(a_0 / D_0) D formed in FP32;
//   the collapse and EdS tests take Df: the FP32 and the polished root fall on
//     the same side of D_top or D_0 except within ~1e-7 of them, where the two
//     sides give the same a (a_max at D_top; the spline is continuous at D_0);
//   FP32 -> FP64: for a collapsing point Df and v are positive normal
//     numbers, 1/A_1' a negative one (A_1 is strictly decreasing on D > 0
//     when l1 > 0, so A_1' < 0 at Df and at the positive iterate before it)
//     and t0 >= 0 (the interval search is exact, D_k = e_k, and on the
//     EdS segment t0 = Df), so they take the three-instruction to_f64_pos /
//     to_f64_neg (a result that is not used may be any finite number; a zero
//     t0 becomes 2^-127); c3 Df + c2 and lo(a_0 / D_0) D take to_f64_normal,
//     where a zero shifts A_1 or a by less than 2^-126.
// kEds = false: the caller sends EdS collapses (res.eds) elsewhere and uses
// only the other results, so the EdS operand selects are left out; every
// result with res.eds false is the same as with kEds = true.
// rdA: the reciprocal of A_1' near Df (newton_f32_r's, or at Df itself).
template <bool kEds = true>
__device__ __forceinline__ MixedResult mixed_finish_r(const MixedEigen& m, const MixedCoef& k, float Df, float rdA,
                                                      const Coef4* __restrict__ coef, const float* __restrict__ Dkf,
                                                      const unsigned short* __restrict__ bucket, const DevTable& tab,
                                                      const float4* __restrict__ seg) {
  MixedResult res;
  res.refined = false;
  res.fp64 = m.fp64;
  const double D0 = to_f64_pos(Df);
  const double A1 = fma(fma(to_f64_normal(fmaf(k.c3f, Df, k.c2f)), D0, -m.lam1), D0, 1.0);
  res.collapsed = m.lam1f > 0.0f && Df > 0.0f && Df <= tab.Dtopf;
  const float Dcf = res.collapsed ? Df : tab.Dtopf;
  const int kk = spline_interval(Dkf, bucket, tab, Dcf);
  res.eds = res.collapsed && Df < Dkf[0];
  const float4 s0 = seg[2 * kk];      // {hi(c0), lo(c0), hi(c1), lo(c1)}
  const float4 s1 = seg[2 * kk + 1];  // {c2, c3, hi(D_k), lo(D_k)}
  const bool eds = kEds && res.eds;
  const float t0 = eds ? Dcf : __fsub_rn(__fsub_rn(Dcf, s1.z), s1.w);
  const float v = eds ? tab.eds_hi : fmaf(fmaf(s1.y, t0, s1.x), t0, s0.z);
  const double head = eds ? to_f64_normal(tab.eds_lo * Dcf) : coef[kk].c0;
  const double t = fma(-A1, to_f64_neg(rdA), to_f64_pos(t0));
  const double av = fma(to_f64_pos(v), t, head);
  res.a = res.collapsed ? av : kInf;
  res.F = res.collapsed ? to_f64(1.0f / to_f32_trunc(av)) : 0.0;
  return res;
}

// The same with A_1' taken at Df.
template <bool kEds = true>
__device__ __forceinline__ MixedResult mixed_finish(const MixedEigen& m, const MixedCoef& k, float Df,
                                                    const Coef4* __restrict__ coef, const float* __restrict__ Dkf,
                                                    const unsigned short* __restrict__ bucket, const DevTable& tab,
                                                    const float4* __restrict__ seg) {
  const float dAf = fmaf(fmaf(3.0f * k.c3f, Df, 2.0f * k.c2f), Df, -k.l1f);
  return mixed_finish_r<kEds>(m, k, Df, rcp_seed(dAf), coef, Dkf, bucket, tab, seg);
}

__device__ __forceinline__ MixedResult full_fp64(float xx, float yy, float zz, float xy, float xz, float yz,
                                                 const double* __restrict__ Dk, const Coef4* __restrict__ coef,
                                                 const float* __restrict__ Dkf,
                                                 const unsigned short* __restrict__ bucket, const DevTable& tab) {
  const PointResult r64 =
      collapse_point_fp64(to_f64(xx), to_f64(yy), to_f64(zz), to_f64(xy), to_f64(xz), to_f64(yz), Dk, coef, Dkf, bucket, tab);
  MixedResult res;
  res.F = r64.F;
  res.a = r64.a;
  res.collapsed = r64.collapsed;
  res.eds = r64.eds;
  res.refined = r64.refined;
  res.fp64 = true;
  return res;
}

__device__ __forceinline__ MixedResult collapse_point_mixed(
    float xx, float yy, float zz, float xy, float xz, float yz, float tri_thr,
    const double* __restrict__ Dk, const Coef4* __restrict__ coef, const float* __restrict__ Dkf,
    const unsigned short* __restrict__ bucket, const DevTable& tab) {
  const MixedEigen m = mixed_eigen(xx, yy, zz, xy, xz, yz, tri_thr);
  if (m.full) return full_fp64(xx, yy, zz, xy, xz, yz, Dk, coef, Dkf, bucket, tab);
  const MixedCoef k = mixed_coef(m);
  // FP32 closed-form root of u^3 - l1 u^2 + c2 u + c3 (u = 1/D), one FP32
  // Newton step on A_1 (the seed is within ~1e-5, one step within ~2e-7, and
  // the FP64 polish squares that)
  const float uf = cubic_largest_root_seed(-k.l1f, k.c2f, k.c3f);
  const RootF32 rt = newton_f32_r(k, __fdividef(1.0f, uf));
  return mixed_finish_r(m, k, rt.D, rt.rdA, coef, Dkf, bucket, tab, tab.dfseg);
}

// ---------------------------------------------------------------------------
// Tabulated collapse (Sec. 3 "Tabulated" option; Sec. 4.2: cubic spline along
// delta at the four (x, y) corners of the cell, bilinear blend). The table holds
// u = 1/D_c; outside it the R-LPT root is used.

// An integer that orders like the FP64 value v (NaN aside): the bit pattern b
// for b >= 0; for b < 0, minus its magnitude bits, so -0.0 and +0.0 both give 0.
__host__ __device__ __forceinline__ long long order_key(double v) {
#ifdef __CUDA_ARCH__
  const long long b = __double_as_longlong(v);
#else
  long long b;
  std::memcpy(&b, &v, sizeof(b));
#endif
  return b < 0 ? -static_cast<long long>(static_cast<unsigned long long>(b) - 0x8000000000000000ull) : b;
}

__device__ __forceinline__ double horner(const Coef4& c, double t) {
  return fma(fma(fma(c.c3, t, c.c2), t, c.c1), t, c.c0);
}

// u(delta, x, y) from the table; ax is the axes image (shared memory), x, y >= 0.
// Cells in x and y are found on FP64 bit patterns (exact: bilinear interpolation
// is only continuous across cell edges); the delta interval by an FP32 search
// (the spline is C2 across its knots).
__device__ __forceinline__ double tab_interp(const TabDev& td, const double* __restrict__ ax,
                                             const Coef4* __restrict__ tcoef, double delta, double x, double y) {
  const double* dg = ax;
  const double* xg = dg + td.nd;
  const double* yg = xg + td.nx;
  const double* ihx = yg + td.ny;
  const double* ihy = ihx + (td.nx - 1);
  const double* cx = ihy + (td.ny - 1);  // -x_i / h_i
  const double* cy = cx + (td.nx - 1);
  const float* dgf = reinterpret_cast<const float*>(cy + (td.ny - 1));
  const long long bx = bits(x), by = bits(y);
  int ix = 0, iy = 0, kd = 0;
  for (int step = td.x_steps; step > 0; step >>= 1) {
    const int j = ix + step;
    ix = (j <= td.nx - 2 && bits(xg[j]) <= bx) ? j : ix;
  }
  for (int step = td.y_steps; step > 0; step >>= 1) {
    const int j = iy + step;
    iy = (j <= td.ny - 2 && bits(yg[j]) <= by) ? j : iy;
  }
  const float df = to_f32_trunc(delta);
  for (int step = td.d_steps; step > 0; step >>= 1) {
    const int j = kd + step;
    kd = (j <= td.nd - 2 && dgf[j] <= df) ? j : kd;
  }
  CC_DBG_CLAMP(ix, 0, td.nx - 2, td.dbg);
  CC_DBG_CLAMP(iy, 0, td.ny - 2, td.dbg);
  CC_DBG_CLAMP(kd, 0, td.nd - 2, td.dbg);
  const double t = delta - dg[kd];
  const size_t nseg = static_cast<size_t>(td.nd - 1);
  const size_t s00 = (static_cast<size_t>(ix) * td.ny + iy) * nseg + kd;
  const size_t sx = static_cast<size_t>(td.ny) * nseg;
  const double z00 = horner(tcoef[s00], t);
  const double z10 = horner(tcoef[s00 + sx], t);
  const double z01 = horner(tcoef[s00 + nseg], t);
  const double z11 = horner(tcoef[s00 + sx + nseg], t);
  // (x - x_i) / h_i in one FMA from the cell's 1/h_i and -x_i / h_i (the
  // offset's rounding is eps x_i / h_i, far below the table's own error)
  const double tx = fma(x, ihx[ix], cx[ix]);
  const double ty = fma(y, ihy[iy], cy[iy]);
  const double z0 = fma(tx, z10 - z00, z00);
  const double z1 = fma(tx, z11 - z01, z01);
  return fma(ty, z1 - z0, z0);
}

struct TabResult {
  double F, a;  // as PointResult
  bool collapsed, eds, refined, outside;
};

__device__ __forceinline__ TabResult collapse_point_tab(
    double xx, double yy, double zz, double xy, double xz, double yz, const double* __restrict__ Dk,
    const Coef4* __restrict__ coef, const float* __restrict__ Dkf, const unsigned short* __restrict__ bucket,
    const DevTable& tab, const TabDev& td, const double* __restrict__ ax, const Coef4* __restrict__ tcoef) {
  TabResult res;
  const EigenTop e = eigen_top_fp64(xx, yy, zz, xy, xz, yz);
  res.refined = e.refined;
  const double q = e.q, x = e.x, p2x3 = e.p2x3;
  const double lam1 = q + x;
  // x = l1 - l2 and y = l2 - l3 from the traceless part alone: the other two
  // roots of x^3 - 3p^2 x - det are (-x +- y) / 2 with
  // y^2 = (x2 - x3)^2 = (x2 + x3)^2 - 4 x2 x3 = x^2 - 4 (x^2 - 3p^2) = 4 (3p^2) - 3x^2
  // (Vieta), so nothing cancels against the trace; x = 1.5 x - y / 2. Near
  // x2 = x3 (y below ~3.5e-5 p, where y^2 cancels) the pair is re-solved by
  // deflation around the isolated l1 (and stays at (l2 + l3) / 2 each when no
  // eigenvalue is isolated, p = 0 included); the test is in FP32.
  const double D2 = fma(x * -3.0, x, 4.0 * p2x3);
  const float D2f = to_f32_trunc(D2);
  double yv, xv;
  if (D2f <= 1e-10f * (4.0f * to_f32_trunc(p2x3))) {
    double l2 = 0.5 * fma(2.0, q, -x), l3 = l2;
    refine_top_pair(xx, yy, zz, xy, xz, yz, lam1, l2, l3);
    res.refined = true;
    yv = l2 - l3;
    xv = lam1 - l2;
  } else {
    // sqrt(D2): FP32 seed, one FP64 Newton step (relative error ~1e-13)
    const float yf = sqrt_seed(D2f);
    const double y0 = to_f64(yf);
    yv = fma(fma(-y0, y0, D2), to_f64(0.5f * rcp_seed(yf)), y0);
    xv = fma(yv, -0.5, 1.5 * x);
  }
  yv = bits(yv) > 0 ? yv : 0.0;
  xv = bits(xv) > 0 ? xv : 0.0;
  const double delta = e.s;  // the trace
  // inside the hull [d_0, d_last] x [x_0, x_last] x [y_0, y_last]: xv, yv and
  // the axis bounds are >= 0, so their bit patterns order like their values;
  // delta by its order key (a NaN of either sign falls outside)
  const long long dkey = order_key(delta);
  res.outside = !(dkey >= td.d_lo_key && dkey <= td.d_hi_key && bits(xv) >= bits(td.x_lo) && bits(xv) <= bits(td.x_hi) &&
                  bits(yv) >= bits(td.y_lo) && bits(yv) <= bits(td.y_hi));
  double D;
  bool root = true;
  if (!res.outside) {
    const double u = tab_interp(td, ax, tcoef, delta, xv, yv);
    const double r0 = to_f64(rcp_seed(to_f32_trunc(u)));
    D = fma(r0, fma(-u, r0, 1.0), r0);  // 1/u: FP32 reciprocal + one FP64 Newton step
    root = bits(u) > 0;
  } else {
    const double Pp = fma(q, q - x, fma(x, x, -p2x3));  // l2 l3
    D = rlpt_root_fp64(lam1, Pp, fma(2.0, q, -x)).D;    // l2 + l3
  }
  const long long bD = bits(D);
  res.collapsed = bits(lam1) > 0 && root && bD > 0 && bD <= bits(tab.Dtop);
  const double Dc = res.collapsed ? D : tab.Dtop;
  const int k = spline_interval(Dkf, bucket, tab, to_f32_trunc(Dc));
  res.eds = res.collapsed && bits(Dc) < bits(tab.D0);
  const double av = spline_a(coef[k], Dk[k], Dc, res.eds, tab);
  res.a = res.collapsed ? av : kInf;
  res.F = res.collapsed ? recip_fp64(av) : 0.0;
  return res;
}

}  // namespace cc
