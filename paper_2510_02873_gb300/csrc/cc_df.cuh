// cc_df.cuh -- FP64-accurate collapse value in float-float arithmetic
// (arXiv:2510.02873, Sec. 3 and 4.1, computed without the FP64 unit).
//
// GB300 runs FP64 at 1/64 of the FP32 rate. A float-float number is an
// unevaluated sum hi + lo of two FP32 numbers with |lo| <= ulp(hi)/2: 48
// significant bits, relative rounding about 2^-47 per operation (FP64:
// 2^-53). Sums and products are built from the error-free transformations
// TwoSum (Knuth), Fast2Sum (Dekker) and TwoProduct through the FMA
// (a b - RN(a b) is exact), so every operation costs 3-10 FP32
// instructions, which issue at 64 times the FP64 rate. The collapse value
// below follows the same steps as collapse_point_fp64 (invariants, FP32
// trigonometric seed, two Newton corrections of l1, R-LPT coefficients,
// FP32 root and one Newton correction, spline) with every FP64 operation
// replaced by its float-float counterpart; the only FP64 instructions left
// are the rare near-degenerate pair (deflation, as in the FP64 path). Inputs
// in FP64 are split into float-float on the integer pipes (their five lowest
// mantissa bits are rounded away: a relative perturbation below 2^-48).
#pragma once

#include "cc_device.cuh"

namespace cc {
namespace dfl {

struct f2 {
  float hi, lo;
};

// The error-free steps use the _rn intrinsics, which the compiler never
// contracts into an FMA or reassociates.
__device__ __forceinline__ f2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ f2 fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ f2 make(float v) { return {v, 0.0f}; }
__device__ __forceinline__ f2 neg(f2 a) { return {-a.hi, -a.lo}; }
// a + b with absolute error ~2^-47 (|a| + |b|)
__device__ __forceinline__ f2 add(f2 a, f2 b) {
  const f2 s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ f2 sub(f2 a, f2 b) { return add(a, neg(b)); }
// the same sum left unnormalised: only for sums that cannot cancel (terms of
// one sign, or a small correction to a large value), whose hi stays the
// rounded sum and whose lo stays a few ulp(hi). After a cancelling sum lo can
// be as large as hi, and the products that follow would lose that precision.
__device__ __forceinline__ f2 addu(f2 a, f2 b) {
  const f2 s = two_sum(a.hi, b.hi);
  return {s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo))};
}
// Products are returned unnormalised: {RN(ab), the rest}, |lo| a few ulp(hi)
// at most. Every sum renormalises (Fast2Sum), and only sums are compared, so
// the renormalisation a product would need is left to the sum that consumes it.
__device__ __forceinline__ f2 mul(f2 a, f2 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  return {p, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, fmaf(a.hi, b.hi, -p)))};
}
__device__ __forceinline__ f2 mul(f2 a, float b) {
  const float p = __fmul_rn(a.hi, b);
  return {p, fmaf(a.lo, b, fmaf(a.hi, b, -p))};
}
__device__ __forceinline__ f2 sqr(f2 a) {
  const float p = __fmul_rn(a.hi, a.hi);
  return {p, fmaf(2.0f * a.hi, a.lo, fmaf(a.hi, a.hi, -p))};
}
__device__ __forceinline__ f2 two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ f2 norm(f2 a) { return fast_two_sum(a.hi, a.lo); }
// exact scaling by a power of two
__device__ __forceinline__ f2 scale(f2 a, float pow2) { return {a.hi * pow2, a.lo * pow2}; }
// order of two normalised float-float numbers (hi first, then lo)
__device__ __forceinline__ bool less(f2 a, f2 b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool less_equal(f2 a, f2 b) { return a.hi < b.hi || (a.hi == b.hi && a.lo <= b.lo); }

// FP64 -> float-float on the integer pipes: hi = the top 24 significant bits
// (truncated), lo = the remaining 29 bits rounded to FP32. Values below 2^-74
// keep only hi (relative error < 2^-23 of a number that small); infinities
// and NaNs become NaN (no collapse, as in the FP64 path).
__device__ __forceinline__ f2 split(double v) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v));
  const float hi = ((b >> 52) & 0x7ff) == 0x7ff ? __int_as_float(0x7fffffff) : to_f32_trunc(v);
  const int se = static_cast<int>((b >> 52) & 0x7ff) - 1075 + 127;  // FP32 exponent of 2^(E - 1075)
  float lo = __uint2float_rn(static_cast<unsigned>(b & 0x1fffffffull)) * __int_as_float(max(se, 1) << 23);
  lo = (se >= 1) ? lo : 0.0f;
  return {hi, (b >> 63) ? -lo : lo};
}
__device__ __forceinline__ f2 split(float v) { return {v, 0.0f}; }

// float-float -> FP64 (exact: hi + lo has at most 48 significant bits)
__device__ __forceinline__ double to_double(f2 a) { return to_f64(a.hi) + to_f64(a.lo); }

// compile-time float-float constants
struct cf2 {
  float hi, lo;
};
constexpr cf2 make_const(double v) {
  return {static_cast<float>(v), static_cast<float>(v - static_cast<double>(static_cast<float>(v)))};
}
__device__ __forceinline__ f2 k(cf2 c) { return {c.hi, c.lo}; }
constexpr cf2 kThird = make_const(1.0 / 3.0);
constexpr cf2 kM3_7 = make_const(-3.0 / 7.0);
constexpr cf2 kM5_21 = make_const(-5.0 / 21.0);
constexpr cf2 k37_63 = make_const(37.0 / 63.0);

struct Result {
  f2 a;  // a_c (meaningful when collapsed)
  bool collapsed, eds, refined;
};

// One evaluation. seg: the spline image in float-float, two float4 per interval
// ({c0 hi, c0 lo, c1 hi, c1 lo}, {c2, c3, D_k hi, D_k lo}).
template <typename T>
__device__ __forceinline__ Result collapse_point(const T* __restrict__ h, int64_t ps, const float4* __restrict__ seg,
                                                 const float* __restrict__ Dkf, const unsigned short* __restrict__ bucket,
                                                 const DevTable& tab) {
  Result res;
  const f2 xx = split(__ldg(h)), yy = split(__ldg(h + ps)), zz = split(__ldg(h + 2 * ps));
  const f2 xy = split(__ldg(h + 3 * ps)), xz = split(__ldg(h + 4 * ps)), yz = split(__ldg(h + 5 * ps));
  // ---- invariants of M = A - qI
  // sums of one sign stay unnormalised (addu); sums that can cancel are renormalised
  const f2 q = mul(add(add(xx, yy), zz), k(kThird));
  const f2 a = sub(xx, q), b = sub(yy, q), c = sub(zz, q);
  const f2 diag = addu(addu(sqr(a), sqr(b)), sqr(c));
  const f2 off = addu(addu(sqr(xy), sqr(xz)), sqr(yz));
  const f2 p2x3 = addu(scale(diag, 0.5f), off);  // 3 p^2
  const f2 det = add(sub(mul(a, sub(mul(b, c), sqr(yz))), mul(xy, sub(mul(xy, c), mul(yz, xz)))),
                     mul(xz, sub(mul(xy, yz), mul(b, xz))));
  // ---- FP32 trigonometric seed of x = l1 - q
  const float p2f = p2x3.hi * (1.0f / 3.0f);
  const float pf = sqrt_seed(p2f);
  float rf = (p2f > 0.0f) ? __fdividef(det.hi, 2.0f * p2f * pf) : 0.0f;
  rf = fminf(1.0f, fmaxf(-1.0f, rf));
  const float x1f = 2.0f * pf * cos_third_acos(rf);
  // ---- two Newton corrections on x (x^2 - 3p^2) - det (FP32 derivative at each iterate)
  f2 x;
  {
    const float gpf = 3.0f * fmaf(x1f, x1f, -p2f);
    const float yg = (gpf != 0.0f) ? __fdividef(1.0f, gpf) : 0.0f;
    const f2 g = sub(mul(sub(two_prod(x1f, x1f), p2x3), x1f), det);
    x = addu(make(x1f), mul(g, -yg));  // a small correction
  }
  {
    const float gpf = 3.0f * fmaf(x.hi, x.hi, -p2f);
    const float yg = (gpf != 0.0f) ? __fdividef(1.0f, gpf) : 0.0f;
    const f2 g = sub(mul(x, sub(sqr(x), p2x3)), det);
    x = addu(x, mul(g, -yg));
  }
  f2 qq = q;
  res.refined = (1.0f + rf) < kPairTauF && p2f > 0.0f;
  if (res.refined) {
    // l1 ~ l2: the FP64 deflation of the FP64 path, on the original values
    const EigenTop e = eigen_top_fp64(static_cast<double>(__ldg(h)), static_cast<double>(__ldg(h + ps)),
                                      static_cast<double>(__ldg(h + 2 * ps)), static_cast<double>(__ldg(h + 3 * ps)),
                                      static_cast<double>(__ldg(h + 4 * ps)), static_cast<double>(__ldg(h + 5 * ps)));
    qq = split(e.q);
    x = split(e.x);
  }
  // ---- R-LPT coefficients: l1, l2 l3, l2 + l3
  const f2 lam1 = add(qq, x);
  const f2 Pp = add(mul(qq, sub(qq, x)), sub(sqr(x), p2x3));
  const f2 S = sub(scale(qq, 2.0f), x);
  const f2 c2 = mul(Pp, k(kM3_7));
  const f2 c3 = mul(lam1, add(mul(sqr(S), k(kM5_21)), mul(Pp, k(k37_63))));
  // ---- FP32 root (closed form in u = 1/D, two Newton steps), one float-float Newton correction
  const float uf = cubic_largest_root_seed(-lam1.hi, c2.hi, c3.hi);
  float Df = __fdividef(1.0f, uf);
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const float Af = fmaf(fmaf(fmaf(c3.hi, Df, c2.hi), Df, -lam1.hi), Df, 1.0f);
    const float dAf = fmaf(fmaf(3.0f * c3.hi, Df, 2.0f * c2.hi), Df, -lam1.hi);
    Df -= __fdividef(Af, dAf);
  }
  const float dAf = fmaf(fmaf(3.0f * c3.hi, Df, 2.0f * c2.hi), Df, -lam1.hi);
  const f2 A1 = add(mul(add(mul(add(mul(c3, Df), c2), Df), neg(lam1)), Df), make(1.0f));
  const f2 D = fast_two_sum(Df, -__fdividef(A1.hi, dAf));  // the correction is ~1e-7 D
  // ---- collapse test: l1 > 0, 0 < D <= D_top
  const f2 Dtop = {tab.Dtop_hi, tab.Dtop_lo};
  res.collapsed = lam1.hi > 0.0f && D.hi > 0.0f && less_equal(D, Dtop);
  const f2 Dc = res.collapsed ? D : Dtop;
  // ---- a(D): interval from the FP32 value, float-float Horner (c2, c3 terms in FP32)
  const int kk = spline_interval(Dkf, bucket, tab, Dc.hi);
  const float4 s0 = seg[2 * kk], s1 = seg[2 * kk + 1];
  const f2 t = sub(Dc, f2{s1.z, s1.w});
  const float u = fmaf(s1.y, t.hi, s1.x);
  const f2 v = addu(f2{s0.z, s0.w}, mul(t, u));  // c1 dominates
  res.a = add(f2{s0.x, s0.y}, mul(t, v));
  res.eds = res.collapsed && less(Dc, f2{tab.D0_hi, tab.D0_lo});
  if (res.eds) res.a = norm(mul(Dc, f2{tab.eds_hi, tab.eds_lo}));
  return res;
}

// running minimum of a_c in float-float; F = 1/a in FP64 once per point
struct MinA2 {
  f2 a = {__builtin_inff(), 0.0f};
  int r = -1;
  __device__ __forceinline__ void add(bool collapsed, f2 av, int radius) {
    if (collapsed && less(av, a)) {
      a = av;
      r = radius;
    }
  }
  __device__ __forceinline__ void store(double* F_max, int32_t* idx, int32_t scale_idx0) const {
    if (r < 0) return;
    const double F = recip_fp64(to_double(a));
    if (bits(F) > bits(*F_max)) {
      *F_max = F;
      *idx = scale_idx0 + r;
    }
  }
};

}  // namespace dfl
}  // namespace cc
