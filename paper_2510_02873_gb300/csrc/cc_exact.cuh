// cc_exact.cuh -- the collapse condition with exact-background growth ratios
// (CC_MODE_EXACT_GROWTH; arXiv:2510.02873, Sec. 3 gives the collapse time by
// third-order LPT on the cosmology's own growth; the R-LPT reading takes the
// second- and third-order growth factors in their EdS ratios to D1, this mode
// takes them from their ODEs in the actual background).
//
//   A_1(D) = 1 - l1 D + r2(D) l2 l3 D^2 + [r3a(D) u3 + r3b(D) v3] D^3,
//   u3 = -l1 l2 l3 / 3,  v3 = -l1 (l2^2 + l3^2) / 2,
// with r2 = D2/D1^2, r3a = D3a/D1^3, r3b = D3b/D1^3 natural splines in D over
// the growth-table knots (EdS values below the first knot, the last value
// beyond the last knot, where no root counts as a collapse). The root starts
// from the EdS root (closed form, FP32), takes three FP32 Newton steps with the
// FP32 ratio splines and their derivatives, then one FP64 Newton step with the
// FP64 splines; the a(D) spline follows as in the FP64 path.
#pragma once

#include "cc_device.cuh"

namespace cc {
namespace exact {

// EdS ratios (below the first knot)
constexpr double kEds2 = -3.0 / 7.0, kEds3a = -1.0 / 3.0, kEds3b = 10.0 / 21.0;

// A_1 and its derivative in FP32 at D (ratios from the FP32 splines)
__device__ __forceinline__ void stretch_f32(const DevTable& tab, const float* __restrict__ Dkf,
                                            const unsigned short* __restrict__ bucket, float D, float l1, float u2,
                                            float u3, float v3, float& A, float& dA) {
  float r[3], dr[3];
  if (D < Dkf[0]) {
    r[0] = static_cast<float>(kEds2);
    r[1] = static_cast<float>(kEds3a);
    r[2] = static_cast<float>(kEds3b);
    dr[0] = dr[1] = dr[2] = 0.0f;
  } else {
    // beyond the last knot the ratios are held at their last value: an
    // iterate there never collapses, and the spline must not extrapolate
    const bool above = D > tab.Dtopf;
    const float Dr = above ? tab.Dtopf : D;
    const int k = spline_interval(Dkf, bucket, tab, Dr);
    const float t = Dr - Dkf[k];
#pragma unroll
    for (int o = 0; o < 3; ++o) {
      const float4 c = __ldg(tab.rc32 + o * (tab.n - 1) + k);
      r[o] = fmaf(fmaf(fmaf(c.w, t, c.z), t, c.y), t, c.x);
      dr[o] = above ? 0.0f : fmaf(fmaf(3.0f * c.w, t, 2.0f * c.z), t, c.y);
    }
  }
  const float w3 = fmaf(r[1], u3, r[2] * v3);
  const float dw3 = fmaf(dr[1], u3, dr[2] * v3);
  const float D2 = D * D;
  A = fmaf(fmaf(fmaf(w3, D, r[0] * u2), D, -l1), D, 1.0f);
  // d/dD [r2 u2 D^2 + w3 D^3] = (dr2 D^2 + 2 r2 D) u2 + dw3 D^3 + 3 w3 D^2
  dA = fmaf(fmaf(dr[0], D2, 2.0f * r[0] * D), u2, fmaf(dw3 * D, D2, fmaf(3.0f * w3, D2, -l1)));
}

struct Result {
  double a;
  bool collapsed, eds, refined;
};

__device__ __forceinline__ Result collapse_point(double xx, double yy, double zz, double xy, double xz, double yz,
                                                 const double* __restrict__ Dk, const Coef4* __restrict__ coef,
                                                 const float* __restrict__ Dkf,
                                                 const unsigned short* __restrict__ bucket, const DevTable& tab) {
  Result res;
  const EigenTop e = eigen_top_fp64(xx, yy, zz, xy, xz, yz);
  res.refined = e.refined;
  const double q = e.q, x = e.x, p2x3 = e.p2x3;
  const double lam1 = q + x;
  const double Pp = fma(q, q - x, fma(x, x, -p2x3));  // l2 l3
  const double S = fma(2.0, q, -x);                    // l2 + l3
  const double Q = fma(S, S, -2.0 * Pp);               // l2^2 + l3^2
  const double u3 = lam1 * (Pp * (-1.0 / 3.0));
  const double v3 = lam1 * (Q * -0.5);
  // ---- FP32: EdS root, then three Newton steps with the exact ratios
  const float l1f = to_f32_trunc(lam1), u2f = to_f32_trunc(Pp), u3f = to_f32_trunc(u3), v3f = to_f32_trunc(v3);
  const float c3f = fmaf(static_cast<float>(kEds3a), u3f, static_cast<float>(kEds3b) * v3f);
  const float uf = cubic_largest_root_seed(-l1f, static_cast<float>(kEds2) * u2f, c3f);
  float Df = __fdividef(1.0f, uf);
  float A, dA;
#pragma unroll
  for (int it = 0; it < 3; ++it) {
    stretch_f32(tab, Dkf, bucket, Df, l1f, u2f, u3f, v3f, A, dA);
    Df -= __fdividef(A, dA);
  }
  stretch_f32(tab, Dkf, bucket, Df, l1f, u2f, u3f, v3f, A, dA);
  // ---- one FP64 Newton step with the FP64 ratio splines (FP32 derivative)
  const double D0 = to_f64(Df);
  double r[3];
  if (Df < Dkf[0]) {
    r[0] = kEds2;
    r[1] = kEds3a;
    r[2] = kEds3b;
  } else {
    // r = c0 + t (c1 + t (c2 + c3 t)): c2 + c3 t in FP32 (the FP32 copies of
    // the coefficients, t from the FP32 root and knot), the rest in FP64. Over
    // one interval a ratio moves by at most 4.4e-4 of its value, nearly all of
    // it in the c1 term; the FP32 part moves r by ~1e-12 relative at most.
    const bool above = Df > tab.Dtopf;
    const float Dr = above ? tab.Dtopf : Df;
    const int k = spline_interval(Dkf, bucket, tab, Dr);
    const double t = (above ? tab.Dtop : D0) - Dk[k];
    const float tf = Dr - Dkf[k];
#pragma unroll
    for (int o = 0; o < 3; ++o) {
      const float4 cf = __ldg(tab.rc32 + o * (tab.n - 1) + k);
      const Coef4 c = tab.rc64[o * (tab.n - 1) + k];
      r[o] = fma(fma(to_f64(fmaf(cf.w, tf, cf.z)), t, c.c1), t, c.c0);
    }
  }
  const double w3 = fma(r[1], u3, r[2] * v3);
  const double A1 = fma(fma(fma(w3, D0, r[0] * Pp), D0, -lam1), D0, 1.0);
  const double D = fma(-A1, to_f64(__fdividef(1.0f, dA)), D0);
  // ---- collapse test, a(D) as in the FP64 path
  const long long bD = bits(D);
  res.collapsed = bits(lam1) > 0 && bD > 0 && bD <= bits(tab.Dtop);
  const double Dc = res.collapsed ? D : tab.Dtop;
  const int kk = spline_interval(Dkf, bucket, tab, res.collapsed ? to_f32_trunc(D) : tab.Dtopf);
  res.eds = res.collapsed && bits(Dc) < bits(tab.D0);
  const double av = spline_a(coef[kk], Dk[kk], Dc, res.eds, tab);
  res.a = res.collapsed ? av : kInf;
  return res;
}

}  // namespace exact
}  // namespace cc
