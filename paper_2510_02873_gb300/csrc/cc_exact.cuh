// cc_exact.cuh -- the collapse condition with exact-background growth ratios
// (CC_MODE_EXACT_GROWTH; arXiv:2510.02873, Sec. 3 gives the collapse time by
// third-order LPT on the cosmology's own growth; the R-LPT reading takes the
// second- and third-order growth factors in their EdS ratios to D1, this mode
// takes them from their ODEs in the actual background).
//
//   A_1(D) = 1 - l1 D + r2(D) l2 l3 D^2 + l1 [r3a'(D) l2 l3 + r3b'(D) (l2^2 + l3^2)] D^3,
//   r3a' = -r3a / 3,  r3b' = -r3b / 2,
// with r2 = D2/D1^2, r3a = D3a/D1^3, r3b = D3b/D1^3. With
// l2^2 + l3^2 = (l2 + l3)^2 - 2 l2 l3 the bracket is ra l2 l3 + rb (l2 + l3)^2,
// ra = r3a' - 2 r3b', rb = r3b': r2, ra and rb are natural splines in D over
// the growth-table knots (EdS values below the first knot, the last value
// beyond the last knot, where no root counts as a collapse). In EdS
// r3a' = 1/9 and r3b' = -5/21, the R-LPT coefficients, so ra = 37/63. The
// root starts from the EdS root (closed form, FP32), takes three FP32 Newton
// steps with the FP32 ratio splines and their derivatives, then one FP64 Newton
// step with the FP64 splines that yields t = D - e_k for the a(D) spline
// directly, as in the FP64 path.
#pragma once

#include "cc_device.cuh"

namespace cc {
namespace exact {

// EdS ratios (below the first knot): r2, ra = r3a' - 2 r3b', rb = r3b'
constexpr double kEds2 = -3.0 / 7.0, kEdsA = 37.0 / 63.0, kEdsB = -5.0 / 21.0;

// A_1 and its derivative in FP32 at D (ratios from the FP32 splines);
// u2 = l2 l3, Q = (l2 + l3)^2
__device__ __forceinline__ void stretch_f32(const DevTable& tab, const float* __restrict__ Dkf,
                                            const unsigned short* __restrict__ bucket, float D, float l1, float u2,
                                            float Q, float& A, float& dA) {
  float r[3], dr[3];
  if (D < Dkf[0]) {
    r[0] = static_cast<float>(kEds2);
    r[1] = static_cast<float>(kEdsA);
    r[2] = static_cast<float>(kEdsB);
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
  const float w3 = l1 * fmaf(r[1], u2, r[2] * Q);
  const float dw3 = l1 * fmaf(dr[1], u2, dr[2] * Q);
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
  (void)Dk;
  Result res;
  const EigenTop e = eigen_top_fp64(xx, yy, zz, xy, xz, yz);
  res.refined = e.refined;
  const double s = e.s, x = e.x, p2x3 = e.p2x3;
  const double lam1 = fma(s, 1.0 / 3.0, x);
  const double Pp = fma(e.q, fma(s, 1.0 / 3.0, -x), fma(x, x, -p2x3));  // l2 l3
  const double S = fma(s, 2.0 / 3.0, -x);                               // l2 + l3
  const double Q = S * S;                                               // (l2 + l3)^2
  // ---- FP32: EdS root, then three Newton steps with the exact ratios
  const float l1f = to_f32_trunc(lam1), u2f = to_f32_trunc(Pp), Qf = to_f32_trunc(Q);
  const float c3f = l1f * fmaf(static_cast<float>(kEdsA), u2f, static_cast<float>(kEdsB) * Qf);
  const float uf = cubic_largest_root_seed(-l1f, static_cast<float>(kEds2) * u2f, c3f);
  float Df = __fdividef(1.0f, uf);
  float A, dA;
#pragma unroll
  for (int it = 0; it < 3; ++it) {
    stretch_f32(tab, Dkf, bucket, Df, l1f, u2f, Qf, A, dA);
    Df -= __fdividef(A, dA);
  }
  stretch_f32(tab, Dkf, bucket, Df, l1f, u2f, Qf, A, dA);
  // ---- one FP64 Newton step with the FP64 ratio splines (FP32 derivative)
  const double D0 = to_f64(Df);
  const int k = spline_interval(Dkf, bucket, tab, Df);
  const bool below = Df < Dkf[0];
  double r[3];
  if (below) {
    r[0] = kEds2;
    r[1] = kEdsA;
    r[2] = kEdsB;
  } else {
    // r = c0 + t (c1 + t (c2 + c3 t)): c2 + c3 t in FP32 (the FP32 copies of
    // the coefficients), the rest in FP64. Over one interval a ratio moves by
    // at most 4.4e-4 of its value, nearly all of it in the c1 term; the FP32
    // part moves r by ~1e-12 relative at most. t = D0 - e_k is exact in FP32
    // (the splines are expanded about the FP32 knots e_k); beyond the last
    // knot the ratios are taken at the FP32 D_top (no collapse there, but an
    // FP64 step may land back within ~1e-7 of it: a point then on the a_max
    // edge, where F ~ 1 either way).
    const bool above = Df > tab.Dtopf;
    const float tf = (above ? tab.Dtopf : Df) - Dkf[k];
    const double t = to_f64(tf);
#pragma unroll
    for (int o = 0; o < 3; ++o) {
      const float4 cf = __ldg(tab.rc32 + o * (tab.n - 1) + k);
      const Coef4 c = tab.rc64[o * (tab.n - 1) + k];
      r[o] = fma(fma(to_f64(fmaf(cf.w, tf, cf.z)), t, c.c1), t, c.c0);
    }
  }
  const double w3 = lam1 * fma(r[1], Pp, r[2] * Q);
  const double A1 = fma(fma(fma(w3, D0, r[0] * Pp), D0, -lam1), D0, 1.0);
  // ---- the step lands on t = D - e_k (on the EdS segment t = D), and the
  // collapse test and a(D) follow as in collapse_point_fp64
  const float t0 = below ? Df : __fsub_rn(Df, Dkf[k]);
  const double t = fma(-A1, to_f64(rcp_seed(dA)), to_f64_normal(t0));
  res.collapsed = bits(lam1) > 0 && Df > 0.0f && (k < tab.n - 2 || bits(t) <= bits(tab.Dtop_t)) && finite_bits(t);
  res.eds = below && res.collapsed;
  const double av = spline_a_t(coef[k], t, res.eds, tab);
  res.a = res.collapsed ? av : kInf;
  return res;
}

}  // namespace exact
}  // namespace cc
