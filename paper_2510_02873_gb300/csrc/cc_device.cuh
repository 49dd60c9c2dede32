// cc_device.cuh -- FP64 device arithmetic of the collapse-time path.
//
// Per point (arXiv:2510.02873, Sec. 3): eigenvalues of the symmetric 3x3
// Hessian (closed-form trigonometric solve, sorted descending), the
// third-order LPT collapse condition solved as a cubic, and the natural cubic
// spline a(D) of the inverse growth function. Control flow is predicated
// where the paper asks for masked execution (Sec. 4.1); the only real branch
// is the rare near-degenerate eigenvalue pair.
#pragma once

#include "cc_internal.h"

namespace cc {

constexpr double kSqrt3 = 1.7320508075688772935;
// 1 + r below this: l1 and l2 nearly coincide and acos(r) loses accuracy in
// the pair; they are re-solved by deflation (1 + r ~ 4.5 theta^2, eigenvalue
// error ~ 0.2 eps p / theta, so 1e-8 keeps it below ~1e-12 p).
constexpr double kPairTau = 1e-8;

// Re-solve l1 >= l2 when they are nearly equal: l3 (isolated, accurate from
// the trigonometric solve) gives an eigenvector v3 as the largest cross
// product of two rows of A - l3 I; A restricted to the plane orthogonal to v3
// is a 2x2 symmetric matrix whose eigenvalues follow without cancellation.
__device__ __noinline__ void refine_top_pair(double xx, double yy, double zz, double xy, double xz,
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
  if (!(nv > 0.0)) return;  // l3 not isolated either: all equal, keep the trigonometric values
  const double iv = rsqrt(nv);
  vx *= iv; vy *= iv; vz *= iv;
  // u orthogonal to v, then w = v x u
  double ux, uy, uz;
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

// Eigenvalues l1 >= l2 >= l3 of [[xx,xy,xz],[xy,yy,yz],[xz,yz,zz]] by the
// trigonometric solution of the characteristic cubic (Smith 1961):
//   q = tr/3, p^2 = (|A - qI|_F^2)/6, r = det(A - qI) / (2 p^3),
//   phi = acos(r)/3, l1 = q + 2p cos(phi), l3 = q + 2p cos(phi + 2pi/3),
//   l2 = q + 2p cos(phi - 2pi/3);
// the two shifted cosines come from one sincos by the angle-sum identity.
// Returns true when the near-degenerate top pair was re-solved.
__device__ __forceinline__ bool eigen_sym3(double xx, double yy, double zz, double xy, double xz,
                                           double yz, double& l1, double& l2, double& l3) {
  const double q = (xx + yy + zz) * (1.0 / 3.0);
  const double a = xx - q, b = yy - q, c = zz - q;
  const double p2 = (a * a + b * b + c * c + 2.0 * (xy * xy + xz * xz + yz * yz)) * (1.0 / 6.0);
  const double p = sqrt(p2);
  const double det = a * (b * c - yz * yz) - xy * (xy * c - yz * xz) + xz * (xy * yz - b * xz);
  double r = (p2 > 0.0) ? det / (2.0 * p2 * p) : 0.0;
  r = fmin(1.0, fmax(-1.0, r));
  const double phi = acos(r) * (1.0 / 3.0);
  double s, co;
  sincos(phi, &s, &co);
  l1 = fma(2.0 * p, co, q);
  l2 = fma(p, fma(kSqrt3, s, -co), q);   // q + 2p cos(phi - 2pi/3)
  l3 = fma(-p, fma(kSqrt3, s, co), q);   // q + 2p cos(phi + 2pi/3)
  const bool pair = (1.0 + r) < kPairTau && p2 > 0.0;
  if (pair) refine_top_pair(xx, yy, zz, xy, xz, yz, l3, l1, l2);
  return pair;
}

// Collapse growth factor (Sec. 3, Classic: third-order LPT stretch of the
// axis with the largest eigenvalue). With u = 1/D the condition A_1(D) = 0
// becomes the monic cubic
//   P(u) = u^3 - l1 u^2 + c2 u + c3,  c2 = -3/7 l2 l3,
//   c3 = l1 (l2 l3 / 9 - 5/21 (l2^2 + l3^2)).
// For l1 > 0 the collapse root is unique (A_1 is strictly decreasing on D > 0),
// so D_c = 1/u* with u* the largest real root of P: closed form (Cardano when
// one root is real, trigonometric when three are), then Newton polish.
__device__ __forceinline__ double collapse_u_fp64(double l1, double l2, double l3) {
  const double b = -l1;
  const double c = (-3.0 / 7.0) * (l2 * l3);
  const double d = l1 * ((l2 * l3) * (1.0 / 9.0) - (5.0 / 21.0) * (l2 * l2 + l3 * l3));
  const double b3 = b * (1.0 / 3.0);
  const double pp = c - b * b3;                                  // c - b^2/3
  const double qq = b3 * (2.0 * b3 * b3 - c) + d;                 // 2b^3/27 - bc/3 + d
  const double disc = 0.25 * qq * qq + pp * pp * pp * (1.0 / 27.0);
  double t;
  if (disc > 0.0) {
    const double A = cbrt(0.5 * fabs(qq) + sqrt(disc));
    const double C = (qq > 0.0) ? -A : A;
    t = (C != 0.0) ? C - pp / (3.0 * C) : 0.0;
  } else {
    const double m = sqrt(-pp * (1.0 / 3.0));
    double arg = (m > 0.0) ? (-0.5 * qq) / (m * m * m) : 0.0;
    arg = fmin(1.0, fmax(-1.0, arg));
    t = 2.0 * m * cos(acos(arg) * (1.0 / 3.0));
  }
  double u = t - b3;
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const double P = fma(fma(u + b, u, c), u, d);
    const double dP = fma(fma(3.0, u, 2.0 * b), u, c);
    u = (dP != 0.0) ? u - P / dP : u;
  }
  return u;
}

// a(D) from the natural spline; interval k = largest with D_k <= D (clamped),
// found by a branch-free binary search; below the first knot a = a0 D / D0.
__device__ __forceinline__ double a_of_D_fp64(const double* __restrict__ Dk,
                                              const Coef4* __restrict__ coef,
                                              const DevTable& tab, double D, bool& eds) {
  int k = 0;
  for (int step = tab.search_steps; step > 0; step >>= 1) {
    const int j = k + step;
    k = (j <= tab.n - 2 && Dk[j] <= D) ? j : k;
  }
  const double t = D - Dk[k];
  const Coef4 cf = coef[k];
  const double a_spl = fma(fma(fma(cf.c3, t, cf.c2), t, cf.c1), t, cf.c0);
  eds = D < tab.D0;
  return eds ? tab.eds_slope * D : a_spl;
}

struct PointResult {
  double F;
  bool collapsed, eds, refined;
};

// Full per-point collapse value F = 1/a_c (or 0 for no collapse).
__device__ __forceinline__ PointResult collapse_point_fp64(double xx, double yy, double zz, double xy,
                                                           double xz, double yz,
                                                           const double* __restrict__ Dk,
                                                           const Coef4* __restrict__ coef,
                                                           const DevTable& tab) {
  PointResult res;
  double l1, l2, l3;
  res.refined = eigen_sym3(xx, yy, zz, xy, xz, yz, l1, l2, l3);
  const double u = collapse_u_fp64(l1, l2, l3);
  const double Dc = 1.0 / u;
  res.collapsed = (l1 > 0.0) && (u > 0.0) && (Dc <= tab.Dtop);
  bool eds;
  const double a = a_of_D_fp64(Dk, coef, tab, res.collapsed ? Dc : tab.Dtop, eds);
  res.eds = eds && res.collapsed;
  res.F = res.collapsed ? 1.0 / a : 0.0;
  return res;
}

}  // namespace cc
