// hessgen.cu -- device-side seeded synthetic Hessian planes (input generation only).
//
// Same definition as hessgen/__init__.py: Philox-4x32-10 (Salmon et al. 2011)
// with counter (lo32(4p+k), hi32(4p+k), radius, realization) and key
// (lo32(seed), hi32(seed)), 52-bit uniforms u = (m + 0.5) 2^-52, Box-Muller
// pairs, and the isotropic-field mixing
//   d_ii = s (c2 g_i + c1 g0),  d_ij = s (c1 g_ij),  c1 = sqrt(1/15), c2 = sqrt(2/15).
// The mixing uses explicitly rounded products and sums (no FMA contraction) so
// it matches the host version operation by operation; only the Box-Muller
// log/sin/cos of the two math libraries may differ in the last bits.
// Correlated radii (hg_fill_correlated): a unit-rms field G_r per radius,
// G_0 = N_0, G_r = rho G_{r-1} + sqrt(1 - rho^2) N_r (an AR(1) chain over the
// radii, kept in an FP64 state buffer), planes = s_r G_r.
// This file holds none of the collapse-time arithmetic.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

__device__ __forceinline__ void philox_round(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& c3,
                                             uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t hi0 = __umulhi(M0, c0), lo0 = M0 * c0;
  const uint32_t hi1 = __umulhi(M1, c2), lo1 = M1 * c2;
  const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
  c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
}

__device__ __forceinline__ void philox10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    philox_round(c[0], c[1], c[2], c[3], k0, k1);
  }
}

template <typename T, bool kCorr>
__global__ void fill_kernel(uint64_t seed, uint32_t realization, uint32_t radius, double s, double c1,
                            double c2, int64_t n, int64_t point_offset, T* __restrict__ out,
                            int64_t plane_stride, double rho, double crho, double* __restrict__ state,
                            int first) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint64_t p = static_cast<uint64_t>(point_offset + i);
    uint32_t w[16];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint64_t ctr = p * 4u + static_cast<uint64_t>(k);
      uint32_t c[4] = {static_cast<uint32_t>(ctr), static_cast<uint32_t>(ctr >> 32), radius, realization};
      philox10(c, static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
#pragma unroll
      for (int j = 0; j < 4; ++j) w[4 * k + j] = c[j];
    }
    double g[8];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      double u[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint32_t hi = w[2 * (2 * j + h)], lo = w[2 * (2 * j + h) + 1];
        const uint64_t m = (static_cast<uint64_t>(hi & 0xFFFFFu) << 32) | lo;
        u[h] = __dmul_rn(__dadd_rn(static_cast<double>(m), 0.5), 0x1p-52);
      }
      const double r = __dsqrt_rn(__dmul_rn(-2.0, log(u[0])));
      const double t = __dmul_rn(6.283185307179586, u[1]);
      double sn, cs;
      sincos(t, &sn, &cs);
      g[2 * j] = __dmul_rn(r, cs);
      g[2 * j + 1] = __dmul_rn(r, sn);
    }
    double unit[6];
#pragma unroll
    for (int a = 0; a < 3; ++a) unit[a] = __dadd_rn(__dmul_rn(c2, g[1 + a]), __dmul_rn(c1, g[0]));
#pragma unroll
    for (int a = 0; a < 3; ++a) unit[3 + a] = __dmul_rn(c1, g[4 + a]);
#pragma unroll
    for (int a = 0; a < 6; ++a) {
      double v = unit[a];
      if constexpr (kCorr) {
        double* st = state + a * n + i;
        v = first ? v : __dadd_rn(__dmul_rn(rho, *st), __dmul_rn(crho, v));
        *st = v;
      }
      out[a * plane_stride + i] = static_cast<T>(__dmul_rn(s, v));
    }
  }
}

// unit white noise: the first Gaussian of the point's draws (counter 4p, the
// given stream slot as the radius word)
__global__ void white_kernel(uint64_t seed, uint32_t realization, uint32_t slot, int64_t n, double* __restrict__ out) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint64_t ctr = static_cast<uint64_t>(i) * 4u;
    uint32_t c[4] = {static_cast<uint32_t>(ctr), static_cast<uint32_t>(ctr >> 32), slot, realization};
    philox10(c, static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
    double u[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint64_t m = (static_cast<uint64_t>(c[2 * h] & 0xFFFFFu) << 32) | c[2 * h + 1];
      u[h] = __dmul_rn(__dadd_rn(static_cast<double>(m), 0.5), 0x1p-52);
    }
    const double r = __dsqrt_rn(__dmul_rn(-2.0, log(u[0])));
    out[i] = __dmul_rn(r, cos(__dmul_rn(6.283185307179586, u[1])));
  }
}

}  // namespace

extern "C" __attribute__((visibility("default"))) int hg_white(uint64_t seed, uint32_t realization, uint32_t slot,
                                                              int64_t n, double* out, void* stream) {
  if (n <= 0) return 0;
  if (out == nullptr) return 1;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t need = (n + 255) / 256;
  const int64_t cap = static_cast<int64_t>(sms > 0 ? sms : 1) * 16;
  white_kernel<<<static_cast<int>(need < cap ? need : cap), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      seed, realization, slot, n, out);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

extern "C" __attribute__((visibility("default"))) int hg_fill(uint64_t seed, uint32_t realization,
                                                             uint32_t radius, double s, double c1,
                                                             double c2, int64_t n, int64_t point_offset,
                                                             void* out, int64_t plane_stride, int dtype,
                                                             void* stream) {
  if (n <= 0) return 0;
  if (out == nullptr || plane_stride < n || (dtype != 8 && dtype != 4)) return 1;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t need = (n + 255) / 256;
  const int64_t cap = static_cast<int64_t>(sms > 0 ? sms : 1) * 16;
  const int grid = static_cast<int>(need < cap ? need : cap);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (dtype == 8)
    fill_kernel<double, false><<<grid, 256, 0, st>>>(seed, realization, radius, s, c1, c2, n, point_offset,
                                                     static_cast<double*>(out), plane_stride, 0.0, 0.0, nullptr, 1);
  else
    fill_kernel<float, false><<<grid, 256, 0, st>>>(seed, realization, radius, s, c1, c2, n, point_offset,
                                                    static_cast<float*>(out), plane_stride, 0.0, 0.0, nullptr, 1);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

// Correlated radii: state is a device FP64 (6, n) buffer holding G_{r-1}
// (overwritten with G_r); first != 0 starts the chain (G_0 = N_0).
extern "C" __attribute__((visibility("default"))) int hg_fill_correlated(
    uint64_t seed, uint32_t realization, uint32_t radius, double s, double c1, double c2, double rho,
    double crho, int64_t n, void* out, int64_t plane_stride, int dtype, double* state, int first, void* stream) {
  if (n <= 0) return 0;
  if (out == nullptr || state == nullptr || plane_stride < n || (dtype != 8 && dtype != 4)) return 1;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t need = (n + 255) / 256;
  const int64_t cap = static_cast<int64_t>(sms > 0 ? sms : 1) * 16;
  const int grid = static_cast<int>(need < cap ? need : cap);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (dtype == 8)
    fill_kernel<double, true><<<grid, 256, 0, st>>>(seed, realization, radius, s, c1, c2, n, 0,
                                                    static_cast<double*>(out), plane_stride, rho, crho, state, first);
  else
    fill_kernel<float, true><<<grid, 256, 0, st>>>(seed, realization, radius, s, c1, c2, n, 0,
                                                   static_cast<float*>(out), plane_stride, rho, crho, state, first);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}
