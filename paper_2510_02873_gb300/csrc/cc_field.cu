// cc_field.cu -- device-resident field -> smoothed Hessian planes, the FFT
// stage ahead of the collapse computation (arXiv:2510.02873, Sec. 3: the
// second derivatives of the potential come from FFTs, and the planned step is
// to keep them on the device between the FFTs and the collapse kernel).
//
// Field: unit white noise w on an N^3 periodic grid (side `box`, C order),
// delta_k = DFT(w) sqrt(P(k)) with P(k) = A k^n exp(-(k/k_cut)^2), Nyquist
// modes and k = 0 zeroed. Hessian at radius R: H_ij = IDFT[(k_i k_j / k^2)
// G(kR) delta_k] with G(kR) = exp(-k^2 R^2 / 2) (trace = smoothed density).
// The transforms are cuFFT (D2Z once per field; six Z2D, or C2R for FP32
// planes, per radius as one batched plan writing straight into the caller's
// planes); the k-space products are this file's kernels. The Gaussian factor is
// separable, G = g(k_x) g(k_y) g(k_z), so the per-mode work is products of
// three table entries (host FP64 exp per axis) instead of an exp per mode. The
// colouring and the rms s(R) work on shells of equal k^2 (sqrt(P) per shell;
// weighted mode counts per shell, built once) instead of on every mode.
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>

#include "cc_internal.h"

namespace cc {
namespace {

constexpr int kFieldMaxN = 1024;

int check_cufft(cufftResult r, const char* what) {
  if (r == CUFFT_SUCCESS) return CC_OK;
  return set_error(r == CUFFT_ALLOC_FAILED ? CC_ENOMEM : CC_ECUDA,
                   std::string(what) + " failed (cuFFT status " + std::to_string(static_cast<int>(r)) + ")");
}

// per-axis tables: signed wavenumbers of the full axes and of the half axis,
// and the per-axis Gaussian factors (1 when only the wavenumbers are needed)
struct AxisTables {
  double k[kFieldMaxN];        // k(m), m = 0..N-1 (signed frequency)
  double g[kFieldMaxN];        // exp(-k(m)^2 R^2 / 2)
  double gz[kFieldMaxN / 2 + 1];
  int N, Nz;
  double kz0;                  // 2 pi / box (k_z = kz0 * iz)
};

__device__ __forceinline__ void decompose(int64_t idx, int N, int Nz, int& ix, int& iy, int& iz) {
  iz = static_cast<int>(idx % Nz);
  const int64_t r = idx / Nz;
  iy = static_cast<int>(r % N);
  ix = static_cast<int>(r / N);
}

// sqrt(P(k)) per shell n2 (k^2 = kf2 n2; shell 0, k = 0, gets 0)
__global__ void shell_amp_kernel(int n_shells, double kf2, double A, double n_idx, double k_cut,
                                 double* __restrict__ amp) {
  const int stride = gridDim.x * blockDim.x;
  for (int n2 = blockIdx.x * blockDim.x + threadIdx.x; n2 < n_shells; n2 += stride) {
    const double k2 = kf2 * n2;
    amp[n2] = (n2 > 0) ? sqrt(A * pow(sqrt(k2), n_idx) * exp(-k2 / (k_cut * k_cut))) : 0.0;
  }
}

// delta_k = DFT(w) sqrt(P(k)) from the shell table; Nyquist modes zeroed
__global__ void color_kernel(double2* __restrict__ dk, int64_t nc, int N, int Nz,
                             const double* __restrict__ amp) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int h = N / 2;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < nc; i += stride) {
    int ix, iy, iz;
    decompose(i, N, Nz, ix, iy, iz);
    double a = 0.0;
    if (ix != h && iy != h && iz != h) {
      const int sx = ix < h ? ix : ix - N, sy = iy < h ? iy : iy - N;
      a = __ldg(amp + (sx * sx + sy * sy + iz * iz));
    }
    double2 v = dk[i];
    v.x *= a;
    v.y *= a;
    dk[i] = v;
  }
}

// the six k-space products of one radius (component order xx yy zz xy xz yz),
// scaled by 1/N^3 for the unnormalised inverse transform, in FP64 for FP64
// planes and in FP32 (from the FP32 copy of the tables) for FP32 planes
template <typename C, typename R, typename Tab>
__global__ void hessian_k_kernel(const double2* __restrict__ dk, int64_t nc, const Tab t, R scale,
                                 C* __restrict__ out) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < nc; i += stride) {
    int ix, iy, iz;
    decompose(i, t.N, t.Nz, ix, iy, iz);
    const R kx = t.k[ix], ky = t.k[iy], kz = t.kz0 * static_cast<R>(iz);
    const R k2 = fma(kx, kx, fma(ky, ky, kz * kz));
    const R w = (k2 > R(0)) ? (t.g[ix] * t.g[iy] * t.gz[iz]) * scale / k2 : R(0);
    const double2 d = dk[i];
    R re, im;
    if constexpr (sizeof(R) == 8) {
      re = d.x * w;
      im = d.y * w;
    } else {
      re = __double2float_rn(d.x) * w;
      im = __double2float_rn(d.y) * w;
    }
    const R f[6] = {kx * kx, ky * ky, kz * kz, kx * ky, kx * kz, ky * kz};
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      C o;
      o.x = re * f[c];
      o.y = im * f[c];
      out[c * nc + i] = o;
    }
  }
}

// FP32 copy of the axis tables (FP32 planes)
struct AxisTables32 {
  float k[kFieldMaxN];
  float g[kFieldMaxN];
  float gz[kFieldMaxN / 2 + 1];
  int N, Nz;
  float kz0;
};

// P(k) G(kR)^2 depends on a mode only through the integer
// n2 = sx^2 + sy^2 + sz^2 of its signed frequencies (k^2 = (2 pi / box)^2 n2).
// shell_count_kernel adds each mode's weight over the full grid (modes with
// 0 < iz < N/2 stand for their mirror images too, so 2; iz = 0 counts 1;
// Nyquist modes and k = 0 are excluded) to its shell n2, once per field;
// sigma_shell_kernel then sums one term per shell for each R.
__global__ void shell_count_kernel(int64_t nc, int N, int Nz, unsigned long long* __restrict__ cnt) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int h = N / 2;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < nc; i += stride) {
    int ix, iy, iz;
    decompose(i, N, Nz, ix, iy, iz);
    if (ix == h || iy == h || iz == h) continue;
    const int sx = ix < h ? ix : ix - N, sy = iy < h ? iy : iy - N;
    const int n2 = sx * sx + sy * sy + iz * iz;
    if (n2 == 0) continue;
    atomicAdd(cnt + n2, iz == 0 ? 1ull : 2ull);
  }
}

__global__ void sigma_shell_kernel(const unsigned long long* __restrict__ cnt, int n_shells, double kf2, double A,
                                   double n_idx, double k_cut, double R, double* __restrict__ acc) {
  double s = 0.0;
  const int stride = gridDim.x * blockDim.x;
  for (int n2 = blockIdx.x * blockDim.x + threadIdx.x; n2 < n_shells; n2 += stride) {
    const unsigned long long c = cnt[n2];
    if (c == 0ull) continue;
    const double k2 = kf2 * n2;
    s += static_cast<double>(c) * (A * pow(sqrt(k2), n_idx) * exp(-k2 / (k_cut * k_cut)) * exp(-k2 * R * R));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(acc, s);
}

int grid_for(int64_t n, int num_sms) {
  return static_cast<int>(std::min<int64_t>((n + 255) / 256, static_cast<int64_t>(num_sms) * 8));
}

}  // namespace
}  // namespace cc

using namespace cc;

struct cc_field {
  cc_ctx* ctx = nullptr;
  int N = 0;
  cc_spectrum spec{};
  int64_t nc = 0;                 // N * N * (N / 2 + 1)
  double2* dk = nullptr;          // delta_k (FP64; the FP32 products are rounded from it)
  void* work = nullptr;           // six k-space products
  size_t work_bytes = 0;
  double* acc = nullptr;          // sigma accumulator
  unsigned long long* shells = nullptr;  // weighted mode count per n2 (built at the first sigma call)
  int n_shells = 0;
  std::map<std::pair<int, int64_t>, cufftHandle> inv_plans;  // (dtype, plane_stride) -> batched inverse
};

namespace {

AxisTables axis_tables(const cc_field* f, double R) {
  AxisTables t;
  const int N = f->N;
  t.N = N;
  t.Nz = N / 2 + 1;
  t.kz0 = 2.0 * 3.14159265358979323846 / f->spec.box;
  for (int m = 0; m < N; ++m) {
    const int s = (m < (N + 1) / 2) ? m : m - N;  // signed frequency (numpy fftfreq order)
    t.k[m] = t.kz0 * s;
    t.g[m] = std::exp(-0.5 * t.k[m] * t.k[m] * R * R);
  }
  for (int m = 0; m < t.Nz; ++m) t.gz[m] = std::exp(-0.5 * (t.kz0 * m) * (t.kz0 * m) * R * R);
  return t;
}

}  // namespace

extern "C" {

int cc_field_create(cc_ctx* ctx, const double* white, int32_t N, const cc_spectrum* spec, cc_field** out,
                    void* stream) {
  if (!ctx || !white || !spec || !out) return set_error(CC_EINVAL, "ctx, white, spec and out must be non-NULL");
  *out = nullptr;
  if (N < 4 || N > kFieldMaxN || N % 2) return set_error(CC_EINVAL, "N must be even, 4 <= N <= 1024");
  if (!(spec->box > 0.0) || !(spec->amplitude > 0.0) || !(spec->k_cut > 0.0) || !std::isfinite(spec->index) ||
      !std::isfinite(spec->box) || !std::isfinite(spec->amplitude) || !std::isfinite(spec->k_cut))
    return set_error(CC_EINVAL, "spectrum: box, amplitude, k_cut > 0 and finite index");
  if (reinterpret_cast<uintptr_t>(white) % 16) return set_error(CC_EINVAL, "white must be 16-byte aligned");
  if (int rc = select_device(ctx)) return rc;
  cc_field* f = new (std::nothrow) cc_field();
  if (!f) return set_error(CC_ENOMEM, "host allocation failed");
  f->ctx = ctx;
  f->N = N;
  f->spec = *spec;
  f->nc = static_cast<int64_t>(N) * N * (N / 2 + 1);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = check_cuda(cudaMalloc(&f->dk, sizeof(double2) * f->nc), "cudaMalloc(delta_k)");
  if (!rc) rc = check_cuda(cudaMalloc(&f->acc, sizeof(double)), "cudaMalloc(accumulator)");
  cufftHandle fwd = 0;
  bool have_plan = false;
  if (!rc) {
    rc = check_cufft(cufftPlan3d(&fwd, N, N, N, CUFFT_D2Z), "cufftPlan3d(D2Z)");
    have_plan = !rc;
  }
  if (!rc) rc = check_cufft(cufftSetStream(fwd, st), "cufftSetStream");
  // an out-of-place real-to-complex transform leaves its input unchanged
  if (!rc) rc = check_cufft(cufftExecD2Z(fwd, const_cast<double*>(white), reinterpret_cast<cufftDoubleComplex*>(f->dk)),
                            "cufftExecD2Z");
  // sqrt(P) per shell n2 of the non-Nyquist modes (the shells of s(R))
  const int h = N / 2;
  const int n_shells = 3 * (h - 1) * (h - 1) + 1;
  double* amp = nullptr;
  if (!rc) rc = check_cuda(cudaMalloc(&amp, sizeof(double) * n_shells), "cudaMalloc(shell amplitudes)");
  if (!rc) {
    const double kf = 2.0 * 3.14159265358979323846 / spec->box;
    shell_amp_kernel<<<grid_for(n_shells, ctx->num_sms), 256, 0, st>>>(n_shells, kf * kf, spec->amplitude,
                                                                        spec->index, spec->k_cut, amp);
    rc = check_cuda(cudaGetLastError(), "shell_amp_kernel launch");
  }
  if (!rc) {
    color_kernel<<<grid_for(f->nc, ctx->num_sms), 256, 0, st>>>(f->dk, f->nc, N, h + 1, amp);
    rc = check_cuda(cudaGetLastError(), "color_kernel launch");
  }
  // the plan and the shell table may be released only after the kernels have run
  if (have_plan || amp) {
    const int rs = check_cuda(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    if (!rc) rc = rs;
  }
  if (have_plan) cufftDestroy(fwd);
  if (amp) cudaFree(amp);
  if (rc) {
    cc_field_destroy(f);
    return rc;
  }
  *out = f;
  return CC_OK;
}

int cc_field_sigma(cc_field* f, double R, double* sigma, void* stream) {
  if (!f || !sigma) return set_error(CC_EINVAL, "field and sigma must be non-NULL");
  if (!(R >= 0.0) || !std::isfinite(R)) return set_error(CC_EINVAL, "R must be finite and >= 0");
  if (int rc = select_device(f->ctx)) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!f->shells) {
    const int h = f->N / 2;
    const int n_shells = 3 * (h - 1) * (h - 1) + 1;  // largest n2 of a non-Nyquist mode, plus one
    unsigned long long* cnt = nullptr;
    if (int rc = check_cuda(cudaMalloc(&cnt, sizeof(unsigned long long) * n_shells), "cudaMalloc(shell counts)"))
      return rc;
    int rc = check_cuda(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * n_shells, st), "cudaMemsetAsync");
    if (!rc) {
      shell_count_kernel<<<grid_for(f->nc, f->ctx->num_sms), 256, 0, st>>>(f->nc, f->N, h + 1, cnt);
      rc = check_cuda(cudaGetLastError(), "shell_count_kernel launch");
    }
    if (rc) {
      cudaFree(cnt);
      return rc;
    }
    f->shells = cnt;
    f->n_shells = n_shells;
  }
  if (int rc = check_cuda(cudaMemsetAsync(f->acc, 0, sizeof(double), st), "cudaMemsetAsync")) return rc;
  const double kf = 2.0 * 3.14159265358979323846 / f->spec.box;
  sigma_shell_kernel<<<grid_for(f->n_shells, f->ctx->num_sms), 256, 0, st>>>(
      f->shells, f->n_shells, kf * kf, f->spec.amplitude, f->spec.index, f->spec.k_cut, R, f->acc);
  if (int rc = check_cuda(cudaGetLastError(), "sigma_shell_kernel launch")) return rc;
  double s = 0.0;
  if (int rc = check_cuda(cudaMemcpyAsync(&s, f->acc, sizeof(double), cudaMemcpyDeviceToHost, st), "D2H sigma")) return rc;
  if (int rc = check_cuda(cudaStreamSynchronize(st), "cudaStreamSynchronize")) return rc;
  const double n3 = static_cast<double>(f->N) * f->N * f->N;
  *sigma = std::sqrt(s / n3);
  return CC_OK;
}

int cc_field_hessian(cc_field* f, double R, void* planes, int32_t dtype, int64_t plane_stride, void* stream) {
  if (!f || !planes) return set_error(CC_EINVAL, "field and planes must be non-NULL");
  if (dtype != CC_F64 && dtype != CC_F32) return set_error(CC_EINVAL, "dtype must be CC_F64 or CC_F32");
  if (!(R >= 0.0) || !std::isfinite(R)) return set_error(CC_EINVAL, "R must be finite and >= 0");
  const int64_t n3 = static_cast<int64_t>(f->N) * f->N * f->N;
  if (plane_stride < n3) return set_error(CC_EINVAL, "plane_stride must be >= N^3");
  if ((plane_stride * dtype) % 16 || reinterpret_cast<uintptr_t>(planes) % 16)
    return set_error(CC_EINVAL, "planes must start on 16 bytes and plane_stride * element size be a multiple of 16");
  if (int rc = select_device(f->ctx)) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t elem = (dtype == CC_F64) ? sizeof(double2) : sizeof(float2);
  const size_t need = elem * 6 * static_cast<size_t>(f->nc);
  if (need > f->work_bytes) {
    if (f->work) cudaFree(f->work);
    f->work = nullptr;
    f->work_bytes = 0;
    if (int rc = check_cuda(cudaMalloc(&f->work, need), "cudaMalloc(field work)")) return rc;
    f->work_bytes = need;
  }
  const auto key = std::make_pair(static_cast<int>(dtype), plane_stride);
  auto it = f->inv_plans.find(key);
  if (it == f->inv_plans.end()) {
    cufftHandle p = 0;
    int n[3] = {f->N, f->N, f->N};
    int inembed[3] = {f->N, f->N, f->N / 2 + 1};
    int onembed[3] = {f->N, f->N, f->N};
    // odist may exceed the int range of cufftPlanMany only for planes above 2^31 elements
    if (plane_stride > INT32_MAX || f->nc > INT32_MAX) return set_error(CC_ERANGE, "grid too large for one batched plan");
    if (int rc = check_cufft(cufftPlanMany(&p, 3, n, inembed, 1, static_cast<int>(f->nc), onembed, 1,
                                           static_cast<int>(plane_stride), dtype == CC_F64 ? CUFFT_Z2D : CUFFT_C2R, 6),
                             "cufftPlanMany(inverse)"))
      return rc;
    it = f->inv_plans.emplace(key, p).first;
  }
  if (int rc = check_cufft(cufftSetStream(it->second, st), "cufftSetStream")) return rc;
  const AxisTables t = axis_tables(f, R);
  const double scale = 1.0 / static_cast<double>(n3);
  const int grid = grid_for(f->nc, f->ctx->num_sms);
  if (dtype == CC_F64) {
    hessian_k_kernel<double2, double, AxisTables><<<grid, 256, 0, st>>>(f->dk, f->nc, t, scale,
                                                                        static_cast<double2*>(f->work));
    if (int rc = check_cuda(cudaGetLastError(), "hessian_k_kernel launch")) return rc;
    return check_cufft(cufftExecZ2D(it->second, static_cast<cufftDoubleComplex*>(f->work), static_cast<double*>(planes)),
                       "cufftExecZ2D");
  }
  AxisTables32 t32;
  t32.N = t.N;
  t32.Nz = t.Nz;
  t32.kz0 = static_cast<float>(t.kz0);
  for (int m = 0; m < t.N; ++m) {
    t32.k[m] = static_cast<float>(t.k[m]);
    t32.g[m] = static_cast<float>(t.g[m]);
  }
  for (int m = 0; m < t.Nz; ++m) t32.gz[m] = static_cast<float>(t.gz[m]);
  hessian_k_kernel<float2, float, AxisTables32><<<grid, 256, 0, st>>>(f->dk, f->nc, t32, static_cast<float>(scale),
                                                                      static_cast<float2*>(f->work));
  if (int rc = check_cuda(cudaGetLastError(), "hessian_k_kernel launch")) return rc;
  return check_cufft(cufftExecC2R(it->second, static_cast<cufftComplex*>(f->work), static_cast<float*>(planes)),
                     "cufftExecC2R");
}

void cc_field_destroy(cc_field* f) {
  if (!f) return;
  if (f->ctx) select_device(f->ctx);
  for (auto& kv : f->inv_plans) cufftDestroy(kv.second);
  if (f->dk) cudaFree(f->dk);
  if (f->work) cudaFree(f->work);
  if (f->acc) cudaFree(f->acc);
  if (f->shells) cudaFree(f->shells);
  delete f;
}

}  // extern "C"
