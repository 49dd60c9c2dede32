// cc_api.cu -- the C-ABI of libcollapse: context, argument checks, launches.
//
// The calls follow the paper's statement of the problem (arXiv:2510.02873,
// Sec. 4.1): tables are built once and kept on the device (Sec. 4.2, "spline
// object constructed once and reused"), device arrays are initialised on the
// device, and each smoothing radius runs one kernel on the caller's stream
// with F_max/idx resident (the OpenMP "target enter data" / "nowait" pattern
// of Sec. 4.1 maps to caller-owned device buffers and an explicit stream).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "cc_internal.h"

namespace cc {

namespace {
thread_local std::string g_last_error;
}

int set_error(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int check_cuda(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return CC_OK;
  char buf[512];
  std::snprintf(buf, sizeof(buf), "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
  return set_error(e == cudaErrorMemoryAllocation ? CC_ENOMEM : CC_ECUDA, buf);
}

namespace {

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int check_planes(const void* hess, int32_t dtype, int64_t n, int64_t plane_stride,
                 int64_t radius_stride, int R) {
  if (dtype != CC_F64 && dtype != CC_F32) return set_error(CC_EINVAL, "dtype must be CC_F64 or CC_F32");
  if (n < 0) return set_error(CC_EINVAL, "n must be >= 0");
  if (n > 0 && hess == nullptr) return set_error(CC_EINVAL, "hess is NULL");
  if (plane_stride < n) return set_error(CC_EINVAL, "plane_stride < n");
  if (R > 1 && radius_stride < 6 * plane_stride)
    return set_error(CC_EINVAL, "radius_stride < 6 * plane_stride");
  if (!aligned16(hess)) return set_error(CC_EINVAL, "hess must be 16-byte aligned");
  if ((plane_stride * dtype) % 16 != 0)
    return set_error(CC_EINVAL, "plane_stride * element size must be a multiple of 16 bytes");
  if (R > 1 && (radius_stride * dtype) % 16 != 0)
    return set_error(CC_EINVAL, "radius_stride * element size must be a multiple of 16 bytes");
  return CC_OK;
}

int check_outputs(const double* F_max, const int32_t* idx, int64_t n) {
  if (n > 0 && (F_max == nullptr || idx == nullptr))
    return set_error(CC_EINVAL, "F_max and idx must be non-NULL");
  return CC_OK;
}

// Records of the mixed path's points with hard radii (cc::HardRec). On
// isotropic-field Hessians ~0.5 % of evaluations are hard, so ~1 - 0.995^R of
// the points need a record; the capacity allows n (0.006 R + 0.02) + 1024
// (at most n), and points beyond it are recomputed in radius order by the
// second kernel instead. Record indices travel as 32-bit numbers, so the
// capacity is also below 2^32. Grows on demand; never shrinks.
int ensure_hard_records(cc_ctx* ctx, int64_t n, int R) {
  const int Rl = R < kMaxRadiiPerLaunch ? R : kMaxRadiiPerLaunch;
  const double frac = 0.006 * Rl + 0.02;
  int64_t want = frac >= 1.0 ? n : static_cast<int64_t>(static_cast<double>(n) * frac) + 1024;
  if (want > n) want = n;
  if (want > static_cast<int64_t>(UINT32_MAX)) want = static_cast<int64_t>(UINT32_MAX);
  if (!ctx->d_hard_ctr) {
    if (int rc = check_cuda(cudaMalloc(reinterpret_cast<void**>(&ctx->d_hard_ctr),
                                       kHardCounters * sizeof(unsigned long long)),
                            "cudaMalloc(hard record counters)"))
      return rc;
  }
  if (want <= ctx->hard_cap) return CC_OK;
  if (ctx->d_hard) {
    cudaFree(ctx->d_hard);
    ctx->d_hard = nullptr;
    ctx->hard_cap = 0;
  }
  if (ctx->d_hard_full) {
    cudaFree(ctx->d_hard_full);
    ctx->d_hard_full = nullptr;
  }
  if (int rc = check_cuda(cudaMalloc(reinterpret_cast<void**>(&ctx->d_hard), sizeof(HardRec) * static_cast<size_t>(want)),
                          "cudaMalloc(hard records)"))
    return rc;
  if (int rc = check_cuda(cudaMalloc(reinterpret_cast<void**>(&ctx->d_hard_full), sizeof(uint32_t) * static_cast<size_t>(want)),
                          "cudaMalloc(hard record list)"))
    return rc;
  ctx->hard_cap = want;
  return CC_OK;
}

int run_collapse(cc_ctx* ctx, cc_mode mode, const void* hess, int32_t dtype, int64_t n,
                 int64_t plane_stride, int64_t radius_stride, const double* sigma, int32_t R,
                 double* F_max, int32_t* idx, int32_t scale_idx0, void* stream) {
  if (ctx == nullptr) return set_error(CC_EINVAL, "ctx is NULL");
  if (mode < CC_MODE_FP64 || mode > CC_MODE_EXACT_GROWTH) return set_error(CC_EINVAL, "unknown mode");
  if (R < 1) return set_error(CC_EINVAL, "R must be >= 1");
  if (sigma == nullptr) return set_error(CC_EINVAL, "sigma is NULL");
  for (int r = 0; r < R; ++r)
    if (!(sigma[r] > 0.0) || !std::isfinite(sigma[r])) return set_error(CC_EINVAL, "sigma must be finite and > 0");
  if (scale_idx0 < 0 || static_cast<int64_t>(scale_idx0) + R - 1 > INT32_MAX)
    return set_error(CC_EINVAL, "scale indices must be in [0, INT32_MAX]");
  if (int rc = check_planes(hess, dtype, n, plane_stride, radius_stride, R)) return rc;
  if (int rc = check_outputs(F_max, idx, n)) return rc;
  if (n == 0) return CC_OK;
  if (int rc = select_device(ctx)) return rc;
  LaunchArgs a{hess, dtype, n, plane_stride, radius_stride, R, scale_idx0, F_max, idx,
               ctx->d_counters, static_cast<cudaStream_t>(stream), ctx->num_sms};
  switch (mode) {
    case CC_MODE_FP64:
      return launch_fp64(a, ctx->tab);
    case CC_MODE_MIXED: {
      if (int rc = ensure_hard_records(ctx, n, R)) return rc;
      return launch_mixed(a, ctx->tab, sigma, HardWork{ctx->d_hard, ctx->hard_cap, ctx->d_hard_ctr, ctx->d_hard_full});
    }
    case CC_MODE_TABULATED:
      return launch_tab_checked(ctx, a);
    case CC_MODE_SURROGATE:
      return launch_surrogate_checked(ctx, a, sigma);
    case CC_MODE_F32X2:
      return launch_f32x2(a, ctx->tab);
    case CC_MODE_EXACT_GROWTH:
      return launch_exact(a, ctx->tab);
  }
  return set_error(CC_EINVAL, "unknown mode");
}

int ensure_staging(cc_ctx* ctx, size_t stage_bytes, int64_t n) {
  if (!ctx->copy_stream) {
    if (int rc = check_cuda(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking),
                            "cudaStreamCreate(copy)"))
      return rc;
    for (int b = 0; b < 2; ++b) {
      if (int rc = check_cuda(cudaEventCreateWithFlags(&ctx->ev_copied[b], cudaEventDisableTiming), "cudaEventCreate"))
        return rc;
      if (int rc = check_cuda(cudaEventCreateWithFlags(&ctx->ev_consumed[b], cudaEventDisableTiming), "cudaEventCreate"))
        return rc;
    }
  }
  if (stage_bytes > ctx->stage_bytes) {
    for (int b = 0; b < 2; ++b) {
      if (ctx->d_stage[b]) { cudaFree(ctx->d_stage[b]); ctx->d_stage[b] = nullptr; }
    }
    ctx->stage_bytes = 0;
    for (int b = 0; b < 2; ++b)
      if (int rc = check_cuda(cudaMalloc(&ctx->d_stage[b], stage_bytes), "cudaMalloc(staging)")) return rc;
    ctx->stage_bytes = stage_bytes;
  }
  if (n > ctx->out_cap) {
    if (ctx->d_F) { cudaFree(ctx->d_F); ctx->d_F = nullptr; }
    if (ctx->d_idx) { cudaFree(ctx->d_idx); ctx->d_idx = nullptr; }
    ctx->out_cap = 0;
    if (int rc = check_cuda(cudaMalloc(reinterpret_cast<void**>(&ctx->d_F), sizeof(double) * n), "cudaMalloc(F)")) return rc;
    if (int rc = check_cuda(cudaMalloc(reinterpret_cast<void**>(&ctx->d_idx), sizeof(int32_t) * n), "cudaMalloc(idx)")) return rc;
    ctx->out_cap = n;
  }
  return CC_OK;
}

}  // namespace

int select_device(const cc_ctx* ctx) {
  int cur = -1;
  if (int rc = check_cuda(cudaGetDevice(&cur), "cudaGetDevice")) return rc;
  if (cur != ctx->device) return check_cuda(cudaSetDevice(ctx->device), "cudaSetDevice");
  return CC_OK;
}

}  // namespace cc

using namespace cc;

extern "C" {

int cc_version(void) { return 100; }

const char* cc_strerror(int code) {
  switch (code) {
    case CC_OK: return "CC_OK";
    case CC_EINVAL: return "CC_EINVAL: invalid argument";
    case CC_ECUDA: return "CC_ECUDA: CUDA runtime error";
    case CC_ENOMEM: return "CC_ENOMEM: out of memory";
    case CC_ETIMEOUT: return "CC_ETIMEOUT: bounded device wait timed out";
    case CC_ERANGE: return "CC_ERANGE: value out of range";
    case CC_ENOTSUP: return "CC_ENOTSUP: not supported";
    default: return "unknown status code";
  }
}

const char* cc_last_error_message(void) { return g_last_error.c_str(); }

int cc_create(cc_ctx** out, const cc_cosmology* cosmo, int device) {
  if (out == nullptr || cosmo == nullptr) return set_error(CC_EINVAL, "out and cosmo must be non-NULL");
  *out = nullptr;
  int ndev = 0;
  if (int rc = check_cuda(cudaGetDeviceCount(&ndev), "cudaGetDeviceCount")) return rc;
  if (device < 0 || device >= ndev) return set_error(CC_EINVAL, "device index out of range");
  cc_ctx* ctx = new (std::nothrow) cc_ctx();
  if (!ctx) return set_error(CC_ENOMEM, "host allocation failed");
  ctx->device = device;
  ctx->cosmo = *cosmo;
  int rc = build_growth_table(*cosmo, ctx->a_k, ctx->D_k);
  if (rc) { delete ctx; return set_error(rc, "growth table: invalid cosmology or knot range"); }
  rc = build_natural_spline(ctx->D_k, ctx->a_k, ctx->coef);
  if (rc) { delete ctx; return set_error(rc, "spline build failed"); }
  if (f32_knots_within_factor2(cosmo->n_knots, ctx->D_k.data())) {
    delete ctx;
    return set_error(CC_EINVAL, "growth-table knots too coarse: D may at most double between neighbouring knots "
                                "(raise n_knots)");
  }
  // the device polynomials are expanded about the FP32 knots e_k
  std::vector<double> e_k(cosmo->n_knots);
  for (int k = 0; k < cosmo->n_knots; ++k) e_k[k] = static_cast<double>(static_cast<float>(ctx->D_k[k]));
  expand_about_f32_knots(cosmo->n_knots, ctx->D_k.data(), ctx->coef.data());
  if ((rc = check_cuda(cudaSetDevice(device), "cudaSetDevice"))) { delete ctx; return rc; }
  if ((rc = check_cuda(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device),
                       "cudaDeviceGetAttribute"))) { delete ctx; return rc; }
  const int n = cosmo->n_knots;
  // FP32 interval search: buckets over the FP32 bit patterns of D, each holding
  // the largest knot index k with D_k <= the bucket's lower edge
  std::vector<float> df(n);
  for (int k = 0; k < n; ++k) df[k] = static_cast<float>(ctx->D_k[k]);
  std::vector<unsigned short> bucket(kBucketsPerKnot * n);
  int nb = 0, b_shift = 0;
  unsigned b0 = 0;
  if (bit_buckets_into(n, df.data(), kBucketsPerKnot * n, bucket.data(), &nb, &b_shift, &b0) != CC_OK) {
    delete ctx;
    return set_error(CC_EINVAL, "growth-table knots too irregular for the interval search buckets");
  }
  // device layout: coef[n-1] (32-byte aligned) | D[n] | Df[n] | bucket[nb]
  const size_t coef_bytes = sizeof(Coef4) * (n - 1);
  const size_t d_bytes = sizeof(double) * n;
  const size_t df_bytes = sizeof(float) * n;
  const size_t b_bytes = sizeof(unsigned short) * nb;
  const size_t main_bytes = coef_bytes + d_bytes + df_bytes + b_bytes;
  const size_t seg_off = ((main_bytes + 15) / 16) * 16;
  const size_t seg_bytes = sizeof(float) * 8 * (n - 1);
  const size_t total = seg_off + seg_bytes;
  if ((rc = check_cuda(cudaMalloc(&ctx->d_table, total), "cudaMalloc(table)"))) { delete ctx; return rc; }
  if ((rc = check_cuda(cudaMalloc(reinterpret_cast<void**>(&ctx->d_counters), sizeof(DevCounters)),
                       "cudaMalloc(counters)"))) {
    cudaFree(ctx->d_table);
    delete ctx;
    return rc;
  }
  std::vector<unsigned char> host(total);
  std::memcpy(host.data(), ctx->coef.data(), coef_bytes);
  std::memcpy(host.data() + coef_bytes, e_k.data(), d_bytes);
  std::memcpy(host.data() + coef_bytes + d_bytes, df.data(), df_bytes);
  std::memcpy(host.data() + coef_bytes + d_bytes + df_bytes, bucket.data(), b_bytes);
  {  // float-float image: value = hi + lo with hi = RN32(value), lo = RN32(value - hi)
    auto split = [](double v, float& hi, float& lo) {
      hi = static_cast<float>(v);
      lo = static_cast<float>(v - static_cast<double>(hi));
    };
    float* seg = reinterpret_cast<float*>(host.data() + seg_off);
    for (int k = 0; k < n - 1; ++k) {
      const double* c = ctx->coef.data() + 4 * k;
      float* s = seg + 8 * k;
      split(c[0], s[0], s[1]);
      split(c[1], s[2], s[3]);
      s[4] = static_cast<float>(c[2]);
      s[5] = static_cast<float>(c[3]);
      split(e_k[k], s[6], s[7]);  // exact in FP32: lo = 0
    }
  }
  rc = check_cuda(cudaMemcpy(ctx->d_table, host.data(), total, cudaMemcpyHostToDevice), "cudaMemcpy(table)");
  if (!rc) rc = check_cuda(cudaMemset(ctx->d_counters, 0, sizeof(DevCounters)), "cudaMemset(counters)");
  if (rc) { cc_destroy(ctx); return rc; }
  auto* base = static_cast<unsigned char*>(ctx->d_table);
  DevTable& t = ctx->tab;
  t.coef = reinterpret_cast<const Coef4*>(base);
  t.D = reinterpret_cast<const double*>(base + coef_bytes);
  t.Df = reinterpret_cast<const float*>(base + coef_bytes + d_bytes);
  t.bucket = reinterpret_cast<const unsigned short*>(base + coef_bytes + d_bytes + df_bytes);
  t.n = n;
  t.n_buckets = nb;
  t.b0 = b0;
  t.b_shift = b_shift;
  t.a0 = ctx->a_k[0];
  t.D0 = ctx->D_k[0];
  t.Dtop = ctx->D_k[n - 1];
  t.eds_slope = ctx->a_k[0] / ctx->D_k[0];
  t.Dtopf = static_cast<float>(t.Dtop);
  t.Dtop_t = t.Dtop - e_k[n - 2];
  t.dfseg = reinterpret_cast<const float4*>(base + seg_off);
  auto split2 = [](double v, float& hi, float& lo) {
    hi = static_cast<float>(v);
    lo = static_cast<float>(v - static_cast<double>(hi));
  };
  split2(t.Dtop, t.Dtop_hi, t.Dtop_lo);
  split2(t.D0, t.D0_hi, t.D0_lo);
  split2(t.eds_slope, t.eds_hi, t.eds_lo);
  {  // growth-ratio splines (CC_MODE_EXACT_GROWTH)
    std::vector<double> r(3 * n), work(6 * n), c64(3 * 4 * (n - 1));
    rc = growth_ratios_into(*cosmo, r.data(), r.data() + n, r.data() + 2 * n);
    for (int o = 0; o < 3 && !rc; ++o)
      rc = natural_spline_into(n, ctx->D_k.data(), r.data() + o * n, c64.data() + o * 4 * (n - 1), work.data());
    for (int o = 0; o < 3 && !rc; ++o) expand_about_f32_knots(n, ctx->D_k.data(), c64.data() + o * 4 * (n - 1));
    // stored as r2, ra = -r3a / 3 + r3b and rb = -r3b / 2 (splines are linear
    // in their node values, so these are the splines of those combinations):
    // with r3a' = -r3a / 3 and r3b' = -r3b / 2 the third-order term
    // l1 (r3a' l2 l3 + r3b' (l2^2 + l3^2)) is l1 (ra l2 l3 + rb (l2 + l3)^2)
    // (see cc_exact.cuh)
    for (size_t i = 0; i < 4 * static_cast<size_t>(n - 1); ++i) {
      c64[4 * (n - 1) + i] = c64[4 * (n - 1) + i] * (-1.0 / 3.0) + c64[8 * (n - 1) + i];
      c64[8 * (n - 1) + i] *= -0.5;
    }
    if (rc) { cc_destroy(ctx); return set_error(rc, "growth ratio tables failed"); }
    std::vector<float> c32(c64.size());
    for (size_t i = 0; i < c64.size(); ++i) c32[i] = static_cast<float>(c64[i]);
    const size_t b64 = sizeof(double) * c64.size(), b32 = sizeof(float) * c32.size();
    if ((rc = check_cuda(cudaMalloc(&ctx->d_ratio, b64 + b32), "cudaMalloc(ratio tables)"))) { cc_destroy(ctx); return rc; }
    rc = check_cuda(cudaMemcpy(ctx->d_ratio, c64.data(), b64, cudaMemcpyHostToDevice), "cudaMemcpy(ratio tables)");
    if (!rc)
      rc = check_cuda(cudaMemcpy(static_cast<unsigned char*>(ctx->d_ratio) + b64, c32.data(), b32, cudaMemcpyHostToDevice),
                      "cudaMemcpy(ratio tables)");
    if (rc) { cc_destroy(ctx); return rc; }
    t.rc64 = static_cast<const Coef4*>(ctx->d_ratio);
    t.rc32 = reinterpret_cast<const float4*>(static_cast<unsigned char*>(ctx->d_ratio) + b64);
  }
  *out = ctx;
  return CC_OK;
}

void cc_destroy(cc_ctx* ctx) {
  if (!ctx) return;
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != ctx->device) cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  if (ctx->d_table) cudaFree(ctx->d_table);
  if (ctx->d_ratio) cudaFree(ctx->d_ratio);
  if (ctx->d_counters) cudaFree(ctx->d_counters);
  if (ctx->d_hard) cudaFree(ctx->d_hard);
  if (ctx->d_hard_full) cudaFree(ctx->d_hard_full);
  if (ctx->d_hard_ctr) cudaFree(ctx->d_hard_ctr);
  for (int b = 0; b < 2; ++b) {
    if (ctx->d_stage[b]) cudaFree(ctx->d_stage[b]);
    if (ctx->ev_copied[b]) cudaEventDestroy(ctx->ev_copied[b]);
    if (ctx->ev_consumed[b]) cudaEventDestroy(ctx->ev_consumed[b]);
  }
  if (ctx->d_F) cudaFree(ctx->d_F);
  if (ctx->d_idx) cudaFree(ctx->d_idx);
  if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
  if (ctx->d_tab_axes) cudaFree(ctx->d_tab_axes);
  if (ctx->d_tab_coef) cudaFree(ctx->d_tab_coef);
  if (ctx->d_tab_work) cudaFree(ctx->d_tab_work);
  if (ctx->d_spl) cudaFree(ctx->d_spl);
  if (ctx->d_mlp_img) cudaFree(ctx->d_mlp_img);
  if (ctx->d_mlp_param) cudaFree(ctx->d_mlp_param);
  if (ctx->d_train) cudaFree(ctx->d_train);
  if (cur >= 0 && cur != ctx->device) cudaSetDevice(cur);
  delete ctx;
}

int cc_build_growth_table(const cc_cosmology* cosmo, double* a_k, double* D_k) {
  if (!cosmo || !a_k || !D_k) return set_error(CC_EINVAL, "NULL argument");
  std::vector<double> a, D;
  if (int rc = build_growth_table(*cosmo, a, D)) return set_error(rc, "growth table: invalid cosmology or knot range");
  std::memcpy(a_k, a.data(), sizeof(double) * a.size());
  std::memcpy(D_k, D.data(), sizeof(double) * D.size());
  return CC_OK;
}

int cc_get_growth_table(const cc_ctx* ctx, double* a_k, double* D_k, int32_t n) {
  if (!ctx || !a_k || !D_k) return set_error(CC_EINVAL, "NULL argument");
  if (n != ctx->cosmo.n_knots) return set_error(CC_EINVAL, "n must equal n_knots");
  std::memcpy(a_k, ctx->a_k.data(), sizeof(double) * n);
  std::memcpy(D_k, ctx->D_k.data(), sizeof(double) * n);
  return CC_OK;
}

int cc_reset_max(cc_ctx* ctx, double* F_max, int32_t* idx, int64_t n, void* stream) {
  if (!ctx) return set_error(CC_EINVAL, "ctx is NULL");
  if (n < 0) return set_error(CC_EINVAL, "n must be >= 0");
  if (int rc = check_outputs(F_max, idx, n)) return rc;
  if (n == 0) return CC_OK;
  if (int rc = select_device(ctx)) return rc;
  return launch_reset_max(F_max, idx, n, static_cast<cudaStream_t>(stream), ctx->num_sms);
}

int cc_collapse_scale(cc_ctx* ctx, cc_mode mode, const void* hess, int32_t dtype, int64_t n,
                      int64_t plane_stride, double sigma_R, double* F_max, int32_t* idx,
                      int32_t scale_idx, void* stream) {
  return run_collapse(ctx, mode, hess, dtype, n, plane_stride, 6 * plane_stride, &sigma_R, 1, F_max,
                      idx, scale_idx, stream);
}

int cc_collapse_multi(cc_ctx* ctx, cc_mode mode, const void* hess, int32_t dtype, int64_t n,
                      int64_t plane_stride, int64_t radius_stride, const double* sigma, int32_t R,
                      double* F_max, int32_t* idx, int32_t scale_idx0, void* stream) {
  return run_collapse(ctx, mode, hess, dtype, n, plane_stride, radius_stride, sigma, R, F_max, idx,
                      scale_idx0, stream);
}

int cc_collapse_multi_host(cc_ctx* ctx, cc_mode mode, const void* hess_host, int32_t dtype, int64_t n,
                           int64_t plane_stride, int64_t radius_stride, const double* sigma, int32_t R,
                           double* F_max_host, int32_t* idx_host, int32_t scale_idx0, void* stream) {
  if (!ctx) return set_error(CC_EINVAL, "ctx is NULL");
  if (R < 1) return set_error(CC_EINVAL, "R must be >= 1");
  if (!sigma) return set_error(CC_EINVAL, "sigma is NULL");
  if (int rc = check_planes(hess_host, dtype, n, plane_stride, radius_stride, R)) return rc;
  if (int rc = check_outputs(F_max_host, idx_host, n)) return rc;
  if (n == 0) return CC_OK;
  if (int rc = select_device(ctx)) return rc;
  const size_t elem = static_cast<size_t>(dtype);
  const size_t radius_bytes = 6 * static_cast<size_t>(plane_stride) * elem;
  if (int rc = ensure_staging(ctx, radius_bytes, n)) return rc;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  cudaStream_t xs = ctx->copy_stream;
  const char* host = static_cast<const char*>(hess_host);
  if (int rc = check_cuda(cudaMemcpyAsync(ctx->d_F, F_max_host, sizeof(double) * n, cudaMemcpyHostToDevice, cs), "H2D F_max")) return rc;
  if (int rc = check_cuda(cudaMemcpyAsync(ctx->d_idx, idx_host, sizeof(int32_t) * n, cudaMemcpyHostToDevice, cs), "H2D idx")) return rc;
  // the copy stream must not overwrite a buffer still in use by an earlier call on `stream`
  if (int rc = check_cuda(cudaEventRecord(ctx->ev_consumed[0], cs), "cudaEventRecord")) return rc;
  if (int rc = check_cuda(cudaEventRecord(ctx->ev_consumed[1], cs), "cudaEventRecord")) return rc;
  for (int r = 0; r < R; ++r) {
    const int b = r & 1;
    if (int rc = check_cuda(cudaStreamWaitEvent(xs, ctx->ev_consumed[b], 0), "cudaStreamWaitEvent")) return rc;
    if (int rc = check_cuda(cudaMemcpyAsync(ctx->d_stage[b], host + static_cast<size_t>(r) * radius_stride * elem,
                                            radius_bytes, cudaMemcpyHostToDevice, xs), "H2D planes")) return rc;
    if (int rc = check_cuda(cudaEventRecord(ctx->ev_copied[b], xs), "cudaEventRecord")) return rc;
    if (int rc = check_cuda(cudaStreamWaitEvent(cs, ctx->ev_copied[b], 0), "cudaStreamWaitEvent")) return rc;
    if (int rc = run_collapse(ctx, mode, ctx->d_stage[b], dtype, n, plane_stride, 6 * plane_stride, sigma + r, 1,
                              ctx->d_F, ctx->d_idx, scale_idx0 + r, stream)) return rc;
    if (int rc = check_cuda(cudaEventRecord(ctx->ev_consumed[b], cs), "cudaEventRecord")) return rc;
  }
  if (int rc = check_cuda(cudaMemcpyAsync(F_max_host, ctx->d_F, sizeof(double) * n, cudaMemcpyDeviceToHost, cs), "D2H F_max")) return rc;
  if (int rc = check_cuda(cudaMemcpyAsync(idx_host, ctx->d_idx, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, cs), "D2H idx")) return rc;
  return check_cuda(cudaStreamSynchronize(cs), "cudaStreamSynchronize");
}

int cc_get_stats(cc_ctx* ctx, cc_stats* out, void* stream) {
  if (!ctx || !out) return set_error(CC_EINVAL, "NULL argument");
  if (int rc = select_device(ctx)) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (int rc = check_cuda(cudaMemcpyAsync(out, ctx->d_counters, sizeof(cc_stats), cudaMemcpyDeviceToHost, s),
                          "cudaMemcpyAsync(stats)"))
    return rc;
  return check_cuda(cudaStreamSynchronize(s), "cudaStreamSynchronize(stats)");
}

int cc_reset_stats(cc_ctx* ctx, void* stream) {
  if (!ctx) return set_error(CC_EINVAL, "ctx is NULL");
  if (int rc = select_device(ctx)) return rc;
  return check_cuda(cudaMemsetAsync(ctx->d_counters, 0, sizeof(DevCounters), static_cast<cudaStream_t>(stream)),
                    "cudaMemsetAsync(stats)");
}

}  // extern "C"
