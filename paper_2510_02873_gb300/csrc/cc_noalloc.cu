// cc_noalloc.cu -- a context-free variant of cc_collapse_multi that allocates nothing.
//
// Why it exists: cudaMalloc is off limits for some callers. Code that lives
// inside another framework whose caching allocator owns all device memory, and
// tight loops that cannot afford the implicit device synchronisation of
// cudaMalloc/cudaFree, need to hand the library their own input and output
// buffers and nothing more.
// cc_create cannot serve them: it allocates the spline table and the counters.
//
// This entry point keeps its scratch (the spline table image and the launch
// counters) in one file-scope static device array of fixed size instead. Every
// GPU that loads the library holds that array until the process exits. All
// calls on a device share it; it keeps the last call's contents, so the
// counters are cleared at the start of every call, and the table is uploaded
// again whenever the cosmology differs from the one already resident. Calls
// whose work overlaps on the GPU (different streams, or different cosmologies
// in flight at once) race on the array.
//
// The first call on each device looks up the array's device address with
// cudaGetSymbolAddress (that device current) and uploads the table.
#include <cmath>
#include <cstring>
#include <mutex>

#include "cc_internal.h"

namespace cc {

namespace {

constexpr int kStaticMaxKnots = 1024;
constexpr int kStaticMaxBuckets = kBucketsPerKnot * kStaticMaxKnots;
constexpr size_t kStaticTableBytes = sizeof(Coef4) * (kStaticMaxKnots - 1) +
                                     sizeof(double) * kStaticMaxKnots +
                                     sizeof(float) * kStaticMaxKnots +
                                     sizeof(unsigned short) * kStaticMaxBuckets;
constexpr size_t kCountersOffset = (kStaticTableBytes + 255) / 256 * 256;
constexpr size_t kStaticScratchBytes = kCountersOffset + 256;  // 53,504 bytes
constexpr int kMaxDevices = 64;

// the scratch array: table image (coef | D | Df | bucket), then DevCounters
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

struct DeviceState {
  void* scratch = nullptr;  // device address of g_static_scratch on this device
  bool table_valid = false;
  cc_cosmology cosmo{};     // cosmology of the resident table
  DevTable tab{};
};

std::mutex g_mutex;
DeviceState g_state[kMaxDevices];
// host staging of one table image and its ingredients (static: no allocation)
double g_a[kStaticMaxKnots], g_D[kStaticMaxKnots];
double g_coef[4 * (kStaticMaxKnots - 1)];
double g_work[6 * kStaticMaxKnots];
float g_scratch_f[kStaticMaxKnots];
unsigned short g_bucket[kStaticMaxBuckets];
alignas(32) unsigned char g_image[kStaticTableBytes];

bool same_cosmology(const cc_cosmology& a, const cc_cosmology& b) {
  return a.omega_m == b.omega_m && a.omega_l == b.omega_l && a.n_knots == b.n_knots &&
         a.a_min == b.a_min && a.a_max == b.a_max;
}

// Build the table image for `c` in host memory and describe it in `tab`
// (device pointers relative to `base`).
int build_image(const cc_cosmology& c, unsigned char* base, DevTable& tab, size_t& bytes) {
  const int n = c.n_knots;
  if (int rc = growth_table_into(c, g_a, g_D)) return rc;
  if (int rc = natural_spline_into(n, g_D, g_a, g_coef, g_work)) return rc;
  if (int rc = f32_knots_within_factor2(n, g_D)) return rc;
  expand_about_f32_knots(n, g_D, g_coef);  // the device polynomials are expanded about the FP32 knots
  float* df = g_scratch_f;
  for (int k = 0; k < n; ++k) df[k] = static_cast<float>(g_D[k]);
  int nb = 0, b_shift = 0;
  unsigned b0 = 0;
  if (int rc = bit_buckets_into(n, df, kBucketsPerKnot * n, g_bucket, &nb, &b_shift, &b0)) return rc;
  const size_t coef_bytes = sizeof(Coef4) * (n - 1);
  const size_t d_bytes = sizeof(double) * n;
  const size_t df_bytes = sizeof(float) * n;
  bytes = coef_bytes + d_bytes + df_bytes + sizeof(unsigned short) * nb;
  std::memcpy(g_image, g_coef, coef_bytes);
  double* e = reinterpret_cast<double*>(g_image + coef_bytes);
  for (int k = 0; k < n; ++k) e[k] = static_cast<double>(static_cast<float>(g_D[k]));
  std::memcpy(g_image + coef_bytes + d_bytes, df, df_bytes);
  std::memcpy(g_image + coef_bytes + d_bytes + df_bytes, g_bucket, sizeof(unsigned short) * nb);
  tab.coef = reinterpret_cast<const Coef4*>(base);
  tab.D = reinterpret_cast<const double*>(base + coef_bytes);
  tab.Df = reinterpret_cast<const float*>(base + coef_bytes + d_bytes);
  tab.bucket = reinterpret_cast<const unsigned short*>(base + coef_bytes + d_bytes + df_bytes);
  tab.n = n;
  tab.n_buckets = nb;
  tab.b0 = b0;
  tab.b_shift = b_shift;
  tab.a0 = g_a[0];
  tab.D0 = g_D[0];
  tab.Dtop = g_D[n - 1];
  tab.eds_slope = g_a[0] / g_D[0];
  tab.Dtopf = static_cast<float>(tab.Dtop);
  tab.Dtop_t = tab.Dtop - static_cast<double>(static_cast<float>(g_D[n - 2]));
  return CC_OK;
}

}  // namespace
}  // namespace cc

using namespace cc;

extern "C" int cc_collapse_multi_noalloc(const cc_cosmology* cosmo, cc_mode mode, const void* hess,
                                         int32_t dtype, int64_t n, int64_t plane_stride,
                                         int64_t radius_stride, const double* sigma, int32_t R,
                                         double* F_max, int32_t* idx, int32_t scale_idx0,
                                         cc_stats* stats, void* stream) {
  if (cosmo == nullptr) return set_error(CC_EINVAL, "cosmo is NULL");
  if (cosmo->n_knots < 2 || cosmo->n_knots > kStaticMaxKnots)
    return set_error(CC_EINVAL, "n_knots must be in [2, 1024] for cc_collapse_multi_noalloc "
                                "(its table lives in a fixed 53.5 KB static device array)");
  if (mode != CC_MODE_FP64) return set_error(CC_ENOTSUP, "cc_collapse_multi_noalloc supports CC_MODE_FP64 only");
  if (R < 1) return set_error(CC_EINVAL, "R must be >= 1");
  if (sigma == nullptr) return set_error(CC_EINVAL, "sigma is NULL");
  for (int r = 0; r < R; ++r)
    if (!(sigma[r] > 0.0) || !std::isfinite(sigma[r])) return set_error(CC_EINVAL, "sigma must be finite and > 0");
  if (scale_idx0 < 0 || static_cast<int64_t>(scale_idx0) + R - 1 > INT32_MAX)
    return set_error(CC_EINVAL, "scale indices must be in [0, INT32_MAX]");
  if (dtype != CC_F64 && dtype != CC_F32) return set_error(CC_EINVAL, "dtype must be CC_F64 or CC_F32");
  if (n < 0) return set_error(CC_EINVAL, "n must be >= 0");
  if (n > 0 && (hess == nullptr || F_max == nullptr || idx == nullptr))
    return set_error(CC_EINVAL, "hess, F_max and idx must be non-NULL");
  if (plane_stride < n) return set_error(CC_EINVAL, "plane_stride < n");
  if (R > 1 && radius_stride < 6 * plane_stride) return set_error(CC_EINVAL, "radius_stride < 6 * plane_stride");
  if ((reinterpret_cast<uintptr_t>(hess) & 15u) != 0) return set_error(CC_EINVAL, "hess must be 16-byte aligned");
  if ((plane_stride * dtype) % 16 != 0)
    return set_error(CC_EINVAL, "plane_stride * element size must be a multiple of 16 bytes");
  if (R > 1 && (radius_stride * dtype) % 16 != 0)
    return set_error(CC_EINVAL, "radius_stride * element size must be a multiple of 16 bytes");

  int dev = -1;
  if (int rc = check_cuda(cudaGetDevice(&dev), "cudaGetDevice")) return rc;
  if (dev < 0 || dev >= kMaxDevices) return set_error(CC_EINVAL, "device index beyond 64");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lock(g_mutex);
  DeviceState& ds = g_state[dev];
  if (ds.scratch == nullptr) {  // once per device, with that device current
    void* ptr = nullptr;
    if (int rc = check_cuda(cudaGetSymbolAddress(&ptr, g_static_scratch), "cudaGetSymbolAddress")) return rc;
    ds.scratch = ptr;
  }
  unsigned char* base = static_cast<unsigned char*>(ds.scratch);
  if (!ds.table_valid || !same_cosmology(ds.cosmo, *cosmo)) {
    DevTable tab{};
    size_t bytes = 0;
    if (int rc = build_image(*cosmo, base, tab, bytes))
      return set_error(rc, "growth table: invalid cosmology or knot range");
    // pageable source: the call returns once g_image has been staged
    ds.table_valid = false;
    if (int rc = check_cuda(cudaMemcpyAsync(base, g_image, bytes, cudaMemcpyHostToDevice, st),
                            "cudaMemcpyAsync(static table)"))
      return rc;
    ds.tab = tab;
    ds.cosmo = *cosmo;
    ds.table_valid = true;
  }
  DevCounters* counters = reinterpret_cast<DevCounters*>(base + kCountersOffset);
  if (int rc = check_cuda(cudaMemsetAsync(counters, 0, sizeof(DevCounters), st), "cudaMemsetAsync(counters)"))
    return rc;
  if (n > 0) {
    int sms = 0;
    if (int rc = check_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "cudaDeviceGetAttribute"))
      return rc;
    LaunchArgs a{hess, dtype, n, plane_stride, radius_stride, R, scale_idx0, F_max, idx, counters, st, sms};
    if (int rc = launch_fp64(a, ds.tab)) return rc;
  }
  if (stats != nullptr) {
    if (int rc = check_cuda(cudaMemcpyAsync(stats, counters, sizeof(cc_stats), cudaMemcpyDeviceToHost, st),
                            "cudaMemcpyAsync(stats)"))
      return rc;
    return check_cuda(cudaStreamSynchronize(st), "cudaStreamSynchronize");
  }
  return CC_OK;
}
