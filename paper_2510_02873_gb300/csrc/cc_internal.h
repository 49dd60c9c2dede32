// cc_internal.h -- internal types of libcollapse (not part of the C-ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/collapse.h"

namespace cc {

constexpr int kMaxKnots = 4096;
constexpr int kThreads = 256;            // threads per block of the collapse kernels
constexpr int kSmemTableMaxBytes = 64 * 1024;
constexpr int kBucketsPerKnot = 4;  // log2-D buckets per knot (bucket finer than knot spacing)

// Bits of cc_stats.error_flags.
constexpr unsigned kErrWait = 1u;   // a bounded tensor-core wait ran out (CC_SURROGATE_TCGEN05)
constexpr unsigned kErrIndex = 2u;  // debug builds: an index left its table (clamped, see CC_DBG_CLAMP)

// Debug builds (compiled with -DCC_DEBUG): an index outside [lo, hi] sets
// kErrIndex in the launch's error flags and is clamped into range, so the
// access stays inside its table and the launch completes; release builds
// compile the check away. `flags` is the launch's &counters->error_flags.
#ifdef CC_DEBUG
#define CC_DBG_CLAMP(i, lo, hi, flags)                       \
  do {                                                        \
    if ((i) < (lo) || (i) > (hi)) {                           \
      if ((flags) != nullptr) atomicOr((flags), cc::kErrIndex); \
      (i) = ((i) < (lo)) ? (lo) : (hi);                       \
    }                                                         \
  } while (0)
#else
#define CC_DBG_CLAMP(i, lo, hi, flags) \
  do {                                 \
  } while (0)
#endif

// Device-side counters; same layout as cc_stats.
struct DevCounters {
  unsigned long long evaluations;
  unsigned long long collapsed;
  unsigned long long eds_branch;
  unsigned long long refined;
  unsigned long long fp64_branch;
  unsigned long long fallback;
  unsigned int error_flags;
  unsigned int reserved;
};
static_assert(sizeof(DevCounters) == sizeof(cc_stats), "counter layout must match cc_stats");

// Cubic on one spline interval: c0 + c1 t + c2 t^2 + c3 t^3.
struct alignas(32) Coef4 {
  double c0, c1, c2, c3;
};

// Inverse growth spline on the device: knots D_k (n) and per-interval
// polynomial coefficients a = c0 + c1 t + c2 t^2 + c3 t^3 (n - 1), expanded
// about e_k = D_k rounded to FP32, t = D - e_k; the image's D array holds e_k
// (D0 and Dtop below are the exact first and last knots).
struct DevTable {
  const Coef4* coef;              // n - 1 intervals
  const double* D;                // n knots
  const float* Df;                // FP32 copy of the knots (interval search)
  const unsigned short* bucket;   // n_buckets: largest k with D_k <= bucket's lower edge
  int n;
  int n_buckets;                  // uniform buckets in the FP32 bit pattern of D over [D_0, D_top]
  unsigned b0;                    // FP32 bit pattern of the first knot
  int b_shift;                    // bucket = (bits(D) - b0) >> b_shift
  double a0, D0, Dtop;            // first scale factor, first and last knot
  double eds_slope;               // a0 / D0
  float Dtopf;                    // D_top rounded to FP32 (interval search)
  double Dtop_t;                  // D_top - e_{n-2}: t of D_top on the last interval
  // float-float image of the spline (CC_MODE_F32X2): two float4 per interval,
  // {c0 hi, c0 lo, c1 hi, c1 lo}, {c2, c3, D_k hi, D_k lo}, stored right after
  // the table image at offset round_up(bytes(), 16); nullptr when absent
  const float4* dfseg;
  float Dtop_hi, Dtop_lo, D0_hi, D0_lo, eds_hi, eds_lo;  // float-float constants
  // exact-background growth ratios as natural splines in D over the same
  // knots (CC_MODE_EXACT_GROWTH), stored as r2, -r3a / 3 + r3b and -r3b / 2:
  // rc64[o * (n - 1) + k] (FP64) and rc32[...] (FP32 copies, {c0, c1, c2,
  // c3}); nullptr when absent
  const Coef4* rc64;
  const float4* rc32;
  unsigned int* dbg;              // the launch's error flags (index checks of debug builds)
  // bytes of the table image (coef | D | Df | bucket), staged in shared memory
  __host__ __device__ size_t bytes() const {
    return sizeof(Coef4) * (n - 1) + sizeof(double) * n + sizeof(float) * n +
           sizeof(unsigned short) * n_buckets;
  }
};

// Tabulated collapse: table of u = 1/D_c over (delta, x = l1 - l2, y = l2 - l3),
// natural cubic splines along delta (per-interval coefficients, built on the
// device), bilinear in (x, y).
constexpr int kTabMaxD = 256;
constexpr int kTabMaxXY = 256;
struct TabDev {
  const double* axes;  // image: dg[nd] | xg[nx] | yg[ny] | 1/hx[nx-1] | 1/hy[ny-1] | -xg/hx[nx-1] | -yg/hy[ny-1] | dgf (float)[nd]
  const Coef4* coef;   // [(ix * ny + iy) * (nd - 1) + k]
  int nd, nx, ny;
  int d_steps, x_steps, y_steps;  // largest power of two <= n - 2 (branch-free searches)
  double d_lo, d_hi, x_lo, x_hi, y_lo, y_hi;  // the table's hull (first and last knot of each axis)
  long long d_lo_key, d_hi_key;                // order keys of d_lo, d_hi (order_key in cc_device.cuh)
  unsigned int* dbg;                          // the launch's error flags (index checks of debug builds)
  __host__ __device__ size_t axes_bytes() const {
    return sizeof(double) * (nd + nx + ny + 2 * (nx - 1) + 2 * (ny - 1)) + sizeof(float) * nd;
  }
};

// host tables (cc_tables.cpp)
int build_growth_table(const cc_cosmology& c, std::vector<double>& a_k, std::vector<double>& D_k);
int build_natural_spline(const std::vector<double>& x, const std::vector<double>& y,
                         std::vector<double>& coef);
// the same, into caller-provided arrays (no allocation); work holds 6 n doubles
int growth_table_into(const cc_cosmology& c, double* a_k, double* D_k);
int natural_spline_into(int n, const double* x, const double* y, double* coef, double* work);
// r2 = D2/D1^2, r3a = D3a/D1^3, r3b = D3b/D1^3 at the knots of growth_table_into
int growth_ratios_into(const cc_cosmology& c, double* r2, double* r3a, double* r3b);
// The device evaluates every per-interval polynomial in t = D - e_k with
// e_k = the knot x_k rounded to FP32, so that an FP32 root Df in interval k
// gives t = Df - e_k exactly (Sterbenz) when e_{k+1} <= 2 e_k.
// f32_knots_within_factor2: CC_OK when the FP32 knots are positive, increasing
// and within a factor 2 of their neighbours, CC_EINVAL otherwise.
int f32_knots_within_factor2(int n, const double* x);
// re-expand the n - 1 cubics c0 + c1 t + c2 t^2 + c3 t^3 (t = D - x_k) about e_k
void expand_about_f32_knots(int n, const double* x, double* coef);
// Interval search buckets over the FP32 knots xf (positive, increasing):
// bucket b covers the FP32 bit patterns [b0 + (b << shift), b0 + ((b + 1) << shift))
// of D and holds the largest k <= n - 2 with xf[k] <= its lower edge; shift is
// the largest with at most two knots x_1 .. x_{n-2} in any bucket, so two
// predicated steps always reach the interval. CC_EINVAL when that needs more
// than max_nb buckets.
int bit_buckets_into(int n, const float* xf, int max_nb, unsigned short* bucket, int* nb, int* shift, unsigned* b0);

// error reporting (cc_api.cu)
int set_error(int code, const std::string& msg);
int check_cuda(cudaError_t e, const char* what);

// per-radius parameters of one launch (kernel-parameter space)
constexpr int kMaxRadiiPerLaunch = 256;
struct RadiusParams {
  float tri_thr[kMaxRadiiPerLaunch];    // MIXED: 1e-4 s(R), the all-three-close threshold
  float inv_sigma[kMaxRadiiPerLaunch];  // SURROGATE: 1 / s(R), the input normalisation
};

// surrogate network (BF16 image) and its training hull, as kernel parameters
struct SurDev {
  const unsigned char* img;
  float lo[3], hi[3];
};

// kernel launchers (cc_kernels.cu)
struct LaunchArgs {
  const void* hess;
  int dtype;
  int64_t n;
  int64_t plane_stride;
  int64_t radius_stride;
  int R;
  int32_t scale_idx0;
  double* F_max;
  int32_t* idx;
  DevCounters* counters;
  cudaStream_t stream;
  int num_sms;
};
// Mixed path: points with evaluations that need FP64 work beyond the polish
// and the spline (the FP64 refinement of l1, or the whole FP64 path near
// degeneracy) leave the main kernel as records; a second kernel evaluates
// those radii and finishes the point. A record holds the point, the running
// minimum of a_c over its other radii and the radius it came from, and the
// hard radii below 32 as a bit mask (bit 16 of r1 flags hard radii >= 32,
// which the second kernel finds again).
struct HardRec {
  int64_t p;
  double a;       // running minimum of a_c over the point's other radii (+inf: none collapsed)
  uint32_t mask;  // hard radii 0..31
  int32_t r1;     // (radius of a) + 1 in bits 0..15; bit 16: hard radii >= 32
};
static_assert(sizeof(HardRec) == 24, "record layout");
// the records of one launch: capacity, and ctr[0] = records requested,
// ctr[1] = nonzero when some did not fit (those points carry idx = -(idx + 3)
// and are recomputed in radius order by the second kernel), ctr[2] = entries
// of `full`: the records that still have radii needing the whole FP64 path
// after the second kernel (the third kernel finishes them)
struct HardWork {
  HardRec* rec;
  int64_t cap;
  unsigned long long* ctr;
  uint32_t* full;
};
constexpr int kHardCounters = 3;

int launch_fp64(const LaunchArgs& a, const DevTable& tab);
int launch_mixed(const LaunchArgs& a, const DevTable& tab, const double* sigma, const HardWork& hw);
int launch_tab(const LaunchArgs& a, const DevTable& tab, const TabDev& td);
int launch_f32x2(const LaunchArgs& a, const DevTable& tab);
int launch_exact(const LaunchArgs& a, const DevTable& tab);
int launch_reset_max(double* F_max, int32_t* idx, int64_t n, cudaStream_t stream, int num_sms);

}  // namespace cc

struct cc_ctx;
namespace cc {
int select_device(const cc_ctx* ctx);  // make ctx's device current (cc_api.cu)
int launch_tab_checked(cc_ctx* ctx, const LaunchArgs& a);                          // cc_tab.cu
int launch_surrogate_checked(cc_ctx* ctx, const LaunchArgs& a, const double* sigma);  // cc_surrogate.cu
}

struct cc_ctx {
  int device = -1;
  int num_sms = 0;
  cc_cosmology cosmo{};
  std::vector<double> a_k, D_k, coef;
  void* d_table = nullptr;  // coef[n-1] | D[n] | Df[n] | bucket[n_buckets]
  void* d_ratio = nullptr;  // growth-ratio splines: FP64 Coef4[3 (n-1)] | FP32 float4[3 (n-1)]
  cc::DevCounters* d_counters = nullptr;
  cc::DevTable tab{};
  // staging of cc_collapse_multi_host (allocated on first use)
  void* d_stage[2] = {nullptr, nullptr};
  size_t stage_bytes = 0;
  double* d_F = nullptr;
  int32_t* d_idx = nullptr;
  int64_t out_cap = 0;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_copied[2] = {nullptr, nullptr};
  cudaEvent_t ev_consumed[2] = {nullptr, nullptr};
  // tabulated mode (cc_set_table)
  bool tab_valid = false;
  void* d_tab_axes = nullptr;
  size_t tab_axes_cap = 0;
  cc::Coef4* d_tab_coef = nullptr;
  size_t tab_coef_cap = 0;
  double* d_tab_work = nullptr;  // node values and tridiagonal scratch
  size_t tab_work_cap = 0;
  cc::TabDev tabdev{};
  // surrogate (cc_surrogate_train / cc_load_surrogate)
  bool sur_valid = false;
  int sur_engine = 1;  // cc_surrogate_engine: CC_SURROGATE_TCGEN05
  unsigned char* d_mlp_img = nullptr;
  float* d_mlp_param = nullptr;  // params | adam m | adam v | grad | loss, stats
  void* d_train = nullptr;       // training records (float4) | count | hull
  size_t train_cap = 0;
  float sur_hull[6] = {0, 0, 0, 0, 0, 0};
  // training state (cc_surrogate_train / _resume / _restore): configuration,
  // Adam steps taken and the length of the learning-rate schedule
  bool sur_trained = false;
  cc_train_config sur_cfg{};
  int64_t sur_step = 0, sur_schedule = 0;
  // interpolation toy (cc_spline_eval)
  void* d_spl = nullptr;
  size_t spl_cap = 0;
  // mixed path: records of points with hard evaluations (allocated on first
  // use at a size; see cc::HardRec) and their two counters
  cc::HardRec* d_hard = nullptr;
  uint32_t* d_hard_full = nullptr;
  int64_t hard_cap = 0;
  unsigned long long* d_hard_ctr = nullptr;
};
