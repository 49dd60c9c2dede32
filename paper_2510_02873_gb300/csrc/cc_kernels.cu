// cc_kernels.cu -- the collapse kernels (arXiv:2510.02873, Sec. 4.1, "Classic"
// kernel) in FP64 and mixed precision, and the device-array initialisation kernel.
//
// One thread per grid point (Sec. 4.1: "assigning the computation at each grid
// point to an individual GPU-thread"), structure-of-arrays planes so that
// consecutive threads read consecutive elements, the spline knots and
// coefficients staged in shared memory once per block, and the running
// maximum over the radii of one launch kept in registers: F_max/idx are read
// and written once per point per launch.
#include "cc_df.cuh"
#include "cc_exact.cuh"
#include "cc_mixed.cuh"

namespace cc {

namespace {

template <typename T>
__device__ __forceinline__ double ld(const T* p) {
  return static_cast<double>(__ldg(p));
}

template <typename T>
__device__ __forceinline__ float ldf(const T* p) {
  return static_cast<float>(__ldg(p));
}

__device__ __forceinline__ void add_counters(DevCounters* cnt, unsigned evals, unsigned coll,
                                             unsigned eds, unsigned refined, unsigned fp64) {
  evals = __reduce_add_sync(0xffffffffu, evals);
  coll = __reduce_add_sync(0xffffffffu, coll);
  eds = __reduce_add_sync(0xffffffffu, eds);
  refined = __reduce_add_sync(0xffffffffu, refined);
  fp64 = __reduce_add_sync(0xffffffffu, fp64);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&cnt->evaluations, static_cast<unsigned long long>(evals));
    if (coll) atomicAdd(&cnt->collapsed, static_cast<unsigned long long>(coll));
    if (eds) atomicAdd(&cnt->eds_branch, static_cast<unsigned long long>(eds));
    if (refined) atomicAdd(&cnt->refined, static_cast<unsigned long long>(refined));
    if (fp64) atomicAdd(&cnt->fp64_branch, static_cast<unsigned long long>(fp64));
  }
}

constexpr int kModeFP64 = 0, kModeMixed = 1, kModeTab = 2, kModeF32x2 = 3, kModeExact = 4;
constexpr int kFp64Radii = 2;  // radii per loop iteration of the FP64 path

// ---- mixed path: the main kernel (collapse_kernel) marks the hard radii and
// writes records; mixed_hard_kernel and mixed_full_kernel finish those points
// (see cc_mixed.cuh).
constexpr int kHardThreads = 128;

template <typename T>
__global__ void __launch_bounds__(kHardThreads)
mixed_hard_kernel(const T* __restrict__ hess, int64_t n, int64_t plane_stride, int64_t radius_stride, int R,
                  int32_t scale_idx0, DevTable tab, RadiusParams rp, HardWork hw, double* __restrict__ F_max,
                  int32_t* __restrict__ idx, DevCounters* __restrict__ cnt) {
  const LaunchSrc<T> src{hess, plane_stride, radius_stride, R, rp, F_max, idx, scale_idx0};
  const unsigned long long req = hw.ctr[0];
  const int64_t nrec = req < static_cast<unsigned long long>(hw.cap) ? static_cast<int64_t>(req) : hw.cap;
  const bool overflow = hw.ctr[1] != 0ull;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t t0 = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  MixedCounts cn;
  for (int64_t i = t0; i < nrec; i += stride) {
    const HardRec rec = hw.rec[i];
    int64_t p = rec.p;
    CC_DBG_CLAMP(p, static_cast<int64_t>(0), n - 1, tab.dbg);
    hard_record(src, rec, p, i, hw, tab, cn);
  }
  if (overflow) {
    for (int64_t p = t0; p < n; p += stride) {
      const int32_t mark = idx[p];
      if (mark > -2) continue;
      idx[p] = -mark - 3;
      recompute_marked(src, p, tab, cn);
    }
  }
  add_counters(cnt, 0u, cn.coll, cn.eds, cn.ref, cn.fp64);
}

template <typename T>
__global__ void __launch_bounds__(kHardThreads)
mixed_full_kernel(const T* __restrict__ hess, int64_t plane_stride, int64_t radius_stride, int R,
                  int32_t scale_idx0, DevTable tab, RadiusParams rp, HardWork hw, double* __restrict__ F_max,
                  int32_t* __restrict__ idx, DevCounters* __restrict__ cnt) {
  const LaunchSrc<T> src{hess, plane_stride, radius_stride, R, rp, F_max, idx, scale_idx0};
  const int64_t nfull = static_cast<int64_t>(hw.ctr[2]);
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  MixedCounts cn;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < nfull; i += stride) {
    int64_t ri = hw.full[i];
    CC_DBG_CLAMP(ri, static_cast<int64_t>(0), hw.cap - 1, tab.dbg);
    const HardRec rec = hw.rec[ri];
    full_record(src, rec, rec.p, tab, cn);
  }
  add_counters(cnt, 0u, cn.coll, cn.eds, cn.ref, cn.fp64);
}

// One thread per point (grid-stride), all R radii of the launch in registers.
// kMode selects collapse_point_fp64, the mixed path (FP32 bulk, its rare
// FP64-heavy radii left to mixed_hard_kernel through records), the
// float-float path (dfl::collapse_point), the exact-growth path
// (exact::collapse_point) or collapse_point_tab (tabulated 1/D_c; its axes
// follow the spline table in shared memory).
// FP64 path: two radii per iteration at 2 blocks of 256 threads per SM (94
// registers, no spill): 1.3 % faster than one radius at 4 blocks and 64
// registers; 3 or 4 radii per iteration, or 1 block, measured the same.
// Mixed path: 5 blocks per SM at 48 registers, each staging the table image
// and the FP32 segment image (the finish's two float4 per evaluation) in
// shared memory, 39 KB (2 % faster than 6 blocks at 40 registers reading the
// segments through L1; 8 blocks at 32 registers spill and run 4 % slower).
// The tabulated path keeps its 98 registers.
template <typename T, bool kSmem, int kMode>
__global__ void __launch_bounds__(kThreads, kMode == 2 ? 1 : (kMode == 1 ? 5 : (kMode == 0 ? 2 : 4)))
collapse_kernel(const T* __restrict__ hess, int64_t n, int64_t plane_stride,
                int64_t radius_stride, int R, int32_t scale_idx0, DevTable tab, RadiusParams rp,
                TabDev td, HardWork hw, double* __restrict__ F_max, int32_t* __restrict__ idx,
                DevCounters* __restrict__ cnt) {
  extern __shared__ Coef4 smem_tab[];
  const Coef4* coef = tab.coef;
  const double* Dk = tab.D;
  const float* Dkf = tab.Df;
  const unsigned short* bucket = tab.bucket;
  const float4* seg = tab.dfseg;
  if constexpr (kSmem) {
    // the table image (coef | D | Df | bucket [| pad | float-float image]) is
    // contiguous: copy it in 16-byte words
    const int words = (kMode == kModeF32x2 || kMode == kModeMixed) ? static_cast<int>((tab.bytes() + 15) / 16) + 2 * (tab.n - 1)
                                            : static_cast<int>(tab.bytes() / 16);
    const uint4* src = reinterpret_cast<const uint4*>(tab.coef);
    uint4* dst = reinterpret_cast<uint4*>(smem_tab);
    for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
    if constexpr (kMode != kModeF32x2 && kMode != kModeMixed) {
      const size_t tail = tab.bytes() & 15;
      if (threadIdx.x < tail)
        reinterpret_cast<unsigned char*>(dst + words)[threadIdx.x] =
            reinterpret_cast<const unsigned char*>(src + words)[threadIdx.x];
    }
    __syncthreads();
    coef = smem_tab;
    Dk = reinterpret_cast<const double*>(smem_tab + (tab.n - 1));
    Dkf = reinterpret_cast<const float*>(Dk + tab.n);
    bucket = reinterpret_cast<const unsigned short*>(Dkf + tab.n);
    seg = reinterpret_cast<const float4*>(smem_tab) + (tab.bytes() + 15) / 16;
  }
  const double* tax = nullptr;
  if constexpr (kMode == kModeTab) {
    // axes image after the spline image (16-byte aligned offset)
    double* dst = reinterpret_cast<double*>(reinterpret_cast<unsigned char*>(smem_tab) + ((tab.bytes() + 15) / 16) * 16);
    const int nwords = static_cast<int>((td.axes_bytes() + 7) / 8);
    for (int i = threadIdx.x; i < nwords; i += blockDim.x) dst[i] = td.axes[i];
    __syncthreads();
    tax = dst;
  }
  unsigned n_eval = 0, n_coll = 0, n_eds = 0, n_ref = 0, n_fp64 = 0;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  // whole warps stay in the loop together so the warp-level counter reduction
  // at the end sees all 32 lanes
  const int64_t n_round = (n + 31) & ~static_cast<int64_t>(31);
  for (int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; p < n_round;
       p += stride) {
    const bool active = p < n;
    if (kMode == kModeF32x2 && active) {
      dfl::MinA2 best;
      for (int r = 0; r < R; ++r) {
        const dfl::Result res =
            dfl::collapse_point(hess + p + static_cast<int64_t>(r) * radius_stride, plane_stride, seg, Dkf, bucket, tab);
        n_coll += res.collapsed;
        n_eds += res.eds;
        n_ref += res.refined;
        best.add(res.collapsed, res.a, r);
      }
      best.store(F_max + p, idx + p, scale_idx0);
      n_eval += R;
    } else if constexpr (kMode == kModeMixed) {
      MinA best;
      MixedCounts cn;
      uint32_t mask = 0;
      bool hi = false;
      const double F_old = active ? F_max[p] : 0.0;
      if (active) {
        for (int r = 0; r < R; ++r) {
          const T* h = hess + p + static_cast<int64_t>(r) * radius_stride;
          const float xx = ldf(h), yy = ldf(h + plane_stride), zz = ldf(h + 2 * plane_stride);
          const float xy = ldf(h + 3 * plane_stride), xz = ldf(h + 4 * plane_stride);
          const float yz = ldf(h + 5 * plane_stride);
          const MixedEigen m = mixed_eigen_f32(xx, yy, zz, xy, xz, yz, rp.tri_thr[r]);
          bool later = m.full || m.need64;
          if (!later) {
            // collapse before the first knot (the EdS segment) also goes to
            // the second kernel, so that this loop carries no EdS selects
            const MixedResult res = mixed_easy<false>(m, coef, Dkf, bucket, tab, seg);
            later = res.eds;
            cn.coll += res.collapsed && !later;
            best.add(res.collapsed && !later, res.a, r);
          }
          if (later) {
            if (r < 32) mask |= 1u << r;
            else hi = true;
          }
        }
        n_eval += R;
      }
      n_coll += cn.coll;
      mixed_record_or_store(active, p, best, mask, hi, hw, F_max + p, idx + p, scale_idx0, F_old);
    } else if (kMode == kModeFP64 && active) {
      // kFp64Radii radii per iteration: independent FP64 chains that the
      // compiler interleaves, so the FP64 unit meets fewer gaps while a warp
      // is in its FP32 seeds and integer conversions (the running minimum
      // still takes the radii in order)
      MinA best;
      const T* base = hess + p;
      int r = 0;
      for (; r + kFp64Radii <= R; r += kFp64Radii) {
        PointResult rs[kFp64Radii];
#pragma unroll
        for (int j = 0; j < kFp64Radii; ++j) {
          const T* h = base + static_cast<int64_t>(r + j) * radius_stride;
          rs[j] = collapse_point_fp64(ld(h), ld(h + plane_stride), ld(h + 2 * plane_stride), ld(h + 3 * plane_stride),
                                      ld(h + 4 * plane_stride), ld(h + 5 * plane_stride), Dk, coef, Dkf, bucket, tab);
        }
#pragma unroll
        for (int j = 0; j < kFp64Radii; ++j) {
          n_coll += rs[j].collapsed;
          n_eds += rs[j].eds;
          n_ref += rs[j].refined;
          best.add(rs[j].collapsed, rs[j].a, r + j);
        }
      }
      for (; r < R; ++r) {
        const T* h = base + static_cast<int64_t>(r) * radius_stride;
        const PointResult res = collapse_point_fp64(ld(h), ld(h + plane_stride), ld(h + 2 * plane_stride),
                                                    ld(h + 3 * plane_stride), ld(h + 4 * plane_stride),
                                                    ld(h + 5 * plane_stride), Dk, coef, Dkf, bucket, tab);
        n_coll += res.collapsed;
        n_eds += res.eds;
        n_ref += res.refined;
        best.add(res.collapsed, res.a, r);
      }
      best.store<false>(F_max + p, idx + p, scale_idx0);
      n_eval += R;
    } else if (kMode != kModeF32x2 && active) {
      MinA best;
      const T* base = hess + p;
      for (int r = 0; r < R; ++r) {
        const T* h = base + static_cast<int64_t>(r) * radius_stride;
        double a;
        bool coll;
        if constexpr (kMode == kModeMixed) {
          const float xx = ldf(h), yy = ldf(h + plane_stride), zz = ldf(h + 2 * plane_stride);
          const float xy = ldf(h + 3 * plane_stride), xz = ldf(h + 4 * plane_stride);
          const float yz = ldf(h + 5 * plane_stride);
          const MixedResult res =
              collapse_point_mixed(xx, yy, zz, xy, xz, yz, rp.tri_thr[r], Dk, coef, Dkf, bucket, tab);
          n_coll += res.collapsed;
          n_eds += res.eds;
          n_ref += res.refined;
          n_fp64 += res.fp64;
          a = res.a;
          coll = res.collapsed;
        } else if constexpr (kMode == kModeTab) {
          const double xx = ld(h), yy = ld(h + plane_stride), zz = ld(h + 2 * plane_stride);
          const double xy = ld(h + 3 * plane_stride), xz = ld(h + 4 * plane_stride);
          const double yz = ld(h + 5 * plane_stride);
          const TabResult res = collapse_point_tab(xx, yy, zz, xy, xz, yz, Dk, coef, Dkf, bucket, tab, td, tax, td.coef);
          n_coll += res.collapsed;
          n_eds += res.eds;
          n_ref += res.refined;
          n_fp64 += res.outside;
          a = res.a;
          coll = res.collapsed;
        } else if constexpr (kMode == kModeExact) {
          const double xx = ld(h), yy = ld(h + plane_stride), zz = ld(h + 2 * plane_stride);
          const double xy = ld(h + 3 * plane_stride), xz = ld(h + 4 * plane_stride);
          const double yz = ld(h + 5 * plane_stride);
          const exact::Result res = exact::collapse_point(xx, yy, zz, xy, xz, yz, Dk, coef, Dkf, bucket, tab);
          n_coll += res.collapsed;
          n_eds += res.eds;
          n_ref += res.refined;
          a = res.a;
          coll = res.collapsed;
        } else {
          const double xx = ld(h), yy = ld(h + plane_stride), zz = ld(h + 2 * plane_stride);
          const double xy = ld(h + 3 * plane_stride), xz = ld(h + 4 * plane_stride);
          const double yz = ld(h + 5 * plane_stride);
          const PointResult res = collapse_point_fp64(xx, yy, zz, xy, xz, yz, Dk, coef, Dkf, bucket, tab);
          n_coll += res.collapsed;
          n_eds += res.eds;
          n_ref += res.refined;
          a = res.a;
          coll = res.collapsed;
        }
        best.add(coll, a, r);
      }
      best.store<kMode == kModeMixed>(F_max + p, idx + p, scale_idx0);
      n_eval += R;
    }
  }
  add_counters(cnt, n_eval, n_coll, n_eds, n_ref, n_fp64);
}

__global__ void reset_max_kernel(double* __restrict__ F_max, int32_t* __restrict__ idx, int64_t n) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; p < n; p += stride) {
    F_max[p] = 0.0;
    idx[p] = -1;
  }
}

template <typename T, bool kSmem, int kMode>
int launch_typed(const LaunchArgs& a, const DevTable& tab, const RadiusParams& rp, const TabDev& td,
                 const HardWork& hw) {
  auto kern = collapse_kernel<T, kSmem, kMode>;
  size_t smem = kSmem ? ((tab.bytes() + 15) / 16) * 16 : 0;
  if (kMode == kModeTab) smem = ((tab.bytes() + 15) / 16) * 16 + ((td.axes_bytes() + 15) / 16) * 16;
  if ((kMode == kModeF32x2 || kMode == kModeMixed) && kSmem) smem = ((tab.bytes() + 15) / 16) * 16 + sizeof(float4) * 2 * (tab.n - 1);
  // resident blocks per SM, cached per shared-memory size (tables differ between contexts)
  static thread_local int occ = 0;
  static thread_local size_t occ_smem = ~size_t{0};
  if (smem != occ_smem) occ = 0;
  if (kSmem && smem > 48 * 1024) {
    if (int rc = check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 static_cast<int>(smem)),
                            "cudaFuncSetAttribute"))
      return rc;
  }
  if (occ == 0) {
    int blocks_per_sm = 0;
    if (int rc = check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern,
                                                                          kThreads, smem),
                            "occupancy query"))
      return rc;
    occ = blocks_per_sm > 0 ? blocks_per_sm : 1;
    occ_smem = smem;
  }
  const int64_t need = (a.n + kThreads - 1) / kThreads;
  const int64_t cap = static_cast<int64_t>(a.num_sms) * occ;
  const int grid = static_cast<int>(need < cap ? need : cap);
  DevTable t = tab;  // the index checks of debug builds report into this launch's flags
  t.dbg = &a.counters->error_flags;
  TabDev tdl = td;
  tdl.dbg = t.dbg;
  kern<<<grid, kThreads, smem, a.stream>>>(static_cast<const T*>(a.hess), a.n, a.plane_stride,
                                           a.radius_stride, a.R, a.scale_idx0, t, rp, tdl, hw, a.F_max,
                                           a.idx, a.counters);
  if (int rc = check_cuda(cudaGetLastError(), "collapse_kernel launch")) return rc;
  if constexpr (kMode == kModeMixed) {
    // the recorded points: a grid of a few blocks per SM strides over them
    mixed_hard_kernel<T><<<4 * a.num_sms, kHardThreads, 0, a.stream>>>(
        static_cast<const T*>(a.hess), a.n, a.plane_stride, a.radius_stride, a.R, a.scale_idx0, t, rp, hw,
        a.F_max, a.idx, a.counters);
    if (int rc = check_cuda(cudaGetLastError(), "mixed_hard_kernel launch")) return rc;
    mixed_full_kernel<T><<<4 * a.num_sms, kHardThreads, 0, a.stream>>>(
        static_cast<const T*>(a.hess), a.plane_stride, a.radius_stride, a.R, a.scale_idx0, t, rp, hw, a.F_max,
        a.idx, a.counters);
    return check_cuda(cudaGetLastError(), "mixed_full_kernel launch");
  }
  return CC_OK;
}

template <int kMode>
int launch_mode(const LaunchArgs& a, const DevTable& tab, const RadiusParams& rp, const TabDev& td,
                const HardWork& hw = HardWork{}) {
  const size_t staged = (kMode == kModeF32x2 || kMode == kModeMixed) ? ((tab.bytes() + 15) / 16) * 16 + sizeof(float4) * 2 * (tab.n - 1)
                                               : tab.bytes();
  const bool smem = staged <= static_cast<size_t>(kSmemTableMaxBytes);
  if (kMode == kModeTab) {  // the tabulated kernel always stages both images
    if (a.dtype == CC_F64) return launch_typed<double, true, kMode>(a, tab, rp, td, hw);
    return launch_typed<float, true, kMode>(a, tab, rp, td, hw);
  }
  if (a.dtype == CC_F64)
    return smem ? launch_typed<double, true, kMode>(a, tab, rp, td, hw) : launch_typed<double, false, kMode>(a, tab, rp, td, hw);
  return smem ? launch_typed<float, true, kMode>(a, tab, rp, td, hw) : launch_typed<float, false, kMode>(a, tab, rp, td, hw);
}

}  // namespace

int launch_fp64(const LaunchArgs& a, const DevTable& tab) {
  return launch_mode<kModeFP64>(a, tab, RadiusParams{}, TabDev{});
}

int launch_f32x2(const LaunchArgs& a, const DevTable& tab) {
  if (tab.dfseg == nullptr) return set_error(CC_ENOTSUP, "CC_MODE_F32X2 needs the float-float spline image");
  return launch_mode<kModeF32x2>(a, tab, RadiusParams{}, TabDev{});
}

int launch_exact(const LaunchArgs& a, const DevTable& tab) {
  if (tab.rc64 == nullptr || tab.rc32 == nullptr)
    return set_error(CC_ENOTSUP, "CC_MODE_EXACT_GROWTH needs the growth-ratio tables");
  return launch_mode<kModeExact>(a, tab, RadiusParams{}, TabDev{});
}

int launch_tab(const LaunchArgs& a, const DevTable& tab, const TabDev& td) {
  return launch_mode<kModeTab>(a, tab, RadiusParams{}, td);
}

int launch_mixed(const LaunchArgs& a, const DevTable& tab, const double* sigma, const HardWork& hw) {
  // at most kMaxRadiiPerLaunch radii per launch (their thresholds ride in the
  // kernel parameters); longer radius lists run as consecutive launches
  for (int r0 = 0; r0 < a.R; r0 += kMaxRadiiPerLaunch) {
    LaunchArgs c = a;
    c.R = (a.R - r0 < kMaxRadiiPerLaunch) ? a.R - r0 : kMaxRadiiPerLaunch;
    c.hess = static_cast<const unsigned char*>(a.hess) + static_cast<size_t>(r0) * a.radius_stride * a.dtype;
    c.scale_idx0 = a.scale_idx0 + r0;
    RadiusParams rp;
    for (int r = 0; r < c.R; ++r) rp.tri_thr[r] = static_cast<float>(1e-4 * sigma[r0 + r]);
    if (int rc = check_cuda(cudaMemsetAsync(hw.ctr, 0, kHardCounters * sizeof(unsigned long long), a.stream),
                            "cudaMemsetAsync(hard records)"))
      return rc;
    if (int rc = launch_mode<kModeMixed>(c, tab, rp, TabDev{}, hw)) return rc;
  }
  return CC_OK;
}

int launch_reset_max(double* F_max, int32_t* idx, int64_t n, cudaStream_t stream, int num_sms) {
  const int64_t need = (n + 255) / 256;
  const int64_t cap = static_cast<int64_t>(num_sms) * 8;
  const int grid = static_cast<int>(need < cap ? need : cap);
  reset_max_kernel<<<grid, 256, 0, stream>>>(F_max, idx, n);
  return check_cuda(cudaGetLastError(), "reset_max_kernel launch");
}

}  // namespace cc
