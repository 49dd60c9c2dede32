// cc_mixed.cuh -- the mixed path's hard radii, shared by the per-launch
// kernels (cc_kernels.cu) and the batched kernel (cc_batch.cu).
//
// About 0.5 % of the mixed path's evaluations need FP64 work beyond the
// polish and the spline (the FP64 refinement of l1, or the whole FP64 path
// near degeneracy), and a few collapse on the EdS segment below the first
// knot. A main kernel that evaluated them in place, or from a per-warp queue,
// carried that code next to its radius loop and spilled at the register
// budget its occupancy needs. Instead the main kernel marks those radii (a
// bit per radius below 32, a flag for the others) and, at the end of a point
// that has any, writes a record (HardRec) in place of its result. A second
// kernel evaluates the marked radii (hard_record) and stores the point, or,
// when some radius needs the whole FP64 path, hands the record to a third
// kernel (full_record). The running minimum merges them out of radius order
// with ties to the smaller radius, so F_max and idx are those of the in-order
// loop. A point beyond the record capacity marks idx as -(idx + 3) and is
// recomputed in radius order (recompute_marked).
#pragma once

#include "cc_device.cuh"

namespace cc {

template <typename T>
__device__ __forceinline__ float ld32(const T* p) {
  return static_cast<float>(__ldg(p));
}

struct MixedCounts {
  unsigned coll = 0, eds = 0, ref = 0, fp64 = 0;
  __device__ __forceinline__ void add(const MixedResult& res) {
    coll += res.collapsed;
    eds += res.eds;
    ref += res.refined;
    fp64 += res.fp64;
  }
};

// One radius that needs nothing beyond the FP32 stages, the FP64 polish and
// the spline (m from mixed_eigen_f32 with neither m.full nor m.need64, or
// after mixed_refine64): the same steps, and so the same result, as
// collapse_point_mixed. kEds = false leaves out the EdS segment (see
// mixed_finish): the caller then sends radii with res.eds elsewhere.
template <bool kEds = true>
__device__ __forceinline__ MixedResult mixed_easy(const MixedEigen& m, const Coef4* __restrict__ coef,
                                                  const float* __restrict__ Dkf,
                                                  const unsigned short* __restrict__ bucket, const DevTable& tab,
                                                  const float4* __restrict__ seg) {
  const MixedCoef k = mixed_coef(m);
  const float uf = cubic_largest_root_seed(-k.l1f, k.c2f, k.c3f);
  const RootF32 rt = newton_f32_r(k, __fdividef(1.0f, uf));
  return mixed_finish_r<kEds>(m, k, rt.D, rt.rdA, coef, Dkf, bucket, tab, seg);
}

constexpr int32_t kHardHigh = 0x10000;  // HardRec::r1: marked radii >= 32

// The six FP32 components of one point at one radius.
struct Planes6 {
  float xx, yy, zz, xy, xz, yz;
};
template <typename T>
__device__ __forceinline__ Planes6 load6(const T* h, int64_t ps) {
  return Planes6{ld32(h), ld32(h + ps), ld32(h + 2 * ps), ld32(h + 3 * ps), ld32(h + 4 * ps), ld32(h + 5 * ps)};
}

// End of a point in a main kernel. All 32 lanes of the warp call this. A point
// without marked radii stores its result; the others take consecutive record
// slots (one atomic per warp) under `key` (the point, or the point and its
// batch item). A point whose slot is beyond the capacity keeps F_max and marks
// idx as -(idx + 3) (idx is -1 or a scale index, so the mark is <= -2).
// F_old: the point's F_max, read before its radii so that the load's latency
// is hidden behind them (only this thread reads or writes that entry).
__device__ __forceinline__ void mixed_record_or_store(bool active, int64_t key, const MinA& best, uint32_t mask,
                                                      bool hi, const HardWork& hw, double* __restrict__ F_max,
                                                      int32_t* __restrict__ idx, int32_t scale_idx0, double F_old) {
  const bool need = active && (mask != 0u || hi);
  const unsigned bal = __ballot_sync(0xffffffffu, need);
  if (bal != 0u) {
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(bal) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(hw.ctr, static_cast<unsigned long long>(__popc(bal)));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (need) {
      const unsigned long long slot = base + static_cast<unsigned>(__popc(bal & ((1u << lane) - 1u)));
      if (slot < static_cast<unsigned long long>(hw.cap)) {
        HardRec rec;
        rec.p = key;
        rec.a = best.a;
        rec.mask = mask;
        rec.r1 = (best.r + 1) | (hi ? kHardHigh : 0);
        hw.rec[slot] = rec;
      } else {
        *idx = -*idx - 3;
        atomicOr(hw.ctr + 1, 1ull);
      }
    }
  }
  if (active && !need) best.store_vs<true>(F_old, F_max, idx, scale_idx0);
}

// Where the record workers find a point's planes, thresholds and outputs.
// LaunchSrc: one launch (thresholds in the kernel's parameter space);
// ItemSrc: one item of a batch (thresholds in device memory).
template <typename T>
struct LaunchSrc {
  const T* hess;
  int64_t ps, rs;
  int R;
  const RadiusParams& rp;
  double* F_max;
  int32_t* idx;
  int32_t s0;
  __device__ __forceinline__ Planes6 planes(int64_t p, int r) const {
    return load6(hess + p + static_cast<int64_t>(r) * rs, ps);
  }
  __device__ __forceinline__ float thr(int r) const { return rp.tri_thr[r]; }
};
template <typename T>
struct ItemSrc {
  const T* hess;
  int64_t ps, rs;
  int R;
  const float* tri_thr;
  double* F_max;
  int32_t* idx;
  int32_t s0;
  __device__ __forceinline__ Planes6 planes(int64_t p, int r) const {
    return load6(hess + p + static_cast<int64_t>(r) * rs, ps);
  }
  __device__ __forceinline__ float thr(int r) const { return __ldg(tri_thr + r); }
};

// Second kernel, one record (index i) of point p: the marked radii through
// mixed_eigen (the FP64 refinement of l1 where flagged) and the full mixed
// finish; radii that need the whole FP64 path stay in the record, which then
// joins hw.full for the third kernel. Beyond radius 32 every radius is taken
// again: the refined and EdS ones are new, and merging one the main kernel
// kept leaves the minimum as it is. Counts the evaluations the main kernel
// left out.
template <class Src>
__device__ __forceinline__ void hard_record(const Src& src, HardRec rec, int64_t p, int64_t i, const HardWork& hw,
                                            const DevTable& tab, MixedCounts& cn) {
  MinA best;
  best.a = rec.a;
  best.r = (rec.r1 & 0xffff) - 1;
  uint32_t full = 0;
  bool full_hi = false;
  for (uint32_t m = rec.mask; m != 0u; m &= m - 1u) {
    const int r = __ffs(m) - 1;
    const Planes6 v = src.planes(p, r);
    const MixedEigen me = mixed_eigen(v.xx, v.yy, v.zz, v.xy, v.xz, v.yz, src.thr(r));
    if (me.full) {
      full |= 1u << r;
      continue;
    }
    const MixedResult res = mixed_easy(me, tab.coef, tab.Df, tab.bucket, tab, tab.dfseg);
    cn.add(res);
    best.add_any_order(res.collapsed, res.a, r);
  }
  if (rec.r1 & kHardHigh) {
    for (int r = 32; r < src.R; ++r) {
      const Planes6 v = src.planes(p, r);
      const MixedEigen me = mixed_eigen_f32(v.xx, v.yy, v.zz, v.xy, v.xz, v.yz, src.thr(r));
      if (me.full) {
        full_hi = true;
        continue;
      }
      MixedEigen mr = me;
      if (me.need64) mixed_refine64(mr, v.xx, v.yy, v.zz, v.xy, v.xz, v.yz);
      const MixedResult res = mixed_easy(mr, tab.coef, tab.Df, tab.bucket, tab, tab.dfseg);
      if (me.need64 || res.eds) cn.add(res);
      best.add_any_order(res.collapsed, res.a, r);
    }
  }
  if (full != 0u || full_hi) {
    rec.a = best.a;
    rec.mask = full;
    rec.r1 = (best.r + 1) | (full_hi ? kHardHigh : 0);
    hw.rec[i] = rec;
    int64_t k = static_cast<int64_t>(atomicAdd(hw.ctr + 2, 1ull));
    CC_DBG_CLAMP(k, static_cast<int64_t>(0), hw.cap - 1, tab.dbg);
    hw.full[k] = static_cast<uint32_t>(i);
  } else {
    best.store<true>(src.F_max + p, src.idx + p, src.s0);
  }
}

// Third kernel, one record of point p: the radii on the whole FP64 path
// through full_fp64 (what collapse_point_mixed runs for them), merged into
// the record's running minimum; then the point's result is stored.
template <class Src>
__device__ __forceinline__ void full_record(const Src& src, const HardRec& rec, int64_t p, const DevTable& tab,
                                            MixedCounts& cn) {
  MinA best;
  best.a = rec.a;
  best.r = (rec.r1 & 0xffff) - 1;
  for (uint32_t m = rec.mask; m != 0u; m &= m - 1u) {
    const int r = __ffs(m) - 1;
    const Planes6 v = src.planes(p, r);
    const MixedResult res = full_fp64(v.xx, v.yy, v.zz, v.xy, v.xz, v.yz, tab.D, tab.coef, tab.Df, tab.bucket, tab);
    cn.add(res);
    best.add_any_order(res.collapsed, res.a, r);
  }
  if (rec.r1 & kHardHigh) {
    for (int r = 32; r < src.R; ++r) {
      const Planes6 v = src.planes(p, r);
      if (!mixed_eigen_f32(v.xx, v.yy, v.zz, v.xy, v.xz, v.yz, src.thr(r)).full) continue;
      const MixedResult res = full_fp64(v.xx, v.yy, v.zz, v.xy, v.xz, v.yz, tab.D, tab.coef, tab.Df, tab.bucket, tab);
      cn.add(res);
      best.add_any_order(res.collapsed, res.a, r);
    }
  }
  best.store<true>(src.F_max + p, src.idx + p, src.s0);
}

// A point marked after an overflow (idx already restored): every radius in
// order, each path in place. Counts the evaluations the main kernel left out.
template <class Src>
__device__ __forceinline__ void recompute_marked(const Src& src, int64_t p, const DevTable& tab, MixedCounts& cn) {
  MinA best;
  for (int r = 0; r < src.R; ++r) {
    const Planes6 v = src.planes(p, r);
    const MixedEigen me = mixed_eigen_f32(v.xx, v.yy, v.zz, v.xy, v.xz, v.yz, src.thr(r));
    MixedResult res;
    if (me.full || me.need64) {
      res = collapse_point_mixed(v.xx, v.yy, v.zz, v.xy, v.xz, v.yz, src.thr(r), tab.D, tab.coef, tab.Df, tab.bucket,
                                 tab);
      cn.add(res);
    } else {
      res = mixed_easy(me, tab.coef, tab.Df, tab.bucket, tab, tab.dfseg);
      if (res.eds) cn.add(res);
    }
    best.add(res.collapsed, res.a, r);
  }
  best.store<true>(src.F_max + p, src.idx + p, src.s0);
}

}  // namespace cc
