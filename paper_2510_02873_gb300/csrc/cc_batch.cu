// cc_batch.cu -- many realizations of uneven size in one persistent launch.
//
// The paper evaluates one grid per launch (Sec. 4.1); a campaign of many
// realizations (Sec. 5.5: thousands of runs) with different grid sizes and
// radius counts would pay a launch, a ramp-up and a tail per realization. Here
// the CTAs of a single persistent kernel (one wave: SMs x resident blocks) take
// tiles of points from a device work counter until every tile of every
// realization is done; a tile runs all radii of its realization for its points
// with the running maximum in registers, exactly as the per-realization
// kernel does. The work counter is the only shared state: CTAs never wait on
// one another. Tile sizes per size class and the block size come from a small
// timing autotuner; the launch can be replayed from a captured CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "cc_mixed.cuh"

namespace cc {

struct BatchItemDev {
  const void* hess;
  int64_t n, plane_stride, radius_stride;
  int64_t tile_begin;  // first global tile index of this item
  double* F_max;
  int32_t* idx;
  const float* tri_thr;  // R per-radius thresholds (mixed mode)
  int32_t R, scale_idx0, dtype, tile_points;
};

namespace {

template <typename T>
__device__ __forceinline__ double ldd(const T* p) { return static_cast<double>(__ldg(p)); }

// The launch's counts, reduced per warp and added once per warp.
__device__ __forceinline__ void batch_counters(DevCounters* cnt, unsigned n_eval, unsigned n_coll, unsigned n_eds,
                                               unsigned n_ref, unsigned n_fp64) {
  n_eval = __reduce_add_sync(0xffffffffu, n_eval);
  n_coll = __reduce_add_sync(0xffffffffu, n_coll);
  n_eds = __reduce_add_sync(0xffffffffu, n_eds);
  n_ref = __reduce_add_sync(0xffffffffu, n_ref);
  n_fp64 = __reduce_add_sync(0xffffffffu, n_fp64);
  if ((threadIdx.x & 31) == 0) {
    if (n_eval) atomicAdd(&cnt->evaluations, static_cast<unsigned long long>(n_eval));
    if (n_coll) atomicAdd(&cnt->collapsed, static_cast<unsigned long long>(n_coll));
    if (n_eds) atomicAdd(&cnt->eds_branch, static_cast<unsigned long long>(n_eds));
    if (n_ref) atomicAdd(&cnt->refined, static_cast<unsigned long long>(n_ref));
    if (n_fp64) atomicAdd(&cnt->fp64_branch, static_cast<unsigned long long>(n_fp64));
  }
}

// FP64 mode: one point, all radii in order.
template <typename T>
__device__ __forceinline__ void run_point_fp64(const BatchItemDev& it, int64_t p, const double* Dk, const Coef4* coef,
                                               const float* Dkf, const unsigned short* bucket, const DevTable& tab,
                                               unsigned& n_coll, unsigned& n_eds, unsigned& n_ref) {
  MinA best;
  const T* base = static_cast<const T*>(it.hess) + p;
  const int64_t ps = it.plane_stride;
  for (int r = 0; r < it.R; ++r) {
    const T* h = base + static_cast<int64_t>(r) * it.radius_stride;
    const PointResult res = collapse_point_fp64(ldd(h), ldd(h + ps), ldd(h + 2 * ps), ldd(h + 3 * ps),
                                                ldd(h + 4 * ps), ldd(h + 5 * ps), Dk, coef, Dkf, bucket, tab);
    n_coll += res.collapsed;
    n_eds += res.eds;
    n_ref += res.refined;
    best.add(res.collapsed, res.a, r);
  }
  best.store<false>(it.F_max + p, it.idx + p, it.scale_idx0);
}

// Mixed mode: one point, as the per-launch mixed kernel does it: the hard and
// EdS radii are marked, and a point with any leaves a record (key: batch item
// << kItemShift | point) for the two follow-up kernels (cc_mixed.cuh). All 32
// lanes of the warp call this (inactive lanes with active = false).
constexpr int kItemShift = 40;
template <typename T>
__device__ __forceinline__ void run_point_mixed(const BatchItemDev& it, int item, int64_t p, bool active,
                                                const Coef4* coef, const float* Dkf, const unsigned short* bucket,
                                                const DevTable& tab, const HardWork& hw, unsigned& n_coll) {
  MinA best;
  uint32_t mask = 0;
  bool hi = false;
  const double F_old = active ? it.F_max[p] : 0.0;
  if (active) {
    const T* base = static_cast<const T*>(it.hess) + p;
    for (int r = 0; r < it.R; ++r) {
      const Planes6 v = load6(base + static_cast<int64_t>(r) * it.radius_stride, it.plane_stride);
      const MixedEigen m = mixed_eigen_f32(v.xx, v.yy, v.zz, v.xy, v.xz, v.yz, __ldg(it.tri_thr + r));
      bool later = m.full || m.need64;
      if (!later) {
        const MixedResult res = mixed_easy<false>(m, coef, Dkf, bucket, tab, tab.dfseg);
        later = res.eds;
        n_coll += res.collapsed && !later;
        best.add(res.collapsed && !later, res.a, r);
      }
      if (later) {
        if (r < 32) mask |= 1u << r;
        else hi = true;
      }
    }
  }
  const int64_t key = (static_cast<int64_t>(item) << kItemShift) | p;
  mixed_record_or_store(active, key, best, mask, hi, hw, it.F_max + (active ? p : 0), it.idx + (active ? p : 0),
                        it.scale_idx0, F_old);
}

template <bool kMixed, int kBlock>
__global__ void __launch_bounds__(kBlock, (kMixed ? 1536 : 1024) / kBlock)
batched_kernel(const BatchItemDev* __restrict__ items, int nitems, int64_t total_tiles,
               unsigned long long* __restrict__ work, DevTable tab, HardWork hw, DevCounters* __restrict__ cnt) {
  extern __shared__ Coef4 smem_tab[];
  __shared__ long long s_tile;
  __shared__ int s_item;
  __shared__ BatchItemDev s_it;
  {  // table image to shared memory (16-byte words)
    const int words = static_cast<int>(tab.bytes() / 16);
    const uint4* src = reinterpret_cast<const uint4*>(tab.coef);
    uint4* dst = reinterpret_cast<uint4*>(smem_tab);
    for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
    const size_t tail = tab.bytes() & 15;
    if (threadIdx.x < tail)
      reinterpret_cast<unsigned char*>(dst + words)[threadIdx.x] =
          reinterpret_cast<const unsigned char*>(src + words)[threadIdx.x];
  }
  const Coef4* coef = smem_tab;
  const double* Dk = reinterpret_cast<const double*>(smem_tab + (tab.n - 1));
  const float* Dkf = reinterpret_cast<const float*>(Dk + tab.n);
  const unsigned short* bucket = reinterpret_cast<const unsigned short*>(Dkf + tab.n);
  unsigned n_eval = 0, n_coll = 0, n_eds = 0, n_ref = 0;
  for (;;) {
    if (threadIdx.x == 0) {
      const long long t = static_cast<long long>(atomicAdd(work, 1ULL));
      int lo = 0, hi = nitems - 1;  // last item with tile_begin <= t
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (items[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
      }
      s_tile = t;
      s_item = lo;
      if (t < total_tiles) s_it = items[lo];
    }
    __syncthreads();  // also orders the table staging before first use
    const long long t = s_tile;
    if (t >= total_tiles) break;
    const BatchItemDev& it = s_it;  // read from shared memory (keeps registers for the point)
    const int64_t p0 = (t - it.tile_begin) * it.tile_points;
    const int64_t p1 = min(p0 + it.tile_points, it.n);
    if constexpr (kMixed) {
      // whole warps step together (the record step is warp-wide)
      for (int64_t pb = p0; pb < p1; pb += kBlock) {
        const int64_t p = pb + threadIdx.x;
        const bool active = p < p1;
        if (it.dtype == CC_F32)
          run_point_mixed<float>(it, s_item, p, active, coef, Dkf, bucket, tab, hw, n_coll);
        else
          run_point_mixed<double>(it, s_item, p, active, coef, Dkf, bucket, tab, hw, n_coll);
        if (active) n_eval += it.R;
      }
    } else {
      for (int64_t p = p0 + threadIdx.x; p < p1; p += kBlock) {
        if (it.dtype == CC_F32)
          run_point_fp64<float>(it, p, Dk, coef, Dkf, bucket, tab, n_coll, n_eds, n_ref);
        else
          run_point_fp64<double>(it, p, Dk, coef, Dkf, bucket, tab, n_coll, n_eds, n_ref);
        n_eval += it.R;
      }
    }
    __syncthreads();  // every thread is done with s_it before thread 0 takes the next tile
  }
  batch_counters(cnt, n_eval, n_coll, n_eds, n_ref, 0u);
}

// The mixed batch's recorded points (second kernel) and, after an overflow,
// its marked points; see hard_record and recompute_marked.
constexpr int kHardThreads = 128;
constexpr int64_t kPointMask = (int64_t{1} << kItemShift) - 1;

__global__ void __launch_bounds__(kHardThreads)
batch_hard_kernel(const BatchItemDev* __restrict__ items, int nitems, DevTable tab, HardWork hw,
                  DevCounters* __restrict__ cnt) {
  const unsigned long long req = hw.ctr[0];
  const int64_t nrec = req < static_cast<unsigned long long>(hw.cap) ? static_cast<int64_t>(req) : hw.cap;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t t0 = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  MixedCounts cn;
  for (int64_t i = t0; i < nrec; i += stride) {
    const HardRec rec = hw.rec[i];
    int item = static_cast<int>(rec.p >> kItemShift);
    CC_DBG_CLAMP(item, 0, nitems - 1, tab.dbg);
    const BatchItemDev& it = items[item];
    const int64_t p = rec.p & kPointMask;
    if (it.dtype == CC_F32)
      hard_record(ItemSrc<float>{static_cast<const float*>(it.hess), it.plane_stride, it.radius_stride, it.R,
                                 it.tri_thr, it.F_max, it.idx, it.scale_idx0}, rec, p, i, hw, tab, cn);
    else
      hard_record(ItemSrc<double>{static_cast<const double*>(it.hess), it.plane_stride, it.radius_stride, it.R,
                                  it.tri_thr, it.F_max, it.idx, it.scale_idx0}, rec, p, i, hw, tab, cn);
  }
  if (hw.ctr[1] != 0ull) {
    for (int item = 0; item < nitems; ++item) {
      const BatchItemDev& it = items[item];
      for (int64_t p = t0; p < it.n; p += stride) {
        const int32_t mark = it.idx[p];
        if (mark > -2) continue;
        it.idx[p] = -mark - 3;
        if (it.dtype == CC_F32)
          recompute_marked(ItemSrc<float>{static_cast<const float*>(it.hess), it.plane_stride, it.radius_stride, it.R,
                                          it.tri_thr, it.F_max, it.idx, it.scale_idx0}, p, tab, cn);
        else
          recompute_marked(ItemSrc<double>{static_cast<const double*>(it.hess), it.plane_stride, it.radius_stride,
                                           it.R, it.tri_thr, it.F_max, it.idx, it.scale_idx0}, p, tab, cn);
      }
    }
  }
  batch_counters(cnt, 0u, cn.coll, cn.eds, cn.ref, cn.fp64);
}

// The mixed batch's records left with radii on the whole FP64 path (third kernel).
__global__ void __launch_bounds__(kHardThreads)
batch_full_kernel(const BatchItemDev* __restrict__ items, int nitems, DevTable tab, HardWork hw,
                  DevCounters* __restrict__ cnt) {
  const int64_t nfull = static_cast<int64_t>(hw.ctr[2]);
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  MixedCounts cn;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < nfull; i += stride) {
    int64_t ri = hw.full[i];
    CC_DBG_CLAMP(ri, static_cast<int64_t>(0), hw.cap - 1, tab.dbg);
    const HardRec rec = hw.rec[ri];
    int item = static_cast<int>(rec.p >> kItemShift);
    CC_DBG_CLAMP(item, 0, nitems - 1, tab.dbg);
    const BatchItemDev& it = items[item];
    const int64_t p = rec.p & kPointMask;
    if (it.dtype == CC_F32)
      full_record(ItemSrc<float>{static_cast<const float*>(it.hess), it.plane_stride, it.radius_stride, it.R,
                                 it.tri_thr, it.F_max, it.idx, it.scale_idx0}, rec, p, tab, cn);
    else
      full_record(ItemSrc<double>{static_cast<const double*>(it.hess), it.plane_stride, it.radius_stride, it.R,
                                  it.tri_thr, it.F_max, it.idx, it.scale_idx0}, rec, p, tab, cn);
  }
  batch_counters(cnt, 0u, cn.coll, cn.eds, cn.ref, cn.fp64);
}

constexpr int kTileCandidates[] = {256, 512, 1024, 2048, 4096, 8192};
constexpr int kBlockCandidates[] = {128, 256};

int size_class(int64_t n) {
  int c = 0;
  while ((int64_t{1} << c) < n) ++c;
  return c;
}

}  // namespace
}  // namespace cc

using namespace cc;

struct cc_batch {
  cc_ctx* ctx = nullptr;
  cc_mode mode = CC_MODE_FP64;
  std::vector<cc_batch_item> items;
  std::vector<std::vector<float>> thr;  // per item, per radius
  std::vector<int> tile;                // per item
  int block = 256;
  BatchItemDev* d_items = nullptr;
  float* d_thr = nullptr;
  unsigned long long* d_work = nullptr;
  // mixed mode: records of the points with hard radii (cc::HardRec, shared
  // by every item; the key packs the item above bit 40)
  cc::HardRec* d_hard = nullptr;
  uint32_t* d_hard_full = nullptr;
  int64_t hard_cap = 0;
  unsigned long long* d_hard_ctr = nullptr;
  int64_t total_tiles = 0;
  bool dirty = true;                    // device item table needs an upload
  cudaGraphExec_t graph_exec = nullptr;
  cudaGraph_t graph = nullptr;
};

namespace cc {
namespace {

int upload_items(cc_batch* b, cudaStream_t st) {
  std::vector<BatchItemDev> dev(b->items.size());
  int64_t tiles = 0;
  size_t thr_off = 0;
  for (size_t i = 0; i < b->items.size(); ++i) {
    const cc_batch_item& it = b->items[i];
    BatchItemDev& d = dev[i];
    d.hess = it.hess;
    d.n = it.n;
    d.plane_stride = it.plane_stride;
    d.radius_stride = it.radius_stride;
    d.F_max = it.F_max;
    d.idx = it.idx;
    d.R = it.R;
    d.scale_idx0 = it.scale_idx0;
    d.dtype = it.dtype;
    d.tile_points = b->tile[i];
    d.tile_begin = tiles;
    d.tri_thr = b->d_thr + thr_off;
    thr_off += static_cast<size_t>(it.R);
    tiles += (it.n + b->tile[i] - 1) / b->tile[i];
  }
  b->total_tiles = tiles;
  // synchronous copy: the host vector is released when this function returns
  if (int rc = check_cuda(cudaStreamSynchronize(st), "cudaStreamSynchronize")) return rc;
  if (int rc = check_cuda(cudaMemcpy(b->d_items, dev.data(), sizeof(BatchItemDev) * dev.size(),
                                     cudaMemcpyHostToDevice), "cudaMemcpy(batch items)"))
    return rc;
  b->dirty = false;
  return CC_OK;
}

template <bool kMixed, int kBlock>
int launch_batch_t(cc_batch* b, cudaStream_t st) {
  auto kern = batched_kernel<kMixed, kBlock>;
  const DevTable& tab = b->ctx->tab;
  const size_t smem = ((tab.bytes() + 15) / 16) * 16;
  if (smem > 48 * 1024) {
    if (int rc = check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 static_cast<int>(smem)), "cudaFuncSetAttribute"))
      return rc;
  }
  int occ = 0;
  if (int rc = check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kBlock, smem), "occupancy"))
    return rc;
  const int64_t want = b->total_tiles;
  const int64_t cap = static_cast<int64_t>(b->ctx->num_sms) * (occ > 0 ? occ : 1);
  const int grid = static_cast<int>(want < cap ? want : cap);
  if (int rc = check_cuda(cudaMemsetAsync(b->d_work, 0, sizeof(unsigned long long), st), "cudaMemsetAsync(work)"))
    return rc;
  if (grid <= 0) return CC_OK;
  DevTable t = tab;  // the index checks of debug builds report into the context's flags
  t.dbg = &b->ctx->d_counters->error_flags;
  const HardWork hw{b->d_hard, b->hard_cap, b->d_hard_ctr, b->d_hard_full};
  const int nitems = static_cast<int>(b->items.size());
  if (kMixed)
    if (int rc = check_cuda(cudaMemsetAsync(b->d_hard_ctr, 0, kHardCounters * sizeof(unsigned long long), st),
                            "cudaMemsetAsync(hard records)"))
      return rc;
  kern<<<grid, kBlock, smem, st>>>(b->d_items, nitems, b->total_tiles, b->d_work, t, hw, b->ctx->d_counters);
  if (int rc = check_cuda(cudaGetLastError(), "batched_kernel launch")) return rc;
  if (kMixed) {
    const int g2 = 4 * b->ctx->num_sms;
    batch_hard_kernel<<<g2, kHardThreads, 0, st>>>(b->d_items, nitems, t, hw, b->ctx->d_counters);
    if (int rc = check_cuda(cudaGetLastError(), "batch_hard_kernel launch")) return rc;
    batch_full_kernel<<<g2, kHardThreads, 0, st>>>(b->d_items, nitems, t, hw, b->ctx->d_counters);
    return check_cuda(cudaGetLastError(), "batch_full_kernel launch");
  }
  return CC_OK;
}

int launch_batch(cc_batch* b, cudaStream_t st) {
  if (b->ctx->tab.bytes() > static_cast<size_t>(kSmemTableMaxBytes))
    return set_error(CC_ENOTSUP, "batched launch needs the spline table in shared memory (<= 64 KB)");
  const bool mixed = b->mode == CC_MODE_MIXED;
  if (b->block == 128) return mixed ? launch_batch_t<true, 128>(b, st) : launch_batch_t<false, 128>(b, st);
  return mixed ? launch_batch_t<true, 256>(b, st) : launch_batch_t<false, 256>(b, st);
}

void drop_graph(cc_batch* b) {
  if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->graph_exec = nullptr;
  b->graph = nullptr;
}

std::string gpu_name(int dev) {
  cudaDeviceProp prop{};
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown";
  std::string s = prop.name;
  for (char& c : s)
    if (c == ' ') c = '_';
  return s;
}

}  // namespace
}  // namespace cc

extern "C" {

int cc_batch_create(cc_ctx* ctx, cc_mode mode, const cc_batch_item* items, int32_t nitems, cc_batch** out) {
  if (!out) return set_error(CC_EINVAL, "out is NULL");
  *out = nullptr;
  if (!ctx || !items || nitems < 1) return set_error(CC_EINVAL, "ctx, items and nitems >= 1 are required");
  if (nitems >= (1 << 23)) return set_error(CC_EINVAL, "at most 2^23 - 1 items");
  if (mode != CC_MODE_FP64 && mode != CC_MODE_MIXED)
    return set_error(CC_ENOTSUP, "batched launch supports CC_MODE_FP64 and CC_MODE_MIXED");
  size_t total_r = 0;
  int64_t hard_want = 0, points = 0;
  for (int i = 0; i < nitems; ++i) {
    const cc_batch_item& it = items[i];
    char where[64];
    std::snprintf(where, sizeof(where), "item %d: ", i);
    if (it.dtype != CC_F64 && it.dtype != CC_F32) return set_error(CC_EINVAL, std::string(where) + "bad dtype");
    if (it.n < 1 || !it.hess || !it.F_max || !it.idx) return set_error(CC_EINVAL, std::string(where) + "n >= 1 and non-NULL pointers required");
    if (it.n >= (int64_t{1} << kItemShift)) return set_error(CC_EINVAL, std::string(where) + "n must be below 2^40");
    if (it.R < 1 || it.R > kMaxRadiiPerLaunch || !it.sigma) return set_error(CC_EINVAL, std::string(where) + "R must be in [1, 256] with sigma");
    if (it.plane_stride < it.n || (it.R > 1 && it.radius_stride < 6 * it.plane_stride))
      return set_error(CC_EINVAL, std::string(where) + "strides too small");
    if ((reinterpret_cast<uintptr_t>(it.hess) & 15u) || (it.plane_stride * it.dtype) % 16 ||
        (it.R > 1 && (it.radius_stride * it.dtype) % 16))
      return set_error(CC_EINVAL, std::string(where) + "planes must be 16-byte aligned");
    if (it.scale_idx0 < 0) return set_error(CC_EINVAL, std::string(where) + "scale_idx0 < 0");
    for (int r = 0; r < it.R; ++r)
      if (!(it.sigma[r] > 0.0) || !std::isfinite(it.sigma[r])) return set_error(CC_EINVAL, std::string(where) + "sigma must be > 0");
    total_r += static_cast<size_t>(it.R);
    // record capacity of the mixed mode: as for one launch (cc_api.cu)
    const double frac = 0.006 * it.R + 0.02;
    hard_want += frac >= 1.0 ? it.n : static_cast<int64_t>(static_cast<double>(it.n) * frac);
    points += it.n;
  }
  hard_want += 1024;
  if (hard_want > points) hard_want = points;
  if (hard_want > static_cast<int64_t>(UINT32_MAX)) hard_want = static_cast<int64_t>(UINT32_MAX);
  int cur = -1;
  if (int rc = check_cuda(cudaGetDevice(&cur), "cudaGetDevice")) return rc;
  if (cur != ctx->device)
    if (int rc = check_cuda(cudaSetDevice(ctx->device), "cudaSetDevice")) return rc;
  cc_batch* b = new (std::nothrow) cc_batch();
  if (!b) return set_error(CC_ENOMEM, "host allocation failed");
  b->ctx = ctx;
  b->mode = mode;
  b->items.assign(items, items + nitems);
  b->tile.assign(nitems, 1024);
  std::vector<float> thr_flat;
  thr_flat.reserve(total_r);
  for (int i = 0; i < nitems; ++i)
    for (int r = 0; r < items[i].R; ++r) thr_flat.push_back(static_cast<float>(1e-4 * items[i].sigma[r]));
  int rc = check_cuda(cudaMalloc(reinterpret_cast<void**>(&b->d_items), sizeof(BatchItemDev) * nitems), "cudaMalloc(items)");
  if (!rc) rc = check_cuda(cudaMalloc(reinterpret_cast<void**>(&b->d_thr), sizeof(float) * total_r), "cudaMalloc(thresholds)");
  if (!rc) rc = check_cuda(cudaMalloc(reinterpret_cast<void**>(&b->d_work), sizeof(unsigned long long)), "cudaMalloc(work)");
  if (!rc && mode == CC_MODE_MIXED) {
    b->hard_cap = hard_want;
    rc = check_cuda(cudaMalloc(reinterpret_cast<void**>(&b->d_hard), sizeof(HardRec) * static_cast<size_t>(hard_want)),
                    "cudaMalloc(hard records)");
    if (!rc) rc = check_cuda(cudaMalloc(reinterpret_cast<void**>(&b->d_hard_full), sizeof(uint32_t) * static_cast<size_t>(hard_want)),
                             "cudaMalloc(hard record list)");
    if (!rc) rc = check_cuda(cudaMalloc(reinterpret_cast<void**>(&b->d_hard_ctr), kHardCounters * sizeof(unsigned long long)),
                             "cudaMalloc(hard record counters)");
  }
  if (!rc) rc = check_cuda(cudaMemcpy(b->d_thr, thr_flat.data(), sizeof(float) * total_r, cudaMemcpyHostToDevice), "cudaMemcpy(thresholds)");
  if (!rc) rc = upload_items(b, nullptr);
  if (rc) { cc_batch_destroy(b); return rc; }
  *out = b;
  return CC_OK;
}

void cc_batch_destroy(cc_batch* b) {
  if (!b) return;
  cudaDeviceSynchronize();
  drop_graph(b);
  if (b->d_items) cudaFree(b->d_items);
  if (b->d_thr) cudaFree(b->d_thr);
  if (b->d_work) cudaFree(b->d_work);
  if (b->d_hard) cudaFree(b->d_hard);
  if (b->d_hard_full) cudaFree(b->d_hard_full);
  if (b->d_hard_ctr) cudaFree(b->d_hard_ctr);
  delete b;
}

int cc_batch_run(cc_batch* b, void* stream) {
  if (!b) return set_error(CC_EINVAL, "batch is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (b->dirty)
    if (int rc = upload_items(b, st)) return rc;
  return launch_batch(b, st);
}

int cc_batch_run_graph(cc_batch* b, void* stream) {
  if (!b) return set_error(CC_EINVAL, "batch is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (b->dirty) {
    drop_graph(b);
    if (int rc = upload_items(b, st)) return rc;
  }
  if (!b->graph_exec) {
    if (st == nullptr) return set_error(CC_EINVAL, "graph capture needs a non-default stream");
    cudaStreamCaptureStatus status;
    if (int rc = check_cuda(cudaStreamIsCapturing(st, &status), "cudaStreamIsCapturing")) return rc;
    if (status != cudaStreamCaptureStatusNone) return set_error(CC_EINVAL, "stream is already capturing");
    if (int rc = check_cuda(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture"))
      return rc;
    const int lrc = launch_batch(b, st);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(st, &g);
    if (lrc) { if (g) cudaGraphDestroy(g); return lrc; }
    if (int rc = check_cuda(e, "cudaStreamEndCapture")) return rc;
    b->graph = g;
    if (int rc = check_cuda(cudaGraphInstantiate(&b->graph_exec, g, 0), "cudaGraphInstantiate")) {
      drop_graph(b);
      return rc;
    }
  }
  return check_cuda(cudaGraphLaunch(b->graph_exec, st), "cudaGraphLaunch");
}

int cc_batch_get_config(const cc_batch* b, int32_t* threads_per_block, int32_t* tile_points, int32_t nitems) {
  if (!b) return set_error(CC_EINVAL, "batch is NULL");
  if (threads_per_block) *threads_per_block = b->block;
  if (tile_points) {
    if (nitems != static_cast<int32_t>(b->items.size())) return set_error(CC_EINVAL, "nitems must match the batch");
    for (int i = 0; i < nitems; ++i) tile_points[i] = b->tile[i];
  }
  return CC_OK;
}

int cc_batch_autotune(cc_batch* b, const char* cache_path, void* stream) {
  if (!b) return set_error(CC_EINVAL, "batch is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const std::string gpu = gpu_name(b->ctx->device);
  const char* mode_name = b->mode == CC_MODE_MIXED ? "mixed" : "fp64";
  // cached choices: "gpu mode class block tile" per line; class -1 holds the block size
  std::map<int, int> cached_tile;
  int cached_block = 0;
  if (cache_path) {
    if (FILE* f = std::fopen(cache_path, "r")) {
      char g[256], m[32];
      int cls, blk, tl;
      while (std::fscanf(f, "%255s %31s %d %d %d", g, m, &cls, &blk, &tl) == 5) {
        if (gpu != g || std::strcmp(m, mode_name) != 0) continue;
        if (cls < 0) cached_block = blk; else cached_tile[cls] = tl;
      }
      std::fclose(f);
    }
  }
  const std::vector<cc_batch_item> all = b->items;
  const std::vector<int> all_tile = b->tile;
  std::map<int, std::vector<int>> classes;  // class -> item indices
  for (size_t i = 0; i < all.size(); ++i) classes[size_class(all[i].n)].push_back(static_cast<int>(i));
  cudaEvent_t e0, e1;
  if (int rc = check_cuda(cudaEventCreate(&e0), "cudaEventCreate")) return rc;
  if (int rc = check_cuda(cudaEventCreate(&e1), "cudaEventCreate")) { cudaEventDestroy(e0); return rc; }
  // time the current configuration restricted to the given items
  auto time_items = [&](const std::vector<int>& sel, float* ms) -> int {
    b->items.clear();
    std::vector<int> tiles;
    for (int i : sel) { b->items.push_back(all[i]); tiles.push_back(b->tile[i]); }
    const std::vector<int> saved = b->tile;
    b->tile = tiles;
    // the thresholds of a sub-batch are those of its items: rebuild their offsets
    std::vector<float> thr;
    for (int i : sel)
      for (int r = 0; r < all[i].R; ++r) thr.push_back(static_cast<float>(1e-4 * all[i].sigma[r]));
    int rc = check_cuda(cudaMemcpy(b->d_thr, thr.data(), sizeof(float) * thr.size(), cudaMemcpyHostToDevice), "cudaMemcpy");
    if (!rc) rc = upload_items(b, st);
    if (!rc) rc = launch_batch(b, st);  // warm-up
    if (!rc) rc = check_cuda(cudaEventRecord(e0, st), "cudaEventRecord");
    for (int rep = 0; rep < 2 && !rc; ++rep) rc = launch_batch(b, st);
    if (!rc) rc = check_cuda(cudaEventRecord(e1, st), "cudaEventRecord");
    if (!rc) rc = check_cuda(cudaEventSynchronize(e1), "cudaEventSynchronize");
    if (!rc) rc = check_cuda(cudaEventElapsedTime(ms, e0, e1), "cudaEventElapsedTime");
    b->tile = saved;
    return rc;
  };
  int rc = CC_OK;
  // block size for the whole batch: timed on one item of the largest class
  if (cached_block) {
    b->block = cached_block;
  } else {
    const std::vector<int> probe = {classes.rbegin()->second.front()};
    float best = 1e30f;
    int best_block = b->block;
    for (int blk : kBlockCandidates) {
      b->block = blk;
      float ms = 0.f;
      if ((rc = time_items(probe, &ms))) break;
      if (ms < best) { best = ms; best_block = blk; }
    }
    b->block = best_block;
  }
  std::map<int, int> chosen;
  for (auto& kv : classes) {
    if (rc) break;
    auto hit = cached_tile.find(kv.first);
    if (hit != cached_tile.end()) { chosen[kv.first] = hit->second; continue; }
    float best = 1e30f;
    int best_tile = 1024;
    for (int tl : kTileCandidates) {
      if (tl < b->block) continue;
      for (int i : kv.second) b->tile[i] = tl;
      float ms = 0.f;
      if ((rc = time_items(kv.second, &ms))) break;
      if (ms < best) { best = ms; best_tile = tl; }
    }
    chosen[kv.first] = best_tile;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // restore the full batch with the chosen shapes
  b->items = all;
  b->tile = all_tile;
  for (size_t i = 0; i < all.size(); ++i) {
    auto c = chosen.find(size_class(all[i].n));
    if (c != chosen.end()) b->tile[i] = c->second;
  }
  std::vector<float> thr;
  for (const auto& it : all)
    for (int r = 0; r < it.R; ++r) thr.push_back(static_cast<float>(1e-4 * it.sigma[r]));
  int rc2 = check_cuda(cudaMemcpy(b->d_thr, thr.data(), sizeof(float) * thr.size(), cudaMemcpyHostToDevice), "cudaMemcpy");
  if (!rc2) rc2 = upload_items(b, st);
  drop_graph(b);
  if (rc) return rc;
  if (rc2) return rc2;
  if (cache_path) {
    if (FILE* f = std::fopen(cache_path, "a")) {
      if (!cached_block) std::fprintf(f, "%s %s -1 %d 0\n", gpu.c_str(), mode_name, b->block);
      for (auto& kv : chosen)
        if (!cached_tile.count(kv.first)) std::fprintf(f, "%s %s %d %d %d\n", gpu.c_str(), mode_name, kv.first, b->block, kv.second);
      std::fclose(f);
    }
  }
  return CC_OK;
}

}  // extern "C"
