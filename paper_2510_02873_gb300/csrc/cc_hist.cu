// cc_hist.cu -- counts of F_max per bin (arXiv:2510.02873, Sec. 5.5: the
// number of collapsed particles per redshift bin, with F = 1 + z_c).
//
// HBM-bound reduction: 8 bytes read per point. F >= 0 and the edges are
// positive, so bins are found on the FP64 bit patterns as integers (integer
// order is value order for non-negative doubles): no FP64 instruction. A
// point's bucket, (bits(F) - kb) >> shift with kb the first edge's pattern
// rounded down to a multiple of 2^shift, gives the number of edges at or
// below the bucket's lower end, and the edges inside the bucket finish the
// count. The host picks the largest shift that leaves at most two edges in a
// bucket; when that shift is 32 or more the kernel takes the bucket from the
// top 32 bits of F and finishes with two predicated steps, otherwise (edges
// a few patterns apart, or clustered within 1/2048 of their range) it takes
// the whole pattern and scans.
// Each block counts with shared-memory atomics and adds its counts to the
// global ones once. (Per-thread private rows and warp-aggregated atomics were
// both measured slower at 16.8M points.)
#include <algorithm>
#include <cstring>

#include "cc_internal.h"

namespace cc {
namespace {

constexpr int kHistMaxEdges = 1024;
constexpr int kHistMaxBuckets = 2048;
constexpr int kHistUnroll = 4;

// Bucket j >= 0 covers the bit patterns [kb + j 2^shift, kb + (j + 1) 2^shift)
// with kb = bits(edge_0) rounded down to a multiple of 2^shift; first[j + 1]
// is the number of edges at or below its lower end and first[0] = 0 serves
// patterns below kb. Two sentinels (the largest pattern) follow the edges.
struct HistEdges {
  long long key[kHistMaxEdges + 2];
  unsigned short first[kHistMaxBuckets + 1];
  long long kb;
  int n_edges;
  int n_buckets;
  int shift;
  int fast;  // shift >= 32 and at most two edges per bucket
};

// kFast: the bucket from the top 32 bits of F, then two predicated steps
// (no bucket holds more than two edges beyond its lower end). Otherwise the
// bucket from the whole pattern and a scan, for edges clustered more tightly
// than the table resolves.
template <bool kFast>
__global__ void __launch_bounds__(256) histogram_kernel(const double* __restrict__ F, int64_t n, const HistEdges e,
                                                        unsigned long long* __restrict__ counts) {
  __shared__ long long skey[kHistMaxEdges + 2];
  __shared__ unsigned short sfirst[kHistMaxBuckets + 1];
  __shared__ unsigned int sc[kHistMaxEdges + 1];
  const int nc = e.n_edges + 1;
  for (int i = threadIdx.x; i < e.n_edges + 2; i += blockDim.x) skey[i] = e.key[i];
  for (int i = threadIdx.x; i <= e.n_buckets; i += blockDim.x) sfirst[i] = e.first[i];
  for (int i = threadIdx.x; i < nc; i += blockDim.x) sc[i] = 0u;
  __syncthreads();
  const long long kb = e.kb;
  const int last = e.n_buckets - 1;
  const int hib = static_cast<int>(kb >> 32), s2 = e.shift - 32;
  // b = number of edges <= F (0 .. n_edges): count slot b. Patterns with the
  // sign bit (-0.0, or negative F against the contract) land below edge 0;
  // NaN patterns above the last edge.
  auto count = [&](long long k) {
    int b;
    if constexpr (kFast) {
      const int hi = static_cast<int>(k >> 32);
      int j = min((hi - hib) >> s2, last);  // hi >= 0: no overflow; below kb: negative
      j = hi < 0 ? -1 : max(j, -1);
      b = sfirst[j + 1];
      b += skey[b] <= k;
      b += skey[b] <= k;
      b = min(b, e.n_edges);
    } else {
      b = 0;
      if (k >= kb) {
        const unsigned long long j = static_cast<unsigned long long>(k - kb) >> e.shift;
        b = sfirst[1 + (j < static_cast<unsigned long long>(last) ? static_cast<int>(j) : last)];
        while (b < e.n_edges && skey[b] <= k) ++b;
      }
    }
    atomicAdd(&sc[b], 1u);
  };
  // kHistUnroll independent loads in flight per thread: one 8-byte load per
  // thread at a time leaves too few bytes in flight to cover HBM latency
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  for (; p + (kHistUnroll - 1) * stride < n; p += kHistUnroll * stride) {
    long long k[kHistUnroll];
#pragma unroll
    for (int u = 0; u < kHistUnroll; ++u) k[u] = __double_as_longlong(__ldg(F + p + u * stride));
#pragma unroll
    for (int u = 0; u < kHistUnroll; ++u) count(k[u]);
  }
  for (; p < n; p += stride) count(__double_as_longlong(__ldg(F + p)));
  __syncthreads();
  for (int i = threadIdx.x; i < nc; i += blockDim.x)
    if (sc[i]) atomicAdd(&counts[i], static_cast<unsigned long long>(sc[i]));
}

}  // namespace
}  // namespace cc

using namespace cc;

extern "C" {

int cc_histogram(cc_ctx* ctx, const double* F_max, int64_t n, const double* edges, int32_t nbins,
                 unsigned long long* counts, void* stream) {
  if (!ctx) return set_error(CC_EINVAL, "ctx is NULL");
  if (!edges || nbins < 1 || nbins + 1 > kHistMaxEdges)
    return set_error(CC_EINVAL, "need 1 <= nbins <= 1023 and nbins + 1 host edges");
  if (!counts) return set_error(CC_EINVAL, "counts is NULL");
  if (n < 0 || (n > 0 && !F_max)) return set_error(CC_EINVAL, "bad F_max array");
  if (reinterpret_cast<uintptr_t>(F_max) % 8 || reinterpret_cast<uintptr_t>(counts) % 8)
    return set_error(CC_EINVAL, "F_max and counts must be 8-byte aligned");
  HistEdges e;
  e.n_edges = nbins + 1;
  for (int i = 0; i < e.n_edges; ++i) {
    if (!(edges[i] > 0.0) || !(edges[i] < __builtin_huge_val()))
      return set_error(CC_EINVAL, "edges must be positive and finite");
    if (i > 0 && !(edges[i] > edges[i - 1])) return set_error(CC_EINVAL, "edges must be strictly increasing");
    long long k;
    std::memcpy(&k, &edges[i], sizeof(k));
    e.key[i] = k;
  }
  e.key[e.n_edges] = e.key[e.n_edges + 1] = 0x7fffffffffffffffll;  // sentinels
  // buckets of 2^shift bit patterns: the largest shift that leaves at most
  // two edges in any bucket (each block copies the table out of the
  // parameter space, so fewer buckets cost less), else the smallest shift
  // whose buckets fit the table
  const long long k0 = e.key[0], kN = e.key[e.n_edges - 1];
  auto n_buckets = [&](int sh) { return (kN >> sh) - (k0 >> sh) + 1; };
  int min_shift = 0;
  while (n_buckets(min_shift) > kHistMaxBuckets) ++min_shift;
  e.shift = min_shift;
  e.fast = 0;
  for (int sh = 62; sh >= min_shift; --sh) {
    int run = 1, worst = 1;
    for (int i = 1; i < e.n_edges; ++i) {
      run = (e.key[i] >> sh) == (e.key[i - 1] >> sh) ? run + 1 : 1;
      worst = std::max(worst, run);
    }
    if (worst <= 2) {
      e.shift = sh;
      e.fast = sh >= 32;
      break;
    }
  }
  e.n_buckets = static_cast<int>(n_buckets(e.shift));
  e.kb = (k0 >> e.shift) << e.shift;
  e.first[0] = 0;
  for (int j = 0, b = 0; j < e.n_buckets; ++j) {
    const long long lo = e.kb + (static_cast<long long>(j) << e.shift);
    while (b < e.n_edges && e.key[b] <= lo) ++b;
    e.first[j + 1] = static_cast<unsigned short>(b);
  }
  if (int rc = select_device(ctx)) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (int rc = check_cuda(cudaMemsetAsync(counts, 0, sizeof(unsigned long long) * (nbins + 2), st),
                          "cudaMemsetAsync(counts)"))
    return rc;
  if (n == 0) return CC_OK;
  const int64_t need = (n + 255) / 256;
  const int grid = static_cast<int>(std::min<int64_t>(need, static_cast<int64_t>(ctx->num_sms) * 8));
  if (e.fast)
    histogram_kernel<true><<<grid, 256, 0, st>>>(F_max, n, e, counts);
  else
    histogram_kernel<false><<<grid, 256, 0, st>>>(F_max, n, e, counts);
  return check_cuda(cudaGetLastError(), "histogram_kernel launch");
}

}  // extern "C"
