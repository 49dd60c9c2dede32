// cc_surrogate.cu -- the learned surrogate (no counterpart in the paper).
//
// An MLP (3 -> 64 -> 64 -> 64 -> 1, SiLU) maps normalised eigenvalues
// z = (l1, l2, l3) / sigma to f ~ log(D_c sigma), the log of the growth factor
// at collapse in units of 1/sigma (D_c is homogeneous of degree -1 in the
// eigenvalues, so one network serves every radius). It is trained here, on the
// GPU, by this file's forward/backward kernels on BF16 tensor cores with FP32
// accumulation and an FP32 Adam; the training targets come from the exact FP64
// path of this library. In CC_MODE_SURROGATE the network's output only seeds
// the Newton iteration of the collapse condition: a residual certificate
// decides whether the refined root is used, and otherwise (or outside the
// training hull) the exact FP64 path is, so results stay within the mixed
// path's accuracy.
#include <cmath>
#include <cstring>
#include <vector>

#include "cc_device.cuh"
#include "cc_mlp.cuh"
#include "cc_umma.cuh"

namespace cc {
namespace {

using namespace mlp;

constexpr int kTrainWarps = 2;
constexpr int kRowsPad = 40;  // transposed tiles: 32 rows + 8 padding (bank-conflict free)

struct WarpScratch {
  float dsl[3][32][H];                 // silu'(u_l) of layers 1..3, [row][unit]
  __nv_bfloat16 zT[16][kRowsPad];      // inputs, [feature][row] (features 3..15 zero)
  __nv_bfloat16 aT[3][H][kRowsPad];    // activations a1..a3, [unit][row]
  __nv_bfloat16 dT[3][H][kRowsPad];    // deltas d1..d3, [unit][row]
  float df[32];                        // dLoss/df per row
};
constexpr int kGradBytes = ((NPARAM * 4 + 15) / 16) * 16;
constexpr size_t kTrainSmem = ALL_BYTES + kGradBytes + sizeof(WarpScratch) * kTrainWarps;

// ---- image of the network for the tensor-memory kernel (collapse_sur_tc_kernel):
// the four weight matrices as MMA B operands (N rows = output units, K
// columns), K-major core-matrix layout (cc_umma.cuh). Layers 1-3 are halved
// (their accumulators are then h = v / 2, see silu2_half); each layer's bias
// rides on two extra K columns, hi = RN_bf16(b) and lo = RN_bf16(b - hi),
// which meet two columns of ones in the activation tile.
namespace tc {
constexpr int kRows = 128;                          // tile rows = threads = tensor-memory lanes
constexpr int kKA = 80;                             // activation tile: 64 units | 1 | 1 | 14 zeros
constexpr int kSboA = 16 * kKA;                     // row-group stride of K = 80 operands
constexpr int kSbo1 = 16 * 16;                      // of the K = 16 first layer
constexpr int kW1 = 0;                              // 64 x 16: W1^T / 2, b1 / 2 at k = 3, 4
constexpr int kW2 = kW1 + 64 * 16 * 2;              // 64 x 80: W2^T / 2, b2 / 2 at k = 64, 65
constexpr int kW3 = kW2 + 64 * kKA * 2;             // 64 x 80
constexpr int kW4 = kW3 + 64 * kKA * 2;             // 8 x 80: row 0 = W4, b4 at k = 64, 65; the
                                                    // N = 16 MMA reads it with row-group stride 0,
                                                    // so rows 8-15 repeat rows 0-7
constexpr int kImgBytes = kW4 + 8 * kKA * 2;
constexpr int kA = kImgBytes;                       // the groups' activation tiles follow in shared memory
constexpr int kATileBytes = kRows * kKA * 2;
constexpr int kGroups = 8;                          // groups of 128 threads per CTA, sharing the weights
constexpr int kTab = kA + kGroups * kATileBytes;    // then the spline table (coef | D | Df | bucket)
constexpr int kSmemBytes = kTab;                    // + the table's bytes, rounded to 16
constexpr int kTmemCols = 64;
constexpr int kWaitTries = 1 << 22;                 // polls of an mbarrier before giving up
constexpr int kCtasPerSm = 1;                       // ~208 KB shared memory, 512 TMEM columns, 64 registers
constexpr int OFF_TC = IMG_BYTES;                   // in the global image
constexpr int IMG_TOTAL = OFF_TC + kImgBytes;
static_assert(OFF_TC % 16 == 0 && kImgBytes % 16 == 0, "bulk copy alignment");
}  // namespace tc

__device__ __forceinline__ uint64_t mix64(uint64_t x) {  // splitmix64 finaliser
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

__device__ __forceinline__ int ordered(float f) {  // monotone int image of a float
  const int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7FFFFFFF;
}
__host__ __device__ __forceinline__ float unordered(int i) {
  const int j = i >= 0 ? i : i ^ 0x7FFFFFFF;
  float f;
  memcpy(&f, &j, sizeof(f));
  return f;
}

// ---- training data: z = l / sigma, t = log(D_c sigma) from the exact FP64 path
template <typename T>
__global__ void sur_data_kernel(const T* __restrict__ hess, int64_t n, int64_t ps, double sigma,
                                float4* __restrict__ out, unsigned long long* __restrict__ count, int64_t cap,
                                int* __restrict__ hull) {
  const double inv = 1.0 / sigma;
  for (int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; p < n;
       p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const T* h = hess + p;
    const double xx = h[0], yy = h[ps], zz = h[2 * ps], xy = h[3 * ps], xz = h[4 * ps], yz = h[5 * ps];
    const EigenTop e = eigen_top_fp64(xx, yy, zz, xy, xz, yz);
    const double lam1 = e.q + e.x;
    if (!(lam1 > 0.0)) continue;
    const double Pp = fma(e.q, e.q - e.x, fma(e.x, e.x, -e.p2x3));
    const double S = fma(2.0, e.q, -e.x);
    const double D = rlpt_root_fp64(lam1, Pp, S).D;
    const double Ds = D * sigma;
    if (!(Ds > 0.0) || !(Ds < 1e4)) continue;
    const double y = sqrt(fmax(fma(S, S, -4.0 * Pp), 0.0));
    const float4 v = make_float4(static_cast<float>(lam1 * inv), static_cast<float>(0.5 * (S + y) * inv),
                                 static_cast<float>(0.5 * (S - y) * inv), static_cast<float>(log(Ds)));
    const unsigned long long slot = atomicAdd(count, 1ULL);
    if (static_cast<int64_t>(slot) < cap) {
      out[slot] = v;
      atomicMin(hull + 0, ordered(v.x)); atomicMax(hull + 3, ordered(v.x));
      atomicMin(hull + 1, ordered(v.y)); atomicMax(hull + 4, ordered(v.y));
      atomicMin(hull + 2, ordered(v.z)); atomicMax(hull + 5, ordered(v.z));
    }
  }
}

__device__ __forceinline__ void stage(unsigned char* dst, const unsigned char* src, int bytes) {
  for (int i = threadIdx.x; i < bytes / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(dst)[i] = reinterpret_cast<const uint4*>(src)[i];
}

__device__ __forceinline__ float bf(const __nv_bfloat16& v) { return __bfloat162float(v); }

// store one layer's pre-activations (C layout of one tile) as silu' and activations
__device__ __forceinline__ void store_layer(WarpScratch& w, int l, int tile, const float (&c)[8][4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int r0 = 16 * tile + g, r1 = r0 + 8;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int n0 = 8 * j + 2 * t;
    w.dsl[l][r0][n0] = dsilu(c[j][0]);
    w.dsl[l][r0][n0 + 1] = dsilu(c[j][1]);
    w.dsl[l][r1][n0] = dsilu(c[j][2]);
    w.dsl[l][r1][n0 + 1] = dsilu(c[j][3]);
    w.aT[l][n0][r0] = __float2bfloat16_rn(silu(c[j][0]));
    w.aT[l][n0 + 1][r0] = __float2bfloat16_rn(silu(c[j][1]));
    w.aT[l][n0][r1] = __float2bfloat16_rn(silu(c[j][2]));
    w.aT[l][n0 + 1][r1] = __float2bfloat16_rn(silu(c[j][3]));
  }
}

// delta of layer l from its upstream gradient (C layout) times silu'; stored
// transposed and returned packed as the A fragments of the next product
__device__ __forceinline__ void delta_layer(WarpScratch& w, int l, int tile, float (&c)[8][4], uint32_t (&a)[4][4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int r0 = 16 * tile + g, r1 = r0 + 8;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int n0 = 8 * j + 2 * t;
    c[j][0] *= w.dsl[l][r0][n0];
    c[j][1] *= w.dsl[l][r0][n0 + 1];
    c[j][2] *= w.dsl[l][r1][n0];
    c[j][3] *= w.dsl[l][r1][n0 + 1];
    w.dT[l][n0][r0] = __float2bfloat16_rn(c[j][0]);
    w.dT[l][n0 + 1][r0] = __float2bfloat16_rn(c[j][1]);
    w.dT[l][n0][r1] = __float2bfloat16_rn(c[j][2]);
    w.dT[l][n0 + 1][r1] = __float2bfloat16_rn(c[j][3]);
  }
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    a[s][0] = pack(c[2 * s][0], c[2 * s][1]);
    a[s][1] = pack(c[2 * s][2], c[2 * s][3]);
    a[s][2] = pack(c[2 * s + 1][0], c[2 * s + 1][1]);
    a[s][3] = pack(c[2 * s + 1][2], c[2 * s + 1][3]);
  }
}

// upstream gradient of the previous layer: c = d W^T (W stored [in][out] in the image)
__device__ __forceinline__ void back_mma(const uint32_t (&a)[4][4], const unsigned char* img, int off_wb,
                                         float (&c)[8][4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    c[j][0] = c[j][1] = c[j][2] = c[j][3] = 0.0f;
    const int row = off_wb + (8 * j + g) * STR * 2;
#pragma unroll
    for (int s = 0; s < 4; ++s)
      mma(c[j], a[s], ld32(img, row + (16 * s + 2 * t) * 2), ld32(img, row + (16 * s + 8 + 2 * t) * 2));
  }
}

// weight gradient dW[in][out] += sum_rows act[row][in] delta[row][out] over the
// warp's 32 rows (K), from the transposed tiles; m_tiles tiles of 16 inputs
__device__ __forceinline__ void wgrad(const __nv_bfloat16 (*actT)[kRowsPad], const __nv_bfloat16 (*dT)[kRowsPad],
                                      int m_tiles, int n_in, float* gW) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  for (int i = 0; i < m_tiles; ++i) {
    float c[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) c[j][0] = c[j][1] = c[j][2] = c[j][3] = 0.0f;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      uint32_t a[4];
      a[0] = *reinterpret_cast<const uint32_t*>(&actT[16 * i + g][16 * s + 2 * t]);
      a[1] = *reinterpret_cast<const uint32_t*>(&actT[16 * i + g + 8][16 * s + 2 * t]);
      a[2] = *reinterpret_cast<const uint32_t*>(&actT[16 * i + g][16 * s + 8 + 2 * t]);
      a[3] = *reinterpret_cast<const uint32_t*>(&actT[16 * i + g + 8][16 * s + 8 + 2 * t]);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const uint32_t b0 = *reinterpret_cast<const uint32_t*>(&dT[8 * j + g][16 * s + 2 * t]);
        const uint32_t b1 = *reinterpret_cast<const uint32_t*>(&dT[8 * j + g][16 * s + 8 + 2 * t]);
        uint32_t aa[4] = {a[0], a[1], a[2], a[3]};
        mma(c[j], aa, b0, b1);
      }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int in0 = 16 * i + g, in1 = in0 + 8, o = 8 * j + 2 * t;
      if (in0 < n_in) { atomicAdd(gW + in0 * H + o, c[j][0]); atomicAdd(gW + in0 * H + o + 1, c[j][1]); }
      if (in1 < n_in) { atomicAdd(gW + in1 * H + o, c[j][2]); atomicAdd(gW + in1 * H + o + 1, c[j][3]); }
    }
  }
}

// One minibatch step: each warp takes 32 samples (indices hashed from seed and
// step, or consecutive when `sequential`), runs forward and backward and adds
// its gradient (already divided by the batch size) to grad_g; loss_g += mean r^2.
__global__ void __launch_bounds__(32 * kTrainWarps)
sur_train_kernel(const float4* __restrict__ data, int64_t ntrain, uint64_t seed, int step, int sequential,
                 float inv_batch, const unsigned char* __restrict__ img_g, float* __restrict__ grad_g,
                 float* __restrict__ loss_g) {
  extern __shared__ __align__(16) unsigned char sm[];
  unsigned char* img = sm;
  float* grad = reinterpret_cast<float*>(sm + ALL_BYTES);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  WarpScratch& w = reinterpret_cast<WarpScratch*>(sm + ALL_BYTES + kGradBytes)[warp];
  stage(img, img_g, ALL_BYTES);
  for (int i = threadIdx.x; i < kGradBytes / 4; i += blockDim.x) grad[i] = 0.0f;
  __syncthreads();
  const int64_t gi = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t sid = sequential ? gi : static_cast<int64_t>(mix64(seed ^ mix64(static_cast<uint64_t>(step) * 0x100000001ull + gi)) %
                                                              static_cast<uint64_t>(ntrain));
  const bool valid = sid < ntrain;
  const float4 d = valid ? data[sid] : make_float4(0.f, 0.f, 0.f, 0.f);
  const float* bias = reinterpret_cast<const float*>(img + OFF_B);
  float fo = 0.0f;
  // ---- forward, keeping silu' and the activations
#pragma unroll 1
  for (int tile = 0; tile < 2; ++tile) {
    float c[8][4];
    uint32_t a[4][4];
    layer1(d.x, d.y, d.z, tile, img, c);
    store_layer(w, 0, tile, c);
    act_pack(c, a);
    layer64(a, img, OFF_W2T, bias + 64, c);
    store_layer(w, 1, tile, c);
    act_pack(c, a);
    layer64(a, img, OFF_W3T, bias + 128, c);
    store_layer(w, 2, tile, c);
    act_pack(c, a);
    float o0, o1;
    layer4(a, img, o0, o1);
    const int src = (lane & 7) * 4;
    const float v0 = __shfl_sync(0xffffffffu, o0, src), v1 = __shfl_sync(0xffffffffu, o1, src);
    if ((lane >> 4) == tile) fo = ((lane & 15) < 8) ? v0 : v1;
  }
  w.zT[0][lane] = __float2bfloat16_rn(d.x);
  w.zT[1][lane] = __float2bfloat16_rn(d.y);
  w.zT[2][lane] = __float2bfloat16_rn(d.z);
  for (int k = 3; k < 16; ++k) w.zT[k][lane] = __float2bfloat16_rn(0.0f);
  const float r = valid ? fo - d.w : 0.0f;
  const float df = 2.0f * r * inv_batch;
  w.df[lane] = df;
  float l2 = r * r;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) l2 += __shfl_xor_sync(0xffffffffu, l2, o);
  if (lane == 0) atomicAdd(loss_g, l2 * inv_batch);
  __syncwarp();
  // ---- backward through the layers, per tile
#pragma unroll 1
  for (int tile = 0; tile < 2; ++tile) {
    const int r0 = 16 * tile + g, r1 = r0 + 8;
    const float d0 = w.df[r0], d1 = w.df[r1];
    float c[8][4];
    uint32_t a[4][4];
    const __nv_bfloat16* w4 = reinterpret_cast<const __nv_bfloat16*>(img + OFF_W4T);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int n0 = 8 * j + 2 * t;
      c[j][0] = d0 * bf(w4[n0]);
      c[j][1] = d0 * bf(w4[n0 + 1]);
      c[j][2] = d1 * bf(w4[n0]);
      c[j][3] = d1 * bf(w4[n0 + 1]);
    }
    delta_layer(w, 2, tile, c, a);     // d3
    back_mma(a, img, OFF_W3B, c);      // d3 W3^T
    delta_layer(w, 1, tile, c, a);     // d2
    back_mma(a, img, OFF_W2B, c);      // d2 W2^T
    delta_layer(w, 0, tile, c, a);     // d1
  }
  __syncwarp();
  // ---- weight gradients on tensor cores, biases and the last layer on CUDA cores
  wgrad(w.aT[1], w.dT[2], 4, H, grad + P_W3);
  wgrad(w.aT[0], w.dT[1], 4, H, grad + P_W2);
  wgrad(w.zT, w.dT[0], 1, 3, grad + P_W1);
  for (int k = lane; k < H; k += 32) {
    float s4 = 0.f, sb1 = 0.f, sb2 = 0.f, sb3 = 0.f;
    for (int row = 0; row < 32; ++row) {
      s4 += bf(w.aT[2][k][row]) * w.df[row];
      sb1 += bf(w.dT[0][k][row]);
      sb2 += bf(w.dT[1][k][row]);
      sb3 += bf(w.dT[2][k][row]);
    }
    atomicAdd(grad + P_W4 + k, s4);
    atomicAdd(grad + P_B1 + k, sb1);
    atomicAdd(grad + P_B2 + k, sb2);
    atomicAdd(grad + P_B3 + k, sb3);
  }
  if (lane == 0) {
    float sb4 = 0.f;
    for (int row = 0; row < 32; ++row) sb4 += w.df[row];
    atomicAdd(grad + P_B4, sb4);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NPARAM; i += blockDim.x)
    if (grad[i] != 0.0f) atomicAdd(grad_g + i, grad[i]);
}

// parameter i -> its places in the BF16 image
// the tensor-memory kernel's image (tc namespace): weight (n, k) of the
// operand at byte base, and a bias as its hi and lo halves at k and k + 1
__device__ __forceinline__ void put_tc(unsigned char* tci, int base, int sbo, int n, int k, float v) {
  *reinterpret_cast<__nv_bfloat16*>(tci + base + umma::offset(n, k, sbo)) = __float2bfloat16_rn(v);
}
__device__ __forceinline__ void put_tc_bias(unsigned char* tci, int base, int sbo, int n, int k, float v) {
  const __nv_bfloat16 hi = __float2bfloat16_rn(v);
  *reinterpret_cast<__nv_bfloat16*>(tci + base + umma::offset(n, k, sbo)) = hi;
  *reinterpret_cast<__nv_bfloat16*>(tci + base + umma::offset(n, k + 1, sbo)) =
      __float2bfloat16_rn(v - __bfloat162float(hi));
}

__device__ __forceinline__ void put_image(int i, float v, unsigned char* img) {
  unsigned char* tci = img + tc::OFF_TC;
  if (i < P_B1) {
    put_tc(tci, tc::kW1, tc::kSbo1, i % H, i / H, 0.5f * v);
  } else if (i < P_W2) {
    put_tc_bias(tci, tc::kW1, tc::kSbo1, i - P_B1, 3, 0.5f * v);
  } else if (i < P_B2) {
    put_tc(tci, tc::kW2, tc::kSboA, (i - P_W2) % H, (i - P_W2) / H, 0.5f * v);
  } else if (i < P_W3) {
    put_tc_bias(tci, tc::kW2, tc::kSboA, i - P_B2, 64, 0.5f * v);
  } else if (i < P_B3) {
    put_tc(tci, tc::kW3, tc::kSboA, (i - P_W3) % H, (i - P_W3) / H, 0.5f * v);
  } else if (i < P_W4) {
    put_tc_bias(tci, tc::kW3, tc::kSboA, i - P_B3, 64, 0.5f * v);
  } else if (i < P_B4) {
    put_tc(tci, tc::kW4, tc::kSboA, 0, i - P_W4, v);
  } else {
    put_tc_bias(tci, tc::kW4, tc::kSboA, 0, 64, v);
  }
  // training image (unscaled) and inference image (layers 1-3 halved)
  const bool half = i < P_W4;
  const __nv_bfloat16 b = __float2bfloat16_rn(v);
  const __nv_bfloat16 bi = __float2bfloat16_rn(half ? 0.5f * v : v);
  const float vi = half ? 0.5f * v : v;
  auto at = [&](int off) {
    *reinterpret_cast<__nv_bfloat16*>(img + off) = b;
  };
  auto at_fwd = [&](int off) {
    *reinterpret_cast<__nv_bfloat16*>(img + off) = b;
    *reinterpret_cast<__nv_bfloat16*>(img + OFF_INF + off) = bi;
  };
  auto bias = [&](int k) {
    reinterpret_cast<float*>(img + OFF_B)[k] = v;
    reinterpret_cast<float*>(img + OFF_INF + OFF_B)[k] = vi;
  };
  if (i < P_B1) {
    const int k = i / H, n = i % H;
    at_fwd(OFF_W1T + (n * STR1 + k) * 2);
  } else if (i < P_W2) {
    bias(i - P_B1);
  } else if (i < P_B2) {
    const int k = (i - P_W2) / H, n = (i - P_W2) % H;
    at_fwd(OFF_W2T + (n * STR + k) * 2);
    at(OFF_W2B + (k * STR + n) * 2);
  } else if (i < P_W3) {
    bias(64 + i - P_B2);
  } else if (i < P_B3) {
    const int k = (i - P_W3) / H, n = (i - P_W3) % H;
    at_fwd(OFF_W3T + (n * STR + k) * 2);
    at(OFF_W3B + (k * STR + n) * 2);
  } else if (i < P_W4) {
    bias(128 + i - P_B3);
  } else if (i < P_B4) {
    at_fwd(OFF_W4T + (i - P_W4) * 2);
  } else {
    bias(192);
  }
}

__global__ void sur_image_kernel(const float* __restrict__ p, unsigned char* __restrict__ img) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < NPARAM) put_image(i, p[i], img);
}

// Adam (FP32 master weights), then the BF16 image; the gradient is cleared
__global__ void sur_adam_kernel(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                                float* __restrict__ grad, float lr, float b1t, float b2t,
                                unsigned char* __restrict__ img) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NPARAM) return;
  const float gi = grad[i];
  grad[i] = 0.0f;
  const float mi = 0.9f * m[i] + 0.1f * gi;
  const float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float pi = p[i] - lr * (mi / (1.0f - b1t)) / (sqrtf(vi / (1.0f - b2t)) + 1e-8f);
  p[i] = pi;
  put_image(i, pi, img);
}

// f for n inputs z (stride 3 or the float4 training records): out and/or error statistics
__global__ void sur_eval_kernel(const float* __restrict__ z, int zstride, int64_t n, const unsigned char* __restrict__ img_g,
                                float* __restrict__ out, float* __restrict__ sumsq, int* __restrict__ maxerr) {
  extern __shared__ __align__(16) unsigned char sm[];
  stage(sm, img_g + OFF_INF, FWD_BYTES);
  __syncthreads();
  const int64_t n_round = (n + 31) & ~static_cast<int64_t>(31);
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n_round;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const bool ok = i < n;
    const float* zi = z + (ok ? i : 0) * zstride;
    const float f = forward_warp(zi[0], zi[1], zi[2], sm);
    if (!ok) continue;
    if (out) out[i] = f;
    if (sumsq) {
      const float e = f - zi[3];
      atomicAdd(sumsq, e * e);
      atomicMax(maxerr, __float_as_int(fabsf(e)));
    }
  }
}

// ---- inference: CC_MODE_SURROGATE collapse kernels.
constexpr float kCertTol = 1e-6f;  // accepted when the last Newton step is below 1e-6 D

// From the FP32 eigen stage and the network's output f = log(D sigma): three
// FP32 Newton steps from D = exp(f) / sigma, accepted when the residual
// certificate holds (and the input lies in the training hull), then the FP64
// polish and spline of the mixed path; the exact FP64 path otherwise.
__device__ __forceinline__ MixedResult sur_finish(const MixedEigen& m, float f, float is, bool inside, float xx,
                                                  float yy, float zz, float xy, float xz, float yz,
                                                  const double* __restrict__ Dk, const Coef4* __restrict__ coef,
                                                  const float* __restrict__ Dkf,
                                                  const unsigned short* __restrict__ bucket, const DevTable& tab,
                                                  unsigned& n_fb) {
  MixedResult res;
  if (m.full) {
    res = full_fp64(xx, yy, zz, xy, xz, yz, Dk, coef, Dkf, bucket, tab);
  } else if (!(m.lam1f > 0.0f)) {
    res.F = 0.0;
    res.a = kInf;
    res.collapsed = res.eds = res.refined = false;
    res.fp64 = m.fp64;
  } else {
    const MixedCoef k = mixed_coef(m);
    bool ok = inside;
    float Df = 0.0f;
    if (ok) {
      Df = newton_f32<3>(k, __expf(f) * is);
      const float Af = fmaf(fmaf(fmaf(k.c3f, Df, k.c2f), Df, -k.l1f), Df, 1.0f);
      const float dAf = fmaf(fmaf(3.0f * k.c3f, Df, 2.0f * k.c2f), Df, -k.l1f);
      ok = Df > 0.0f && isfinite(Df) && fabsf(Af) <= kCertTol * fabsf(dAf * Df);
    }
    if (ok) {
      res = mixed_finish(m, k, Df, coef, Dkf, bucket, tab, tab.dfseg);
    } else {
      res = full_fp64(xx, yy, zz, xy, xz, yz, Dk, coef, Dkf, bucket, tab);
      ++n_fb;
    }
  }
  return res;
}

__device__ __forceinline__ void sur_counters(DevCounters* cnt, unsigned n_eval, unsigned n_coll, unsigned n_eds,
                                             unsigned n_ref, unsigned n_fp64, unsigned n_fb) {
  n_eval = __reduce_add_sync(0xffffffffu, n_eval);
  n_coll = __reduce_add_sync(0xffffffffu, n_coll);
  n_eds = __reduce_add_sync(0xffffffffu, n_eds);
  n_ref = __reduce_add_sync(0xffffffffu, n_ref);
  n_fp64 = __reduce_add_sync(0xffffffffu, n_fp64);
  n_fb = __reduce_add_sync(0xffffffffu, n_fb);
  if ((threadIdx.x & 31) == 0) {
    if (n_eval) atomicAdd(&cnt->evaluations, static_cast<unsigned long long>(n_eval));
    if (n_coll) atomicAdd(&cnt->collapsed, static_cast<unsigned long long>(n_coll));
    if (n_eds) atomicAdd(&cnt->eds_branch, static_cast<unsigned long long>(n_eds));
    if (n_ref) atomicAdd(&cnt->refined, static_cast<unsigned long long>(n_ref));
    if (n_fp64) atomicAdd(&cnt->fp64_branch, static_cast<unsigned long long>(n_fp64));
    if (n_fb) atomicAdd(&cnt->fallback, static_cast<unsigned long long>(n_fb));
  }
}

// The warp-level form: mma.sync m16n8k16 on register fragments. All lanes of
// a warp stay in the loops so that the warp-wide MLP sees 32 rows every radius.

template <typename T>
__global__ void __launch_bounds__(kThreads, 3)
collapse_sur_kernel(const T* __restrict__ hess, int64_t n, int64_t ps, int64_t rs, int R, int32_t scale_idx0,
                    DevTable tab, RadiusParams rp, SurDev sd, double* __restrict__ F_max, int32_t* __restrict__ idx,
                    DevCounters* __restrict__ cnt) {
  extern __shared__ __align__(16) unsigned char sm[];
  const size_t tb = ((tab.bytes() + 15) / 16) * 16;
  {
    const int words = static_cast<int>(tab.bytes() / 16);
    const uint4* src = reinterpret_cast<const uint4*>(tab.coef);
    uint4* dst = reinterpret_cast<uint4*>(sm);
    for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
    const size_t tail = tab.bytes() & 15;
    if (threadIdx.x < tail)
      reinterpret_cast<unsigned char*>(dst + words)[threadIdx.x] = reinterpret_cast<const unsigned char*>(src + words)[threadIdx.x];
  }
  stage(sm + tb, sd.img + OFF_INF, FWD_BYTES);
  __syncthreads();
  const Coef4* coef = reinterpret_cast<const Coef4*>(sm);
  const double* Dk = reinterpret_cast<const double*>(coef + (tab.n - 1));
  const float* Dkf = reinterpret_cast<const float*>(Dk + tab.n);
  const unsigned short* bucket = reinterpret_cast<const unsigned short*>(Dkf + tab.n);
  const unsigned char* img = sm + tb;
  unsigned n_eval = 0, n_coll = 0, n_eds = 0, n_ref = 0, n_fp64 = 0, n_fb = 0;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t n_round = (n + 31) & ~static_cast<int64_t>(31);
  for (int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; p < n_round; p += stride) {
    const bool active = p < n;
    MinA best;
    const T* base = hess + (active ? p : 0);
    for (int r = 0; r < R; ++r) {
      const T* h = base + static_cast<int64_t>(r) * rs;
      float xx = 0.f, yy = 0.f, zz = 0.f, xy = 0.f, xz = 0.f, yz = 0.f;
      if (active) {
        xx = static_cast<float>(__ldg(h)); yy = static_cast<float>(__ldg(h + ps));
        zz = static_cast<float>(__ldg(h + 2 * ps)); xy = static_cast<float>(__ldg(h + 3 * ps));
        xz = static_cast<float>(__ldg(h + 4 * ps)); yz = static_cast<float>(__ldg(h + 5 * ps));
      }
      const MixedEigen m = mixed_eigen(xx, yy, zz, xy, xz, yz, rp.tri_thr[r]);
      const float is = rp.inv_sigma[r];
      const float z0 = m.lam1f * is, z1 = (m.q + m.x2) * is, z2 = (m.q + m.x3) * is;
      const bool inside = z0 >= sd.lo[0] && z0 <= sd.hi[0] && z1 >= sd.lo[1] && z1 <= sd.hi[1] &&
                          z2 >= sd.lo[2] && z2 <= sd.hi[2];
      __syncwarp();
      const float f = mlp::forward_warp(z0, z1, z2, img);
      if (!active) continue;
      const MixedResult res = sur_finish(m, f, is, inside, xx, yy, zz, xy, xz, yz, Dk, coef, Dkf, bucket, tab, n_fb);
      n_coll += res.collapsed;
      n_eds += res.eds;
      n_ref += res.refined;
      n_fp64 += res.fp64;
      best.add(res.collapsed, res.a, r);
    }
    if (active) {
      best.store<true>(F_max + p, idx + p, scale_idx0);
      n_eval += R;
    }
  }
  sur_counters(cnt, n_eval, n_coll, n_eds, n_ref, n_fp64, n_fb);
}

// barrier of the 128 threads of group g (named barrier 1 + g); returns the OR
// of v over them
__device__ __forceinline__ int group_sync_or(int g, int v) {
  int r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.s32 p, %1, 0;\n\t"
      "bar.red.or.pred q, %2, 128, p;\n\t"
      "selp.s32 %0, 1, 0, q;\n\t}\n"
      : "=r"(r)
      : "r"(v), "r"(g + 1)
      : "memory");
  return r;
}

// The tensor-memory form (tcgen05). A CTA holds kGroups groups of 128
// threads that share one copy of the weights (one bulk copy per CTA) and run
// independently: a group owns a tile of 128 consecutive points, thread i the
// point tile * 128 + i, for all the radii of the launch. Per radius each
// thread writes its point's network input as row i of the group's activation
// tile in shared memory; one thread of the group issues the layer's M = 128
// MMAs (K = 16 for layer 1, 80 for the others, N = 64, or 16 for the last
// layer) into the group's 64 tensor-memory columns and commits them to the
// group's mbarrier; every thread then loads its row of the accumulator
// (tcgen05.ld; the group's warps cover the four lane quadrants), applies SiLU
// and writes the row back as the next layer's input. The bias of every layer
// is an extra pair of K columns (hi, lo) against two columns of ones, so the
// accumulators need no initialisation and the epilogue no adds. One CTA of
// eight groups per SM (1024 threads at 64 registers, all 512 tensor-memory
// columns, the weights and the spline table staged once in shared memory)
// keeps other groups' SiLU and FP32 work running while one waits for its
// MMAs. Every wait is bounded; a wait that runs out stops the group and sets
// an error bit.
template <typename T>
__global__ void __launch_bounds__(tc::kRows * tc::kGroups, tc::kCtasPerSm)
collapse_sur_tc_kernel(const T* __restrict__ hess, int64_t n, int64_t ps, int64_t rs, int R, int32_t scale_idx0,
                       DevTable tab, RadiusParams rp, SurDev sd, double* __restrict__ F_max,
                       int32_t* __restrict__ idx, DevCounters* __restrict__ cnt) {
  using namespace tc;
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ __align__(8) uint64_t bar_ld, bar_mma[kGroups];
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int g = tid >> 7, row = tid & (kRows - 1);
  unsigned char* sA = sm + kA + g * kATileBytes;
  if (tid == 0) {
    umma::mbar_init(&bar_ld, 1);
    for (int i = 0; i < kGroups; ++i) umma::mbar_init(&bar_mma[i], 1);
  }
  __syncwarp();
  if (warp == 0) umma::tmem_alloc<kTmemCols * kGroups>(&tmem_slot);
  // the constant columns of this thread's activation row: 64, 65 = 1 (bias hi, lo), 66..79 = 0
  *reinterpret_cast<uint4*>(sA + umma::offset(row, 64, kSboA)) = make_uint4(pack(1.0f, 1.0f), 0u, 0u, 0u);
  *reinterpret_cast<uint4*>(sA + umma::offset(row, 72, kSboA)) = make_uint4(0u, 0u, 0u, 0u);
  {  // the spline table (coef | D | Df | bucket) into shared memory, 16-byte words
    const int words = static_cast<int>((tab.bytes() + 15) / 16);
    const uint4* src = reinterpret_cast<const uint4*>(tab.coef);
    uint4* dst = reinterpret_cast<uint4*>(sm + kTab);
    for (int i = tid; i < words; i += blockDim.x) dst[i] = src[i];
  }
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  if (tid == 0) umma::bulk_load(sm, sd.img + OFF_TC, kImgBytes, &bar_ld);
  int bad = umma::mbar_wait(&bar_ld, 0, kWaitTries) ? 0 : 1;
  const Coef4* coef = reinterpret_cast<const Coef4*>(sm + kTab);
  const double* Dk = reinterpret_cast<const double*>(coef + (tab.n - 1));
  const float* Dkf = reinterpret_cast<const float*>(Dk + tab.n);
  const unsigned short* bucket = reinterpret_cast<const unsigned short*>(Dkf + tab.n);
  // columns g * 64 .. g * 64 + 63; lanes 32 (warp % 4) .. + 31
  const uint32_t tmem = tmem_slot + static_cast<uint32_t>(g * kTmemCols);
  const uint32_t trow = tmem + (static_cast<uint32_t>((warp & 3) * 32) << 16);
  const uint32_t aA = umma::smem_addr(sA), aW = umma::smem_addr(sm);
  uint64_t* bar = &bar_mma[g];
  constexpr uint32_t kIdesc64 = umma::idesc_bf16_f32(kRows, 64), kIdesc16 = umma::idesc_bf16_f32(kRows, 16);
  uint32_t phase = 0;
  unsigned n_eval = 0, n_coll = 0, n_eds = 0, n_ref = 0, n_fp64 = 0, n_fb = 0;
  const int64_t ntiles = (n + kRows - 1) / kRows;
  const int64_t tstride = static_cast<int64_t>(gridDim.x) * kGroups;
  for (int64_t tile = static_cast<int64_t>(blockIdx.x) * kGroups + g; tile < ntiles; tile += tstride) {
    bad = group_sync_or(g, bad);
    if (bad) break;
    const int64_t p = tile * kRows + row;
    const bool active = p < n;
    MinA best;
    const T* base = hess + (active ? p : 0);
    for (int r = 0; r < R; ++r) {
      const T* h = base + static_cast<int64_t>(r) * rs;
      float xx = 0.f, yy = 0.f, zz = 0.f, xy = 0.f, xz = 0.f, yz = 0.f;
      if (active) {
        xx = static_cast<float>(__ldg(h)); yy = static_cast<float>(__ldg(h + ps));
        zz = static_cast<float>(__ldg(h + 2 * ps)); xy = static_cast<float>(__ldg(h + 3 * ps));
        xz = static_cast<float>(__ldg(h + 4 * ps)); yz = static_cast<float>(__ldg(h + 5 * ps));
      }
      const MixedEigen m = mixed_eigen(xx, yy, zz, xy, xz, yz, rp.tri_thr[r]);
      const float is = rp.inv_sigma[r];
      const float z0 = m.lam1f * is, z1 = (m.q + m.x2) * is, z2 = (m.q + m.x3) * is;
      const bool inside = z0 >= sd.lo[0] && z0 <= sd.hi[0] && z1 >= sd.lo[1] && z1 <= sd.hi[1] &&
                          z2 >= sd.lo[2] && z2 <= sd.hi[2];
      // layer-1 input row: z0 z1 z2, ones at k = 3, 4 (bias hi, lo), zeros to k = 15
      *reinterpret_cast<uint4*>(sA + umma::offset(row, 0, kSboA)) =
          make_uint4(pack(z0, z1), pack(z2, 1.0f), pack(1.0f, 0.0f), 0u);
      *reinterpret_cast<uint4*>(sA + umma::offset(row, 8, kSboA)) = make_uint4(0u, 0u, 0u, 0u);
      float f = 0.0f;
#pragma unroll
      for (int layer = 0; layer < 4; ++layer) {
        // the rows written by every thread of the group (generic proxy) become
        // MMA operands (async proxy)
        umma::fence_smem_async();
        umma::fence_before_sync();
        bad = group_sync_or(g, bad);
        umma::fence_after_sync();
        if (bad) break;
        if (row == 0) {
          if (layer == 0) {
            umma::mma_bf16(tmem, umma::desc(aA, 128, kSboA), umma::desc(aW + kW1, 128, kSbo1), kIdesc64, false);
          } else {
            const uint32_t w = aW + (layer == 1 ? kW2 : layer == 2 ? kW3 : kW4);
#pragma unroll
            for (int s = 0; s < kKA / 16; ++s)
              umma::mma_bf16(tmem, umma::desc(aA + 256 * s, 128, kSboA),
                             umma::desc(w + 256 * s, 128, layer == 3 ? 0 : kSboA), layer == 3 ? kIdesc16 : kIdesc64,
                             s > 0);
          }
          umma::commit(bar);
        }
        // every thread watches the mbarrier (measured faster than one warp
        // watching and a barrier releasing the others)
        if (!umma::mbar_wait(bar, phase, kWaitTries)) bad = 1;
        phase ^= 1u;
        __syncwarp();
        umma::fence_after_sync();
        if (layer < 3) {
          // h = (pre-activation) / 2 of this thread's 64 units -> SiLU -> next input row
#pragma unroll
          for (int c0 = 0; c0 < 64; c0 += 16) {
            uint32_t v[16];
            umma::ld16(trow + c0, v);
            umma::wait_ld();
            uint32_t w[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) w[j] = silu2_half(__uint_as_float(v[2 * j]), __uint_as_float(v[2 * j + 1]));
            *reinterpret_cast<uint4*>(sA + umma::offset(row, c0, kSboA)) = make_uint4(w[0], w[1], w[2], w[3]);
            *reinterpret_cast<uint4*>(sA + umma::offset(row, c0 + 8, kSboA)) = make_uint4(w[4], w[5], w[6], w[7]);
          }
        } else {
          f = __uint_as_float(umma::ld1(trow));
          umma::wait_ld();
        }
        // this thread's accumulator loads are complete before the next MMA overwrites them
        umma::fence_before_sync();
      }
      bad = group_sync_or(g, bad);
      if (bad) break;
      if (!active) continue;
      const MixedResult res =
          sur_finish(m, f, is, inside, xx, yy, zz, xy, xz, yz, Dk, coef, Dkf, bucket, tab, n_fb);
      n_coll += res.collapsed;
      n_eds += res.eds;
      n_ref += res.refined;
      n_fp64 += res.fp64;
      best.add(res.collapsed, res.a, r);
    }
    if (bad) break;
    if (active) {
      best.store<true>(F_max + p, idx + p, scale_idx0);
      n_eval += R;
    }
  }
  sur_counters(cnt, n_eval, n_coll, n_eds, n_ref, n_fp64, n_fb);
  if (bad && row == 0) atomicOr(&cnt->error_flags, kErrWait);
  // every tensor-memory load of the CTA has completed and every MMA was waited
  // for (or its group gave up on it): the tensor memory can go
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  if (warp == 0) umma::tmem_free<kTmemCols * kGroups>(tmem_slot);
}

int launch_grid(int64_t n, int threads, int cap) {
  const int64_t need = (n + threads - 1) / threads;
  return static_cast<int>(need < cap ? need : cap);
}

struct SurState {
  unsigned char* img = nullptr;
  float* p = nullptr;  // p | m | v | grad | loss(2)
};

int ensure_surrogate(cc_ctx* ctx) {
  if (ctx->d_mlp_img) return CC_OK;
  if (int rc = check_cuda(cudaMalloc(reinterpret_cast<void**>(&ctx->d_mlp_img), tc::IMG_TOTAL), "cudaMalloc(mlp image)")) return rc;
  if (int rc = check_cuda(cudaMalloc(reinterpret_cast<void**>(&ctx->d_mlp_param), sizeof(float) * (4 * NPARAM + 8)),
                          "cudaMalloc(mlp params)"))
    return rc;
  if (int rc = check_cuda(cudaMemset(ctx->d_mlp_img, 0, tc::IMG_TOTAL), "cudaMemset")) return rc;
  return check_cuda(cudaMemset(ctx->d_mlp_param, 0, sizeof(float) * (4 * NPARAM + 8)), "cudaMemset");
}

// LeCun-uniform initial weights (variance 1/fan_in) from a seeded xorshift; biases 0, b4 = mean target
void init_params(std::vector<float>& p, uint64_t seed, float b4) {
  p.assign(NPARAM, 0.0f);
  uint64_t s = seed * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
  auto uni = [&]() {
    s ^= s << 13; s ^= s >> 7; s ^= s << 17;
    return static_cast<float>((s >> 11) * (1.0 / 9007199254740992.0)) * 2.0f - 1.0f;
  };
  auto fill = [&](int off, int fan_in, int count) {
    const float bound = std::sqrt(3.0f / static_cast<float>(fan_in));
    for (int i = 0; i < count; ++i) p[off + i] = bound * uni();
  };
  fill(P_W1, 3, 3 * H);
  fill(P_W2, H, H * H);
  fill(P_W3, H, H * H);
  fill(P_W4, H, H);
  p[P_B4] = b4;
}

template <typename T>
int launch_sur_typed(cc_ctx* ctx, const LaunchArgs& a, const RadiusParams& rp) {
  SurDev sd;
  sd.img = ctx->d_mlp_img;
  for (int i = 0; i < 3; ++i) {
    sd.lo[i] = ctx->sur_hull[i];
    sd.hi[i] = ctx->sur_hull[3 + i];
  }
  if (ctx->sur_engine == CC_SURROGATE_TCGEN05) {
    auto kern = collapse_sur_tc_kernel<T>;
    if (int rc = check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100),
                            "cudaFuncSetAttribute"))
      return rc;
    const size_t smem = tc::kSmemBytes + ((ctx->tab.bytes() + 15) / 16) * 16;
    if (int rc = check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 static_cast<int>(smem)),
                            "cudaFuncSetAttribute"))
      return rc;
    // resident CTAs per SM from the shared-memory footprint (the occupancy
    // calculator does not follow the carveout preference set above)
    const int64_t need = ((a.n + tc::kRows - 1) / tc::kRows + tc::kGroups - 1) / tc::kGroups;
    const int64_t cap = static_cast<int64_t>(a.num_sms) * tc::kCtasPerSm;
    const int grid = static_cast<int>(need < cap ? need : cap);
    DevTable t = ctx->tab;  // the index checks of debug builds report into this launch's flags
    t.dbg = &a.counters->error_flags;
    kern<<<grid, tc::kRows * tc::kGroups, smem, a.stream>>>(static_cast<const T*>(a.hess), a.n, a.plane_stride,
                                                         a.radius_stride, a.R, a.scale_idx0, t, rp, sd,
                                                         a.F_max, a.idx, a.counters);
    return check_cuda(cudaGetLastError(), "collapse_sur_tc_kernel launch");
  }
  auto kern = collapse_sur_kernel<T>;
  const size_t smem = ((ctx->tab.bytes() + 15) / 16) * 16 + FWD_BYTES;
  if (smem > 48 * 1024)
    if (int rc = check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)),
                            "cudaFuncSetAttribute"))
      return rc;
  int occ = 0;
  if (int rc = check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, smem), "occupancy")) return rc;
  const int64_t need = (a.n + kThreads - 1) / kThreads;
  const int64_t cap = static_cast<int64_t>(a.num_sms) * (occ > 0 ? occ : 1);
  const int grid = static_cast<int>(need < cap ? need : cap);
  DevTable t = ctx->tab;
  t.dbg = &a.counters->error_flags;
  kern<<<grid, kThreads, smem, a.stream>>>(static_cast<const T*>(a.hess), a.n, a.plane_stride, a.radius_stride, a.R,
                                           a.scale_idx0, t, rp, sd, a.F_max, a.idx, a.counters);
  return check_cuda(cudaGetLastError(), "collapse_sur_kernel launch");
}

}  // namespace

int launch_surrogate_checked(cc_ctx* ctx, const LaunchArgs& a, const double* sigma) {
  if (!ctx->sur_valid) return set_error(CC_EINVAL, "CC_MODE_SURROGATE needs a trained or loaded surrogate");
  for (int r0 = 0; r0 < a.R; r0 += kMaxRadiiPerLaunch) {
    LaunchArgs c = a;
    c.R = (a.R - r0 < kMaxRadiiPerLaunch) ? a.R - r0 : kMaxRadiiPerLaunch;
    c.hess = static_cast<const unsigned char*>(a.hess) + static_cast<size_t>(r0) * a.radius_stride * a.dtype;
    c.scale_idx0 = a.scale_idx0 + r0;
    RadiusParams rp;
    for (int r = 0; r < c.R; ++r) {
      rp.tri_thr[r] = static_cast<float>(1e-4 * sigma[r0 + r]);
      rp.inv_sigma[r] = static_cast<float>(1.0 / sigma[r0 + r]);
    }
    const int rc = (a.dtype == CC_F64) ? launch_sur_typed<double>(ctx, c, rp) : launch_sur_typed<float>(ctx, c, rp);
    if (rc) return rc;
  }
  return CC_OK;
}

// ---- training (shared by cc_surrogate_train and cc_surrogate_train_resume)
struct TrainSet {
  float4* recs = nullptr;  // training records (z, target), then the held-out ones
  int64_t total = 0, ntrain = 0, nval = 0;
  float hull[6] = {0, 0, 0, 0, 0, 0};
};

// Samples of the exact FP64 path on the caller's planes (every point with
// l1 > 0 and D_c s < 1e4), the last val_fraction of them held out.
int build_training_set(cc_ctx* ctx, const void* hess, int32_t dtype, int64_t n, int64_t plane_stride, double sigma,
                       float val_fraction, TrainSet& ts, void* stream) {
  if (dtype != CC_F64 && dtype != CC_F32) return set_error(CC_EINVAL, "dtype must be CC_F64 or CC_F32");
  if (n < 1024 || plane_stride < n || !(sigma > 0.0)) return set_error(CC_EINVAL, "need n >= 1024, plane_stride >= n, sigma > 0");
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != ctx->device) cudaSetDevice(ctx->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (int rc = ensure_surrogate(ctx)) return rc;
  const size_t rec_bytes = sizeof(float4) * static_cast<size_t>(n);
  if (rec_bytes > ctx->train_cap) {
    if (ctx->d_train) cudaFree(ctx->d_train);
    ctx->d_train = nullptr;
    ctx->train_cap = 0;
    if (int rc = check_cuda(cudaMalloc(&ctx->d_train, rec_bytes + 64), "cudaMalloc(training set)")) return rc;
    ctx->train_cap = rec_bytes;
  }
  float4* recs = static_cast<float4*>(ctx->d_train);
  unsigned long long* count = reinterpret_cast<unsigned long long*>(static_cast<unsigned char*>(ctx->d_train) + rec_bytes);
  int* hull = reinterpret_cast<int*>(count + 1);
  const int hull_init[6] = {0x7FFFFFFF, 0x7FFFFFFF, 0x7FFFFFFF, static_cast<int>(0x80000000), static_cast<int>(0x80000000),
                            static_cast<int>(0x80000000)};
  if (int rc = check_cuda(cudaMemsetAsync(count, 0, sizeof(unsigned long long), st), "cudaMemsetAsync")) return rc;
  if (int rc = check_cuda(cudaMemcpyAsync(hull, hull_init, sizeof(hull_init), cudaMemcpyHostToDevice, st), "H2D hull")) return rc;
  const int grid = launch_grid(n, 256, ctx->num_sms * 8);
  if (dtype == CC_F64)
    sur_data_kernel<double><<<grid, 256, 0, st>>>(static_cast<const double*>(hess), n, plane_stride, sigma, recs, count, n, hull);
  else
    sur_data_kernel<float><<<grid, 256, 0, st>>>(static_cast<const float*>(hess), n, plane_stride, sigma, recs, count, n, hull);
  if (int rc = check_cuda(cudaGetLastError(), "sur_data_kernel launch")) return rc;
  unsigned long long cnt = 0;
  int hull_h[6];
  if (int rc = check_cuda(cudaMemcpyAsync(&cnt, count, sizeof(cnt), cudaMemcpyDeviceToHost, st), "D2H count")) return rc;
  if (int rc = check_cuda(cudaMemcpyAsync(hull_h, hull, sizeof(hull_h), cudaMemcpyDeviceToHost, st), "D2H hull")) return rc;
  if (int rc = check_cuda(cudaStreamSynchronize(st), "cudaStreamSynchronize")) return rc;
  ts.recs = recs;
  ts.total = static_cast<int64_t>(cnt < static_cast<unsigned long long>(n) ? cnt : n);
  ts.nval = static_cast<int64_t>(ts.total * val_fraction);
  ts.ntrain = ts.total - ts.nval;
  for (int i = 0; i < 6; ++i) ts.hull[i] = unordered(hull_h[i]);
  return CC_OK;
}

// Adam steps ctx->sur_step .. ctx->sur_step + steps - 1 of the warm-up + cosine
// schedule of length ctx->sur_schedule (minibatch indices hashed from the seed
// and the step: the sampler's state is the step), then the held-out error.
int train_and_validate(cc_ctx* ctx, const TrainSet& ts, int64_t steps, cc_train_report* report, cudaStream_t st) {
  const cc_train_config& cfg = ctx->sur_cfg;
  float* P = ctx->d_mlp_param;
  float* Mv = P + NPARAM;
  float* Vv = Mv + NPARAM;
  float* G = Vv + NPARAM;
  float* loss = G + NPARAM;
  if (int rc = check_cuda(cudaFuncSetAttribute(sur_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               static_cast<int>(kTrainSmem)), "cudaFuncSetAttribute"))
    return rc;
  const int blocks = cfg.batch / (32 * kTrainWarps);
  const float inv_batch = 1.0f / static_cast<float>(cfg.batch);
  std::vector<float> losses;
  const int64_t s0 = ctx->sur_step, s1 = s0 + steps;
  ctx->sur_trained = false;  // until the steps are done
  for (int64_t s = s0; s < s1; ++s) {
    const bool record = (s == s0 || s == s1 - 1);
    if (record)
      if (int rc = check_cuda(cudaMemsetAsync(loss, 0, sizeof(float), st), "cudaMemsetAsync")) return rc;
    sur_train_kernel<<<blocks, 32 * kTrainWarps, kTrainSmem, st>>>(ts.recs, ts.ntrain, cfg.seed, static_cast<int>(s), 0,
                                                                   inv_batch, ctx->d_mlp_img, G, loss);
    const double warm = std::min(1.0, (s + 1) / 100.0);
    const double lr = cfg.lr * warm * 0.5 * (1.0 + std::cos(3.141592653589793 * s / ctx->sur_schedule)) + 1e-6;
    const float b1t = static_cast<float>(std::pow(0.9, s + 1)), b2t = static_cast<float>(std::pow(0.999, s + 1));
    sur_adam_kernel<<<(NPARAM + 255) / 256, 256, 0, st>>>(P, Mv, Vv, G, static_cast<float>(lr), b1t, b2t, ctx->d_mlp_img);
    if (record) {
      float l = 0.f;
      if (int rc = check_cuda(cudaMemcpyAsync(&l, loss, sizeof(float), cudaMemcpyDeviceToHost, st), "D2H loss")) return rc;
      if (int rc = check_cuda(cudaStreamSynchronize(st), "cudaStreamSynchronize")) return rc;
      losses.push_back(l);
    }
  }
  if (int rc = check_cuda(cudaGetLastError(), "training launch")) return rc;
  ctx->sur_step = s1;
  ctx->sur_trained = true;
  // ---- validation on the held-out records
  float* stats = loss + 2;
  if (int rc = check_cuda(cudaMemsetAsync(stats, 0, sizeof(float) * 2, st), "cudaMemsetAsync")) return rc;
  sur_eval_kernel<<<launch_grid(ts.nval, 256, ctx->num_sms * 4), 256, FWD_BYTES, st>>>(
      reinterpret_cast<const float*>(ts.recs + ts.ntrain), 4, ts.nval, ctx->d_mlp_img, nullptr, stats,
      reinterpret_cast<int*>(stats + 1));
  float stats_h[2];
  if (int rc = check_cuda(cudaMemcpyAsync(stats_h, stats, sizeof(stats_h), cudaMemcpyDeviceToHost, st), "D2H stats")) return rc;
  if (int rc = check_cuda(cudaStreamSynchronize(st), "cudaStreamSynchronize")) return rc;
  ctx->sur_valid = true;
  if (report) {
    report->samples = ts.total;
    report->train_samples = ts.ntrain;
    report->val_samples = ts.nval;
    report->loss_first = losses.empty() ? 0.f : losses.front();
    report->loss_last = losses.empty() ? 0.f : losses.back();
    report->val_rms = std::sqrt(stats_h[0] / static_cast<float>(ts.nval));
    std::memcpy(&report->val_max, &stats_h[1], sizeof(float));
    for (int i = 0; i < 3; ++i) {
      report->hull_lo[i] = ctx->sur_hull[i];
      report->hull_hi[i] = ctx->sur_hull[3 + i];
    }
  }
  return CC_OK;
}

// ---- checkpoint blob: header, then FP32 parameters, Adam first and second moments
constexpr char kCkptMagic[8] = {'C', 'C', 'S', 'U', 'R', 'C', 'K', '\0'};
constexpr uint32_t kCkptVersion = 1;
struct CkptHeader {
  char magic[8];
  uint32_t version, nparam;
  int64_t step, schedule_steps;  // Adam steps taken, length of the learning-rate schedule
  uint64_t seed;                 // minibatch sampler key (its counter is the step)
  float lr, val_fraction;
  int32_t batch, reserved;
  float hull[6];
};
static_assert(sizeof(CkptHeader) % 8 == 0, "header keeps the arrays 8-byte aligned");
constexpr size_t kCkptBytes = sizeof(CkptHeader) + sizeof(float) * 3 * NPARAM;

}  // namespace cc

using namespace cc;
using namespace cc::mlp;

extern "C" {

int cc_set_surrogate_engine(cc_ctx* ctx, int32_t engine) {
  if (!ctx) return set_error(CC_EINVAL, "ctx is NULL");
  if (engine != CC_SURROGATE_MMA_SYNC && engine != CC_SURROGATE_TCGEN05)
    return set_error(CC_EINVAL, "engine must be CC_SURROGATE_MMA_SYNC or CC_SURROGATE_TCGEN05");
  ctx->sur_engine = engine;
  return CC_OK;
}

int cc_surrogate_train(cc_ctx* ctx, const void* hess, int32_t dtype, int64_t n, int64_t plane_stride, double sigma,
                       const cc_train_config* cfg, cc_train_report* report, void* stream) {
  if (!ctx || !hess || !cfg) return set_error(CC_EINVAL, "ctx, hess and cfg are required");
  if (cfg->steps < 1 || cfg->batch < 64 || cfg->batch % 64 || !(cfg->lr > 0.0f) || !(cfg->val_fraction > 0.0f) ||
      !(cfg->val_fraction < 0.5f))
    return set_error(CC_EINVAL, "train config: steps >= 1, batch a multiple of 64, lr > 0, 0 < val_fraction < 0.5");
  TrainSet ts;
  if (int rc = build_training_set(ctx, hess, dtype, n, plane_stride, sigma, cfg->val_fraction, ts, stream)) return rc;
  if (ts.ntrain < cfg->batch || ts.nval < 32) return set_error(CC_EINVAL, "too few collapsing points to train on");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // ---- initial parameters: b4 = mean target of the first samples
  std::vector<float4> head(static_cast<size_t>(std::min<int64_t>(ts.ntrain, 65536)));
  if (int rc = check_cuda(cudaMemcpy(head.data(), ts.recs, sizeof(float4) * head.size(), cudaMemcpyDeviceToHost), "D2H head")) return rc;
  double tmean = 0.0;
  for (const auto& r : head) tmean += r.w;
  tmean /= static_cast<double>(head.size());
  std::vector<float> p0;
  init_params(p0, cfg->seed, static_cast<float>(tmean));
  float* P = ctx->d_mlp_param;
  if (int rc = check_cuda(cudaMemcpyAsync(P, p0.data(), sizeof(float) * NPARAM, cudaMemcpyHostToDevice, st), "H2D params")) return rc;
  if (int rc = check_cuda(cudaMemsetAsync(P + NPARAM, 0, sizeof(float) * (3 * NPARAM + 8), st), "cudaMemsetAsync")) return rc;
  sur_image_kernel<<<(NPARAM + 255) / 256, 256, 0, st>>>(P, ctx->d_mlp_img);
  ctx->sur_cfg = *cfg;
  ctx->sur_step = 0;
  ctx->sur_schedule = cfg->steps;
  for (int i = 0; i < 6; ++i) ctx->sur_hull[i] = ts.hull[i];
  return train_and_validate(ctx, ts, cfg->steps, report, st);
}

int cc_surrogate_train_resume(cc_ctx* ctx, const void* hess, int32_t dtype, int64_t n, int64_t plane_stride,
                              double sigma, int32_t steps, int32_t schedule_steps, cc_train_report* report,
                              void* stream) {
  if (!ctx || !hess) return set_error(CC_EINVAL, "ctx and hess are required");
  if (!ctx->sur_trained) return set_error(CC_EINVAL, "no training state: call cc_surrogate_train or cc_surrogate_restore first");
  if (steps < 1) return set_error(CC_EINVAL, "steps must be >= 1");
  const int64_t until = ctx->sur_step + steps;
  if (schedule_steps != 0 && schedule_steps < until)
    return set_error(CC_EINVAL, "schedule_steps must be 0 or at least the steps taken plus the new ones");
  TrainSet ts;
  if (int rc = build_training_set(ctx, hess, dtype, n, plane_stride, sigma, ctx->sur_cfg.val_fraction, ts, stream)) return rc;
  if (ts.ntrain < ctx->sur_cfg.batch || ts.nval < 32) return set_error(CC_EINVAL, "too few collapsing points to train on");
  ctx->sur_schedule = schedule_steps != 0 ? schedule_steps : std::max<int64_t>(ctx->sur_schedule, until);
  for (int i = 0; i < 3; ++i) {  // the hull covers every training set seen
    ctx->sur_hull[i] = std::min(ctx->sur_hull[i], ts.hull[i]);
    ctx->sur_hull[3 + i] = std::max(ctx->sur_hull[3 + i], ts.hull[3 + i]);
  }
  return train_and_validate(ctx, ts, steps, report, static_cast<cudaStream_t>(stream));
}

int cc_surrogate_checkpoint(const cc_ctx* ctx, void* blob, size_t* bytes) {
  if (!ctx || !bytes) return set_error(CC_EINVAL, "ctx and bytes are required");
  if (!blob) {
    *bytes = kCkptBytes;
    return CC_OK;
  }
  if (*bytes < kCkptBytes) return set_error(CC_EINVAL, "blob smaller than the checkpoint (query the size with blob = NULL)");
  if (!ctx->sur_trained) return set_error(CC_EINVAL, "no training state: call cc_surrogate_train or cc_surrogate_restore first");
  CkptHeader h{};
  std::memcpy(h.magic, kCkptMagic, sizeof(h.magic));
  h.version = kCkptVersion;
  h.nparam = NPARAM;
  h.step = ctx->sur_step;
  h.schedule_steps = ctx->sur_schedule;
  h.seed = ctx->sur_cfg.seed;
  h.lr = ctx->sur_cfg.lr;
  h.val_fraction = ctx->sur_cfg.val_fraction;
  h.batch = ctx->sur_cfg.batch;
  std::memcpy(h.hull, ctx->sur_hull, sizeof(h.hull));
  if (int rc = select_device(ctx)) return rc;
  unsigned char* out = static_cast<unsigned char*>(blob);
  std::memcpy(out, &h, sizeof(h));
  if (int rc = check_cuda(cudaMemcpy(out + sizeof(h), ctx->d_mlp_param, sizeof(float) * 3 * NPARAM, cudaMemcpyDeviceToHost),
                          "D2H training state"))
    return rc;
  *bytes = kCkptBytes;
  return CC_OK;
}

int cc_surrogate_restore(cc_ctx* ctx, const void* blob, size_t bytes) {
  if (!ctx || !blob) return set_error(CC_EINVAL, "ctx and blob are required");
  if (bytes < sizeof(CkptHeader)) return set_error(CC_EINVAL, "blob shorter than a checkpoint header");
  CkptHeader h;
  std::memcpy(&h, blob, sizeof(h));
  if (std::memcmp(h.magic, kCkptMagic, sizeof(h.magic)) != 0) return set_error(CC_EINVAL, "not a surrogate checkpoint");
  if (h.version != kCkptVersion) return set_error(CC_ENOTSUP, "checkpoint version not supported by this library");
  if (h.nparam != static_cast<uint32_t>(NPARAM) || bytes != kCkptBytes)
    return set_error(CC_EINVAL, "checkpoint size does not match the network");
  if (h.step < 0 || h.schedule_steps < h.step || h.batch < 64 || h.batch % 64 || !(h.lr > 0.0f) ||
      !(h.val_fraction > 0.0f) || !(h.val_fraction < 0.5f))
    return set_error(CC_EINVAL, "checkpoint header out of range");
  for (int i = 0; i < 3; ++i)
    if (!(h.hull[i] <= h.hull[3 + i])) return set_error(CC_EINVAL, "checkpoint hull: lo <= hi per component");
  const float* arr = reinterpret_cast<const float*>(static_cast<const unsigned char*>(blob) + sizeof(h));
  std::vector<float> state(arr, arr + 3 * NPARAM);
  for (float v : state)
    if (!std::isfinite(v)) return set_error(CC_EINVAL, "checkpoint values must be finite");
  if (int rc = select_device(ctx)) return rc;
  if (int rc = ensure_surrogate(ctx)) return rc;
  if (int rc = check_cuda(cudaMemcpy(ctx->d_mlp_param, state.data(), sizeof(float) * 3 * NPARAM, cudaMemcpyHostToDevice),
                          "H2D training state"))
    return rc;
  sur_image_kernel<<<(NPARAM + 255) / 256, 256>>>(ctx->d_mlp_param, ctx->d_mlp_img);
  if (int rc = check_cuda(cudaDeviceSynchronize(), "sur_image_kernel")) return rc;
  ctx->sur_cfg.steps = static_cast<int32_t>(h.schedule_steps);
  ctx->sur_cfg.batch = h.batch;
  ctx->sur_cfg.lr = h.lr;
  ctx->sur_cfg.seed = h.seed;
  ctx->sur_cfg.val_fraction = h.val_fraction;
  ctx->sur_step = h.step;
  ctx->sur_schedule = h.schedule_steps;
  std::memcpy(ctx->sur_hull, h.hull, sizeof(h.hull));
  ctx->sur_trained = true;
  ctx->sur_valid = true;
  return CC_OK;
}

int cc_surrogate_params(const cc_ctx* ctx, float* params, float* hull) {
  if (!ctx || !params) return set_error(CC_EINVAL, "ctx and params are required");
  if (!ctx->sur_valid) return set_error(CC_EINVAL, "no surrogate: train or load one first");
  if (int rc = check_cuda(cudaMemcpy(params, ctx->d_mlp_param, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost), "D2H params"))
    return rc;
  if (hull) std::memcpy(hull, ctx->sur_hull, sizeof(float) * 6);
  return CC_OK;
}

int cc_load_surrogate(cc_ctx* ctx, const float* params, const float* hull) {
  if (!ctx || !params || !hull) return set_error(CC_EINVAL, "ctx, params and hull are required");
  for (int i = 0; i < NPARAM; ++i)
    if (!std::isfinite(params[i])) return set_error(CC_EINVAL, "parameters must be finite");
  for (int i = 0; i < 3; ++i)
    if (!(hull[i] <= hull[3 + i])) return set_error(CC_EINVAL, "hull: lo <= hi per component");
  if (int rc = ensure_surrogate(ctx)) return rc;
  if (int rc = check_cuda(cudaMemcpy(ctx->d_mlp_param, params, sizeof(float) * NPARAM, cudaMemcpyHostToDevice), "H2D params"))
    return rc;
  sur_image_kernel<<<(NPARAM + 255) / 256, 256>>>(ctx->d_mlp_param, ctx->d_mlp_img);
  if (int rc = check_cuda(cudaDeviceSynchronize(), "sur_image_kernel")) return rc;
  std::memcpy(ctx->sur_hull, hull, sizeof(float) * 6);
  ctx->sur_valid = true;
  ctx->sur_trained = false;  // parameters without optimiser state: nothing to resume
  return CC_OK;
}

int cc_surrogate_eval(cc_ctx* ctx, const float* z, int64_t n, float* out, void* stream) {
  if (!ctx || n < 0 || (n > 0 && (!z || !out))) return set_error(CC_EINVAL, "bad arguments");
  if (!ctx->sur_valid) return set_error(CC_EINVAL, "no surrogate: train or load one first");
  if (n == 0) return CC_OK;
  sur_eval_kernel<<<launch_grid(n, 256, ctx->num_sms * 4), 256, FWD_BYTES, static_cast<cudaStream_t>(stream)>>>(
      z, 3, n, ctx->d_mlp_img, out, nullptr, nullptr);
  return check_cuda(cudaGetLastError(), "sur_eval_kernel launch");
}

int cc_surrogate_grad(cc_ctx* ctx, const float* z, const float* t, int32_t n, float* grad, float* loss_out) {
  if (!ctx || !z || !t || !grad || n < 64 || n % 64) return set_error(CC_EINVAL, "need host z, t, grad and n a multiple of 64");
  if (!ctx->sur_valid) return set_error(CC_EINVAL, "no surrogate: train or load one first");
  std::vector<float4> recs(n);
  for (int i = 0; i < n; ++i) recs[i] = make_float4(z[3 * i], z[3 * i + 1], z[3 * i + 2], t[i]);
  float4* d = nullptr;
  float* g = nullptr;
  if (int rc = check_cuda(cudaMalloc(reinterpret_cast<void**>(&d), sizeof(float4) * n), "cudaMalloc")) return rc;
  int rc = check_cuda(cudaMalloc(reinterpret_cast<void**>(&g), sizeof(float) * (NPARAM + 1)), "cudaMalloc");
  if (!rc) rc = check_cuda(cudaMemcpy(d, recs.data(), sizeof(float4) * n, cudaMemcpyHostToDevice), "H2D");
  if (!rc) rc = check_cuda(cudaMemset(g, 0, sizeof(float) * (NPARAM + 1)), "cudaMemset");
  if (!rc) rc = check_cuda(cudaFuncSetAttribute(sur_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                static_cast<int>(kTrainSmem)), "cudaFuncSetAttribute");
  if (!rc) {
    sur_train_kernel<<<n / (32 * kTrainWarps), 32 * kTrainWarps, kTrainSmem>>>(d, n, 0, 0, 1, 1.0f / n, ctx->d_mlp_img,
                                                                              g, g + NPARAM);
    rc = check_cuda(cudaDeviceSynchronize(), "sur_train_kernel");
  }
  if (!rc) rc = check_cuda(cudaMemcpy(grad, g, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost), "D2H grad");
  if (!rc && loss_out) rc = check_cuda(cudaMemcpy(loss_out, g + NPARAM, sizeof(float), cudaMemcpyDeviceToHost), "D2H loss");
  cudaFree(d);
  cudaFree(g);
  return rc;
}

}  // extern "C"
