// cc_mlp.cuh -- the surrogate MLP (3 -> 64 -> 64 -> 64 -> 1, SiLU) on BF16
// tensor cores with FP32 accumulation (no counterpart in the paper).
//
// One warp evaluates 32 points as two 16-row tiles with mma.sync m16n8k16
// (BF16 in, FP32 accumulate). A layer's accumulator fragments (rows g, g+8;
// columns 2t, 2t+1 of each 8-column tile) are exactly the A-operand fragments
// of the next layer's 16-column k-steps, so activations never leave registers.
// Weights live in shared memory as BF16 rows padded to 72 elements (144 bytes:
// the 32 lanes' 32-bit fragment loads hit 32 different banks).
#pragma once

#include <cuda_bf16.h>

#include "cc_internal.h"

namespace cc {
namespace mlp {

constexpr int H = 64;
constexpr int STR = 72;   // padded row stride (bf16) of 64-wide rows
constexpr int STR1 = 24;  // padded row stride of layer 1's 16-wide (3 used) rows
// parameter offsets in the FP32 master vector (same layout as the oracle's):
// W1[3][64], b1[64], W2[64][64], b2[64], W3[64][64], b3[64], W4[64], b4
constexpr int P_W1 = 0, P_B1 = 192, P_W2 = 256, P_B2 = 4352, P_W3 = 4416, P_B3 = 8512, P_W4 = 8576, P_B4 = 8640;
constexpr int NPARAM = 8641;
// byte offsets of the BF16 image (forward part first)
constexpr int OFF_W1T = 0;                               // [64][STR1]: W1t[n][k] = W1[k][n]
constexpr int OFF_W2T = OFF_W1T + H * STR1 * 2;          // [64][STR]:  W2t[n][k] = W2[k][n]
constexpr int OFF_W3T = OFF_W2T + H * STR * 2;
constexpr int OFF_W4T = OFF_W3T + H * STR * 2;           // [8][STR]: row 0 = W4, rows 1..7 = 0
constexpr int OFF_B = OFF_W4T + 8 * STR * 2;             // FP32 b1[64] b2[64] b3[64] b4 (+pad)
constexpr int FWD_BYTES = OFF_B + 784;
constexpr int OFF_W2B = FWD_BYTES;                       // [64][STR]: W2b[k][n] = W2[k][n] (backward)
constexpr int OFF_W3B = OFF_W2B + H * STR * 2;
constexpr int ALL_BYTES = OFF_W3B + H * STR * 2;
// the inference image: the forward part again with W1..W3 and b1..b3 halved
// (W4 and b4 as they are), read by the inference kernels only
constexpr int OFF_INF = ALL_BYTES;
constexpr int IMG_BYTES = OFF_INF + FWD_BYTES;
static_assert(FWD_BYTES % 16 == 0 && ALL_BYTES % 16 == 0, "16-byte staging");

__device__ __forceinline__ uint32_t pack(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ uint32_t ld32(const unsigned char* base, int byte_off) {
  return *reinterpret_cast<const uint32_t*>(base + byte_off);
}

__device__ __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// the same MMA as a pure register operation, which the scheduler may move
// (the inference layers interleave it with the next fragment loads)
__device__ __forceinline__ void mma_pure(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float silu(float v) { return __fdividef(v, 1.0f + __expf(-v)); }
__device__ __forceinline__ float dsilu(float v) {
  const float s = __fdividef(1.0f, 1.0f + __expf(-v));
  return s * fmaf(v, 1.0f - s, 1.0f);
}

// one 16-row tile through a 64 -> 64 layer: c = A W + b (Wt rows = output units)
__device__ __forceinline__ void layer64(const uint32_t (&a)[4][4], const unsigned char* img, int off_wt,
                                        const float* bias, float (&c)[8][4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float b0 = bias[8 * j + 2 * t], b1 = bias[8 * j + 2 * t + 1];
    c[j][0] = b0; c[j][1] = b1; c[j][2] = b0; c[j][3] = b1;
    const int row = off_wt + (8 * j + g) * STR * 2;
#pragma unroll
    for (int s = 0; s < 4; ++s)
      mma(c[j], a[s], ld32(img, row + (16 * s + 2 * t) * 2), ld32(img, row + (16 * s + 8 + 2 * t) * 2));
  }
}

// SiLU and repack accumulators as the next layer's A fragments
__device__ __forceinline__ void act_pack(const float (&c)[8][4], uint32_t (&a)[4][4]) {
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    a[s][0] = pack(silu(c[2 * s][0]), silu(c[2 * s][1]));
    a[s][1] = pack(silu(c[2 * s][2]), silu(c[2 * s][3]));
    a[s][2] = pack(silu(c[2 * s + 1][0]), silu(c[2 * s + 1][1]));
    a[s][3] = pack(silu(c[2 * s + 1][2]), silu(c[2 * s + 1][3]));
  }
}

// Inference SiLU on packed BF16 pairs: silu(v) = v sigmoid(v) = h + h tanh(h)
// with h = v/2, one tanh.approx.bf16x2 (two results per special-function
// instruction) and one bf16x2 FMA. The inference image holds W1..W3 and
// b1..b3 halved (exact in BF16 and FP32, so the accumulators are exactly
// v/2 = h): a pair costs one pack, one tanh and one FMA. The result is the
// BF16 A fragment either way; the hardware tanh adds an error of the order of
// that rounding. The training kernels keep the FP32 SiLU of act_pack on the
// unscaled image (they need silu' as well).
__device__ __forceinline__ uint32_t silu2_half(float h0, float h1) {
  const uint32_t h = pack(h0, h1);
  uint32_t t, r;
  asm("tanh.approx.bf16x2 %0, %1;" : "=r"(t) : "r"(h));
  asm("fma.rn.bf16x2 %0, %1, %2, %1;" : "=r"(r) : "r"(h), "r"(t));
  return r;
}

// layer 1 (3 inputs, padded to one k16 step) for one tile; rows r0 = 16 tile + g, r1 = r0 + 8
__device__ __forceinline__ void layer1(float z0, float z1, float z2, int tile, const unsigned char* img,
                                       float (&c)[8][4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int r0 = 16 * tile + g, r1 = r0 + 8;
  const float a00 = __shfl_sync(0xffffffffu, z0, r0), a01 = __shfl_sync(0xffffffffu, z1, r0);
  const float a02 = __shfl_sync(0xffffffffu, z2, r0);
  const float a10 = __shfl_sync(0xffffffffu, z0, r1), a11 = __shfl_sync(0xffffffffu, z1, r1);
  const float a12 = __shfl_sync(0xffffffffu, z2, r1);
  uint32_t a[4];
  a[0] = (t == 0) ? pack(a00, a01) : (t == 1) ? pack(a02, 0.0f) : 0u;
  a[1] = (t == 0) ? pack(a10, a11) : (t == 1) ? pack(a12, 0.0f) : 0u;
  a[2] = 0u;
  a[3] = 0u;
  const float* bias = reinterpret_cast<const float*>(img + OFF_B);
  uint32_t aa[4] = {a[0], a[1], a[2], a[3]};
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float b0 = bias[8 * j + 2 * t], b1 = bias[8 * j + 2 * t + 1];
    c[j][0] = b0; c[j][1] = b1; c[j][2] = b0; c[j][3] = b1;
    const int row = OFF_W1T + (8 * j + g) * STR1 * 2;
    mma(c[j], aa, ld32(img, row + (2 * t) * 2), ld32(img, row + (8 + 2 * t) * 2));
  }
}

// last layer (64 -> 1, padded to one 8-column tile): returns the outputs of
// rows r0 (c[0]) and r1 (c[2]) on lanes with t == 0
__device__ __forceinline__ void layer4(const uint32_t (&a)[4][4], const unsigned char* img, float& o0, float& o1) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const float b4 = reinterpret_cast<const float*>(img + OFF_B)[192];
  float c[4] = {b4, b4, b4, b4};
  const int row = OFF_W4T + g * STR * 2;
#pragma unroll
  for (int s = 0; s < 4; ++s)
    mma(c, a[s], ld32(img, row + (16 * s + 2 * t) * 2), ld32(img, row + (16 * s + 8 + 2 * t) * 2));
  o0 = c[0];
  o1 = c[2];
}

// ---- inference, one 16-row tile at a time: each 8-column output tile goes
// through SiLU into the next layer's A fragments as soon as its four k-steps
// are done, so one 4-register accumulator is live instead of a layer's 32.
__device__ __forceinline__ void silu_into(const float (&c)[4], int j, uint32_t (&a)[4][4]) {
  a[j >> 1][(j & 1) * 2] = silu2_half(c[0], c[1]);
  a[j >> 1][(j & 1) * 2 + 1] = silu2_half(c[2], c[3]);
}

// Four 8x8 BF16 matrices from shared memory in one instruction: lanes 8m..8m+7
// give the row addresses of matrix m (16-byte rows), and lane 4g + t receives
// row g, columns 2t and 2t + 1 of each, which is an mma.sync B fragment when
// the rows are output units and the columns 8 consecutive k.
__device__ __forceinline__ void ldsm_x4(const unsigned char* p, uint32_t& r0, uint32_t& r1, uint32_t& r2,
                                        uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(static_cast<uint32_t>(__cvta_generic_to_shared(p))));
}

__device__ __forceinline__ void layer1_act(float z0, float z1, float z2, int tile, const unsigned char* img,
                                           uint32_t (&o)[4][4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int r0 = 16 * tile + g, r1 = r0 + 8;
  const float a00 = __shfl_sync(0xffffffffu, z0, r0), a01 = __shfl_sync(0xffffffffu, z1, r0);
  const float a02 = __shfl_sync(0xffffffffu, z2, r0);
  const float a10 = __shfl_sync(0xffffffffu, z0, r1), a11 = __shfl_sync(0xffffffffu, z1, r1);
  const float a12 = __shfl_sync(0xffffffffu, z2, r1);
  const uint32_t a[4] = {(t == 0) ? pack(a00, a01) : (t == 1) ? pack(a02, 0.0f) : 0u,
                         (t == 0) ? pack(a10, a11) : (t == 1) ? pack(a12, 0.0f) : 0u, 0u, 0u};
  const float* bias = reinterpret_cast<const float*>(img + OFF_B);
  // lanes 0-15 address tile j (k 0-7, 8-15), lanes 16-31 tile j + 1
  const unsigned char* wl = img + OFF_W1T + ((lane & 7) + 8 * (lane >> 4)) * STR1 * 2 + ((lane >> 3) & 1) * 16;
#pragma unroll
  for (int j = 0; j < 8; j += 2) {
    const float2 b0 = *reinterpret_cast<const float2*>(bias + 8 * j + 2 * t);
    const float2 b1 = *reinterpret_cast<const float2*>(bias + 8 * j + 8 + 2 * t);
    float c0[4] = {b0.x, b0.y, b0.x, b0.y}, c1[4] = {b1.x, b1.y, b1.x, b1.y};
    uint32_t w0, w1, v0, v1;
    ldsm_x4(wl + (8 * j) * STR1 * 2, w0, w1, v0, v1);
    mma_pure(c0, a, w0, w1);
    mma_pure(c1, a, v0, v1);
    silu_into(c0, j, o);
    silu_into(c1, j + 1, o);
  }
}

// 64 -> 64 for one tile; two output tiles (j, j + 1) at a time give two
// independent accumulator chains, and each ldmatrix brings the B fragments of
// two k-steps (lane L addresses row L % 8 of the tile, k offset 8 (L / 8)).
__device__ __forceinline__ void layer64_act(const uint32_t (&a)[4][4], const unsigned char* img, int off_wt,
                                            const float* bias, uint32_t (&o)[4][4]) {
  const int lane = threadIdx.x & 31, t = lane & 3;
  const unsigned char* wl = img + off_wt + (lane & 7) * STR * 2 + (lane >> 3) * 16;
#pragma unroll
  for (int j = 0; j < 8; j += 2) {
    const float2 b0 = *reinterpret_cast<const float2*>(bias + 8 * j + 2 * t);
    const float2 b1 = *reinterpret_cast<const float2*>(bias + 8 * j + 8 + 2 * t);
    float c0[4] = {b0.x, b0.y, b0.x, b0.y}, c1[4] = {b1.x, b1.y, b1.x, b1.y};
#pragma unroll
    for (int s = 0; s < 4; s += 2) {
      uint32_t w0, w1, w2, w3, v0, v1, v2, v3;
      ldsm_x4(wl + (8 * j) * STR * 2 + s * 32, w0, w1, w2, w3);
      ldsm_x4(wl + (8 * j + 8) * STR * 2 + s * 32, v0, v1, v2, v3);
      mma_pure(c0, a[s], w0, w1);
      mma_pure(c1, a[s], v0, v1);
      mma_pure(c0, a[s + 1], w2, w3);
      mma_pure(c1, a[s + 1], v2, v3);
    }
    silu_into(c0, j, o);
    silu_into(c1, j + 1, o);
  }
}

// The MLP for the warp's 32 points (inference image, SiLU through silu2_half): lane
// L's input (z0, z1, z2), its output returned. Must be called by all 32 lanes together.
__device__ __forceinline__ float forward_warp(float z0, float z1, float z2, const unsigned char* img) {
  const int lane = threadIdx.x & 31;
  const float* bias = reinterpret_cast<const float*>(img + OFF_B);
  float mine = 0.0f;
#pragma unroll 1
  for (int tile = 0; tile < 2; ++tile) {
    uint32_t x[4][4], y[4][4];
    layer1_act(z0, z1, z2, tile, img, x);
    layer64_act(x, img, OFF_W2T, bias + 64, y);
    layer64_act(y, img, OFF_W3T, bias + 128, x);
    // 64 -> 1 (one 8-column tile, column 0 used)
    const float b4 = bias[192];
    float c[4] = {b4, b4, b4, b4};
    const unsigned char* wl = img + OFF_W4T + (lane & 7) * STR * 2 + (lane >> 3) * 16;
#pragma unroll
    for (int s = 0; s < 4; s += 2) {
      uint32_t w0, w1, w2, w3;
      ldsm_x4(wl + s * 32, w0, w1, w2, w3);
      mma_pure(c, x[s], w0, w1);
      mma_pure(c, x[s + 1], w2, w3);
    }
    // row (lane & 15) of this tile sits on lane 4 (lane & 7), in c[0] (rows 0-7) or c[2] (rows 8-15)
    const int src = (lane & 7) * 4;
    const float v0 = __shfl_sync(0xffffffffu, c[0], src), v1 = __shfl_sync(0xffffffffu, c[2], src);
    if ((lane >> 4) == tile) mine = ((lane & 15) < 8) ? v0 : v1;
  }
  return mine;
}

}  // namespace mlp
}  // namespace cc
