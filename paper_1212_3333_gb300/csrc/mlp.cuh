// Learned segment proposal: a 12-64-64-64-1 MLP (ReLU hidden layers, sigmoid output) that
// predicts a segment's opacity contribution (1 - A_in) alpha_seg = A_out - A_in from
// features the march knows before sampling the segment.  The paper has no counterpart.
//
// Parameters (FP32 master, 9217 floats, in this order): W1[64][12], b1[64], W2[64][64],
// b2[64], W3[64][64], b3[64], W4[1][64], b4[1]  (W[out][in], row-major).
//
// Inference runs on the tensor cores with mma.sync.m16n8k16 BF16 x BF16 -> FP32: a warp
// evaluates its 32 lanes' current segments as a 32-row tile.  A layer's FP32 accumulator
// fragments (bias, ReLU, rounded to BF16) are, register for register, the A fragments of
// the next layer, so activations never leave registers.  Weights live in shared memory as
// BF16 rows padded to a 36-word stride (conflict-free B-fragment loads).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace amr {

constexpr int kMlpIn = 12;
constexpr int kMlpInPad = 16;
constexpr int kMlpH = 64;
constexpr int kMlpParams = kMlpH * kMlpIn + kMlpH + 2 * (kMlpH * kMlpH + kMlpH) + kMlpH + 1;  // 9217
// offsets into the FP32 parameter vector
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kMlpH * kMlpIn;
constexpr int kOffW2 = kOffB1 + kMlpH, kOffB2 = kOffW2 + kMlpH * kMlpH;
constexpr int kOffW3 = kOffB2 + kMlpH, kOffB3 = kOffW3 + kMlpH * kMlpH;
constexpr int kOffW4 = kOffB3 + kMlpH, kOffB4 = kOffW4 + kMlpH;

// packed inference image (BF16 weights with padded rows, FP32 biases); copied verbatim
// into shared memory by the kernels
constexpr int kStride1 = kMlpInPad + 8;  // bf16 per row of W1
constexpr int kStrideH = kMlpH + 8;      // bf16 per row of W2, W3, W4
constexpr int kPackW1 = 0;                                // [64][kStride1]
constexpr int kPackW2 = kPackW1 + kMlpH * kStride1 * 2;   // bytes
constexpr int kPackW3 = kPackW2 + kMlpH * kStrideH * 2;
constexpr int kPackW4 = kPackW3 + kMlpH * kStrideH * 2;   // [8][kStrideH], rows 1..7 zero
constexpr int kPackB = kPackW4 + 8 * kStrideH * 2;        // float b1[64] b2[64] b3[64] b4[4]
constexpr int kPackBytes = kPackB + (3 * kMlpH + 4) * 4;  // multiple of 16

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// One hidden layer for the warp's 32 rows: acc = bias + A * W^T (ReLU follows).  The
// accumulators start at the bias, so the epilogue is only ReLU and packing.
// a: [2 m-tiles][KS k-steps][4] packed BF16 A fragments; W: smem rows of `stride` bf16.
template <int KS>
__device__ __forceinline__ void mlp_layer(const uint32_t (&a)[2][KS][4], const unsigned char* smem,
                                          int woff, int stride, const float* bias, int lane,
                                          float (&acc)[2][8][4]) {
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int n = 0; n < 8; ++n) {
    const float2 b = *reinterpret_cast<const float2*>(bias + 8 * n + 2 * t);
#pragma unroll
    for (int m = 0; m < 2; ++m) {
      acc[m][n][0] = b.x;
      acc[m][n][1] = b.y;
      acc[m][n][2] = b.x;
      acc[m][n][3] = b.y;
    }
  }
#pragma unroll
  for (int n = 0; n < 8; ++n) {
    const uint32_t* row =
        reinterpret_cast<const uint32_t*>(smem + woff + (size_t)(8 * n + g) * stride * 2);
#pragma unroll
    for (int s = 0; s < KS; ++s) {
      const uint32_t b0 = row[8 * s + t];
      const uint32_t b1 = row[8 * s + 4 + t];
#pragma unroll
      for (int m = 0; m < 2; ++m) mma_bf16(acc[m][n], a[m][s], b0, b1);
    }
  }
}

// ReLU of the accumulators, rounded to BF16 and repacked as the next layer's A fragments
// (4 k-steps).  Rounding is monotone and keeps 0, so max(round(x), 0) = round(max(x, 0)):
// the maximum is taken on the packed pairs.
__device__ __forceinline__ uint32_t relu_bf16x2(float lo, float hi) {
  const __nv_bfloat162 v = __hmax2(__floats2bfloat162_rn(lo, hi), __float2bfloat162_rn(0.0f));
  return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ void mlp_relu_pack(const float (&acc)[2][8][4], uint32_t (&a)[2][4][4]) {
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      a[m][s][0] = relu_bf16x2(acc[m][2 * s][0], acc[m][2 * s][1]);
      a[m][s][1] = relu_bf16x2(acc[m][2 * s][2], acc[m][2 * s][3]);
      a[m][s][2] = relu_bf16x2(acc[m][2 * s + 1][0], acc[m][2 * s + 1][1]);
      a[m][s][3] = relu_bf16x2(acc[m][2 * s + 1][2], acc[m][2 * s + 1][3]);
    }
}

// Warp-cooperative forward pass.  xs: this warp's staging rows in shared memory,
// [32][kStride1] bf16, row r = the features of lane r (zero-padded to 16).  All 32 lanes
// must call it together.  Returns the prediction for the calling lane's row.
// An out-of-line call: the pass's accumulator and fragment registers are live only inside
// it, so the learned march around it keeps its ray state in registers (spills 60 -> 16
// bytes per thread; 8 held-out C2 2048^2 views, coarse16 at tau 1e-2: 160.2 -> 154.5 ms).
// Its 152 mma.sync per 32 rows are the bound: about 500 SM cycles per call at full
// throughput (B fragments by ldmatrix instead of 32-bit loads: 526 -> 501, no gain in the
// march).
static __device__ __noinline__ float mlp_forward_warp(const unsigned char* wsm,
                                                      const __nv_bfloat16* xs, float* ys,
                                                      int lane) {
  const int g = lane >> 2, t = lane & 3;
  const float* bias = reinterpret_cast<const float*>(wsm + kPackB);
  uint32_t a1[2][1][4];
#pragma unroll
  for (int m = 0; m < 2; ++m) {
    const uint32_t* r0 = reinterpret_cast<const uint32_t*>(xs + (16 * m + g) * kStride1);
    const uint32_t* r8 = reinterpret_cast<const uint32_t*>(xs + (16 * m + g + 8) * kStride1);
    a1[m][0][0] = r0[t];
    a1[m][0][1] = r8[t];
    a1[m][0][2] = r0[4 + t];
    a1[m][0][3] = r8[4 + t];
  }
  float acc[2][8][4];
  uint32_t a[2][4][4];
  mlp_layer<1>(a1, wsm, kPackW1, kStride1, bias, lane, acc);
  mlp_relu_pack(acc, a);
  mlp_layer<4>(a, wsm, kPackW2, kStrideH, bias + kMlpH, lane, acc);
  mlp_relu_pack(acc, a);
  mlp_layer<4>(a, wsm, kPackW3, kStrideH, bias + 2 * kMlpH, lane, acc);
  mlp_relu_pack(acc, a);
  // output layer: one n-tile whose column 0 is the logit
  const uint32_t* w4 = reinterpret_cast<const uint32_t*>(wsm + kPackW4 + (size_t)g * kStrideH * 2);
  float o[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const uint32_t b0 = w4[8 * s + t], b1 = w4[8 * s + 4 + t];
#pragma unroll
    for (int m = 0; m < 2; ++m) mma_bf16(o[m], a[m][s], b0, b1);
  }
  const float b4 = bias[3 * kMlpH];
  if (t == 0) {
#pragma unroll
    for (int m = 0; m < 2; ++m) {
      ys[16 * m + g] = 1.0f / (1.0f + __expf(-(o[m][0] + b4)));
      ys[16 * m + g + 8] = 1.0f / (1.0f + __expf(-(o[m][2] + b4)));
    }
  }
  __syncwarp();
  const float y = ys[lane];
  __syncwarp();
  return y;
}

// Octahedral encoding of a direction: two coordinates in [-1, 1].
__device__ __forceinline__ void octahedral(float x, float y, float z, float& u, float& v) {
  const float inv = 1.0f / (fabsf(x) + fabsf(y) + fabsf(z));
  x *= inv;
  y *= inv;
  z *= inv;
  if (z < 0.0f) {
    const float ox = (1.0f - fabsf(y)) * (x >= 0.0f ? 1.0f : -1.0f);
    const float oy = (1.0f - fabsf(x)) * (y >= 0.0f ? 1.0f : -1.0f);
    x = ox;
    y = oy;
  }
  u = x;
  v = y;
}

}  // namespace amr
