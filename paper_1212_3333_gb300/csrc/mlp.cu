// MLP kernels of the learned segment proposal: packing, tensor-core inference, training
// (loss + gradient) and Adam.  Declarations and contracts: include/amr.h.
#include <cstring>

#include "ctx.h"
#include "mlp.cuh"

static_assert(amr::kPackBytes == AMR_MLP_PACKED_BYTES, "packed MLP image size");
static_assert(amr::kMlpParams == AMR_MLP_PARAMS, "MLP parameter count");
static_assert(amr::kMlpIn == AMR_MLP_FEATURES, "MLP feature count");

namespace amr {
namespace {

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// FP32 master parameters -> inference image (BF16 weights, padded rows, FP32 biases)
__global__ void pack_kernel(const float* __restrict__ p, unsigned char* __restrict__ out) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  __nv_bfloat16* w1 = reinterpret_cast<__nv_bfloat16*>(out + kPackW1);
  __nv_bfloat16* w2 = reinterpret_cast<__nv_bfloat16*>(out + kPackW2);
  __nv_bfloat16* w3 = reinterpret_cast<__nv_bfloat16*>(out + kPackW3);
  __nv_bfloat16* w4 = reinterpret_cast<__nv_bfloat16*>(out + kPackW4);
  float* b = reinterpret_cast<float*>(out + kPackB);
  if (tid < kMlpH * kStride1) {
    const int o = tid / kStride1, i = tid % kStride1;
    w1[tid] = __float2bfloat16_rn(i < kMlpIn ? p[kOffW1 + o * kMlpIn + i] : 0.0f);
  }
  if (tid < kMlpH * kStrideH) {
    const int o = tid / kStrideH, i = tid % kStrideH;
    w2[tid] = __float2bfloat16_rn(i < kMlpH ? p[kOffW2 + o * kMlpH + i] : 0.0f);
    w3[tid] = __float2bfloat16_rn(i < kMlpH ? p[kOffW3 + o * kMlpH + i] : 0.0f);
  }
  if (tid < 8 * kStrideH) {
    const int o = tid / kStrideH, i = tid % kStrideH;
    w4[tid] = __float2bfloat16_rn(o == 0 && i < kMlpH ? p[kOffW4 + i] : 0.0f);
  }
  if (tid < 3 * kMlpH + 4) {
    float v = 0.0f;
    if (tid < kMlpH) v = p[kOffB1 + tid];
    else if (tid < 2 * kMlpH) v = p[kOffB2 + tid - kMlpH];
    else if (tid < 3 * kMlpH) v = p[kOffB3 + tid - 2 * kMlpH];
    else if (tid == 3 * kMlpH) v = p[kOffB4];
    b[tid] = v;
  }
}

// Inference on n rows of 12 features through the same warp routine the march uses.
__global__ void __launch_bounds__(128) forward_kernel(const unsigned char* __restrict__ packed,
                                                      const float* __restrict__ x, int64_t n,
                                                      float* __restrict__ y) {
  extern __shared__ __align__(16) unsigned char sm[];
  unsigned char* wsm = sm;
  for (int k = threadIdx.x; k < kPackBytes / 16; k += blockDim.x)
    reinterpret_cast<uint4*>(wsm)[k] = reinterpret_cast<const uint4*>(packed)[k];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __nv_bfloat16* xs = reinterpret_cast<__nv_bfloat16*>(sm + kPackBytes) + warp * 32 * kStride1;
  float* ys = reinterpret_cast<float*>(sm + kPackBytes + 4 * 32 * kStride1 * 2) + warp * 32;
  const int64_t tiles = (n + 31) / 32;
  for (int64_t tile = (int64_t)blockIdx.x * 4 + warp; tile < tiles; tile += (int64_t)gridDim.x * 4) {
    const int64_t r = tile * 32 + lane;
#pragma unroll
    for (int k = 0; k < kMlpInPad; ++k)
      xs[lane * kStride1 + k] = __float2bfloat16_rn(r < n && k < kMlpIn ? x[r * kMlpIn + k] : 0.0f);
    __syncwarp();
    const float v = mlp_forward_warp(wsm, xs, ys, lane);
    if (r < n) y[r] = v;
    __syncwarp();
  }
}

// Loss and gradient, one row per thread over tiles of 128 rows.  The forward rounds
// weights and activations to BF16 exactly as inference does; everything else is FP32.
// Shared memory: weights (9217 floats), activations A1..A3 and one delta buffer
// (128 x 64 floats each), features (128 x 12), output deltas (128).
constexpr int kGradThreads = 128;
constexpr int kRow = kMlpH + 1;    // activation row stride: per-thread rows hit distinct banks
constexpr int kXRow = kMlpIn + 1;  // feature row stride
constexpr size_t kGradSmem =
    (size_t)(kMlpParams + 4 * kGradThreads * kRow + kGradThreads * kXRow + kGradThreads) * 4;

__global__ void __launch_bounds__(kGradThreads, 1)
    grad_kernel(const float* __restrict__ params, const float* __restrict__ x,
                const float* __restrict__ tgt, int64_t n_total, int64_t first, int64_t n,
                int64_t perm_a, int64_t perm_b, float* __restrict__ partial,
                float* __restrict__ loss_part) {
  extern __shared__ __align__(16) float fs[];
  float* W = fs;                                        // BF16-rounded weights, FP32 biases
  float* A1 = W + kMlpParams;
  float* A2 = A1 + kGradThreads * kRow;
  float* A3 = A2 + kGradThreads * kRow;
  float* D = A3 + kGradThreads * kRow;
  float* X = D + kGradThreads * kRow;
  float* d4 = X + kGradThreads * kXRow;
  const int tid = threadIdx.x;
  for (int k = tid; k < kMlpParams; k += kGradThreads) {
    const bool bias = (k >= kOffB1 && k < kOffW2) || (k >= kOffB2 && k < kOffW3) ||
                      (k >= kOffB3 && k < kOffW4) || k == kOffB4;
    W[k] = bias ? params[k] : bf16r(params[k]);
  }
  __syncthreads();
  // gradient entries owned by this thread: k = tid + 128 j
  constexpr int kOwn = (kMlpParams + kGradThreads - 1) / kGradThreads;
  float g[kOwn];
#pragma unroll
  for (int j = 0; j < kOwn; ++j) g[j] = 0.0f;
  float loss = 0.0f;
  const float inv_n = 1.0f / (float)n;
  const int64_t tiles = (n + kGradThreads - 1) / kGradThreads;
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t rb = tile * kGradThreads + tid;  // row of the batch
    const bool valid = rb < n;
    const int64_t r = valid ? (perm_a * (first + rb) + perm_b) % n_total : 0;  // dataset row
    // ---- forward (this thread's row)
    float xr[kMlpIn];
#pragma unroll
    for (int i = 0; i < kMlpIn; ++i) {
      xr[i] = valid ? bf16r(x[r * kMlpIn + i]) : 0.0f;
      X[tid * kXRow + i] = xr[i];
    }
    for (int o = 0; o < kMlpH; ++o) {
      float s = W[kOffB1 + o];
#pragma unroll
      for (int i = 0; i < kMlpIn; ++i) s = fmaf(W[kOffW1 + o * kMlpIn + i], xr[i], s);
      A1[tid * kRow + o] = bf16r(fmaxf(s, 0.0f));
    }
    for (int o = 0; o < kMlpH; ++o) {
      float s = W[kOffB2 + o];
      for (int i = 0; i < kMlpH; ++i) s = fmaf(W[kOffW2 + o * kMlpH + i], A1[tid * kRow + i], s);
      A2[tid * kRow + o] = bf16r(fmaxf(s, 0.0f));
    }
    for (int o = 0; o < kMlpH; ++o) {
      float s = W[kOffB3 + o];
      for (int i = 0; i < kMlpH; ++i) s = fmaf(W[kOffW3 + o * kMlpH + i], A2[tid * kRow + i], s);
      A3[tid * kRow + o] = bf16r(fmaxf(s, 0.0f));
    }
    float z4 = W[kOffB4];
    for (int i = 0; i < kMlpH; ++i) z4 = fmaf(W[kOffW4 + i], A3[tid * kRow + i], z4);
    const float y = 1.0f / (1.0f + expf(-z4));
    const float t = valid ? tgt[r] : 0.0f;
    if (valid) {
      const float sp = z4 > 0.0f ? z4 + log1pf(expf(-z4)) : log1pf(expf(z4));
      loss += sp - t * z4;
    }
    d4[tid] = valid ? (y - t) * inv_n : 0.0f;
    // ---- output-layer delta into hidden layer 3
    for (int o = 0; o < kMlpH; ++o)
      D[tid * kRow + o] = A3[tid * kRow + o] > 0.0f ? d4[tid] * W[kOffW4 + o] : 0.0f;
    __syncthreads();
    // ---- weight gradients of layers 4 and 3 (sums over the tile's rows)
#pragma unroll
    for (int j = 0; j < kOwn; ++j) {
      const int k = tid + kGradThreads * j;
      float s = 0.0f;
      if (k >= kOffW4 && k < kOffB4) {
        const int i = k - kOffW4;
        for (int q = 0; q < kGradThreads; ++q) s = fmaf(d4[q], A3[q * kRow + i], s);
      } else if (k == kOffB4) {
        for (int q = 0; q < kGradThreads; ++q) s += d4[q];
      } else if (k >= kOffW3 && k < kOffB3) {
        const int o = (k - kOffW3) / kMlpH, i = (k - kOffW3) % kMlpH;
        for (int q = 0; q < kGradThreads; ++q) s = fmaf(D[q * kRow + o], A2[q * kRow + i], s);
      } else if (k >= kOffB3 && k < kOffW4) {
        const int o = k - kOffB3;
        for (int q = 0; q < kGradThreads; ++q) s += D[q * kRow + o];
      } else {
        continue;
      }
      g[j] += s;
    }
    __syncthreads();
    // ---- delta into hidden layer 2 (reuses A3's buffer)
    for (int o = 0; o < kMlpH; ++o) {
      float s = 0.0f;
      for (int k = 0; k < kMlpH; ++k) s = fmaf(D[tid * kRow + k], W[kOffW3 + k * kMlpH + o], s);
      A3[tid * kRow + o] = A2[tid * kRow + o] > 0.0f ? s : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kOwn; ++j) {
      const int k = tid + kGradThreads * j;
      float s = 0.0f;
      if (k >= kOffW2 && k < kOffB2) {
        const int o = (k - kOffW2) / kMlpH, i = (k - kOffW2) % kMlpH;
        for (int q = 0; q < kGradThreads; ++q) s = fmaf(A3[q * kRow + o], A1[q * kRow + i], s);
      } else if (k >= kOffB2 && k < kOffW3) {
        const int o = k - kOffB2;
        for (int q = 0; q < kGradThreads; ++q) s += A3[q * kRow + o];
      } else {
        continue;
      }
      g[j] += s;
    }
    __syncthreads();
    // ---- delta into hidden layer 1 (into D)
    for (int o = 0; o < kMlpH; ++o) {
      float s = 0.0f;
      for (int k = 0; k < kMlpH; ++k) s = fmaf(A3[tid * kRow + k], W[kOffW2 + k * kMlpH + o], s);
      D[tid * kRow + o] = A1[tid * kRow + o] > 0.0f ? s : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kOwn; ++j) {
      const int k = tid + kGradThreads * j;
      float s = 0.0f;
      if (k >= kOffW1 && k < kOffB1) {
        const int o = (k - kOffW1) / kMlpIn, i = (k - kOffW1) % kMlpIn;
        for (int q = 0; q < kGradThreads; ++q) s = fmaf(D[q * kRow + o], X[q * kXRow + i], s);
      } else if (k >= kOffB1 && k < kOffW2) {
        const int o = k - kOffB1;
        for (int q = 0; q < kGradThreads; ++q) s += D[q * kRow + o];
      } else {
        continue;
      }
      g[j] += s;
    }
    __syncthreads();
  }
  // this block's partial sums, reduced over the blocks in a fixed order by reduce_kernel
  // (no atomics: the gradient is the same bit for bit on every call)
  float* part = partial + (size_t)blockIdx.x * kMlpParams;
#pragma unroll
  for (int j = 0; j < kOwn; ++j) {
    const int k = tid + kGradThreads * j;
    if (k < kMlpParams) part[k] = g[j];
  }
  for (int off = 16; off > 0; off >>= 1) loss += __shfl_down_sync(0xffffffffu, loss, off);
  __shared__ float wl[kGradThreads / 32];
  if ((tid & 31) == 0) wl[tid >> 5] = loss;
  __syncthreads();
  if (tid == 0) {
    float s = 0.0f;
    for (int w = 0; w < kGradThreads / 32; ++w) s += wl[w];
    loss_part[blockIdx.x] = s * inv_n;
  }
}

// grad[k] = sum of the blocks' partials in block order; loss likewise (thread kMlpParams).
__global__ void reduce_kernel(const float* __restrict__ partial, const float* __restrict__ loss_part,
                              int blocks, float* __restrict__ grad, float* __restrict__ loss) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < kMlpParams) {
    float s = 0.0f;
    for (int b = 0; b < blocks; ++b) s += partial[(size_t)b * kMlpParams + k];
    grad[k] = s;
  } else if (k == kMlpParams) {
    float s = 0.0f;
    for (int b = 0; b < blocks; ++b) s += loss_part[b];
    loss[0] = s;
  }
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, int n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float gk = g[k];
  const float mk = fmaf(b1, m[k], (1.0f - b1) * gk);
  const float vk = fmaf(b2, v[k], (1.0f - b2) * gk * gk);
  m[k] = mk;
  v[k] = vk;
  p[k] -= lr * (mk * c1) / (sqrtf(vk * c2) + eps);
}

thread_local std::string g_mlp_error;

amr_status mlp_fail(amr_status s, const std::string& m) {
  g_mlp_error = m;
  return s;
}

}  // namespace

const char* mlp_last_error() { return g_mlp_error.c_str(); }

}  // namespace amr

using namespace amr;

extern "C" {

amr_status amr_mlp_pack(const float* params_dev, void* packed_dev, void* stream) {
  if (!params_dev || !packed_dev || ((uintptr_t)packed_dev & 15))
    return mlp_fail(AMR_ERR_ARG, "params / packed buffer NULL or packed not 16-byte aligned");
  pack_kernel<<<(kMlpH * kStrideH + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
      params_dev, (unsigned char*)packed_dev);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? AMR_OK : mlp_fail(AMR_ERR_CUDA, cudaGetErrorString(e));
}

amr_status amr_mlp_forward(const void* packed_dev, const float* x_dev, int64_t n, float* y_dev,
                           void* stream) {
  if (!packed_dev || !x_dev || !y_dev || n < 0 || ((uintptr_t)packed_dev & 15))
    return mlp_fail(AMR_ERR_ARG, "bad MLP forward arguments");
  if (n == 0) return AMR_OK;
  const size_t smem = kPackBytes + 4 * 32 * kStride1 * 2 + 4 * 32 * 4;
  const int64_t tiles = (n + 31) / 32;
  const int blocks = (int)std::min<int64_t>((tiles + 3) / 4, 152 * 8);
  forward_kernel<<<blocks, 128, smem, (cudaStream_t)stream>>>((const unsigned char*)packed_dev,
                                                              x_dev, n, y_dev);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? AMR_OK : mlp_fail(AMR_ERR_CUDA, cudaGetErrorString(e));
}

amr_status amr_mlp_loss_grad(const float* params_dev, const float* x_dev, const float* t_dev,
                             int64_t n_total, int64_t first, int64_t n, int64_t perm_a,
                             int64_t perm_b, float* grad_dev, float* loss_dev, float* scratch_dev,
                             void* stream) {
  if (!params_dev || !x_dev || !t_dev || !grad_dev || !loss_dev || !scratch_dev || n <= 0 ||
      n_total <= 0 ||
      first < 0 || perm_a <= 0 || perm_b < 0 || perm_a >= ((int64_t)1 << 31) ||
      n_total >= ((int64_t)1 << 31) || first + n >= ((int64_t)1 << 32))
    return mlp_fail(AMR_ERR_ARG, "bad MLP gradient arguments");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaFuncSetAttribute(grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kGradSmem);
  if (e != cudaSuccess) return mlp_fail(AMR_ERR_CUDA, cudaGetErrorString(e));
  const int64_t tiles = (n + kGradThreads - 1) / kGradThreads;
  const int blocks = (int)std::min<int64_t>(tiles, AMR_MLP_GRAD_BLOCKS);
  float* partial = scratch_dev;                                        // [blocks][params]
  float* loss_part = scratch_dev + (size_t)AMR_MLP_GRAD_BLOCKS * kMlpParams;  // [blocks]
  grad_kernel<<<blocks, kGradThreads, kGradSmem, st>>>(params_dev, x_dev, t_dev, n_total, first,
                                                       n, perm_a, perm_b % n_total, partial,
                                                       loss_part);
  reduce_kernel<<<(kMlpParams + 1 + 255) / 256, 256, 0, st>>>(partial, loss_part, blocks, grad_dev,
                                                             loss_dev);
  e = cudaGetLastError();
  return e == cudaSuccess ? AMR_OK : mlp_fail(AMR_ERR_CUDA, cudaGetErrorString(e));
}

amr_status amr_mlp_adam(float* params_dev, const float* grad_dev, float* m_dev, float* v_dev,
                        float lr, float beta1, float beta2, float eps, int32_t step, void* stream) {
  if (!params_dev || !grad_dev || !m_dev || !v_dev || step < 1)
    return mlp_fail(AMR_ERR_ARG, "bad Adam arguments");
  const float c1 = 1.0f / (1.0f - powf(beta1, (float)step));
  const float c2 = 1.0f / (1.0f - powf(beta2, (float)step));
  adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
      params_dev, grad_dev, m_dev, v_dev, kMlpParams, lr, beta1, beta2, eps, c1, c2);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? AMR_OK : mlp_fail(AMR_ERR_CUDA, cudaGetErrorString(e));
}

}  // extern "C"
