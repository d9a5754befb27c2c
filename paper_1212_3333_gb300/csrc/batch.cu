// Batched multi-view rendering: one persistent launch marches many views of one dataset.
//
// The views' pixel tiles form one work queue (items in view order, tiles row-major within
// a view).  Every block pops a tile with one atomic, builds that view's ray arguments in
// shared memory and marches the tile's pixels with the same per-pixel code as the
// single-view kernel, so each view's image is bit-identical to its own amr_render.  Up to
// eight transfer functions are read from global memory (L1-cached); their prefix counts of
// non-transparent entries are staged in shared memory once per block.  With schedule 3
// each warp marches its rays with the deferred-shading loop instead of the per-ray loop.
// The view table travels in the kernel's parameter block, so a call is one memset and one
// launch and can be captured in a CUDA graph.  The paper renders one view per pass; batching is an
// addition for throughput over many small and large views.
#include <cuda_runtime.h>

#include "ctx.h"
#include "march_launch.cuh"

namespace amr {

namespace {

// DEFER: the warp-synchronous march with deferred shading (schedule 3) instead of the
// per-ray loop; each warp's queue area follows the transfer functions in shared memory.
template <int ST, int SHADE, int TW, int TH, bool DEFER>
__global__ void __launch_bounds__(TW * TH,
                                  (128 * (DEFER ? AMR_MIN_BLOCKS_DEFERRED : kMinBlocks<SHADE>)) /
                                      (TW * TH))
    batch_kernel(const __grid_constant__ BatchArgs B) {
  const RenderArgs& A = B.A;
  extern __shared__ float4 smem[];
  const int tf_n = A.tf_n;
  // the transfer functions are read where they are (global memory, cached in L1): staging
  // all of them in every block took up to 160 KB of an SM's shared memory away from the
  // L1 cache that serves the brick reads; only their prefix counts are staged
  int* s_nz = reinterpret_cast<int*>(smem);                        // [n_tf][tf_n + 1]
  __shared__ RayArgs s_ray;
  __shared__ int s_item, s_tf_idx, s_w, s_h, s_item0, s_tiles_x;
  __shared__ long long s_out;
  const int tid = threadIdx.x + TW * threadIdx.y;
  if (tid < B.n_tf) {
    int acc = 0;
    int* nz = s_nz + tid * (tf_n + 1);
    const float4* tf = A.tf + tid * tf_n;
    nz[0] = 0;
    for (int k = 0; k < tf_n; ++k) {
      acc += __ldg(&tf[k].w) != 0.0f ? 1 : 0;
      nz[k + 1] = acc;
    }
  }
  if (tid == 0) s_ray = A.ray;
  __syncthreads();

  unsigned nsamp = 0;
  unsigned long long status = 0;
  const int rpt = B.rays_per_thread;
  // each pass consumes one queue item, so the loop ends after at most n_items passes
  for (;;) {
    if (tid == 0) {
      const unsigned long long q = atomicAdd(A.counters + kQueueCounter, 1ull);
      const int item = q < (unsigned long long)B.n_items ? (int)q : B.n_items;
      if (item < B.n_items) {
        int lo = 0, hi = B.n_views - 1;  // last view whose first item is <= item
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (B.v[mid].item0 <= item) lo = mid;
          else hi = mid - 1;
        }
        const BatchView& bv = B.v[lo];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          s_ray.eye[a] = bv.eye[a];
          s_ray.fwd[a] = bv.fwd[a];
          s_ray.right[a] = bv.right[a];
          s_ray.up[a] = bv.up[a];
        }
        s_ray.tan_half_fov_y = bv.tan_half_fov_y;
        s_ray.width = bv.width;
        s_ray.height = bv.height;
        s_ray.row0 = 0;
        s_ray.rows = bv.height;
        s_ray.lod_scale = bv.lod_scale;
        s_ray.lod_scale_f = bv.lod_scale_f;
        s_tf_idx = bv.tf;
        s_w = bv.width;
        s_h = bv.height;
        s_item0 = bv.item0;
        s_tiles_x = bv.tiles_x;
        s_out = bv.out;
      }
      s_item = item;
    }
    __syncthreads();
    const int item = s_item;
    if (item >= B.n_items) break;
    const int t = item - s_item0;
    const int tx = t % s_tiles_x, ty = t / s_tiles_x;
    const int W = s_w, H = s_h;
    const int i = tx * TW + (int)threadIdx.x;
    const float4* tf = A.tf + s_tf_idx * tf_n;
    const int* nz = s_nz + s_tf_idx * (tf_n + 1);
    float4* out = A.out + s_out;
    for (int r = 0; r < rpt; ++r) {
      const int j = (ty * rpt + r) * TH + (int)threadIdx.y;
      if constexpr (DEFER) {
        // every lane of the warp takes part, with or without a pixel
        const size_t area = ((size_t)B.n_tf * (tf_n + 1) * sizeof(int) + 15) & ~(size_t)15;
        DeferArea& Q = reinterpret_cast<DeferArea*>(reinterpret_cast<char*>(smem) + area)[tid >> 5];
        const bool act = i < W && j < H;
        const float4 c = march_deferred<ST, SHADE>(A, s_ray, i, j, act, tf, nz, Q, nsamp, status);
        if (act) out[(size_t)j * W + i] = c;
      } else if (i < W && j < H) {
        RayF rf;
        out[(size_t)j * W + i] = march_ray<ST, 1, SHADE>(A, s_ray, i, j, tf, nz, rf, nsamp, status);
      }
    }
    __syncthreads();  // s_ray and the tile fields are rewritten by the next pop
  }
  const unsigned total = __reduce_add_sync(0xffffffffu, nsamp);
  if ((tid & 31) == 0 && total) atomicAdd(A.counters, (unsigned long long)total);
  if (status) atomicOr(A.counters + 1, status);
}

template <int ST, int SHADE, int TW, int TH, bool DEFER>
amr_status launch_shape(amr_ctx* c, const BatchArgs& b, int blocks_per_sm, cudaStream_t s) {
  auto k = batch_kernel<ST, SHADE, TW, TH, DEFER>;
  constexpr int kThreads = TW * TH;
  size_t smem = (size_t)b.n_tf * (b.A.tf_n + 1) * sizeof(int);
  if (DEFER) smem = ((smem + 15) & ~(size_t)15) + (kThreads / 32) * sizeof(DeferArea);
  cudaError_t e = cudaSuccess;
  if (smem > 48 * 1024)
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int dev = 0, sms = 0, occ = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = fit_carveout(k, smem, kThreads, occ);
  if (e != cudaSuccess) return fail(c, AMR_ERR_CUDA, std::string("batch launch setup: ") + cudaGetErrorString(e));
  const int per_sm = blocks_per_sm > 0 ? std::min(blocks_per_sm, std::max(occ, 1)) : std::max(occ, 1);
  const int grid = std::max(1, std::min(sms * per_sm, b.n_items));
  k<<<grid, dim3(TW, TH), smem, s>>>(b);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(c, AMR_ERR_CUDA, std::string("batch launch: ") + cudaGetErrorString(e));
  return AMR_OK;
}

template <int ST, int SHADE, bool DEFER>
amr_status launch_st(amr_ctx* c, const BatchArgs& b, const amr_batch_config& cfg, cudaStream_t s) {
  if (cfg.tile_w == 8 && cfg.tile_h == 8)
    return launch_shape<ST, SHADE, 8, 8, DEFER>(c, b, cfg.blocks_per_sm, s);
  if (cfg.tile_w == 16 && cfg.tile_h == 8)
    return launch_shape<ST, SHADE, 16, 8, DEFER>(c, b, cfg.blocks_per_sm, s);
  if (cfg.tile_w == 16 && cfg.tile_h == 16)
    return launch_shape<ST, SHADE, 16, 16, DEFER>(c, b, cfg.blocks_per_sm, s);
  return fail(c, AMR_ERR_ARG, "batch tile must be 8x8, 16x8 or 16x16");
}

}  // namespace

amr_status launch_batch(amr_ctx* c, const BatchArgs& b, int storage, int shade, int schedule,
                        const amr_batch_config& cfg, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const bool mx = (shade & kShadeMaxBit) != 0;  // the stencil-maximum test
  shade &= ~kShadeMaxBit;
  if (storage != ST_PTR) return fail(c, AMR_ERR_ARG, "batched rendering needs the ptr storage (FP32)");
  if (schedule == 3) {
    if (shade == 1) return mx ? launch_st<ST_PTR, 1 | kShadeMaxBit, true>(c, b, cfg, s)
                              : launch_st<ST_PTR, 1, true>(c, b, cfg, s);
    if (shade == 2) return mx ? launch_st<ST_PTR, 2 | kShadeMaxBit, true>(c, b, cfg, s)
                              : launch_st<ST_PTR, 2, true>(c, b, cfg, s);
    return fail(c, AMR_ERR_ARG, "deferred shading renders with shade = 1");
  }
  if (mx) {
    if (shade == 0) return launch_st<ST_PTR, kShadeMaxBit, false>(c, b, cfg, s);
    if (shade == 1) return launch_st<ST_PTR, 1 | kShadeMaxBit, false>(c, b, cfg, s);
    return launch_st<ST_PTR, 2 | kShadeMaxBit, false>(c, b, cfg, s);
  }
  if (shade == 0) return launch_st<ST_PTR, 0, false>(c, b, cfg, s);
  if (shade == 1) return launch_st<ST_PTR, 1, false>(c, b, cfg, s);
  return launch_st<ST_PTR, 2, false>(c, b, cfg, s);
}

}  // namespace amr
