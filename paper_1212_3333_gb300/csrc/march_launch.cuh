// Template launcher shared by the per-storage translation units.
#pragma once
#include <algorithm>

#include "ctx.h"
#include "march.cuh"
#include "march_deferred.cuh"
#include "march_persist.cuh"
#include "march_wave.cuh"

namespace amr {

// Shared-memory carveout: the smallest split that still holds as many blocks per SM as the
// registers allow, so that the rest of the SM's 256 KB serves as L1 cache for the bricks
// (measured on C2, Phong, per-ray loop at 2048^2 / deferred at 1024^2, Gsamples/s: driver's
// choice 81.1 / 46.4, this split 81.8 / 47.7; more L1 matters - the per-ray loop with 28 KB
// of unused shared memory per block ran at 77.6).  Returns the resident blocks per SM.
template <typename K>
cudaError_t fit_carveout(K kernel, size_t smem, int threads, int& occ) {
  int dev = 0, max_smem = 0, reserved = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, smem);
  cudaFuncAttributes fa;
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess || occ <= 0 || max_smem <= 0) return e;
  // a block's shared memory: the dynamic part, the kernel's static arrays, the reserve
  const long long need = (long long)occ * ((long long)smem + (long long)fa.sharedSizeBytes + reserved);
  const int pct = (int)std::min(100LL, (need * 100 + max_smem - 1) / max_smem);
  return cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
}

template <typename K>
cudaError_t launch_one(K kernel, dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       const RenderArgs& a) {
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  {
    int occ = 0;
    cudaError_t e = fit_carveout(kernel, smem, (int)(block.x * block.y * block.z), occ);
    if (e != cudaSuccess) return e;
  }
  kernel<<<grid, block, smem, s>>>(a);
  return cudaGetLastError();
}

// Persistent launch of the refill schedule: the queue head is zeroed, then as many blocks
// as fit on the device start, at most one warp per 8x4 pixel tile.
template <typename K>
cudaError_t launch_persist(K kernel, size_t smem, cudaStream_t s, const RenderArgs& a) {
  cudaError_t e = cudaMemsetAsync(a.counters + kQueueCounter, 0, sizeof(unsigned long long), s);
  if (e == cudaSuccess && smem > 48 * 1024)
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int dev = 0, sms = 0, occ = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, 128, smem);
  if (e != cudaSuccess) return e;
  const long long tiles = (long long)((a.ray.width + 7) / 8) * ((a.ray.rows + 3) / 4);
  const long long grid = std::max(1LL, std::min((long long)sms * std::max(occ, 1), (tiles + 3) / 4));
  kernel<<<(unsigned)grid, dim3(8, 16), smem, s>>>(a, a.samples_per_iter);
  return cudaGetLastError();
}

// Persistent launch of the tile-queue kernels (march_kernel, deferred_kernel): the queue
// head is zeroed (every launch owns its queue, also when a caller renders a frame in
// several bands on one set of counters), then as many 128-thread blocks as are resident at
// once start, at most one warp per 8x4 tile.
template <typename K>
cudaError_t launch_tiles(K kernel, size_t smem, cudaStream_t s, const RenderArgs& a) {
  cudaError_t e = cudaMemsetAsync(a.counters + kQueueCounter, 0, sizeof(unsigned long long), s);
  if (e == cudaSuccess && smem > 48 * 1024)
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int dev = 0, sms = 0, occ = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = fit_carveout(kernel, smem, 128, occ);
  if (e != cudaSuccess) return e;
  const long long tiles = (long long)((a.ray.width + 7) / 8) * ((a.ray.rows + 3) / 4);
  const long long grid = std::max(1LL, std::min((long long)sms * std::max(occ, 1), (tiles + 3) / 4));
  kernel<<<(unsigned)grid, dim3(8, 16), smem, s>>>(a);
  return cudaGetLastError();
}

template <int ST>
amr_status launch_storage(amr_ctx* c, const RenderArgs& a, int interp, int shade, int schedule,
                          cudaStream_t s) {
  const dim3 block(8, 16);
  const dim3 grid((unsigned)((a.ray.width + 7) / 8), (unsigned)((a.ray.rows + 15) / 16));
  const size_t tf_bytes = (size_t)a.tf_n * sizeof(float4) + (size_t)(a.tf_n + 1) * sizeof(int);
  if (grid.x == 0 || grid.y == 0) return AMR_OK;
  // the stencil-maximum opacity test: pointer storages, trilinear, schedules 0 and 3
  constexpr bool kPtr = ST == ST_PTR || ST == ST_PTR_F16 || ST == ST_PTR_BF16;
  const bool mx = kPtr && (shade & kShadeMaxBit) != 0 && interp == 1 &&
                  !(shade & kShadeShadow) && (schedule == 0 || schedule == 3);
  shade &= ~kShadeMaxBit;
  cudaError_t e;
  if (shade & kShadeShadow) {
    // secondary rays to the point light: per-ray schedule (a lane marches its samples'
    // light rays) or deferred shading (the warp marches each queued sample's light ray
    // together); trilinear, FP32 linear storages
    if constexpr (ST == ST_PTR || ST == ST_ATLAS_LINEAR) {
      const int base = shade & 3;
      if (interp != 1 || (schedule != 0 && schedule != 3) || (schedule == 3 && base == 0))
        return fail(c, AMR_ERR_ARG,
                    "secondary rays render trilinear with schedule 0, or 3 with shade = 1");
      if (schedule == 3) {
        const size_t smem = ((tf_bytes + 15) & ~(size_t)15) + 4 * sizeof(DeferArea);
        if (base == 1) e = launch_tiles(deferred_kernel<ST, 1 | kShadeShadow>, smem, s, a);
        else e = launch_tiles(deferred_kernel<ST, 2 | kShadeShadow>, smem, s, a);
      } else {
        const size_t smem = tf_bytes;
        if (base == 0) e = launch_tiles(march_kernel<ST, 1, kShadeShadow>, smem, s, a);
        else if (base == 1) e = launch_tiles(march_kernel<ST, 1, 1 | kShadeShadow>, smem, s, a);
        else e = launch_tiles(march_kernel<ST, 1, 2 | kShadeShadow>, smem, s, a);
      }
    } else {
      return fail(c, AMR_ERR_ARG, "secondary rays need the ptr or atlas_linear storage, FP32 cells");
    }
  } else if (schedule == 3) {
    // warp-synchronous march with deferred shading (trilinear, Phong)
    if (interp != 1 || (shade != 1 && shade != 2))
      return fail(c, AMR_ERR_ARG, "deferred shading renders trilinear with shade = 1");
    const size_t smem = ((tf_bytes + 15) & ~(size_t)15) + 4 * sizeof(DeferArea);
    if constexpr (kPtr) {
      if (mx) {
        if (shade == 1) e = launch_tiles(deferred_kernel<ST, 1 | kShadeMaxBit>, smem, s, a);
        else e = launch_tiles(deferred_kernel<ST, 2 | kShadeMaxBit>, smem, s, a);
        goto launched;
      }
    }
    if (shade == 1) e = launch_tiles(deferred_kernel<ST, 1>, smem, s, a);
    else e = launch_tiles(deferred_kernel<ST, 2>, smem, s, a);
  } else if (schedule == 2) {
    // persistent warps with ray refill (trilinear)
    if (interp != 1) return fail(c, AMR_ERR_ARG, "the refill schedule renders trilinear");
    const size_t smem = tf_bytes;
    if (shade == 0) e = launch_persist(persist_kernel<ST, 1, 0>, smem, s, a);
    else if (shade == 1) e = launch_persist(persist_kernel<ST, 1, 1>, smem, s, a);
    else e = launch_persist(persist_kernel<ST, 1, 2>, smem, s, a);
  } else if constexpr (ST >= ST_PTR_F16) {
    // 16-bit cells: trilinear, per-ray schedule
    if (interp != 1 || schedule != 0)
      return fail(c, AMR_ERR_ARG, "16-bit storage renders trilinear with schedule 0, 2 or 3");
    const size_t smem = tf_bytes;
    if constexpr (kPtr) {
      if (mx) {
        if (shade == 0) e = launch_tiles(march_kernel<ST, 1, kShadeMaxBit>, smem, s, a);
        else if (shade == 1) e = launch_tiles(march_kernel<ST, 1, 1 | kShadeMaxBit>, smem, s, a);
        else e = launch_tiles(march_kernel<ST, 1, 2 | kShadeMaxBit>, smem, s, a);
        goto launched;
      }
    }
    if (shade == 0) e = launch_tiles(march_kernel<ST, 1, 0>, smem, s, a);
    else if (shade == 1) e = launch_tiles(march_kernel<ST, 1, 1>, smem, s, a);
    else e = launch_tiles(march_kernel<ST, 1, 2>, smem, s, a);
  } else if (schedule == 0 && ST == ST_TEXOBJ) {
    // per-patch textures: one block per 8x16 tile (see march_kernel)
    const size_t smem = tf_bytes;
    if (interp == 1 && shade == 0) e = launch_one(march_kernel<ST, 1, 0, false>, grid, block, smem, s, a);
    else if (interp == 1 && shade == 1) e = launch_one(march_kernel<ST, 1, 1, false>, grid, block, smem, s, a);
    else if (interp == 1 && shade == 2) e = launch_one(march_kernel<ST, 1, 2, false>, grid, block, smem, s, a);
    else if (interp == 0 && shade == 0) e = launch_one(march_kernel<ST, 0, 0, false>, grid, block, smem, s, a);
    else e = launch_one(march_kernel<ST, 0, 1, false>, grid, block, smem, s, a);
  } else if (schedule == 0) {
    const size_t smem = tf_bytes;
    if constexpr (kPtr) {
      if (mx) {
        if (shade == 0) e = launch_tiles(march_kernel<ST, 1, kShadeMaxBit>, smem, s, a);
        else if (shade == 1) e = launch_tiles(march_kernel<ST, 1, 1 | kShadeMaxBit>, smem, s, a);
        else e = launch_tiles(march_kernel<ST, 1, 2 | kShadeMaxBit>, smem, s, a);
        goto launched;
      }
    }
    if (interp == 1 && shade == 0) e = launch_tiles(march_kernel<ST, 1, 0>, smem, s, a);
    else if (interp == 1 && shade == 1) e = launch_tiles(march_kernel<ST, 1, 1>, smem, s, a);
    else if (interp == 1 && shade == 2) e = launch_tiles(march_kernel<ST, 1, 2>, smem, s, a);
    else if (interp == 0 && shade == 0) e = launch_tiles(march_kernel<ST, 0, 0>, smem, s, a);
    else e = launch_tiles(march_kernel<ST, 0, 1>, smem, s, a);
  } else {
    const size_t smem = ((tf_bytes + 15) & ~(size_t)15) + 4 * sizeof(WarpArea);
    if (interp == 1 && shade == 0) e = launch_one(wave_kernel<ST, 1, 0>, grid, block, smem, s, a);
    else if (interp == 1 && shade == 1) e = launch_one(wave_kernel<ST, 1, 1>, grid, block, smem, s, a);
    else if (interp == 1 && shade == 2) e = launch_one(wave_kernel<ST, 1, 2>, grid, block, smem, s, a);
    else if (interp == 0 && shade == 0) e = launch_one(wave_kernel<ST, 0, 0>, grid, block, smem, s, a);
    else e = launch_one(wave_kernel<ST, 0, 1>, grid, block, smem, s, a);
  }
launched:
  if (e != cudaSuccess)
    return fail(c, AMR_ERR_CUDA, std::string("march launch: ") + cudaGetErrorString(e));
  return AMR_OK;
}

amr_status launch_ptr(amr_ctx* c, const RenderArgs& a, int interp, int shade, int schedule,
                      cudaStream_t s);
amr_status launch_texobj(amr_ctx* c, const RenderArgs& a, int interp, int shade, int schedule,
                         cudaStream_t s);
amr_status launch_atlas_linear(amr_ctx* c, const RenderArgs& a, int interp, int shade,
                               int schedule, cudaStream_t s);
amr_status launch_atlas_tex3d(amr_ctx* c, const RenderArgs& a, int interp, int shade,
                              int schedule, cudaStream_t s);
amr_status launch_16bit(amr_ctx* c, const RenderArgs& a, int storage, int interp, int shade,
                        int schedule, cudaStream_t s);

}  // namespace amr
