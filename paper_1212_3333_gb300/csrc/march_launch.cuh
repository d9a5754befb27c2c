// Template launcher shared by the per-storage translation units.
#pragma once
#include "ctx.h"
#include "march.cuh"

namespace amr {

template <int ST>
amr_status launch_storage(amr_ctx* c, const RenderArgs& a, int interp, int shade,
                          cudaStream_t s) {
  const dim3 block(8, 16);
  const dim3 grid((unsigned)((a.ray.width + 7) / 8), (unsigned)((a.ray.rows + 15) / 16));
  const size_t smem = (size_t)a.tf_n * sizeof(float4) + (size_t)(a.tf_n + 1) * sizeof(int);
  if (grid.x == 0 || grid.y == 0) return AMR_OK;
  if (interp == 1 && shade == 0) march_kernel<ST, 1, 0><<<grid, block, smem, s>>>(a);
  else if (interp == 1 && shade == 1) march_kernel<ST, 1, 1><<<grid, block, smem, s>>>(a);
  else if (interp == 0 && shade == 0) march_kernel<ST, 0, 0><<<grid, block, smem, s>>>(a);
  else march_kernel<ST, 0, 1><<<grid, block, smem, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return fail(c, AMR_ERR_CUDA, std::string("march launch: ") + cudaGetErrorString(e));
  return AMR_OK;
}

amr_status launch_ptr(amr_ctx* c, const RenderArgs& a, int interp, int shade, cudaStream_t s);
amr_status launch_texobj(amr_ctx* c, const RenderArgs& a, int interp, int shade, cudaStream_t s);
amr_status launch_atlas_linear(amr_ctx* c, const RenderArgs& a, int interp, int shade,
                               cudaStream_t s);
amr_status launch_atlas_tex3d(amr_ctx* c, const RenderArgs& a, int interp, int shade,
                              cudaStream_t s);

}  // namespace amr
