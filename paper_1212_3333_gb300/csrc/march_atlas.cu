// March kernels for the NFDH-packed brick atlas (the paper's memory-pool texture,
// Sec. 4.1), in linear memory and as one 3D texture.
#include "march_launch.cuh"

namespace amr {
amr_status launch_atlas_linear(amr_ctx* c, const RenderArgs& a, int interp, int shade,
                               int schedule, cudaStream_t s) {
  return launch_storage<ST_ATLAS_LINEAR>(c, a, interp, shade, schedule, s);
}
amr_status launch_atlas_tex3d(amr_ctx* c, const RenderArgs& a, int interp, int shade,
                               int schedule, cudaStream_t s) {
  return launch_storage<ST_ATLAS_TEX3D>(c, a, interp, shade, schedule, s);
}
}  // namespace amr
