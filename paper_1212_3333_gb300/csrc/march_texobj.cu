// March kernels for the per-patch table of texture objects (the CUDA counterpart of the
// paper's bindless texture handles, Sec. 4.2).
#include "march_launch.cuh"

namespace amr {
amr_status launch_texobj(amr_ctx* c, const RenderArgs& a, int interp, int shade, int schedule,
                         cudaStream_t s) {
  return launch_storage<ST_TEXOBJ>(c, a, interp, shade, schedule, s);
}
}  // namespace amr
