// March kernels for the per-patch pointer table (bricks in one device pool).
#include "march_launch.cuh"

namespace amr {
amr_status launch_ptr(amr_ctx* c, const RenderArgs& a, int interp, int shade, int schedule,
                         cudaStream_t s) {
  return launch_storage<ST_PTR>(c, a, interp, shade, schedule, s);
}
}  // namespace amr
