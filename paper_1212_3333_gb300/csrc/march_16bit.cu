// March kernels for bricks stored with 16-bit cells (FP16 or BF16; interpolation, gradients
// and compositing in FP32), in the pointer-table and linear-atlas layouts.
#include "march_launch.cuh"

namespace amr {
amr_status launch_16bit(amr_ctx* c, const RenderArgs& a, int storage, int interp, int shade,
                        int schedule, cudaStream_t s) {
  switch (storage) {
    case ST_PTR_F16: return launch_storage<ST_PTR_F16>(c, a, interp, shade, schedule, s);
    case ST_PTR_BF16: return launch_storage<ST_PTR_BF16>(c, a, interp, shade, schedule, s);
    case ST_ATLAS_LINEAR_F16: return launch_storage<ST_ATLAS_LINEAR_F16>(c, a, interp, shade, schedule, s);
    case ST_ATLAS_LINEAR_BF16: return launch_storage<ST_ATLAS_LINEAR_BF16>(c, a, interp, shade, schedule, s);
    default: return fail(c, AMR_ERR_ARG, "unknown 16-bit storage");
  }
}
}  // namespace amr
