// Per-pixel traversal sequences (Sec. 3.3 kd-restart) and the render dispatcher.
#include "march_launch.cuh"

namespace amr {

__global__ void __launch_bounds__(128) trace_kernel(const __grid_constant__ TraceArgs A) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= A.ray.width || j >= A.ray.height) return;
  const size_t p = (size_t)j * A.ray.width + i;
  RayX rx;
  if (!make_ray(A.ray, i, j, rx)) {
    A.seq_len[p] = 0;
    return;
  }
  RayF rf;
  make_frame(A.ray, rx, rf);
  int pid0 = kPidIn;
  float tau0 = 0.0f, e0 = 0.0f;
  uint32_t start = 0;
  int n = 0, prev = -1;
  unsigned long long status = 0;
  while (pid0 != kPidOut) {
    if (n >= A.max_segments) {
      status |= kStatusCapacity;
      break;
    }
    int pid1 = kPidOut;
    float tau1 = rf.tau_out, e1 = exit_bound(rf);
    const int lmin = lod_min_level(A.ray, A.lv, rf, i, j, pid0, tau0, e0);
    const int lid = next_leaf(A.nodes, A.leaves, A.face_node, A.node_box, A.ray, i, j, rf, start,
                              prev, pid0, tau0, e0, pid1, tau1, e1, lmin);
    if (lid < 0) {
      status |= kStatusDevice;
      break;
    }
    prev = lid;
    if (n < A.max_len) {
      const size_t q = p * (size_t)A.max_len + n;
      A.leaf_seq[q] = lid;
      if (A.t_seq) {
        A.t_seq[2 * q] = exact_t(A.ray, rx, pid0);
        A.t_seq[2 * q + 1] = exact_t(A.ray, rx, pid1);
      }
    }
    ++n;
    pid0 = pid1;
    tau0 = tau1;
    e0 = e1;
  }
  A.seq_len[p] = n <= A.max_len ? n : -1;
  if (status) atomicOr(A.counters + 1, status);
}

amr_status launch_trace(amr_ctx* c, const TraceArgs& a, void* stream) {
  const dim3 block(8, 16);
  const dim3 grid((unsigned)((a.ray.width + 7) / 8), (unsigned)((a.ray.height + 15) / 16));
  trace_kernel<<<grid, block, 0, (cudaStream_t)stream>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return fail(c, AMR_ERR_CUDA, std::string("trace launch: ") + cudaGetErrorString(e));
  return AMR_OK;
}

amr_status launch_render(amr_ctx* c, const RenderArgs& a, int storage, int interp, int shade,
                         int schedule, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  switch (storage) {
    case ST_PTR: return launch_ptr(c, a, interp, shade, schedule, s);
    case ST_TEXOBJ: return launch_texobj(c, a, interp, shade, schedule, s);
    case ST_ATLAS_LINEAR: return launch_atlas_linear(c, a, interp, shade, schedule, s);
    case ST_ATLAS_TEX3D: return launch_atlas_tex3d(c, a, interp, shade, schedule, s);
    case ST_PTR_F16:
    case ST_PTR_BF16:
    case ST_ATLAS_LINEAR_F16:
    case ST_ATLAS_LINEAR_BF16: return launch_16bit(c, a, storage, interp, shade, schedule, s);
    default: return fail(c, AMR_ERR_ARG, "unknown storage");
  }
}

}  // namespace amr
