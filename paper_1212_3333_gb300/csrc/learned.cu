// Learned segment proposal fused into the ray march, and the segment log it is trained on.
// The paper has no counterpart; the march itself is Sec. 3.3 as in march.cuh.
//
// learned_kernel gives each warp a 4x8 pixel tile and marches the tile's rays in rounds,
// so that the warp is converged at segment boundaries: every live lane descends to its
// ray's next segment, drops it if exact min/max skipping proves it transparent, and stages
// its 12 features; when some lane's segment has at least learned_min_samples samples the
// warp evaluates the MLP for all 32 lanes on the tensor cores (mlp_forward_warp); such a
// segment whose predicted opacity contribution is below tau is skipped (mode 1) or sampled
// with a coarse_factor times coarser step (mode 2); every other segment is sampled exactly
// as the plain march samples it.
//
// log_kernel is the plain march (no early termination) that records, per segment kept by a
// seeded hash, the same 12 features and the target A_out - A_in = (1 - A_in) alpha_seg.
#include "march_launch.cuh"
#include "mlp.cuh"

namespace amr {

// Features of the segment [tau0, tau1] of leaf lf (all O(1)): entry and exit position in
// root-box units, level / (L-1), leaf value range through the TF domain, accumulated
// opacity, octahedral ray direction.
__device__ __forceinline__ void segment_features(const RenderArgs& A, const RayF& rf, float tau0,
                                                 float tau1, const DLeaf& lf, float Acc,
                                                 float* f) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float lo = (float)A.ray.root_f[a];
    const float inv_ext = 1.0f / (float)(A.ray.root_f[3 + a] - A.ray.root_f[a]);
    f[a] = (fmaf(tau0, rf.Dd[a], rf.Xe[a]) - lo) * inv_ext;
    f[3 + a] = (fmaf(tau1, rf.Dd[a], rf.Xe[a]) - lo) * inv_ext;
  }
  f[6] = (float)lf.level * A.inv_levels;
  f[7] = fminf(fmaxf((lf.vmin - A.vmin) * A.inv_range, 0.0f), 1.0f);
  f[8] = fminf(fmaxf((lf.vmax - A.vmin) * A.inv_range, 0.0f), 1.0f);
  f[9] = Acc;
  octahedral(rf.Dd[0], rf.Dd[1], rf.Dd[2], f[10], f[11]);
}

__device__ __forceinline__ uint32_t mix32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

struct LogArgs {
  float* features;              // [cap][12]
  float* targets;               // [cap]
  long long cap;
  unsigned long long* count;    // running record count (may exceed cap: records dropped)
  float keep_prob;
  uint32_t seed;
  int32_t* counts;              // per pixel of the view: records it keeps (count pass)
  const unsigned long long* offsets;  // per pixel: index of its first record (write pass)
};

// Whether segment seg of pixel (i, j) is logged: a seeded hash, independent of the march.
__device__ __forceinline__ bool log_keep(const LogArgs& L, int i, int j, int seg) {
  const uint32_t h = mix32((uint32_t)i * 0x9E3779B1u ^ mix32((uint32_t)j + L.seed * 0x85EBCA77u) ^
                           ((uint32_t)seg * 0xC2B2AE3Du));
  return (float)(h >> 8) * (1.0f / 16777216.0f) < L.keep_prob;
}

// WRITE = false: count the records each pixel keeps (the segments alone, no sampling);
// WRITE = true: the march, each kept record written at its pixel's offset, so the records
// of a view follow pixel and segment order whatever the thread schedule.
template <int ST, bool WRITE>
__global__ void __launch_bounds__(128) log_kernel(const __grid_constant__ RenderArgs A,
                                                  const LogArgs L) {
  extern __shared__ float4 smem[];
  float4* s_tf = smem;
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  if constexpr (WRITE) {
    for (int k = tid; k < A.tf_n; k += blockDim.x * blockDim.y) s_tf[k] = A.tf[k];
    __syncthreads();
  }
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int jr = blockIdx.y * blockDim.y + threadIdx.y;
  const int j = A.ray.row0 + jr;
  if (i >= A.ray.width || jr >= A.ray.rows || j >= A.ray.height) return;
  const size_t pix = (size_t)jr * A.ray.width + i;
  int kept = 0;
  RayX rx;
  if (!make_ray(A.ray, i, j, rx)) {
    if constexpr (!WRITE) L.counts[pix] = 0;
    return;
  }
  RayF rf;
  make_frame(A.ray, rx, rf);
  float C0 = 0.f, C1 = 0.f, C2 = 0.f, Acc = 0.f;
  unsigned nsamp = 0;
  int pid0 = kPidIn;
  float tau0 = 0.0f, e0 = 0.0f;
  uint32_t start = 0;
  int prev = -1;
  for (int seg = 0; pid0 != kPidOut && seg < A.max_segments; ++seg) {
    int pid1 = kPidOut;
    float tau1 = rf.tau_out, e1 = exit_bound(rf);
    const int lid = next_leaf(A.nodes, A.leaves, A.face_node, A.node_box, A.ray, i, j, rf, start,
                              prev, pid0, tau0, e0, pid1, tau1, e1);
    if (lid < 0) break;
    prev = lid;
    if constexpr (WRITE) {
      const DLeaf lf = A.leaves[lid];
      const DLevel& lv = A.lv[lf.level];
      int n = min(segment_count(A.ray, i, j, rf, pid0, tau0, e0, pid1, tau1, e1, lv),
                  kMaxSamplesPerSegment);
      float f[kMlpIn];
      segment_features(A, rf, tau0, tau1, lf, Acc, f);
      const float a_in = Acc;
      SegSetup g;
      setup_segment(A, rf, lf, lv, lid, pid0, pid1, tau0, e0, tau1, e1, n, i, j, g);
      sample_segment<ST, 1, 0>(A, A.ray, s_tf, nullptr, g, lv, 0.f, 0.f, 0.f, C0, C1, C2, Acc,
                               nsamp);
      if (log_keep(L, i, j, seg)) {
        const unsigned long long idx = L.offsets[pix] + (unsigned long long)kept++;
        if ((long long)idx < L.cap) {
#pragma unroll
          for (int k = 0; k < kMlpIn; ++k) L.features[idx * kMlpIn + k] = f[k];
          L.targets[idx] = Acc - a_in;
        }
      }
    } else if (log_keep(L, i, j, seg)) {
      ++kept;
    }
    pid0 = pid1;
    tau0 = tau1;
    e0 = e1;
  }
  if constexpr (!WRITE) L.counts[pix] = kept;
}

// Exclusive prefix sums of the view's per-pixel record counts, starting at the running
// record count, which then grows by the view's total (one block of 1024 threads, each
// summing a contiguous chunk).
__global__ void __launch_bounds__(1024) log_scan_kernel(const int32_t* __restrict__ counts,
                                                        long long n,
                                                        unsigned long long* __restrict__ offsets,
                                                        unsigned long long* __restrict__ count) {
  __shared__ unsigned long long part[1024];
  const int t = threadIdx.x;
  const long long chunk = (n + 1023) / 1024;
  const long long lo = min(n, (long long)t * chunk), hi = min(n, lo + chunk);
  unsigned long long s = 0;
  for (long long k = lo; k < hi; ++k) s += (unsigned long long)counts[k];
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    unsigned long long run = *count;
    for (int q = 0; q < 1024; ++q) {
      const unsigned long long v = part[q];
      part[q] = run;
      run += v;
    }
    *count = run;
  }
  __syncthreads();
  unsigned long long run = part[t];
  for (long long k = lo; k < hi; ++k) {
    offsets[k] = run;
    run += (unsigned long long)counts[k];
  }
}

// The learned march samples a segment as the plain march does; with stencil-maximum bricks
// it tests every sample's maximum on its own (AMR_LEARNED_GROUP 0) or G at a time.
#ifndef AMR_LEARNED_GROUP
#define AMR_LEARNED_GROUP 0
#endif
template <int ST, int SHADE>
__device__ __forceinline__ bool sample_learned(const RenderArgs& A, const float4* s_tf,
                                               const int* s_nz, const SegSetup& g,
                                               const DLevel& lv, float Lx, float Ly, float Lz,
                                               float& C0, float& C1, float& C2, float& Acc,
                                               unsigned& nsamp) {
  if constexpr ((SHADE & kShadeMaxBit) != 0)
    return sample_segment_grouped<ST, SHADE, AMR_LEARNED_GROUP>(A, A.ray, s_tf, s_nz, g, lv, Lx,
                                                                Ly, Lz, C0, C1, C2, Acc, nsamp);
  else
    return sample_segment<ST, 1, SHADE>(A, A.ray, s_tf, s_nz, g, lv, Lx, Ly, Lz, C0, C1, C2, Acc,
                                        nsamp);
}

#ifndef AMR_LEARNED_TILE_W
#define AMR_LEARNED_TILE_W 4  // pixel tile of one warp: AMR_LEARNED_TILE_W x (32 / it)
#endif
static_assert(AMR_LEARNED_TILE_W == 2 || AMR_LEARNED_TILE_W == 4 || AMR_LEARNED_TILE_W == 8 ||
                  AMR_LEARNED_TILE_W == 16,
              "learned tile width");
template <int ST, int SHADE>
__global__ void __launch_bounds__(128, AMR_MIN_BLOCKS) learned_kernel(const __grid_constant__ RenderArgs A) {
  extern __shared__ float4 smem[];
  float4* s_tf = smem;
  int* s_nz = reinterpret_cast<int*>(smem + A.tf_n);
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int lane = tid & 31, warp = tid >> 5;
  const size_t tf_bytes = (size_t)A.tf_n * sizeof(float4) + (size_t)(A.tf_n + 1) * sizeof(int);
  unsigned char* wsm = reinterpret_cast<unsigned char*>(smem) + ((tf_bytes + 15) & ~(size_t)15);
  __nv_bfloat16* xs = reinterpret_cast<__nv_bfloat16*>(wsm + kPackBytes) + warp * 32 * kStride1;
  float* ys = reinterpret_cast<float*>(wsm + kPackBytes + 4 * 32 * kStride1 * 2) + warp * 32;
  for (int k = tid; k < A.tf_n; k += blockDim.x * blockDim.y) s_tf[k] = A.tf[k];
  for (int k = tid; k < kPackBytes / 16; k += blockDim.x * blockDim.y)
    reinterpret_cast<uint4*>(wsm)[k] = reinterpret_cast<const uint4*>(A.mlp)[k];
  __syncthreads();
  if (tid == 0) {
    int acc = 0;
    s_nz[0] = 0;
    for (int k = 0; k < A.tf_n; ++k) {
      acc += s_tf[k].w != 0.0f ? 1 : 0;
      s_nz[k + 1] = acc;
    }
  }
  __syncthreads();

  unsigned nsamp = 0;
  unsigned long long status = 0;
  // one pixel tile per warp (persistent warps over a tile queue measured slower here: 174
  // against 160 ms for 8 views of C2 at 2048^2, coarse16 at tau 1e-2); tiles 4 wide and 8
  // high keep a warp's rays together through the rounds better than 8 x 4 or 16 x 2
  // (coarse32 at tau 1e-2: 133.8 / 142.2 / 162.1 ms)
  constexpr int TW = AMR_LEARNED_TILE_W, TH = 32 / TW;
  const int tiles_x = (A.ray.width + TW - 1) / TW;
  const int n_tiles = tiles_x * ((A.ray.rows + TH - 1) / TH);
  const int t = (int)blockIdx.x * 4 + (tid >> 5);
  {
    const int i = (t % tiles_x) * TW + lane % TW;
    const int jr = (t / tiles_x) * TH + lane / TW;
    const int j = A.ray.row0 + jr;
    const bool active = t < n_tiles && i < A.ray.width && jr < A.ray.rows && j < A.ray.height;
    float C0 = 0.f, C1 = 0.f, C2 = 0.f, Acc = 0.f;
    RayX rx;
    RayF rf;
    bool live = active && make_ray(A.ray, i, j, rx);
    float Lx = 0.f, Ly = 0.f, Lz = 0.f;
    if (live) {
      make_frame(A.ray, rx, rf);
      const float inv_dn = 1.0f / rf.dn;
      Lx = -rf.Dd[0] * (float)A.ray.hf[0] * inv_dn;
      Ly = -rf.Dd[1] * (float)A.ray.hf[1] * inv_dn;
      Lz = -rf.Dd[2] * (float)A.ray.hf[2] * inv_dn;
    }
    int pid0 = kPidIn;
    float tau0 = 0.0f, e0 = 0.0f;
    uint32_t start = 0;
    int nseg = 0, prev = -1;
    while (__any_sync(0xffffffffu, live)) {
      int n = 0, lid = -1, pid1 = kPidOut;
      float tau1 = 0.0f, e1 = 0.0f;
      {
        float f[kMlpInPad];
#pragma unroll
        for (int k = 0; k < kMlpInPad; ++k) f[k] = 0.0f;
        if (live) {
          if (pid0 == kPidOut) {
            live = false;
          } else if (nseg >= A.max_segments) {
            status |= kStatusCapacity;
            live = false;
          } else {
            ++nseg;
            tau1 = rf.tau_out;
            e1 = exit_bound(rf);
            lid = next_leaf(A.nodes, A.leaves, A.face_node, A.node_box, A.ray, i, j, rf, start,
                            prev, pid0, tau0, e0, pid1, tau1, e1);
            if (lid < 0) {
              status |= kStatusDevice;
              live = false;
            } else {
              prev = lid;
              const DLeaf lf = A.leaves[lid];
              n = segment_count(A.ray, i, j, rf, pid0, tau0, e0, pid1, tau1, e1, A.lv[lf.level]);
              if (n > kMaxSamplesPerSegment) {
                status |= kStatusCapacity;
                n = kMaxSamplesPerSegment;
              }
              if (A.skip && tf_transparent(s_nz, A.tf_n, lf.vmin, lf.vmax, A.vmin, A.inv_range))
                n = 0;
              if (n > 0) segment_features(A, rf, tau0, tau1, lf, Acc, f);
            }
          }
        }
        // stage this lane's features (zero-padded) as its BF16 row of the warp's tile
        uint4* row = reinterpret_cast<uint4*>(xs + lane * kStride1);
        row[0] = make_uint4(pack_bf16(f[0], f[1]), pack_bf16(f[2], f[3]), pack_bf16(f[4], f[5]),
                            pack_bf16(f[6], f[7]));
        row[1] = make_uint4(pack_bf16(f[8], f[9]), pack_bf16(f[10], f[11]),
                            pack_bf16(f[12], f[13]), pack_bf16(f[14], f[15]));
      }
      // evaluate the proposal on the tensor cores, only when some lane has a segment long
      // enough (learned_min_samples) for a skip or a coarser step to save more than the
      // evaluation costs; shorter segments are sampled as is
      const bool ask = n >= A.learned_min_samples;
      if (__any_sync(0xffffffffu, ask)) {
        __syncwarp();
        const float predicted = mlp_forward_warp(wsm, xs, ys, lane);
        if (ask && predicted < A.tau)
          n = A.learned == 1 ? 0 : (n + A.coarse_factor - 1) / A.coarse_factor;
      }
      if (n > 0) {
        const DLeaf lf = A.leaves[lid];  // reloaded: not held across the evaluation
        const DLevel& lv = A.lv[lf.level];
        SegSetup g;
        setup_segment(A, rf, lf, lv, lid, pid0, pid1, tau0, e0, tau1, e1, n, i, j, g);
        if (sample_learned<ST, SHADE>(A, s_tf, s_nz, g, lv, Lx, Ly, Lz, C0, C1, C2, Acc, nsamp))
          live = false;  // early ray termination
      }
      if (lid >= 0) {
        pid0 = pid1;
        tau0 = tau1;
        e0 = e1;
      }
    }
    if (active) A.out[(size_t)jr * A.ray.width + i] = make_float4(C0, C1, C2, Acc);
  }
  const unsigned total = __reduce_add_sync(0xffffffffu, nsamp);
  if (lane == 0 && total) atomicAdd(A.counters, (unsigned long long)total);
  if (status) atomicOr(A.counters + 1, status);
}

size_t learned_smem(int tf_n) {
  const size_t tf_bytes = (size_t)tf_n * sizeof(float4) + (size_t)(tf_n + 1) * sizeof(int);
  return ((tf_bytes + 15) & ~(size_t)15) + kPackBytes + 4 * 32 * kStride1 * 2 + 4 * 32 * 4;
}

amr_status launch_learned(amr_ctx* c, const RenderArgs& a, int storage, int shade, void* stream) {
  if (a.ray.width <= 0 || a.ray.rows <= 0) return AMR_OK;
  constexpr int TW = AMR_LEARNED_TILE_W, TH = 32 / TW;
  const long long tiles = (long long)((a.ray.width + TW - 1) / TW) * ((a.ray.rows + TH - 1) / TH);
  const dim3 grid((unsigned)((tiles + 3) / 4)), block(8, 16);
  const size_t smem = learned_smem(a.tf_n);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  const bool mx = (shade & kShadeMaxBit) != 0;  // stencil-maximum test (pointer storage)
  shade &= ~kShadeMaxBit;
  if (storage == ST_PTR && mx) {
    if (shade == 0) e = launch_one(learned_kernel<ST_PTR, kShadeMaxBit>, grid, block, smem, s, a);
    else if (shade == 1) e = launch_one(learned_kernel<ST_PTR, 1 | kShadeMaxBit>, grid, block, smem, s, a);
    else e = launch_one(learned_kernel<ST_PTR, 2 | kShadeMaxBit>, grid, block, smem, s, a);
  } else if (storage == ST_PTR) {
    if (shade == 0) e = launch_one(learned_kernel<ST_PTR, 0>, grid, block, smem, s, a);
    else if (shade == 1) e = launch_one(learned_kernel<ST_PTR, 1>, grid, block, smem, s, a);
    else e = launch_one(learned_kernel<ST_PTR, 2>, grid, block, smem, s, a);
  } else if (storage == ST_ATLAS_LINEAR) {
    if (shade == 0) e = launch_one(learned_kernel<ST_ATLAS_LINEAR, 0>, grid, block, smem, s, a);
    else if (shade == 1) e = launch_one(learned_kernel<ST_ATLAS_LINEAR, 1>, grid, block, smem, s, a);
    else e = launch_one(learned_kernel<ST_ATLAS_LINEAR, 2>, grid, block, smem, s, a);
  } else {
    return fail(c, AMR_ERR_ARG, "the learned proposal needs the ptr or atlas_linear storage");
  }
  if (e != cudaSuccess)
    return fail(c, AMR_ERR_CUDA, std::string("learned march launch: ") + cudaGetErrorString(e));
  return AMR_OK;
}

amr_status launch_log(amr_ctx* c, const RenderArgs& a, int storage, float* features,
                      float* targets, long long cap, unsigned long long* count, float keep_prob,
                      uint32_t seed, void* stream) {
  const dim3 block(8, 16);
  const dim3 grid((unsigned)((a.ray.width + 7) / 8), (unsigned)((a.ray.rows + 15) / 16));
  if (grid.x == 0 || grid.y == 0) return AMR_OK;
  if (storage != ST_PTR && storage != ST_ATLAS_LINEAR)
    return fail(c, AMR_ERR_ARG, "segment logging needs the ptr or atlas_linear storage");
  // per-pixel counts and offsets of the view (grown as needed, kept with the context)
  const size_t pixels = (size_t)a.ray.width * (size_t)a.ray.rows;
  DeviceState& d = c->dev;
  if (pixels > d.log_pixels) {
    cudaFree(d.log_counts);
    cudaFree(d.log_offsets);
    d.log_counts = nullptr;
    d.log_offsets = nullptr;
    d.log_pixels = 0;
    if (cudaMalloc(&d.log_counts, pixels * sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc(&d.log_offsets, pixels * sizeof(unsigned long long)) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(d.log_counts);
      d.log_counts = nullptr;
      return fail(c, AMR_ERR_OOM, "segment log: per-pixel counts");
    }
    d.log_pixels = pixels;
  }
  LogArgs L{features, targets, cap, count, keep_prob, seed, d.log_counts, d.log_offsets};
  const size_t smem = (size_t)a.tf_n * sizeof(float4);
  cudaStream_t s = (cudaStream_t)stream;
  if (storage == ST_PTR) log_kernel<ST_PTR, false><<<grid, block, 0, s>>>(a, L);
  else log_kernel<ST_ATLAS_LINEAR, false><<<grid, block, 0, s>>>(a, L);
  log_scan_kernel<<<1, 1024, 0, s>>>(d.log_counts, (long long)pixels, d.log_offsets, count);
  if (storage == ST_PTR) log_kernel<ST_PTR, true><<<grid, block, smem, s>>>(a, L);
  else log_kernel<ST_ATLAS_LINEAR, true><<<grid, block, smem, s>>>(a, L);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return fail(c, AMR_ERR_CUDA, std::string("segment log launch: ") + cudaGetErrorString(e));
  return AMR_OK;
}

}  // namespace amr
