// Warp-synchronous frame march with deferred shading (schedule 3).
//
// Under the per-ray loop (march_kernel) the opaque samples of a warp - a few percent of
// all samples - branch into gradient shading a handful of lanes at a time, and when a
// gradient neighbour lies beyond the leaf (a cross-leaf lookup through the tree) the whole
// warp waits for that chain of dependent loads.  Here every lane marches its own pixel as
// before, but the warp moves through one loop in step:
//   fetch  - lanes whose segment ended find their next non-empty segment;
//   sample - lanes with samples left take up to samples_per_iter samples: value, transfer
//            function, opacity and the accumulated alpha (so early ray termination is
//            decided at once); an opaque sample is queued with what its shading needs;
//   shade  - once 32 samples are queued (and at the end), each lane shades one of them
//            (gradient, Phong; with secondary rays the warp first marches each queued
//            sample's light ray together) and every lane then adds its own samples'
//            colours in sample order.
// The colour sum of a pixel sees the same terms in the same order as in the per-ray loop,
// so the image is bit-identical to it; only the moments at which the sums are taken
// change.  (With secondary rays each light ray's transmittance is a product taken in
// another order - 32 samples per round - so those images agree to rounding, not bits.)
#pragma once
#include "march.cuh"

namespace amr {

// An opaque sample waiting for its colour: position and segment, transfer-function colour
// and compositing weight w = (1 - A) alpha.  19 words (odd, so a warp writing one task per
// lane hits distinct banks).
struct ShadeTask {
  float beta[3];  // brick coordinates
  float cr, cg, cb;
  float w;
  float margin;   // bound on the FP32 position error (brick units)
  float Lx, Ly, Lz;
  int leaf;       // packed leaf id and pruning bound
  int pid0, pid1, n, k;
  int px, py;
};

struct DeferArea {
  ShadeTask task[32];
  float3 col[32];
  float T[32];    // secondary rays: transmittance from each task's sample to the light
};

// resident blocks per SM the register budget allows for (measured on C2, Phong, 2048^2 /
// 1024^2 / 512^2 Gsamples/s: 3 blocks 61.3 / 46.1 / 28.9, 4 blocks 55.9 / 41.9 / 24.9)
#ifndef AMR_MIN_BLOCKS_DEFERRED
#define AMR_MIN_BLOCKS_DEFERRED 3
#endif

// The sample of task t in finest-cell units (as composite_sample computes it).
__device__ __forceinline__ float3 task_point(const RenderArgs& A, const ShadeTask& t) {
  const DLeaf& lf = A.leaves[leaf_of(t.leaf)];
  const float sc = (float)A.lv[lf.level].sc;
  return make_float3((t.beta[0] - 0.5f + (float)lf.blo[0]) * sc,
                     (t.beta[1] - 0.5f + (float)lf.blo[1]) * sc,
                     (t.beta[2] - 0.5f + (float)lf.blo[2]) * sc);
}

// Colour of queued sample t (what composite_sample computes for an opaque sample); T is
// its transmittance to the light when SHADOW is set.
template <int ST, int GB, bool SHADOW = false>
__device__ __forceinline__ float3 shade_task(const RenderArgs& A, const RayArgs& R,
                                             const ShadeTask& t, float T = 1.0f) {
  const DLeaf lf = A.leaves[leaf_of(t.leaf)];
  const DLevel& lv = A.lv[lf.level];
  SegState s;
  s.brick = leaf_brick(A.patches, lf);
  s.level = lf.level;
  s.leaf = t.leaf;
  leaf_bounds(lf, lv, s.brick, lod_of(t.leaf), s.leaf_lo, s.bl, s.bh);
  s.margin = t.margin;
  s.pid0 = t.pid0;
  s.pid1 = t.pid1;
  s.n = t.n;
  s.px = t.px;
  s.py = t.py;
  const float beta[3] = {t.beta[0], t.beta[1], t.beta[2]};
  float gr[3];
  gradient<ST, 1, GB>(A, R, s, beta, t.k, lv, gr);
  float cr = t.cr, cg = t.cg, cb = t.cb;
  phong(A, lv, gr, t.Lx, t.Ly, t.Lz, cr, cg, cb);
  if constexpr (SHADOW) {
    const float I = fmaf(1.0f - A.light_ambient, T, A.light_ambient);
    cr *= I;
    cg *= I;
    cb *= I;
  }
  return make_float3(cr, cg, cb);
}

// The march of pixel (i, j) of view R by one lane of a warp whose 32 lanes all call this
// together (lanes without a pixel pass active = false); Q is the warp's queue area.
// Returns premultiplied RGBA (zero for inactive lanes); adds to nsamp and status.
// samples whose stencil maxima the deferred loop loads together (stencil-maximum bricks)
#ifndef AMR_DEFER_GROUP
#define AMR_DEFER_GROUP 8
#endif
constexpr int kDeferGroup = AMR_DEFER_GROUP;

template <int ST, int SHADE>
__device__ __forceinline__ float4 march_deferred(const RenderArgs& A, const RayArgs& R, int i,
                                                 int j, bool active, const float4* s_tf,
                                                 const int* s_nz, DeferArea& Q, unsigned& nsamp,
                                                 unsigned long long& status) {
  constexpr bool MX = (SHADE & kShadeMaxBit) != 0;  // the stencil-maximum test
  const unsigned FULL = 0xffffffffu;
  const int lane = (int)(threadIdx.x + blockDim.x * threadIdx.y) & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  RayF rf;
  float Lx = 0.f, Ly = 0.f, Lz = 0.f;
  bool live = false;
  {
    RayX rx;
    if (active && make_ray(R, i, j, rx)) {
      make_frame(R, rx, rf);
      const float inv_dn = 1.0f / rf.dn;
      Lx = -rf.Dd[0] * (float)R.hf[0] * inv_dn;
      Ly = -rf.Dd[1] * (float)R.hf[1] * inv_dn;
      Lz = -rf.Dd[2] * (float)R.hf[2] * inv_dn;
      live = true;
    }
  }
  float C0 = 0.f, C1 = 0.f, C2 = 0.f, Acc = 0.f;
  int pid0 = kPidIn, seg = 0, prev = -1;
  float tau0 = 0.f, e0 = 0.f;
  uint32_t start = 0;
  SegSetup g;
  g.s.n = 0;
  int k = 0;
  int queued = 0;      // warp-uniform: tasks in the queue
  unsigned mine = 0;   // this lane's queue slots

  // shade every queued task (one per lane), then each lane adds its own colours in order;
  // with secondary rays the whole warp first marches each task's light ray together
  auto drain = [&]() {
    __syncwarp();
    if constexpr ((SHADE & kShadeShadow) != 0) {
      for (int q = 0; q < queued; ++q) {
        const float3 x = task_point(A, Q.task[q]);
        const float T = warp_shadow_transmittance<ST>(A, R, s_tf, x.x, x.y, x.z);
        if (lane == 0) Q.T[q] = T;
      }
      __syncwarp();
    }
    if (lane < queued)
      Q.col[lane] = shade_task<ST, (SHADE & 3) == 2, (SHADE & kShadeShadow) != 0>(
          A, R, Q.task[lane], Q.T[lane]);
    __syncwarp();
    for (unsigned m = mine; m != 0; m &= m - 1) {
      const int q = __ffs(m) - 1;
      const float w = Q.task[q].w;
      const float3 c = Q.col[q];
      C0 = fmaf(w, c.x, C0);
      C1 = fmaf(w, c.y, C1);
      C2 = fmaf(w, c.z, C2);
    }
    __syncwarp();
    queued = 0;
    mine = 0;
  };

  // Every pass either fetches segments for at least one lane or takes samples, and each
  // ray has finitely many of both, so the loop ends with every lane's ray finished.
  for (;;) {
    const unsigned live_mask = __ballot_sync(FULL, live);
    if (live_mask == 0) break;
    // lanes whose segment ended fetch their next non-empty one (measured on C2: fetching
    // as soon as any lane needs beats waiting for a quarter or half of them)
    const bool need = live && k >= g.s.n;
    if (need) {
      for (;;) {
        if (pid0 == kPidOut) {
          live = false;
          break;
        }
        if (seg >= A.max_segments) {
          status |= kStatusCapacity;
          live = false;
          break;
        }
        ++seg;
        int pid1 = kPidOut;
        float tau1 = rf.tau_out, e1 = exit_bound(rf);
        const int lmin = lod_min_level(R, A.lv, rf, i, j, pid0, tau0, e0);
        const int lid = next_leaf(A.nodes, A.leaves, A.face_node, A.node_box, R, i, j, rf,
                                  start, prev, pid0, tau0, e0, pid1, tau1, e1, lmin);
        if (lid < 0) {
          status |= kStatusDevice;
          live = false;
          break;
        }
        prev = lid;
        const DLeaf lf = A.leaves[lid];
        const DLevel& lv = A.lv[lf.level];
        int n = segment_count(R, i, j, rf, pid0, tau0, e0, pid1, tau1, e1, lv);
        if (n > kMaxSamplesPerSegment) {
          status |= kStatusCapacity;
          n = kMaxSamplesPerSegment;
        }
        if (A.skip && tf_transparent(s_nz, A.tf_n, lf.vmin, lf.vmax, A.vmin, A.inv_range)) {
          pid0 = pid1;
          tau0 = tau1;
          e0 = e1;
          continue;
        }
        setup_segment(A, rf, lf, lv, lid, pid0, pid1, tau0, e0, tau1, e1, n, i, j, g, lmin);
        k = 0;
        pid0 = pid1;  // where the next segment starts
        tau0 = tau1;
        e0 = e1;
        break;
      }
    }
    // one sample step of every lane (the queue operations are warp-wide); mj: the sample's
    // stencil maximum when the stencil-maximum test is on
    auto take = [&](float mj) {
      bool opaque = false;
      float beta[3], cr = 0.f, cg = 0.f, cb = 0.f, w = 0.f;
      if (live && k < g.s.n) {
        ++nsamp;
#pragma unroll
        for (int a = 0; a < 3; ++a) beta[a] = fmaf((float)k, g.db[a], g.b0[a]);
        if (!(MX && stencil_transparent(A, s_nz, mj))) {  // else opacity zero
          const float v = trilinear<ST>(A, g.s.brick, beta[0], beta[1], beta[2]);
          const float4 c = tf_lookup(s_tf, A.tf_n, v, A.vmin, A.inv_range);
          if (c.w > 0.0f) {
            const float alpha = -expm1f(-A.kappa * c.w * g.delta);
            w = (1.0f - Acc) * alpha;
            Acc += w;
            cr = c.x;
            cg = c.y;
            cb = c.z;
            opaque = true;
          }
        }
        ++k;
      }
      const unsigned om = __ballot_sync(FULL, opaque);
      if (om != 0) {
        if (queued + __popc(om) > 32) drain();
        if (opaque) {
          const int q = queued + __popc(om & lt_mask);
          ShadeTask& t = Q.task[q];
          t.beta[0] = beta[0];
          t.beta[1] = beta[1];
          t.beta[2] = beta[2];
          t.cr = cr;
          t.cg = cg;
          t.cb = cb;
          t.w = w;
          t.margin = g.s.margin;
          t.Lx = Lx;
          t.Ly = Ly;
          t.Lz = Lz;
          t.leaf = g.s.leaf;
          t.pid0 = g.s.pid0;
          t.pid1 = g.s.pid1;
          t.n = g.s.n;
          t.k = k - 1;
          t.px = i;
          t.py = j;
          mine |= 1u << q;
          if (Acc >= A.ert_thresh) live = false;  // early ray termination
        }
        queued += __popc(om);
      }
    };
    if constexpr (MX) {
      // the stencil maxima of a lane's next kDeferGroup samples are loaded together, then
      // the steps take them in a rolled loop that rotates them through registers
      for (int step = 0; step < A.samples_per_iter;) {
        float m[kDeferGroup];
#pragma unroll
        for (int q = 0; q < kDeferGroup; ++q) {
          m[q] = __int_as_float(0x7f800000);
          if (live && k < g.s.n) {
            const int kk = min(k + q, g.s.n - 1);
            const Stencil<ST> st = stencil_at<ST>(g.s.brick, fmaf((float)kk, g.db[0], g.b0[0]),
                                                  fmaf((float)kk, g.db[1], g.b0[1]),
                                                  fmaf((float)kk, g.db[2], g.b0[2]));
            m[q] = fetch_max<ST>(A, g.s.brick, st.l0);
          }
        }
#pragma unroll 1
        for (int jj = 0; jj < kDeferGroup && step < A.samples_per_iter; ++jj, ++step) {
          const float mj = m[0];
#pragma unroll
          for (int q = 0; q + 1 < kDeferGroup; ++q) m[q] = m[q + 1];
          take(mj);
        }
      }
    } else {
      for (int step = 0; step < A.samples_per_iter; ++step) take(0.0f);
    }
  }
  if (queued != 0) drain();
  return make_float4(C0, C1, C2, Acc);
}

// Schedule 3: persistent warps taking 8x4-pixel tiles from the global queue (as
// march_kernel does for the per-ray loop), each marching its tile with deferred shading.
template <int ST, int SHADE>
__global__ void __launch_bounds__(128, AMR_MIN_BLOCKS_DEFERRED)
    deferred_kernel(const __grid_constant__ RenderArgs A) {
  extern __shared__ float4 smem[];
  float4* s_tf = smem;
  int* s_nz = reinterpret_cast<int*>(smem + A.tf_n);
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const size_t tf_bytes = (size_t)A.tf_n * sizeof(float4) + (size_t)(A.tf_n + 1) * sizeof(int);
  DeferArea& Q = reinterpret_cast<DeferArea*>(reinterpret_cast<char*>(smem) +
                                              ((tf_bytes + 15) & ~(size_t)15))[tid >> 5];
  stage_tf(A.tf, A.tf_n, s_tf, s_nz, tid, blockDim.x * blockDim.y);
  const int lane = tid & 31;
  const RayArgs& R = A.ray;
  const int tiles_x = (R.width + 7) / 8;
  const int n_tiles = tiles_x * ((R.rows + 3) / 4);
  unsigned nsamp = 0;
  unsigned long long status = 0;
  // each pass takes one tile, and the queue hands out every tile once
  for (;;) {
    int t = 0;
    if (lane == 0) {
      const unsigned long long q = atomicAdd(A.counters + kQueueCounter, 1ull);
      t = q < (unsigned long long)n_tiles ? (int)q : n_tiles;
    }
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= n_tiles) break;
    const int i = (t % tiles_x) * 8 + (lane & 7);
    const int jr = (t / tiles_x) * 4 + (lane >> 3);
    const int j = R.row0 + jr;
    const bool active = i < R.width && jr < R.rows && j < R.height;
    const float4 c = march_deferred<ST, SHADE>(A, R, i, j, active, s_tf, s_nz, Q, nsamp, status);
    if (active) A.out[(size_t)jr * R.width + i] = c;
  }
  const unsigned total = __reduce_add_sync(0xffffffffu, nsamp);
  if (lane == 0 && total) atomicAdd(A.counters, (unsigned long long)total);
  if (status) atomicOr(A.counters + 1, status);
}

}  // namespace amr
