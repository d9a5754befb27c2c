// Persistent-warp schedule of the frame march: lanes refill with new rays and warps fetch
// segments in batches, so a warp keeps most of its lanes busy although its rays need
// different numbers of segments and samples.
//
// The per-ray loop (march_kernel) runs each lane's segment loop to completion; lanes whose
// segment or ray ended wait for the others, and the frame kernel ran with about a quarter
// of its lanes active.  Here one loop per warp interleaves three steps:
//   refill  - once at most half the lanes hold a ray, free lanes take the next pixels of
//             the warp's current 8x4 pixel tile, tiles coming from a global queue;
//   fetch   - once at least half of the live lanes (or all of them) finished their
//             segment, those lanes descend to their next non-empty segment together;
//   sample  - lanes with samples left take up to `samples_per_iter` samples.
// Each lane calls the same per-ray functions in the same order as march_kernel, so the
// image is the same; only the interleaving of rays on the warp changes.
#pragma once
#include "march.cuh"

namespace amr {

template <int ST, int INTERP, int SHADE>
__global__ void __launch_bounds__(128, kMinBlocks<SHADE>)
    persist_kernel(const __grid_constant__ RenderArgs A, int samples_per_iter) {
  extern __shared__ float4 smem[];
  float4* s_tf = smem;
  int* s_nz = reinterpret_cast<int*>(smem + A.tf_n);
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  stage_tf(A.tf, A.tf_n, s_tf, s_nz, tid, blockDim.x * blockDim.y);

  const RayArgs& R = A.ray;
  const unsigned FULL = 0xffffffffu;
  const int lane = tid & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  const int W = R.width;
  const int tiles_x = (W + 7) / 8;
  const int n_tiles = tiles_x * ((R.rows + 3) / 4);

  // warp-uniform tile pool
  int tile = 0, handed = 32;
  bool exhausted = false;
  // lane state: the ray, its traversal position, the current segment
  bool live = false;
  int i = 0, jr = 0;
  RayF rf;
  float Lx = 0.f, Ly = 0.f, Lz = 0.f;
  float C0 = 0.f, C1 = 0.f, C2 = 0.f, Acc = 0.f;
  int pid0 = kPidOut, seg = 0, prev = -1;
  float tau0 = 0.f, e0 = 0.f;
  uint32_t start = 0;
  SegSetup g;
  g.s.n = 0;
  int k = 0;
  unsigned nsamp = 0;
  unsigned long long status = 0;

  auto finish = [&]() {
    A.out[(size_t)jr * W + i] = make_float4(C0, C1, C2, Acc);
    live = false;
  };

  // Every pass hands out pixels, fetches segments or takes samples, so the loop ends once
  // the queue is drained and every lane's ray has finished.
  for (;;) {
    // refill
    if (!exhausted && __popc(__ballot_sync(FULL, live)) <= 16) {
      for (;;) {
        const unsigned free = __ballot_sync(FULL, !live);
        if (free == 0) break;
        if (handed >= 32) {
          int t = 0;
          if (lane == 0) t = (int)atomicAdd(A.counters + kQueueCounter, 1ull);
          t = __shfl_sync(FULL, t, 0);
          if (t >= n_tiles) {
            exhausted = true;
            break;
          }
          tile = t;
          handed = 0;
        }
        const int avail = 32 - handed;
        const int rank = __popc(free & lt_mask);
        if (!live && rank < avail) {
          const int p = handed + rank;
          i = (tile % tiles_x) * 8 + (p & 7);
          jr = (tile / tiles_x) * 4 + (p >> 3);
          if (i < W && jr < R.rows) {
            RayX rx;
            C0 = C1 = C2 = Acc = 0.f;
            if (make_ray(R, i, R.row0 + jr, rx)) {
              make_frame(R, rx, rf);
              const float inv_dn = 1.0f / rf.dn;
              Lx = -rf.Dd[0] * (float)R.hf[0] * inv_dn;
              Ly = -rf.Dd[1] * (float)R.hf[1] * inv_dn;
              Lz = -rf.Dd[2] * (float)R.hf[2] * inv_dn;
              pid0 = kPidIn;
              tau0 = 0.f;
              e0 = 0.f;
              start = 0;
              seg = 0;
              prev = -1;
              k = 0;
              g.s.n = 0;
              live = true;
            } else {
              A.out[(size_t)jr * W + i] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
          }
        }
        handed += min(__popc(free), avail);
      }
    }
    const unsigned live_mask = __ballot_sync(FULL, live);
    if (live_mask == 0) {
      if (exhausted) break;
      continue;
    }
    // fetch the next non-empty segment, in batches of lanes
    const bool need = live && k >= g.s.n;
    const unsigned need_mask = __ballot_sync(FULL, need);
    if (need_mask != 0 &&
        (need_mask == live_mask || 2 * __popc(need_mask) >= __popc(live_mask))) {
      if (need) {
        for (;;) {
          if (pid0 == kPidOut) {
            finish();
            break;
          }
          if (seg >= A.max_segments) {
            status |= kStatusCapacity;
            finish();
            break;
          }
          ++seg;
          int pid1 = kPidOut;
          float tau1 = rf.tau_out, e1 = exit_bound(rf);
          const int lmin = lod_min_level(R, A.lv, rf, i, R.row0 + jr, pid0, tau0, e0);
          const int lid = next_leaf(A.nodes, A.leaves, A.face_node, A.node_box, R, i, R.row0 + jr,
                                    rf, start, prev, pid0, tau0, e0, pid1, tau1, e1, lmin);
          if (lid < 0) {
            status |= kStatusDevice;
            finish();
            break;
          }
          prev = lid;
          const DLeaf lf = A.leaves[lid];
          const DLevel& lv = A.lv[lf.level];
          int n = segment_count(R, i, R.row0 + jr, rf, pid0, tau0, e0, pid1, tau1, e1, lv);
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
          setup_segment(A, rf, lf, lv, lid, pid0, pid1, tau0, e0, tau1, e1, n, i, R.row0 + jr, g,
                        lmin);
          k = 0;
          pid0 = pid1;  // where the next segment starts
          tau0 = tau1;
          e0 = e1;
          break;
        }
      }
    }
    // sample
    if (live && k < g.s.n) {
      const DLevel& lv = A.lv[g.s.level];
      for (int q = 0; q < samples_per_iter && k < g.s.n; ++q) {
        ++nsamp;
        const bool ert = sample_one<ST, INTERP, SHADE>(A, R, s_tf, g, lv, k, Lx, Ly, Lz, C0, C1,
                                                       C2, Acc);
        ++k;
        if (ert) {
          finish();
          break;
        }
      }
    }
  }
  const unsigned total = __reduce_add_sync(FULL, nsamp);
  if (lane == 0 && total) atomicAdd(A.counters, (unsigned long long)total);
  if (status) atomicOr(A.counters + 1, status);
}

}  // namespace amr
