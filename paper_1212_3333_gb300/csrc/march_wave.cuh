// Warp-wavefront schedule of the ray march.
//
// The per-ray loop (march_kernel) leaves most lanes idle: segments of the 32 rays of a
// warp hold different numbers of samples, and only samples with non-zero opacity take the
// six-neighbour gradient path.  Here each warp works in rounds:
//   1. every live lane descends to its ray's next segment (Sec. 3.3 kd-restart) and
//      publishes the segment in shared memory;
//   2. a warp prefix sum over the segments' sample counts lays all samples of the round
//      out as one list, which the 32 lanes evaluate evenly (value, transfer function,
//      opacity), chunk by chunk;
//   3. the samples with non-zero opacity are compacted and shaded, again evenly;
//   4. front-to-back compositing is a segmented scan: a sample's weight needs only the
//      transmittance T_k = prod_{j<k} (1 - alpha_j) of its own ray, so each ray's colour is
//      a sum of T_k alpha_k rgb_k, and early termination keeps the samples with T_k > eps.
// Results are the same quantities as the per-ray loop (up to FP32 summation order).
#pragma once
#include "march.cuh"

namespace amr {

constexpr int kChunk = 128;              // sample positions per warp and chunk
constexpr int kPerLane = kChunk / 32;    // contiguous positions per lane when compositing

struct WaveSeg {      // one lane's current segment, published to the warp
  SegState s;
  float b0[3], db[3];
  float delta;
  int pad;
};

struct WarpArea {
  WaveSeg seg[32];
  int start[33];
  int njobs;
  unsigned short jobs[kChunk];
  float alpha[kChunk + kChunk / 8];
  float red[kChunk + kChunk / 8], green[kChunk + kChunk / 8], blue[kChunk + kChunk / 8];
  float dC[32][3];
  int Tend[32];     // float bits; transmittances are >= 0, so integer order is float order
  float Tstart[32];
  int cnt[32];
  float light[32][3];
};

__device__ __forceinline__ int pad_idx(int q) { return q + (q >> 3); }

// owner segment of sample position p: largest lane with start[lane] <= p (starts ascend)
__device__ __forceinline__ int find_owner(const int* start, int p) {
  int lo = 0;
#pragma unroll
  for (int step = 16; step >= 1; step >>= 1)
    if (start[lo + step] <= p) lo += step;
  return lo;
}

template <int ST, int INTERP, int SHADE>
__global__ void __launch_bounds__(128) wave_kernel(const __grid_constant__ RenderArgs A) {
  extern __shared__ float4 smem[];
  float4* s_tf = smem;
  int* s_nz = reinterpret_cast<int*>(smem + A.tf_n);
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  for (int k = tid; k < A.tf_n; k += blockDim.x * blockDim.y) s_tf[k] = A.tf[k];
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
  const int lane = tid & 31;
  const size_t tf_bytes = (size_t)A.tf_n * sizeof(float4) + (size_t)(A.tf_n + 1) * sizeof(int);
  WarpArea* W = reinterpret_cast<WarpArea*>(reinterpret_cast<char*>(smem) +
                                            ((tf_bytes + 15) & ~(size_t)15)) + (tid >> 5);

  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int jr = blockIdx.y * blockDim.y + threadIdx.y;
  const int j = A.ray.row0 + jr;
  const bool active = i < A.ray.width && jr < A.ray.rows && j < A.ray.height;
  float C0 = 0.f, C1 = 0.f, C2 = 0.f, T = 1.0f;
  unsigned nsamp = 0;
  unsigned long long status = 0;
  RayX rx;
  RayF rf;
  bool live = active && make_ray(A.ray, i, j, rx);
  if (live) make_frame(A.ray, rx, rf);
  if (live) {
    const float inv_dn = 1.0f / rf.dn;
    W->light[lane][0] = -rf.Dd[0] * (float)A.ray.hf[0] * inv_dn;
    W->light[lane][1] = -rf.Dd[1] * (float)A.ray.hf[1] * inv_dn;
    W->light[lane][2] = -rf.Dd[2] * (float)A.ray.hf[2] * inv_dn;
  }
  int pid0 = kPidIn;
  float tau0 = 0.0f, e0 = 0.0f;
  uint32_t start = 0;
  int nseg = 0, prev = -1;
  const float one_minus_eps = A.ert_thresh;  // include a sample while 1 - T < 1 - eps

  while (__any_sync(0xffffffffu, live)) {
    // ---- 1. next segment of every live ray
    int n = 0;
    if (live) {
      if (pid0 == kPidOut) {
        live = false;
      } else if (nseg >= A.max_segments) {
        status |= kStatusCapacity;
        live = false;
      } else {
        ++nseg;
        int pid1 = kPidOut;
        float tau1 = rf.tau_out, e1 = exit_bound(rf);
        const int lid = next_leaf(A.nodes, A.leaves, A.face_node, A.node_box, A.ray, i, j, rf,
                                  start, prev, pid0, tau0, e0, pid1, tau1, e1);
        if (lid < 0) {
          status |= kStatusDevice;
          live = false;
        } else {
          prev = lid;
          const DLeaf lf = A.leaves[lid];
          const DLevel& lv = A.lv[lf.level];
          n = segment_count(A.ray, i, j, rf, pid0, tau0, e0, pid1, tau1, e1, lv);
          if (n > kMaxSamplesPerSegment) {
            status |= kStatusCapacity;
            n = kMaxSamplesPerSegment;
          }
          if (A.skip && tf_transparent(s_nz, A.tf_n, lf.vmin, lf.vmax, A.vmin, A.inv_range)) n = 0;
          if (n > 0) {
            WaveSeg& ws = W->seg[lane];
            SegState& s = ws.s;
            s.brick = leaf_brick(A.patches, lf);
            s.level = lf.level;
            s.leaf = pack_leaf(lid, kNoLod);
            s.pid0 = pid0;
            s.pid1 = pid1;
            s.n = n;
            s.px = i;
            s.py = j;
            const float nfl = (float)n;
            const float dtau = (tau1 - tau0) / nfl;
            ws.delta = dtau * rf.dn;
            const float taum = fmaf(0.5f, dtau, tau0);
            const float etau = fmaxf(e0, e1) + ldexpf(tau1 + 1.0f, -21);
            float ex = 0.0f, bmax = 0.0f;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
              const float xm = fmaf(taum, rf.Dd[a], rf.Xe[a]);
              const float lo05 = 0.5f - (float)s.brick.lo[a];
              const float b0 = fmaf(xm, lv.inv_sc, lo05);
              const float db = dtau * rf.Dd[a] * lv.inv_sc;
              ws.b0[a] = b0;
              ws.db[a] = db;
              s.leaf_lo[a] = lf.lo[a];
              s.bl[a] = (float)(lf.lo[a] - s.brick.lo[a] * lv.sc) * lv.inv_sc + 0.5f;
              s.bh[a] = (float)(lf.hi[a] - s.brick.lo[a] * lv.sc) * lv.inv_sc + 0.5f;
              const float ea = fabsf(rf.Dd[a]) * etau +
                               ldexpf(fabsf(rf.Xe[a]) + fabsf(xm) + nfl * fabsf(dtau * rf.Dd[a]) + 1.0f, -21);
              ex = fmaxf(ex, ea);
              bmax = fmaxf(bmax, fabsf(b0) + nfl * fabsf(db) + (float)s.brick.dim[a]);
            }
            s.margin = ex * lv.inv_sc + ldexpf(bmax + 2.0f, -21);
          }
          pid0 = pid1;
          tau0 = tau1;
          e0 = e1;
        }
      }
    }
    // ---- 2. lay the round's samples out as one list
    int incl = n;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += v;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    W->start[lane] = incl - n;
    if (lane == 31) W->start[32] = total;
    __syncwarp();
    for (int base = 0; base < total; base += kChunk) {
      const int cnt = min(kChunk, total - base);
      if (lane == 0) W->njobs = 0;
      __syncwarp();
      // ---- value, transfer function and opacity of every sample
#pragma unroll 1
      for (int r = 0; r < kPerLane; ++r) {
        const int q = lane + 32 * r;
        bool job = false;
        if (q < cnt) {
          const int p = base + q;
          const int o = find_owner(W->start, p);
          const int k = p - W->start[o];
          const WaveSeg& ws = W->seg[o];
          float beta[3];
#pragma unroll
          for (int a = 0; a < 3; ++a) beta[a] = fmaf((float)k, ws.db[a], ws.b0[a]);
          const float v = sample_value<ST, INTERP>(A, A.ray, ws.s, beta, k);
          const float4 c = tf_lookup(s_tf, A.tf_n, v, A.vmin, A.inv_range);
          const float alpha = c.w > 0.0f ? -expm1f(-A.kappa * c.w * ws.delta) : 0.0f;
          const int pq = pad_idx(q);
          W->alpha[pq] = alpha;
          W->red[pq] = c.x;
          W->green[pq] = c.y;
          W->blue[pq] = c.z;
          job = SHADE >= 1 && alpha > 0.0f;
        }
        if constexpr (SHADE >= 1) {
          const unsigned m = __ballot_sync(0xffffffffu, job);
          int b = 0;
          if (lane == 0 && m) b = atomicAdd(&W->njobs, __popc(m));
          b = __shfl_sync(0xffffffffu, b, 0);
          if (job) W->jobs[b + __popc(m & ((1u << lane) - 1u))] = (unsigned short)q;
        }
      }
      __syncwarp();
      // ---- gradient Phong shading of the opaque samples, spread evenly over the lanes
      if constexpr (SHADE >= 1) {
        const int nj = W->njobs;
        for (int t = lane; t < nj; t += 32) {
          const int q = W->jobs[t];
          const int p = base + q;
          const int o = find_owner(W->start, p);
          const int k = p - W->start[o];
          const WaveSeg& ws = W->seg[o];
          float beta[3];
#pragma unroll
          for (int a = 0; a < 3; ++a) beta[a] = fmaf((float)k, ws.db[a], ws.b0[a]);
          const DLevel& lv = A.lv[ws.s.level];
          float g[3];
          gradient<ST, INTERP, (SHADE == 2)>(A, A.ray, ws.s, beta, k, lv, g);
          const float gn = sqrtf(fmaf(g[0], g[0], fmaf(g[1], g[1], g[2] * g[2])));
          const float gf = A.gfloor_num / lv.hmin;
          const float den = fmaxf(gn, gf);
          const float inv = den > 0.0f ? 1.0f / den : 0.0f;
          const float ndl = fabsf((g[0] * W->light[o][0] + g[1] * W->light[o][1] +
                                   g[2] * W->light[o][2]) * inv);
          const float spec = A.ks * __powf(ndl, A.shininess);
          const float diff = fmaf(A.kd, ndl, A.ka);
          const int pq = pad_idx(q);
          W->red[pq] = fminf(fmaxf(fmaf(W->red[pq], diff, spec), 0.0f), 1.0f);
          W->green[pq] = fminf(fmaxf(fmaf(W->green[pq], diff, spec), 0.0f), 1.0f);
          W->blue[pq] = fminf(fmaxf(fmaf(W->blue[pq], diff, spec), 0.0f), 1.0f);
        }
        __syncwarp();
      }
      // ---- front-to-back compositing as a segmented scan over contiguous positions
      W->dC[lane][0] = 0.0f;
      W->dC[lane][1] = 0.0f;
      W->dC[lane][2] = 0.0f;
      W->cnt[lane] = 0;
      W->Tstart[lane] = T;
      W->Tend[lane] = __float_as_int(T);
      __syncwarp();
      const int q0 = lane * kPerLane;
      const int q1 = min(q0 + kPerLane, cnt);
      // product of (1 - alpha) since the last run start (owner change or chunk start) seen
      // in this lane's positions; `head` records whether such a start lies in this lane
      float prod = 1.0f;
      bool head = false;
      for (int q = q0; q < q1; ++q) {
        const int p = base + q;
        if (q == 0 || p == W->start[find_owner(W->start, p)]) {
          prod = 1.0f;
          head = true;
        }
        prod *= 1.0f - W->alpha[pad_idx(q)];
      }
      // segmented inclusive scan of the run products across lanes
      float sp = prod;
      bool sf = head;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const float vp = __shfl_up_sync(0xffffffffu, sp, off);
        const bool vf = __shfl_up_sync(0xffffffffu, sf ? 1 : 0, off) != 0;
        if (lane >= off && !sf) {
          sp *= vp;
          sf = vf;
        }
      }
      float R = __shfl_up_sync(0xffffffffu, sp, 1);  // carried-in run product
      if (lane == 0) R = 1.0f;
      // per-position contributions T_p alpha_p rgb_p of the samples before termination
      float cr[kPerLane], cg[kPerLane], cb[kPerLane], cc[kPerLane];
      float l0 = 0.f, l1 = 0.f, l2 = 0.f, l3 = 0.f;  // sums since the last run start
#pragma unroll
      for (int u = 0; u < kPerLane; ++u) {
        const int q = q0 + u;
        cr[u] = cg[u] = cb[u] = cc[u] = 0.0f;
        if (q < q1) {
          const int p = base + q;
          const int o = find_owner(W->start, p);
          if (q == 0 || p == W->start[o]) {
            R = 1.0f;
            l0 = l1 = l2 = l3 = 0.0f;
          }
          const int pq = pad_idx(q);
          const float a = W->alpha[pq];
          const float Tp = W->Tstart[o] * R;
          const float Tn = Tp * (1.0f - a);
          if (1.0f - Tp < one_minus_eps) {  // not yet terminated before this sample
            const float w = Tp * a;
            cr[u] = w * W->red[pq];
            cg[u] = w * W->green[pq];
            cb[u] = w * W->blue[pq];
            cc[u] = 1.0f;
            // the last included sample of its ray in this chunk records the transmittance
            const bool next_same = p + 1 < min(W->start[o + 1], base + cnt);
            if (!(next_same && 1.0f - Tn < one_minus_eps)) W->Tend[o] = __float_as_int(Tn);
          }
          l0 += cr[u];
          l1 += cg[u];
          l2 += cb[u];
          l3 += cc[u];
          R *= 1.0f - a;
        }
      }
      // segmented inclusive scan of the partial sums across lanes (fixed order)
      float v0 = l0, v1 = l1, v2 = l2, v3 = l3;
      bool vf = head;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const float u0 = __shfl_up_sync(0xffffffffu, v0, off);
        const float u1 = __shfl_up_sync(0xffffffffu, v1, off);
        const float u2 = __shfl_up_sync(0xffffffffu, v2, off);
        const float u3 = __shfl_up_sync(0xffffffffu, v3, off);
        const bool uf = __shfl_up_sync(0xffffffffu, vf ? 1 : 0, off) != 0;
        if (lane >= off && !vf) {
          v0 += u0;
          v1 += u1;
          v2 += u2;
          v3 += u3;
          vf = uf;
        }
      }
      float a0 = __shfl_up_sync(0xffffffffu, v0, 1), a1 = __shfl_up_sync(0xffffffffu, v1, 1);
      float a2 = __shfl_up_sync(0xffffffffu, v2, 1), a3 = __shfl_up_sync(0xffffffffu, v3, 1);
      if (lane == 0) a0 = a1 = a2 = a3 = 0.0f;
      // running sums; the position that ends a ray's run in this chunk writes its total
#pragma unroll
      for (int u = 0; u < kPerLane; ++u) {
        const int q = q0 + u;
        if (q < q1) {
          const int p = base + q;
          const int o = find_owner(W->start, p);
          if (q == 0 || p == W->start[o]) a0 = a1 = a2 = a3 = 0.0f;
          a0 += cr[u];
          a1 += cg[u];
          a2 += cb[u];
          a3 += cc[u];
          if (q == cnt - 1 || p + 1 == W->start[o + 1]) {
            W->dC[o][0] = a0;
            W->dC[o][1] = a1;
            W->dC[o][2] = a2;
            W->cnt[o] = (int)a3;
          }
        }
      }
      __syncwarp();
      C0 += W->dC[lane][0];
      C1 += W->dC[lane][1];
      C2 += W->dC[lane][2];
      nsamp += (unsigned)W->cnt[lane];
      T = __int_as_float(W->Tend[lane]);
      if (live && 1.0f - T >= one_minus_eps) live = false;  // early ray termination
      __syncwarp();
    }
  }
  if (active) A.out[(size_t)jr * A.ray.width + i] = make_float4(C0, C1, C2, 1.0f - T);
  const unsigned tot = __reduce_add_sync(0xffffffffu, nsamp);
  if (lane == 0 && tot) atomicAdd(A.counters, (unsigned long long)tot);
  if (status) atomicOr(A.counters + 1, status);
}

}  // namespace amr
