// Device side of the single-pass AMR raycaster (Sec. 3.3 of Kaehler & Abel).
//
// One thread per pixel; each warp marches 8x4-pixel tiles (taken from a queue by
// persistent warps), so the rays of a warp traverse nearly the same leaves and read nearly
// the same brick cache lines.
//
// Exactness without FP64 throughput.  The reference semantics are FP64: ray parameters of
// split planes t_s = (plane - o) / d decide the kd-restart descent, and the per-segment
// sample count n = max(1, ceil(len / step)) depends on exact t0, t1.  GB300 issues FP64 at
// a small fraction of its FP32 rate, so the kernel works in an FP32 frame
// tau = t - t_in (the ray parameter measured from the root entry point, which keeps the
// magnitudes small) and carries, for every FP32 quantity, a rigorous bound on its distance
// from the FP64 value.  A decision is taken in FP32 only when the bound cannot flip it;
// otherwise the exact FP64 quantities are recomputed from plane ids (each t0 / t1 is
// remembered as the split plane that produced it) and the decision is taken exactly.
// The same filtering guards the cell decisions of cross-leaf gradient lookups and of
// nearest sampling.  The traversal sequence and segment bounds therefore match the FP64
// reference bit for bit while the hot loops issue FP32 only.
//
// Every device loop is bounded; exceeding a bound sets a status bit, never traps.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "amr_device.h"

namespace amr {

// storage strategies; ids 4..7 are the 16-bit-cell variants of the two linear storages
enum {
  ST_PTR = 0, ST_TEXOBJ = 1, ST_ATLAS_LINEAR = 2, ST_ATLAS_TEX3D = 3,
  ST_PTR_F16 = 4, ST_PTR_BF16 = 5, ST_ATLAS_LINEAR_F16 = 6, ST_ATLAS_LINEAR_BF16 = 7
};

// plane ids: split * 4 + axis; the two ray ends use axis field 3
constexpr int kPidIn = 3;
constexpr int kPidOut = 7;

__device__ __forceinline__ double sel3(int a, double x, double y, double z) {
  return a == 0 ? x : (a == 1 ? y : z);
}
__device__ __forceinline__ float sel3f(int a, float x, float y, float z) {
  return a == 0 ? x : (a == 1 ? y : z);
}
__device__ __forceinline__ int sel3i(int a, int x, int y, int z) {
  return a == 0 ? x : (a == 1 ? y : z);
}

// Exact ray (FP64), used by the rare exact paths.
struct RayX {
  double o[3], d[3], inv[3];
  double t_in, t_out;
};

// FP32 frame of the ray.  tau_s(s) = s * B[a] + C[a] approximates t_s - t_in of split
// plane s on axis a within Ef[a]; X(tau) = Xe + tau * Dd approximates the position in
// finest-cell units (x - dlo) / h_f.
struct RayF {
  float B[3], C[3];      // leading parts
  float Bl[3], Cl[3];    // trailing parts (B = B + Bl, C = C + Cl to ~2^-48)
  float Xe[3], Dd[3];
  float tau_out;         // t_out - t_in (its bound: exit_bound)
  float dn;
  float t_in;            // root entry parameter (level-of-detail distance)
  int exact_axes;        // bit a set: planes on axis a are always decided in FP64
};

struct RayFSlot {
  RayF f;
  float pad;
};

// Pixel (i, j) -> exact ray and root interval.  The operation order is part of the
// contract: the FP64 reference evaluates the same expressions in the same order.
__device__ __forceinline__ bool make_ray(const RayArgs& A, int i, int j, RayX& r) {
  const double W = (double)A.width, H = (double)A.height;
  const double aspect = __ddiv_rn(W, H);
  const double u = __dmul_rn(
      __dmul_rn(__dsub_rn(__ddiv_rn(__dmul_rn(2.0, __dadd_rn((double)i, 0.5)), W), 1.0),
                A.tan_half_fov_y),
      aspect);
  const double v = __dmul_rn(
      __dsub_rn(1.0, __ddiv_rn(__dmul_rn(2.0, __dadd_rn((double)j, 0.5)), H)), A.tan_half_fov_y);
  double t_in = 0.0, t_out = __longlong_as_double(0x7ff0000000000000ll);
  bool hit = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    r.o[a] = A.eye[a];
    r.d[a] = __dadd_rn(__dadd_rn(A.fwd[a], __dmul_rn(u, A.right[a])), __dmul_rn(v, A.up[a]));
    const double lo = A.root_w[a], hi = A.root_w[3 + a];
    r.inv[a] = 0.0;
    if (r.d[a] != 0.0) {
      const double inv = __ddiv_rn(1.0, r.d[a]);
      r.inv[a] = inv;
      const double ta = __dmul_rn(__dsub_rn(lo, r.o[a]), inv);
      const double tb = __dmul_rn(__dsub_rn(hi, r.o[a]), inv);
      const double tn = ta < tb ? ta : tb;
      const double tf = ta < tb ? tb : ta;
      if (tn > t_in) t_in = tn;
      if (tf < t_out) t_out = tf;
    } else if (r.o[a] < lo || r.o[a] >= hi) {
      hit = false;
    }
  }
  if (!(t_in < t_out)) hit = false;
  r.t_in = t_in;
  r.t_out = t_out;
  return hit;
}

// Exact FP64 ray parameter of a plane id (the reference's t_s, t_in or t_out).
__device__ __forceinline__ double exact_t(const RayArgs& A, const RayX& r, int pid) {
  if (pid == kPidIn) return r.t_in;
  if (pid == kPidOut) return r.t_out;
  const int ax = pid & 3;
  const int s = pid >> 2;
  const double o = sel3(ax, r.o[0], r.o[1], r.o[2]);
  const double d = sel3(ax, r.d[0], r.d[1], r.d[2]);
  const double sw = __dadd_rn(sel3(ax, A.dlo[0], A.dlo[1], A.dlo[2]),
                              __dmul_rn((double)s, sel3(ax, A.hf[0], A.hf[1], A.hf[2])));
  (void)d;
  return __dmul_rn(__dsub_rn(sw, o), sel3(ax, r.inv[0], r.inv[1], r.inv[2]));
}

// The rare exact paths rebuild the FP64 ray of their pixel (make_ray is deterministic)
// instead of keeping it live, so the hot loops hold FP32 state only.

// Exact descent decision for plane `pid` against (t0, t1) = (pid0, pid1):
// 0 near only, 1 far only, 2 near with t1 = t_s.
static __device__ __noinline__ int exact_decide(const RayArgs& A, int px, int py, int pid,
                                                int pid0, int pid1) {
  atomicAdd(A.counters + 2, 1ull);
  RayX r;
  make_ray(A, px, py, r);
  const double t = exact_t(A, r, pid);
  if (t >= exact_t(A, r, pid1)) return 0;
  if (t <= exact_t(A, r, pid0)) return 1;
  return 2;
}

// Exact sample count n = max(1, ceil(len / step)) of the segment (pid0, pid1).
static __device__ __noinline__ int exact_count(const RayArgs& A, int px, int py, int pid0,
                                               int pid1, double step) {
  atomicAdd(A.counters + 3, 1ull);
  RayX r;
  make_ray(A, px, py, r);
  const double t0 = exact_t(A, r, pid0), t1 = exact_t(A, r, pid1);
  const double dn = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(r.d[0], r.d[0]),
                                                   __dmul_rn(r.d[1], r.d[1])),
                                         __dmul_rn(r.d[2], r.d[2])));
  const double len = __dmul_rn(__dsub_rn(t1, t0), dn);
  const double nf = ceil(__ddiv_rn(len, step));
  return nf < 1.0 ? 1 : (nf > (double)kMaxSamplesPerSegment ? kMaxSamplesPerSegment + 1 : (int)nf);
}

// Position of sample k of the segment (pid0, pid1, n), exactly as the FP64 reference
// computes it: t = t0 + (k + 1/2) (t1 - t0) / n, x = o + t d.
static __device__ __noinline__ double3 sample_x_exact(const RayArgs& A, int px, int py, int pid0,
                                                      int pid1, int n, int k) {
  atomicAdd(A.counters + 4, 1ull);
  RayX r;
  make_ray(A, px, py, r);
  const double t0 = exact_t(A, r, pid0);
  const double t1 = exact_t(A, r, pid1);
  const double dt = __ddiv_rn(__dsub_rn(t1, t0), (double)n);
  const double t = __dadd_rn(t0, __dmul_rn(__dadd_rn((double)k, 0.5), dt));
  return make_double3(__dadd_rn(r.o[0], __dmul_rn(t, r.d[0])),
                      __dadd_rn(r.o[1], __dmul_rn(t, r.d[1])),
                      __dadd_rn(r.o[2], __dmul_rn(t, r.d[2])));
}

// Build the FP32 frame.  tau_s = (s h_f + dlo - o) / d - t_in = s B + C with
// B = h_f / d and C = (dlo - e) / d, e = o + t_in d the root entry point.  B and C are
// kept as two-float pairs, so fma(s, B, C) + fma(s, Bl, Cl) carries only the final
// roundings: |error| <= 2u |tau_s| plus terms below 2^-45 (|s B| + |C|), all inside the
// per-node bound 2^-22 (|tau_s| + 1) while |s B| + |C| < 2^20 (else: exact decisions).
__device__ __forceinline__ void make_frame(const RayArgs& A, const RayX& r, RayF& f) {
  const double dn = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(r.d[0], r.d[0]),
                                                   __dmul_rn(r.d[1], r.d[1])),
                                         __dmul_rn(r.d[2], r.d[2])));
  f.dn = (float)dn;
  f.exact_axes = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double e = r.o[a] + r.t_in * r.d[a];  // entry point (accuracy only)
    const double smax = (double)max(abs(A.root_f[a]), abs(A.root_f[3 + a]));
    if (r.d[a] != 0.0) {
      const double inv = r.inv[a];
      const double B = A.hf[a] * inv;
      const double C = (A.dlo[a] - e) * inv;
      const float bh = (float)B, ch = (float)C;
      // B == 0 must mean d_a == 0: keep the sign of a B that would underflow
      f.B[a] = bh != 0.0f ? bh : copysignf(1e-38f, (float)inv);
      f.C[a] = ch;
      f.Bl[a] = (float)(B - (double)bh);
      f.Cl[a] = (float)(C - (double)ch);
      const bool fits = fabs(B) * smax + fabs(C) < 1048576.0 && fabs(B) > 1e-30;
      if (!fits) f.exact_axes |= 1 << a;
    } else {
      f.B[a] = f.C[a] = f.Bl[a] = f.Cl[a] = 0.0f;
      f.exact_axes |= 1 << a;
    }
    f.Xe[a] = (float)((e - A.dlo[a]) * A.inv_hf[a]);
    f.Dd[a] = (float)(r.d[a] * A.inv_hf[a]);
  }
  const double tau_out = r.t_out - r.t_in;
  f.tau_out = (float)tau_out;
  f.t_in = (float)r.t_in;
}

// error bound of tau_out (recomputed where needed instead of held per ray)
__device__ __forceinline__ float exit_bound(const RayF& f) { return ldexpf(f.tau_out + 1.0f, -22); }

// Level-of-detail pruning (Sec. 3.1: a type-(a) node's region is held by at least two
// levels; Sec. 3.3: the descent may stop there when the coarser cells project small
// enough).  For the segment starting at t0 the bound is X = lod_scale * t0 (a pixel's
// footprint at t0 times the threshold in pixels), and the descent stops at the first inner
// node whose label level l has min_a h^l_a <= X, i.e. l >= lod_min: the smallest such
// level, or kNoLod when pruning is off or no level qualifies.
constexpr int kNoLod = 1 << 20;
// shading variant bits of the kernels' SHADE parameter: 0 none, 1 Phong, 2 Phong with
// gradient bricks, plus kShadeShadow for secondary rays to the point light
constexpr int kShadeShadow = kShadeShadowBit;

static __device__ __noinline__ int lod_min_exact(const RayArgs& R, const DLevel* lv, int px,
                                                 int py, int pid0) {
  RayX r;
  make_ray(R, px, py, r);
  const double X = __dmul_rn(R.lod_scale, exact_t(R, r, pid0));
  for (int l = 0; l < R.levels; ++l)
    if (lv[l].hmin_d <= X) return l;
  return kNoLod;
}

// FP32 filter: t0 ~ t_in + tau0 within e0 and a few roundings; a level within the bound of
// X is decided on the exact FP64 values.
__device__ __forceinline__ int lod_min_level(const RayArgs& R, const DLevel* lv, const RayF& rf,
                                             int px, int py, int pid0, float tau0, float e0) {
  if (!(R.lod_scale_f > 0.0f)) return kNoLod;
  const float t0 = rf.t_in + tau0;
  const float X = R.lod_scale_f * t0;
  const float eX = R.lod_scale_f * (e0 + ldexpf(rf.t_in + fabsf(t0) + 1.0f, -22)) + ldexpf(X, -21);
  for (int l = 0; l < R.levels; ++l) {
    const float hm = lv[l].hmin, eh = ldexpf(hm, -22);
    if (hm + eh < X - eX) return l;  // certainly h <= X
    if (hm - eh > X + eX) continue;  // certainly h > X
    return lod_min_exact(R, lv, px, py, pid0);
  }
  return kNoLod;
}

// Pruned leaf of inner node i for bound lod_min, or -1.
__device__ __forceinline__ int lod_stop(const RayArgs& R, uint32_t i, int lod_min) {
  if (lod_min >= kNoLod) return -1;
  const int q = __ldg(R.lod + i);
  return (q >= 0 && (q & 31) >= lod_min) ? (q >> 5) : -1;
}

// FP32 ray parameter tau_s of split plane s on axis ax and its error bound (infinite on
// the axes whose planes are always decided in FP64).
__device__ __forceinline__ float plane_tau(const RayF& rf, uint32_t ax, int s, float& es) {
  const float sf = (float)s;
  const float ts = fmaf(sf, sel3f(ax, rf.B[0], rf.B[1], rf.B[2]), sel3f(ax, rf.C[0], rf.C[1], rf.C[2])) +
                   fmaf(sf, sel3f(ax, rf.Bl[0], rf.Bl[1], rf.Bl[2]),
                        sel3f(ax, rf.Cl[0], rf.Cl[1], rf.Cl[2]));
  es = ((rf.exact_axes >> ax) & 1) ? __int_as_float(0x7f800000) : ldexpf(fabsf(ts) + 1.0f, -22);
  return ts;
}

// kd-restart descent (Sec. 3.3) for the segment starting at (pid0, tau0): returns the leaf
// holding the ray just after t0 and narrows (pid1, tau1, e1) to the first split plane
// beyond t0.  Near child = the side entered first (d_a > 0: lower); t_s >= t1 -> near
// only; t_s <= t0 -> far only; otherwise near with t1 = t_s; d_a == 0 -> the side holding
// the origin.  Returns -1 on a malformed tree.
//
// Push-down (Horn et al.'s refinement of kd-restart): `start` is the deepest node reached
// before any narrowing, i.e. a node whose box holds the whole remaining ray [t0, t_out].
// Every later restart takes the same one-sided decisions above it (t0 only grows and t1
// is t_out there), so restarting at `start` instead of the root yields the same leaves
// and the same t1 bit for bit.  With level-of-detail pruning on, `start` stays at or above
// every type-(a) node on the path: the pruning bound grows with t0, so a later segment
// may stop at an ancestor that this one passed.
//
// `from` is where the descent begins: `start` itself (push = true), or a node known to hold
// the ray just after t0 whose ancestors' narrowing the caller has already applied (a rope,
// push = false: `start` is left as it is).
__device__ __forceinline__ int descend_from(const DNode* __restrict__ nodes, const RayArgs& A,
                                            int px, int py, const RayF& rf, uint32_t from,
                                            bool push, uint32_t& start, int pid0, float tau0,
                                            float e0, int& pid1, float& tau1, float& e1,
                                            int lod_min) {
  uint32_t i = from;
  bool pushing = push;  // no narrowing yet: the chosen child still holds all of [t0, t_out]
  for (int depth = 0; depth < kMaxDepth; ++depth) {
    const DNode nd = nodes[i];
    const uint32_t ax = nd.meta >> 30;
    const uint32_t idx = nd.meta & kIndexMask;
    if (ax == kLeafAxis) return (int)idx;
    // type-(a) node (pruning on for this ray): stop here if its level is coarse enough;
    // never push the restart below it, since a later segment may stop at it
    const int q = A.lod_scale_f > 0.0f ? __ldg(A.lod + i) : -1;
    if (q >= 0 && (q & 31) >= lod_min) return q >> 5;
    pushing = pushing && q < 0;
    const float B = sel3f(ax, rf.B[0], rf.B[1], rf.B[2]);
    if (B == 0.0f) {  // ray parallel to the plane: the origin's (eye's) side, exactly
      const double o = sel3(ax, A.eye[0], A.eye[1], A.eye[2]);
      const double sw = __dadd_rn(sel3(ax, A.dlo[0], A.dlo[1], A.dlo[2]),
                                  __dmul_rn((double)nd.split, sel3(ax, A.hf[0], A.hf[1], A.hf[2])));
      i = idx + (o < sw ? 0u : 1u);
      if (pushing) start = i;
      continue;
    }
    const int pid = nd.split * 4 + (int)ax;
    const uint32_t near_c = idx + (B > 0.0f ? 0u : 1u);
    const uint32_t far_c = idx + (B > 0.0f ? 1u : 0u);
    bool narrow = false;
    if (pid == pid0) {  // the plane that produced t0: t_s == t0
      i = far_c;
    } else if (pid == pid1) {  // the plane that produced t1: t_s == t1
      i = near_c;
    } else {
      float es;
      const float ts = plane_tau(rf, ax, nd.split, es);
      if (ts - tau1 > es + e1) {
        i = near_c;
      } else if (tau0 - ts > es + e0) {
        i = far_c;
      } else if (tau1 - ts > es + e1 && ts - tau0 > es + e0) {
        i = near_c;
        narrow = true;
      } else {  // too close to call in FP32: decide on the exact FP64 values
        const int dcs = exact_decide(A, px, py, pid, pid0, pid1);
        i = dcs == 1 ? far_c : near_c;
        narrow = dcs == 2;
      }
      if (narrow) {
        pid1 = pid;
        tau1 = ts;
        e1 = es;
      }
    }
    pushing = pushing && !narrow;
    if (pushing) start = i;
  }
  return -1;
}

__device__ __forceinline__ int descend(const DNode* __restrict__ nodes, const RayArgs& A, int px,
                                       int py, const RayF& rf, uint32_t& start, int pid0,
                                       float tau0, float e0, int& pid1, float& tau1, float& e1,
                                       int lod_min = kNoLod) {
  return descend_from(nodes, A, px, py, rf, start, true, start, pid0, tau0, e0, pid1, tau1, e1,
                      lod_min);
}

// Rope restart (neighbour links in the manner of Havran's ropes; the paper restarts every
// segment by kd-restart).  The segment after leaf `prev`, which the ray left through its
// face on plane pid0, begins in node N = the deepest node holding the level cell beyond
// that face (second half of the face table; often a leaf, which the table then names).
// A descent from N reaches the same leaf as one from the root whenever the ray just after
// t0 lies in N's box; and the planes the root descent would narrow (t1) to above N are
// N's ancestors' planes, of which only N's own exit planes can be nearest, so these are
// applied first (the root's faces are t_out already).  Both steps use the FP32 filter,
// narrowing falls back to the exact decision; when containment is too close to call (the
// ray passes near an edge of N) the caller descends from the push-down start.  On the
// exit-face axis the ray is inside N (N's lower side on that axis is the face or behind
// it); on an axis the ray runs parallel to, its coordinate stays inside the face's extent,
// which N holds.  Under level-of-detail pruning the root descent stops at the first
// type-(a) node whose label level reaches lod_min; the rope is taken only when no node
// above N does (N and its subtree the descent from N checks itself).  Returns the leaf when
// N is one (nothing left to descend), -2 - N's slot for an inner node, -1 for no rope.
__device__ __forceinline__ int rope_start(const int32_t* __restrict__ face_node,
                                          const int4* __restrict__ node_box,
                                          const DLeaf* __restrict__ leaves, const RayArgs& R,
                                          int px, int py, const RayF& rf, int prev, int pid0,
                                          float tau0, float e0, int& pid1, float& tau1,
                                          float& e1, int lod_min) {
  const int a = pid0 & 3;
  const bool up = sel3f(a, rf.B[0], rf.B[1], rf.B[2]) > 0.0f;
  const uint32_t ent = (uint32_t)__ldg(face_node + 12 * prev + 6 + 2 * a + (up ? 1 : 0));
  int blo[3], bhi[3], anc;
  if (ent & kFaceLeaf) {
    const int4* w = reinterpret_cast<const int4*>(leaves + (ent & ~kFaceLeaf));
    const int4 w1 = __ldg(w + 1), w2 = __ldg(w + 2);  // lo[3], hi[0] | hi[1], hi[2], lod_anc
    blo[0] = w1.x, blo[1] = w1.y, blo[2] = w1.z;
    bhi[0] = w1.w, bhi[1] = w2.x, bhi[2] = w2.y;
    anc = w2.z;
  } else {
    const int4 lo = __ldg(node_box + 2 * ent), hi = __ldg(node_box + 2 * ent + 1);
    blo[0] = lo.x, blo[1] = lo.y, blo[2] = lo.z;
    bhi[0] = hi.x, bhi[1] = hi.y, bhi[2] = hi.z;
    anc = lo.w;
  }
  if (anc >= lod_min) return -1;  // a node above N may stop the pruned descent
  int pid[3];
  float ts[3], es[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    pid[b] = -1;
    const float Bb = rf.B[b];
    if (Bb == 0.0f) continue;
    const bool fwd = Bb > 0.0f;
    const int s_in = fwd ? blo[b] : bhi[b], s_out = fwd ? bhi[b] : blo[b];
    if (b != a && s_in != (fwd ? R.root_f[b] : R.root_f[3 + b])) {
      float e;
      const float t = plane_tau(rf, b, s_in, e);
      if (!(tau0 - t > e + e0)) return -1;  // N entered at or after t0 on this axis
    }
    if (s_out != (fwd ? R.root_f[3 + b] : R.root_f[b])) {
      ts[b] = plane_tau(rf, b, s_out, es[b]);
      if (b != a && !(ts[b] - tau0 > es[b] + e0)) return -1;  // N left by t0
      pid[b] = s_out * 4 + b;
    }
  }
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    if (pid[b] < 0 || ts[b] - tau1 > es[b] + e1) continue;  // certainly not before t1
    const bool narrow = (tau1 - ts[b] > es[b] + e1 && ts[b] - tau0 > es[b] + e0) ||
                        exact_decide(R, px, py, pid[b], pid0, pid1) == 2;
    if (narrow) {
      pid1 = pid[b];
      tau1 = ts[b];
      e1 = es[b];
    }
  }
  return (ent & kFaceLeaf) ? (int)(ent & ~kFaceLeaf) : -2 - (int)ent;
}

// Leaf of the segment starting at (pid0, tau0) that follows leaf `prev` (-1 on the first
// segment): by rope when prev is a leaf of the unpruned tree, else (or when the rope's
// filter cannot decide, or a node above the rope's target may stop the pruned descent) by
// the push-down descent.  The leaf and the exact t1 are the same either way; only the
// plane id recorded for t1 may differ, between planes whose t1 is the same FP64 value.
__device__ __forceinline__ int next_leaf(const DNode* __restrict__ nodes,
                                         const DLeaf* __restrict__ leaves,
                                         const int32_t* __restrict__ face_node,
                                         const int4* __restrict__ node_box, const RayArgs& R,
                                         int px, int py, const RayF& rf, uint32_t& start,
                                         int prev, int pid0, float tau0, float e0, int& pid1,
                                         float& tau1, float& e1, int lod_min = kNoLod) {
  if (prev >= 0 && prev < R.n_leaves) {
    const int r = rope_start(face_node, node_box, leaves, R, px, py, rf, prev, pid0, tau0, e0,
                             pid1, tau1, e1, lod_min);
    if (r >= 0) return r;
    if (r <= -2)
      return descend_from(nodes, R, px, py, rf, (uint32_t)(-2 - r), false, start, pid0, tau0, e0,
                          pid1, tau1, e1, lod_min);
  }
  return descend(nodes, R, px, py, rf, start, pid0, tau0, e0, pid1, tau1, e1, lod_min);
}

// Node slot where the unpruned point location of finest cell f (inside the root) may start:
// the macro-grid cell's deepest node holding the whole cell.
__device__ __forceinline__ uint32_t macro_start(const RayArgs& R, int f0, int f1, int f2) {
  const int g0 = (f0 - R.root_f[0]) / R.macro_cell;
  const int g1 = (f1 - R.root_f[1]) / R.macro_cell;
  const int g2 = (f2 - R.root_f[2]) / R.macro_cell;
  return __ldg(R.macro + g0 + R.macro_dims[0] * (g1 + R.macro_dims[1] * g2));
}

// Point location by integer finest-cell coordinates (left iff f_a < split), stopping at a
// pruned node when lod_min says so.
__device__ __forceinline__ int locate_cell(const DNode* __restrict__ nodes, const RayArgs& R,
                                           int lod_min, int f0, int f1, int f2) {
  // unpruned: start at the macro-grid cell's node (a pruned descent must pass every
  // type-(a) node above the leaf, so it starts at the root)
  uint32_t i = lod_min >= kNoLod ? macro_start(R, f0, f1, f2) : 0u;
  for (int depth = 0; depth < kMaxDepth; ++depth) {
    const DNode nd = nodes[i];
    const uint32_t ax = nd.meta >> 30;
    const uint32_t idx = nd.meta & kIndexMask;
    if (ax == kLeafAxis) return (int)idx;
    const int pruned = lod_stop(R, i, lod_min);
    if (pruned >= 0) return pruned;
    i = idx + (sel3i(ax, f0, f1, f2) < nd.split ? 0u : 1u);
  }
  return -1;
}

// Point location from node `start` (which must hold the point), unpruned tree.
__device__ __forceinline__ int locate_cell_from(const DNode* __restrict__ nodes, uint32_t start,
                                                int f0, int f1, int f2) {
  uint32_t i = start;
  for (int depth = 0; depth < kMaxDepth; ++depth) {
    const DNode nd = nodes[i];
    const uint32_t ax = nd.meta >> 30;
    const uint32_t idx = nd.meta & kIndexMask;
    if (ax == kLeafAxis) return (int)idx;
    i = idx + (sel3i(ax, f0, f1, f2) < nd.split ? 0u : 1u);
  }
  return -1;
}

// Brick of one patch as held in registers while a segment is sampled.
struct BrickRef {
  long long base;  // pointer / element offset / texture object
  long long gbase; // the same for the gradient brick
  int sy, sz;
  int dim[3];
  int lo[3];
  int org[3];
};

// The brick of a leaf from its record (the 3D-atlas origin, used by that storage only,
// from the patch table).
__device__ __forceinline__ BrickRef leaf_brick(const DPatch* __restrict__ pt, const DLeaf& lf) {
  BrickRef b;
  b.base = lf.base;
  b.gbase = lf.gbase;
  b.sy = lf.sy;
  b.sz = lf.sz;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    b.dim[a] = lf.dim[a];
    b.lo[a] = lf.blo[a];
    b.org[a] = pt[lf.patch].org[a];
  }
  return b;
}

// In-brick element offsets: 32-bit for the per-patch storages (a brick holds fewer than
// 2^31 cells, checked at upload), 64-bit for the atlases, whose strides span the atlas.
template <int ST> struct BrickIndex { using type = long long; };
template <> struct BrickIndex<ST_PTR> { using type = int; };
template <> struct BrickIndex<ST_PTR_F16> { using type = int; };
template <> struct BrickIndex<ST_PTR_BF16> { using type = int; };
template <> struct BrickIndex<ST_TEXOBJ> { using type = int; };

template <int ST>
__device__ __forceinline__ float fetch(const RenderArgs& A, const BrickRef& b,
                                       typename BrickIndex<ST>::type lin, int i,
                                       int j, int k) {
  if constexpr (ST == ST_PTR) {
    return __ldg(reinterpret_cast<const float*>(b.base) + lin);
  } else if constexpr (ST == ST_ATLAS_LINEAR) {
    return __ldg(reinterpret_cast<const float*>(A.pool) + b.base + lin);
  } else if constexpr (ST == ST_PTR_F16) {
    return __half2float(__ldg(reinterpret_cast<const __half*>(b.base) + lin));
  } else if constexpr (ST == ST_PTR_BF16) {
    return __bfloat162float(__ldg(reinterpret_cast<const __nv_bfloat16*>(b.base) + lin));
  } else if constexpr (ST == ST_ATLAS_LINEAR_F16) {
    return __half2float(__ldg(reinterpret_cast<const __half*>(A.pool) + b.base + lin));
  } else if constexpr (ST == ST_ATLAS_LINEAR_BF16) {
    return __bfloat162float(__ldg(reinterpret_cast<const __nv_bfloat16*>(A.pool) + b.base + lin));
  } else if constexpr (ST == ST_TEXOBJ) {
    return tex3D<float>((cudaTextureObject_t)b.base, (float)i + 0.5f, (float)j + 0.5f,
                        (float)k + 0.5f);
  } else {
    return tex3D<float>(A.atlas, (float)(b.org[0] + i) + 0.5f, (float)(b.org[1] + j) + 0.5f,
                        (float)(b.org[2] + k) + 0.5f);
  }
}

// Gradient-brick cell: (V, V(c+x) - V(c-x), V(c+y) - V(c-y), V(c+z) - V(c-z)).
__device__ __forceinline__ float4 unpack_half4(uint2 u) {
  const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
  const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
  return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ float4 unpack_bf164(uint2 u) {
  const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
  const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
  return make_float4(a.x, a.y, b.x, b.y);
}

template <int ST>
__device__ __forceinline__ float4 fetch4(const RenderArgs& A, const BrickRef& b,
                                         typename BrickIndex<ST>::type lin,
                                         int i, int j, int k) {
  if constexpr (ST == ST_PTR) {
    return __ldg(reinterpret_cast<const float4*>(b.gbase) + lin);
  } else if constexpr (ST == ST_ATLAS_LINEAR) {
    return __ldg(A.gpool + b.gbase + lin);
  } else if constexpr (ST == ST_PTR_F16) {
    return unpack_half4(__ldg(reinterpret_cast<const uint2*>(b.gbase) + lin));
  } else if constexpr (ST == ST_PTR_BF16) {
    return unpack_bf164(__ldg(reinterpret_cast<const uint2*>(b.gbase) + lin));
  } else if constexpr (ST == ST_ATLAS_LINEAR_F16) {
    return unpack_half4(__ldg(reinterpret_cast<const uint2*>(A.gpool) + b.gbase + lin));
  } else if constexpr (ST == ST_ATLAS_LINEAR_BF16) {
    return unpack_bf164(__ldg(reinterpret_cast<const uint2*>(A.gpool) + b.gbase + lin));
  } else if constexpr (ST == ST_TEXOBJ) {
    return tex3D<float4>((cudaTextureObject_t)b.gbase, (float)i + 0.5f, (float)j + 0.5f,
                         (float)k + 0.5f);
  } else {
    return tex3D<float4>(A.gatlas, (float)(b.org[0] + i) + 0.5f, (float)(b.org[1] + j) + 0.5f,
                         (float)(b.org[2] + k) + 0.5f);
  }
}

// Trilinear interpolation at brick coordinate beta (brick index = cell - lo + 1, cell
// centres at integer beta).  Coordinates are clamped into the brick, which reproduces edge
// replication where the brick touches the domain boundary.
// The eight cells around a brick position and the interpolation weights: fetched first,
// combined later, so a sample's loads can be issued while the previous sample is shaded.
struct Corners {
  float v[8];
  float wx, wy, wz;
  __device__ __forceinline__ float value() const {
    const float c00 = fmaf(wx, v[1] - v[0], v[0]);
    const float c10 = fmaf(wx, v[3] - v[2], v[2]);
    const float c01 = fmaf(wx, v[5] - v[4], v[4]);
    const float c11 = fmaf(wx, v[7] - v[6], v[6]);
    const float c0 = fmaf(wy, c10 - c00, c00);
    const float c1 = fmaf(wy, c11 - c01, c01);
    return fmaf(wz, c1 - c0, c0);
  }
};

template <int ST>
__device__ __forceinline__ Corners trilinear_fetch(const RenderArgs& A, const BrickRef& b,
                                                   float bx, float by, float bz) {
  bx = fminf(fmaxf(bx, 0.0f), (float)(b.dim[0] - 1));
  by = fminf(fmaxf(by, 0.0f), (float)(b.dim[1] - 1));
  bz = fminf(fmaxf(bz, 0.0f), (float)(b.dim[2] - 1));
  const int ix = min((int)bx, b.dim[0] - 2);
  const int iy = min((int)by, b.dim[1] - 2);
  const int iz = min((int)bz, b.dim[2] - 2);
  Corners c;
  c.wx = bx - (float)ix;
  c.wy = by - (float)iy;
  c.wz = bz - (float)iz;
  using I = typename BrickIndex<ST>::type;
  const I l0 = (I)ix + (I)b.sy * iy + (I)b.sz * iz;
  c.v[0] = fetch<ST>(A, b, l0, ix, iy, iz);
  c.v[1] = fetch<ST>(A, b, l0 + 1, ix + 1, iy, iz);
  c.v[2] = fetch<ST>(A, b, l0 + b.sy, ix, iy + 1, iz);
  c.v[3] = fetch<ST>(A, b, l0 + b.sy + 1, ix + 1, iy + 1, iz);
  c.v[4] = fetch<ST>(A, b, l0 + b.sz, ix, iy, iz + 1);
  c.v[5] = fetch<ST>(A, b, l0 + b.sz + 1, ix + 1, iy, iz + 1);
  c.v[6] = fetch<ST>(A, b, l0 + b.sz + b.sy, ix, iy + 1, iz + 1);
  c.v[7] = fetch<ST>(A, b, l0 + b.sz + b.sy + 1, ix + 1, iy + 1, iz + 1);
  return c;
}

// Trilinear interpolation at brick position (bx, by, bz), clamped into the brick.
template <int ST>
__device__ __forceinline__ float trilinear(const RenderArgs& A, const BrickRef& b, float bx,
                                           float by, float bz) {
  return trilinear_fetch<ST>(A, b, bx, by, bz).value();
}

// The trilinear stencil of a brick position, as trilinear_fetch computes it (clamped into
// the brick): its lower corner's element offset and the weights.
template <int ST>
struct Stencil {
  typename BrickIndex<ST>::type l0;
  float wx, wy, wz;
};

template <int ST>
__device__ __forceinline__ Stencil<ST> stencil_at(const BrickRef& b, float bx, float by, float bz) {
  bx = fminf(fmaxf(bx, 0.0f), (float)(b.dim[0] - 1));
  by = fminf(fmaxf(by, 0.0f), (float)(b.dim[1] - 1));
  bz = fminf(fmaxf(bz, 0.0f), (float)(b.dim[2] - 1));
  const int ix = min((int)bx, b.dim[0] - 2);
  const int iy = min((int)by, b.dim[1] - 2);
  const int iz = min((int)bz, b.dim[2] - 2);
  using I = typename BrickIndex<ST>::type;
  Stencil<ST> st;
  st.wx = bx - (float)ix;
  st.wy = by - (float)iy;
  st.wz = bz - (float)iz;
  st.l0 = (I)ix + (I)b.sy * iy + (I)b.sz * iz;
  return st;
}

// Trilinear value of a stencil (the arithmetic of Corners::value on the same cells).
template <int ST>
__device__ __forceinline__ float stencil_value(const RenderArgs& A, const BrickRef& b,
                                               const Stencil<ST>& st) {
  static_assert(ST == ST_PTR || ST == ST_PTR_F16 || ST == ST_PTR_BF16,
                "stencil-maximum bricks belong to the pointer storage");
  Corners c;
  c.wx = st.wx;
  c.wy = st.wy;
  c.wz = st.wz;
  const auto l0 = st.l0;
  c.v[0] = fetch<ST>(A, b, l0, 0, 0, 0);
  c.v[1] = fetch<ST>(A, b, l0 + 1, 0, 0, 0);
  c.v[2] = fetch<ST>(A, b, l0 + b.sy, 0, 0, 0);
  c.v[3] = fetch<ST>(A, b, l0 + b.sy + 1, 0, 0, 0);
  c.v[4] = fetch<ST>(A, b, l0 + b.sz, 0, 0, 0);
  c.v[5] = fetch<ST>(A, b, l0 + b.sz + 1, 0, 0, 0);
  c.v[6] = fetch<ST>(A, b, l0 + b.sz + b.sy, 0, 0, 0);
  c.v[7] = fetch<ST>(A, b, l0 + b.sz + b.sy + 1, 0, 0, 0);
  return c.value();
}

// The stencil-maximum brick's cell at offset lin (pointer storage; the maximum of the
// eight stencil cells starting there, in the cell type): the value brick shifted by
// A.mdelta bytes.
template <int ST>
__device__ __forceinline__ float fetch_max(const RenderArgs& A, const BrickRef& b,
                                           typename BrickIndex<ST>::type lin) {
  if constexpr (ST == ST_PTR) {
    return __ldg(reinterpret_cast<const float*>(b.base + A.mdelta) + lin);
  } else if constexpr (ST == ST_PTR_F16) {
    return __half2float(__ldg(reinterpret_cast<const __half*>(b.base + A.mdelta) + lin));
  } else if constexpr (ST == ST_PTR_BF16) {
    return __bfloat162float(__ldg(reinterpret_cast<const __nv_bfloat16*>(b.base + A.mdelta) + lin));
  } else {
    return __int_as_float(0x7f800000);  // no maximum bricks: never transparent
  }
}

// Whether every value up to m - and so a trilinear value whose stencil's maximum is m - maps
// to zero opacity: tf_lookup's index of m (the same FP32 arithmetic, monotone in the
// value), plus one entry of margin for the last-bit rounding of the interpolation, and
// every table entry up to the next one after it transparent (nz: prefix counts of the
// non-transparent entries).
__device__ __forceinline__ bool stencil_transparent(const RenderArgs& A, const int* nz, float m) {
  const float u = fminf(fmaxf((m - A.vmin) * A.inv_range, 0.0f), 1.0f) * (float)(A.tf_n - 1);
  return nz[min((int)u + 3, A.tf_n)] == 0;
}

// Nearest cell value at integer brick index (clamped).
template <int ST>
__device__ __forceinline__ float cell_at(const RenderArgs& A, const BrickRef& b, int i, int j,
                                         int k) {
  i = min(max(i, 0), b.dim[0] - 1);
  j = min(max(j, 0), b.dim[1] - 1);
  k = min(max(k, 0), b.dim[2] - 1);
  using I = typename BrickIndex<ST>::type;
  return fetch<ST>(A, b, (I)i + (I)b.sy * j + (I)b.sz * k, i, j, k);
}

// State of the segment being sampled.
struct SegState {
  BrickRef brick;
  int level;
  int leaf;           // leaf id (bits 0..25) and the segment's pruning bound (26..31; 63: none)
  int leaf_lo[3];     // finest cells
  float bl[3], bh[3]; // leaf box in brick coordinates
  float margin;       // bound on |FP32 beta - beta of the exact FP64 sample position|
  int pid0, pid1, n;  // exact segment: t0, t1 by plane id, n samples
  int px, py;         // pixel (the exact paths rebuild its ray)
};

// SegState.leaf packing: the pruning bound rides in the top bits of the leaf id
constexpr uint32_t kLeafBits = 26, kLeafMask = (1u << kLeafBits) - 1u, kLodNone = 63u;
__device__ __forceinline__ int pack_leaf(int leaf, int lod_min) {
  const uint32_t l = lod_min >= kNoLod ? kLodNone : (uint32_t)lod_min;
  return (int)(((uint32_t)leaf & kLeafMask) | (l << kLeafBits));
}
__device__ __forceinline__ int leaf_of(int packed) { return (int)((uint32_t)packed & kLeafMask); }
__device__ __forceinline__ int lod_of(int packed) {
  const uint32_t l = (uint32_t)packed >> kLeafBits;
  return l == kLodNone ? kNoLod : (int)l;
}

// finest cell of an exact point, clamped into the root (the reference's rule)
__device__ __forceinline__ int finest_cell_exact(const RayArgs& A, double x, int a) {
  const double q = floor(__ddiv_rn(__dsub_rn(x, A.dlo[a]), A.hf[a]));
  if (q < (double)A.root_f[a]) return A.root_f[a];
  if (q > (double)(A.root_f[3 + a] - 1)) return A.root_f[3 + a] - 1;
  return (int)q;
}

// Brick index of the level-l cell holding an exact point (nearest sampling).
__device__ __forceinline__ int nearest_index_exact(const RayArgs& A, const DLevel& lv, double x,
                                                   int a, int lo) {
  return (int)floor(__ddiv_rn(__dsub_rn(x, A.dlo[a]), lv.h[a])) - lo + 1;
}

// Cross-leaf gradient neighbour x_k + sign h^l e_a: descend the tree on finest-cell
// coordinates relative to the current leaf corner; a split within the error margin sends
// the decision to FP64.  The current leaf's level and corner come from the caller, so the
// first load of the lookup is the face table.  (x0, x1, x2): the neighbour in finest cells
// from the leaf corner (lo0, lo1, lo2); mf: its error margin in finest cells; beyond: the
// point lies clearly beyond the face (a, sign).  Inlined at its one call site (the rolled
// neighbour loop): as a call, saving and restoring the caller's live registers around
// 18.5 M lookups per C2 2048^2 frame cost more than the lookups (measured 52.8 -> 61.6
// Gsamples/s).
template <int ST, int INTERP>
__device__ __forceinline__ float neighbour_slow(const RenderArgs& A, const RayArgs& R, int px, int py,
                                             int leaf_lod, int level, int lo0, int lo1, int lo2,
                                             int pid0, int pid1, int n, int k, float mf,
                                             float x0, float x1, float x2, int a, float sign,
                                             bool beyond) {
  const int leaf = leaf_of(leaf_lod), lod_min = lod_of(leaf_lod);
  const DLevel& lv = A.lv[level];
  const float xr[3] = {x0, x1, x2};
  const int clo[3] = {lo0, lo1, lo2};
  bool amb = false;
  int lid = -1;
  const bool pruning = lod_min < kNoLod;
  // the neighbour lies in the leaf or in the level cell beyond its face (a, sign): start at
  // the deepest node holding both, or the cell alone when the point is clearly beyond the
  // face, which the face table names directly when it is a leaf.  Under pruning only when
  // no type-(a) node above that start reaches the bound (else from the root), and never
  // from a pruned leaf (the table covers the unpruned leaves)
  uint32_t i = 0;
  if (leaf < R.n_leaves) {
    const uint32_t ent =
        (uint32_t)__ldg(A.face_node + 12 * leaf + (beyond ? 6 : 0) + 2 * a + (sign > 0.0f ? 1 : 0));
    bool ok = true;
    if (pruning) {
      const int anc = (ent & kFaceLeaf) ? __ldg(&A.leaves[ent & ~kFaceLeaf].lod_anc)
                                        : __ldg(&A.node_box[2 * ent].w);
      ok = anc < lod_min;
    }
    if (ok) {
      if (ent & kFaceLeaf) lid = (int)(ent & ~kFaceLeaf);
      else i = ent;
    }
  }
  for (int depth = 0; lid < 0 && depth < kMaxDepth; ++depth) {
    const DNode nd = A.nodes[i];
    const uint32_t ax = nd.meta >> 30;
    const uint32_t idx = nd.meta & kIndexMask;
    if (ax == kLeafAxis) {
      lid = (int)idx;
      break;
    }
    if (pruning) {
      const int pruned = lod_stop(R, i, lod_min);
      if (pruned >= 0) {
        lid = pruned;
        break;
      }
    }
    const float diff = sel3f(ax, xr[0], xr[1], xr[2]) - (float)(nd.split - sel3i(ax, clo[0], clo[1], clo[2]));
    if (fabsf(diff) <= mf) {
      amb = true;
      break;
    }
    i = idx + (diff < 0.0f ? 0u : 1u);
  }
  double xe[3] = {0.0, 0.0, 0.0};
  auto exact_point = [&]() {
    const double3 x = sample_x_exact(R, px, py, pid0, pid1, n, k);
    xe[0] = x.x;
    xe[1] = x.y;
    xe[2] = x.z;
    const double hq = sel3(a, lv.h[0], lv.h[1], lv.h[2]);
    if (a == 0) xe[0] = sign > 0.0f ? __dadd_rn(xe[0], hq) : __dsub_rn(xe[0], hq);
    if (a == 1) xe[1] = sign > 0.0f ? __dadd_rn(xe[1], hq) : __dsub_rn(xe[1], hq);
    if (a == 2) xe[2] = sign > 0.0f ? __dadd_rn(xe[2], hq) : __dsub_rn(xe[2], hq);
  };
  if (amb) {
    exact_point();
    lid = locate_cell(A.nodes, R, lod_min, finest_cell_exact(R, xe[0], 0),
                      finest_cell_exact(R, xe[1], 1),
                      finest_cell_exact(R, xe[2], 2));
  }
  if (lid < 0) return 0.0f;
  const DLeaf lf = A.leaves[lid];
  const BrickRef nb = leaf_brick(A.patches, lf);
  const DLevel& lw = A.lv[lf.level];
  float bq[3];
  if (amb) {
#pragma unroll
    for (int q = 0; q < 3; ++q)
      bq[q] = (float)((xe[q] - R.dlo[q]) * lw.inv_h[q] + (0.5 - (double)nb.lo[q]));
  } else {
#pragma unroll
    for (int q = 0; q < 3; ++q)
      bq[q] = fmaf(xr[q], lw.inv_sc, (float)(clo[q] - nb.lo[q] * lw.sc) * lw.inv_sc + 0.5f);
  }
  if constexpr (INTERP == 1) {
    return trilinear<ST>(A, nb, bq[0], bq[1], bq[2]);
  } else {
    if (!amb) {
      const float fx = bq[0] + 0.5f, fy = bq[1] + 0.5f, fz = bq[2] + 0.5f;
      const float rx = fx - floorf(fx), ry = fy - floorf(fy), rz = fz - floorf(fz);
      const float mq = mf * lw.inv_sc;
      if (fminf(fminf(fminf(rx, 1.0f - rx), fminf(ry, 1.0f - ry)), fminf(rz, 1.0f - rz)) > mq)
        return cell_at<ST>(A, nb, (int)floorf(fx), (int)floorf(fy), (int)floorf(fz));
      exact_point();
    }
    return cell_at<ST>(A, nb, nearest_index_exact(R, lw, xe[0], 0, nb.lo[0]),
                       nearest_index_exact(R, lw, xe[1], 1, nb.lo[1]),
                       nearest_index_exact(R, lw, xe[2], 2, nb.lo[2]));
  }
}

// Exact nearest-cell value of sample k in its own brick (rare path).
template <int ST>
__device__ __noinline__ float nearest_sample_exact(const RenderArgs& A, const RayArgs& R, int px,
                                                   int py, int leaf,
                                                   int pid0, int pid1, int n, int k) {
  const DLeaf cl = A.leaves[leaf];
  const DLevel& lv = A.lv[cl.level];
  const BrickRef b = leaf_brick(A.patches, cl);
  const double3 x = sample_x_exact(R, px, py, pid0, pid1, n, k);
  return cell_at<ST>(A, b, nearest_index_exact(R, lv, x.x, 0, b.lo[0]),
                     nearest_index_exact(R, lv, x.y, 1, b.lo[1]),
                     nearest_index_exact(R, lv, x.z, 2, b.lo[2]));
}

// Value of the AMR field at the gradient neighbour bn = x_k + sg h^l e_ax (Sec. 4: shading
// reads across block boundaries).  Inside the current leaf (beyond the error margin) it is
// the current brick; otherwise the slow path locates the finest leaf holding the point.
template <int ST, int INTERP>
__device__ __forceinline__ float neighbour_at(const RenderArgs& A, const RayArgs& R,
                                              const SegState& s, const DLevel& lv,
                                              const float* bn, int k, int ax, float sg) {
  const float m = s.margin;
  bool inside = true;
#pragma unroll
  for (int q = 0; q < 3; ++q) inside = inside && (bn[q] >= s.bl[q] + m) && (bn[q] < s.bh[q] - m);
  if (inside) {
    if constexpr (INTERP == 1) {
      return trilinear<ST>(A, s.brick, bn[0], bn[1], bn[2]);
    } else {
      const float fx = bn[0] + 0.5f, fy = bn[1] + 0.5f, fz = bn[2] + 0.5f;
      const float rx = fx - floorf(fx), ry = fy - floorf(fy), rz = fz - floorf(fz);
      if (fminf(fminf(fminf(rx, 1.0f - rx), fminf(ry, 1.0f - ry)), fminf(rz, 1.0f - rz)) > m)
        return cell_at<ST>(A, s.brick, (int)floorf(fx), (int)floorf(fy), (int)floorf(fz));
    }
  }
  // finest cells from the leaf corner; beyond the face against the (possibly widened) leaf
  // bound, which only ever errs towards the deeper start node
  const float scf = (float)lv.sc;
  float x[3];
#pragma unroll
  for (int q = 0; q < 3; ++q)
    x[q] = (bn[q] - ((float)(s.leaf_lo[q] - s.brick.lo[q] * lv.sc) * lv.inv_sc + 0.5f)) * scf;
  const float ba = sel3f(ax, bn[0], bn[1], bn[2]);
  const bool beyond = sg > 0.0f ? ba >= sel3f(ax, s.bh[0], s.bh[1], s.bh[2]) + m
                                : ba < sel3f(ax, s.bl[0], s.bl[1], s.bl[2]) - m;
  return neighbour_slow<ST, INTERP>(A, R, s.px, s.py, s.leaf, s.level, s.leaf_lo[0],
                                    s.leaf_lo[1], s.leaf_lo[2], s.pid0, s.pid1, s.n, k,
                                    m * scf, x[0], x[1], x[2], ax, sg, beyond);
}

// Value at the sample itself (the segment's own leaf and level, Sec. 3.3).
template <int ST, int INTERP>
__device__ __forceinline__ float sample_value(const RenderArgs& A, const RayArgs& R,
                                              const SegState& s,
                                              const float* beta, int k) {
  if constexpr (INTERP == 1) {
    return trilinear<ST>(A, s.brick, beta[0], beta[1], beta[2]);
  } else {
    const float fx = beta[0] + 0.5f, fy = beta[1] + 0.5f, fz = beta[2] + 0.5f;
    const float rx = fx - floorf(fx), ry = fy - floorf(fy), rz = fz - floorf(fz);
    if (fminf(fminf(fminf(rx, 1.0f - rx), fminf(ry, 1.0f - ry)), fminf(rz, 1.0f - rz)) > s.margin)
      return cell_at<ST>(A, s.brick, (int)floorf(fx), (int)floorf(fy), (int)floorf(fz));
    return nearest_sample_exact<ST>(A, R, s.px, s.py, leaf_of(s.leaf), s.pid0, s.pid1, s.n, k);
  }
}

__device__ __forceinline__ float4 tf_lookup(const float4* __restrict__ tf, int n, float v,
                                            float vmin, float inv_range) {
  float u = (v - vmin) * inv_range;
  u = fminf(fmaxf(u, 0.0f), 1.0f) * (float)(n - 1);
  const int i = min((int)u, n - 2);
  const float w = u - (float)i;
  const float4 a = tf[i], b = tf[i + 1];
  return make_float4(fmaf(w, b.x - a.x, a.x), fmaf(w, b.y - a.y, a.y), fmaf(w, b.z - a.z, a.z),
                     fmaf(w, b.w - a.w, a.w));
}

// true when the transfer function is fully transparent over [v0, v1] (conservative)
__device__ __forceinline__ bool tf_transparent(const int* __restrict__ nz_prefix, int n, float v0,
                                               float v1, float vmin, float inv_range) {
  float u0 = fminf(fmaxf((v0 - vmin) * inv_range, 0.0f), 1.0f) * (float)(n - 1);
  float u1 = fminf(fmaxf((v1 - vmin) * inv_range, 0.0f), 1.0f) * (float)(n - 1);
  const int i0 = max((int)u0 - 1, 0);
  const int i1 = min((int)u1 + 2, n - 1);
  return nz_prefix[i1 + 1] - nz_prefix[i0] == 0;
}

// Sample count of a segment: n = max(1, ceil(len / step)), len = (t1 - t0) |d|.
// The FP32 estimate decides unless the quotient lies within its error bound of an integer.
__device__ __forceinline__ int segment_count(const RayArgs& R, int px, int py, const RayF& f,
                                             int pid0, float tau0, float e0, int pid1, float tau1,
                                             float e1, const DLevel& lv) {
  const float inv_step = lv.inv_step;
  const float lenf = (tau1 - tau0) * f.dn;
  const float q = lenf * inv_step;
  // |q - exact| <= (e0 + e1) |d| / step + 5u q (subtraction, |d|, product, 1/step roundings)
  const float eq = (e0 + e1) * f.dn * inv_step + ldexpf(q + 1.0f, -21);
  if (q + eq <= 1.0f) return 1;
  const float c = ceilf(q);
  if (c - q > eq && q - (c - 1.0f) > eq && c <= (float)kMaxSamplesPerSegment) return (int)c;
  return exact_count(R, px, py, pid0, pid1, lv.step);
}

// Central-difference gradient g_a = (F(x + h e_a) - F(x - h e_a)) / 2h at sample beta.
// When all six neighbours lie inside the current leaf (beyond the error margin), they are
// trilinear values of the same brick: one interpolation of the gradient brick's per-cell
// differences, or one 32-cell stencil (the differences along an axis are lerps of the two
// outer cell pairs, combined bilinearly in the other axes).  Otherwise each neighbour goes
// through neighbour_at (cross-leaf lookups), in one rolled loop.
// Whether both gradient neighbours of brick position beta on every axis read the segment's
// own brick (beyond the FP32 error margin): then the brick's cells give the gradient.
__device__ __forceinline__ bool gradient_inner(const SegState& s, const float* beta) {
  const float m = s.margin;
  bool inner = true;
#pragma unroll
  for (int q = 0; q < 3; ++q)
    inner = inner && (beta[q] - 1.0f >= s.bl[q] + m) && (beta[q] + 1.0f < s.bh[q] - m);
  return inner;
}

// The eight gradient-brick cells (V, central differences) of the trilinear stencil at an
// inner brick position, and the weights.
struct GradCorners {
  float4 q[8];  // x fastest, then y, then z (as Corners)
  float wx, wy, wz;
  __device__ __forceinline__ float tri(int c) const {  // component c = 1, 2, 3 (y, z, w)
    auto e = [&](int i) { return c == 1 ? q[i].y : c == 2 ? q[i].z : q[i].w; };
    const float c00 = fmaf(wx, e(1) - e(0), e(0)), c10 = fmaf(wx, e(3) - e(2), e(2));
    const float c01 = fmaf(wx, e(5) - e(4), e(4)), c11 = fmaf(wx, e(7) - e(6), e(6));
    const float c0 = fmaf(wy, c10 - c00, c00), c1 = fmaf(wy, c11 - c01, c01);
    return fmaf(wz, c1 - c0, c0);
  }
  __device__ __forceinline__ void gradient(const DLevel& lv, float* g) const {
    g[0] = tri(1) * lv.ginv[0];
    g[1] = tri(2) * lv.ginv[1];
    g[2] = tri(3) * lv.ginv[2];
  }
};

template <int ST>
__device__ __forceinline__ GradCorners grad_fetch(const RenderArgs& A, const BrickRef& b,
                                                  const float* beta) {
  const int ix = min(max((int)beta[0], 1), b.dim[0] - 3);
  const int iy = min(max((int)beta[1], 1), b.dim[1] - 3);
  const int iz = min(max((int)beta[2], 1), b.dim[2] - 3);
  GradCorners c;
  c.wx = beta[0] - (float)ix;
  c.wy = beta[1] - (float)iy;
  c.wz = beta[2] - (float)iz;
  using I = typename BrickIndex<ST>::type;
  const I l0 = (I)ix + (I)b.sy * iy + (I)b.sz * iz;
  c.q[0] = fetch4<ST>(A, b, l0, ix, iy, iz);
  c.q[1] = fetch4<ST>(A, b, l0 + 1, ix + 1, iy, iz);
  c.q[2] = fetch4<ST>(A, b, l0 + b.sy, ix, iy + 1, iz);
  c.q[3] = fetch4<ST>(A, b, l0 + b.sy + 1, ix + 1, iy + 1, iz);
  c.q[4] = fetch4<ST>(A, b, l0 + b.sz, ix, iy, iz + 1);
  c.q[5] = fetch4<ST>(A, b, l0 + b.sz + 1, ix + 1, iy, iz + 1);
  c.q[6] = fetch4<ST>(A, b, l0 + b.sz + b.sy, ix, iy + 1, iz + 1);
  c.q[7] = fetch4<ST>(A, b, l0 + b.sz + b.sy + 1, ix + 1, iy + 1, iz + 1);
  return c;
}

template <int ST, int INTERP, int GB>
__device__ __forceinline__ void gradient(const RenderArgs& A, const RayArgs& R, const SegState& s,
                                         const float* beta,
                                         int k, const DLevel& lv, float* g) {
  if constexpr (INTERP == 1) {
    const bool inner = gradient_inner(s, beta);
    if (GB && inner) {
      // gradient brick: trilinear interpolation of the per-cell central differences
      grad_fetch<ST>(A, s.brick, beta).gradient(lv, g);
      return;
    }
    if (inner) {
      const BrickRef& b = s.brick;
      const int ix = min(max((int)beta[0], 1), b.dim[0] - 3);
      const int iy = min(max((int)beta[1], 1), b.dim[1] - 3);
      const int iz = min(max((int)beta[2], 1), b.dim[2] - 3);
      const float wx = beta[0] - (float)ix, wy = beta[1] - (float)iy, wz = beta[2] - (float)iz;
      using I = typename BrickIndex<ST>::type;
      const I l0 = (I)ix + (I)b.sy * iy + (I)b.sz * iz;
      auto V = [&](int dx, int dy, int dz) {
        return fetch<ST>(A, b, l0 + dx + (I)b.sy * dy + (I)b.sz * dz, ix + dx,
                         iy + dy, iz + dz);
      };
      float c[2][2][2];
#pragma unroll
      for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
          for (int dx = 0; dx < 2; ++dx) c[dz][dy][dx] = V(dx, dy, dz);
      float dxv[2][2], dyv[2][2], dzv[2][2];
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v) {
          // x: at (y = iy + u, z = iz + v)
          const float xm = V(-1, u, v), xp = V(2, u, v);
          dxv[v][u] = fmaf(wx, xp - c[v][u][1], c[v][u][1]) - fmaf(wx, c[v][u][0] - xm, xm);
          // y: at (x = ix + u, z = iz + v)
          const float ym = V(u, -1, v), yp = V(u, 2, v);
          dyv[v][u] = fmaf(wy, yp - c[v][1][u], c[v][1][u]) - fmaf(wy, c[v][0][u] - ym, ym);
          // z: at (x = ix + u, y = iy + v)
          const float zm = V(u, v, -1), zp = V(u, v, 2);
          dzv[v][u] = fmaf(wz, zp - c[1][v][u], c[1][v][u]) - fmaf(wz, c[0][v][u] - zm, zm);
        }
      // bilinear combination in the two transverse axes
      const float gx0 = fmaf(wy, dxv[0][1] - dxv[0][0], dxv[0][0]);
      const float gx1 = fmaf(wy, dxv[1][1] - dxv[1][0], dxv[1][0]);
      const float gy0 = fmaf(wx, dyv[0][1] - dyv[0][0], dyv[0][0]);
      const float gy1 = fmaf(wx, dyv[1][1] - dyv[1][0], dyv[1][0]);
      const float gz0 = fmaf(wx, dzv[0][1] - dzv[0][0], dzv[0][0]);
      const float gz1 = fmaf(wx, dzv[1][1] - dzv[1][0], dzv[1][0]);
      g[0] = fmaf(wz, gx1 - gx0, gx0) * lv.ginv[0];
      g[1] = fmaf(wz, gy1 - gy0, gy0) * lv.ginv[1];
      g[2] = fmaf(wy, gz1 - gz0, gz0) * lv.ginv[2];
      return;
    }
  }
  // one rolled loop over the six neighbours (+x, -x, +y, -y, +z, -z) keeps a single copy
  // of the lookup code in the kernel
  float d[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll 1
  for (int q = 0; q < 6; ++q) {
    const int ax = q >> 1;
    const float sg = (q & 1) ? -1.0f : 1.0f;
    float bn[3] = {beta[0], beta[1], beta[2]};
    bn[0] += ax == 0 ? sg : 0.0f;
    bn[1] += ax == 1 ? sg : 0.0f;
    bn[2] += ax == 2 ? sg : 0.0f;
    const float v = neighbour_at<ST, INTERP>(A, R, s, lv, bn, k, ax, sg);
    d[0] += ax == 0 ? sg * v : 0.0f;
    d[1] += ax == 1 ? sg * v : 0.0f;
    d[2] += ax == 2 ? sg * v : 0.0f;
  }
  g[0] = d[0] * lv.ginv[0];
  g[1] = d[1] * lv.ginv[1];
  g[2] = d[2] * lv.ginv[2];
}

// A segment ready for sampling: its state, first sample position and step in brick
// coordinates, and the world length of one sub-step.
struct SegSetup {
  SegState s;
  float b0[3], db[3];
  float delta;
};

// The leaf's corner and its box in brick coordinates, the region whose gradient neighbours
// read the leaf's own brick.
__device__ __forceinline__ void leaf_bounds(const DLeaf& lf, const DLevel& lv, const BrickRef& b,
                                            int lod_min, int* leaf_lo, float* bl, float* bh) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    leaf_lo[a] = lf.lo[a];
    bl[a] = (float)(lf.lo[a] - b.lo[a] * lv.sc) * lv.inv_sc + 0.5f;
    bh[a] = (float)(lf.hi[a] - b.lo[a] * lv.sc) * lv.inv_sc + 0.5f;
    // a face bit (the far side is the same unrefined patch, or with a two-cell halo any
    // patch of this level) widens the region whose neighbours read this brick by one cell.
    // Under pruning only when the bound is finer than this leaf's level: then no node the
    // pruned descent could stop at overlaps the (level-l) cells beyond the face
    if (lod_min > lf.level) {
      if ((lf.faces >> (2 * a)) & 1) bl[a] -= 1.0f;
      if ((lf.faces >> (2 * a + 1)) & 1) bh[a] += 1.0f;
    }
  }
}

// Sample parameters of segment (pid0, pid1) of leaf `lid` with n midpoint samples, and the
// bound on their FP32 error: the tau ends within max(e0, e1), a few roundings of the tau
// arithmetic, then the position and brick-space roundings.
__device__ __forceinline__ void setup_segment(const RenderArgs& A, const RayF& rf, const DLeaf& lf,
                                              const DLevel& lv, int lid, int pid0, int pid1,
                                              float tau0, float e0, float tau1, float e1, int n,
                                              int px, int py, SegSetup& g,
                                              int lod_min = kNoLod) {
  SegState& s = g.s;
  s.brick = leaf_brick(A.patches, lf);
  s.level = lf.level;
  s.leaf = pack_leaf(lid, lod_min);
  s.pid0 = pid0;
  s.pid1 = pid1;
  s.n = n;
  s.px = px;
  s.py = py;
  const float nfl = (float)n;
  const float dtau = (tau1 - tau0) / nfl;
  g.delta = dtau * rf.dn;
  const float taum = fmaf(0.5f, dtau, tau0);
  const float etau = fmaxf(e0, e1) + ldexpf(tau1 + 1.0f, -21);
  float ex = 0.0f, bmax = 0.0f;
  leaf_bounds(lf, lv, s.brick, lod_min, s.leaf_lo, s.bl, s.bh);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float xm = fmaf(taum, rf.Dd[a], rf.Xe[a]);  // finest units
    const float lo05 = 0.5f - (float)s.brick.lo[a];
    g.b0[a] = fmaf(xm, lv.inv_sc, lo05);
    g.db[a] = dtau * rf.Dd[a] * lv.inv_sc;
    const float ea = fabsf(rf.Dd[a]) * etau +
                     ldexpf(fabsf(rf.Xe[a]) + fabsf(xm) + nfl * fabsf(dtau * rf.Dd[a]) + 1.0f, -21);
    ex = fmaxf(ex, ea);
    bmax = fmaxf(bmax, fabsf(g.b0[a]) + nfl * fabsf(g.db[a]) + (float)s.brick.dim[a]);
  }
  s.margin = ex * lv.inv_sc + ldexpf(bmax + 2.0f, -21);
}

// Secondary ray from a sample to the point light (the global-illumination example of
// Sec. 5): transmittance of the part of the segment X -> light inside the root box, marched
// with n = max(1, ceil(len / light_step)) midpoint samples of the AMR field (the finest
// leaf holding each point, trilinear in its brick), stopping with 0 once T <= 1e-4.
// X in finest-cell units.  LightRay holds what both marchers below share.
struct LightRay {
  float X[3], D[3];  // start and light - start, finest-cell units
  float s_out;       // the path inside the root ends at X + s_out D
  float delta;       // world length of one light step
  int n;             // light samples
};

__device__ __forceinline__ LightRay light_ray(const RenderArgs& A, const RayArgs& R, float x0,
                                              float x1, float x2) {
  LightRay L;
  L.X[0] = x0;
  L.X[1] = x1;
  L.X[2] = x2;
  float s_out = 1.0f, len2 = 0.0f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    L.D[a] = A.light_f[a] - L.X[a];
    if (L.D[a] != 0.0f) {
      const float bound = (float)(L.D[a] > 0.0f ? R.root_f[3 + a] : R.root_f[a]);
      s_out = fminf(s_out, (bound - L.X[a]) / L.D[a]);
    }
    const float w = L.D[a] * (float)R.hf[a];
    len2 = fmaf(w, w, len2);
  }
  L.s_out = fmaxf(s_out, 0.0f);
  const float len = L.s_out * sqrtf(len2);
  L.n = (int)fminf(fmaxf(ceilf(len / A.light_step), 1.0f), 65536.0f);
  L.delta = len / (float)L.n;
  return L;
}

// Point k of the light ray (finest-cell units) and its finest cell, clamped into the root.
__device__ __forceinline__ void light_point(const RayArgs& R, const LightRay& L, int k, float* P,
                                            int* f) {
  const float sk = ((float)k + 0.5f) / (float)L.n * L.s_out;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    P[a] = fmaf(sk, L.D[a], L.X[a]);
    f[a] = min(max((int)floorf(P[a]), R.root_f[a]), R.root_f[3 + a] - 1);
  }
}

// The prefix counts of the transfer function's non-transparent entries, which the frame
// kernels stage right after the transfer function in shared memory (stage_tf).
__device__ __forceinline__ const int* tf_nonzero_prefix(const RenderArgs& A, const float4* s_tf) {
  return reinterpret_cast<const int*>(s_tf + A.tf_n);
}

// Light samples in a leaf whose value range the transfer function maps to zero opacity
// multiply T by exp(-kappa * 0 * delta) = 1 exactly, so both marchers skip them: the same
// T bit for bit, without their stencils.

// A light sample at brick position (bx, by, bz) whose stencil maximum maps to zero
// opacity (stencil-maximum bricks present: mdelta != 0) contributes the factor 1 exactly.
template <int ST>
__device__ __forceinline__ bool light_sample_transparent(const RenderArgs& A, const int* nz,
                                                         const BrickRef& b, float bx, float by,
                                                         float bz) {
  if constexpr (ST == ST_PTR) {
    if (A.mdelta == 0) return false;
    const Stencil<ST> st = stencil_at<ST>(b, bx, by, bz);
    return stencil_transparent(A, nz, fetch_max<ST>(A, b, st.l0));
  } else {
    return false;
  }
}

// One lane marches the whole light ray, sample by sample (the per-ray schedule).
// Consecutive samples usually stay in one leaf, which is reused.
template <int ST>
__device__ __noinline__ float shadow_transmittance(const RenderArgs& A, const RayArgs& R,
                                                   const float4* s_tf, float x0, float x1,
                                                   float x2) {
  const LightRay L = light_ray(A, R, x0, x1, x2);
  const int* s_nz = tf_nonzero_prefix(A, s_tf);
  float T = 1.0f;
  int leaf = -1;
  DLeaf lf;
  BrickRef b;
  float inv_sc = 1.0f;
  bool clear = false;  // the current leaf is fully transparent
  for (int k = 0; k < L.n; ++k) {
    float P[3];
    int f[3];
    light_point(R, L, k, P, f);
    const bool inside = leaf >= 0 && f[0] >= lf.lo[0] && f[0] < lf.hi[0] && f[1] >= lf.lo[1] &&
                        f[1] < lf.hi[1] && f[2] >= lf.lo[2] && f[2] < lf.hi[2];
    if (!inside) {
      leaf = locate_cell(A.nodes, R, kNoLod, f[0], f[1], f[2]);
      if (leaf < 0) return T;
      lf = A.leaves[leaf];
      b = leaf_brick(A.patches, lf);
      inv_sc = A.lv[lf.level].inv_sc;
      clear = tf_transparent(s_nz, A.tf_n, lf.vmin, lf.vmax, A.vmin, A.inv_range);
    }
    if (clear) continue;
    const float bx = fmaf(P[0], inv_sc, 0.5f - (float)b.lo[0]);
    const float by = fmaf(P[1], inv_sc, 0.5f - (float)b.lo[1]);
    const float bz = fmaf(P[2], inv_sc, 0.5f - (float)b.lo[2]);
    if (light_sample_transparent<ST>(A, s_nz, b, bx, by, bz)) continue;  // factor 1
    const float v = trilinear<ST>(A, b, bx, by, bz);
    const float a_tf = tf_lookup(s_tf, A.tf_n, v, A.vmin, A.inv_range).w;
    T *= expf(-A.kappa * a_tf * L.delta);
    if (T <= 1e-4f) return 0.0f;
  }
  return T;
}

// The same transmittance, marched by all 32 lanes of a warp together (the deferred
// schedule; every lane must call it with the same start point).  Round r takes the 32
// consecutive samples 32 r .. 32 r + 31, one per lane: neighbouring lanes read
// neighbouring cells.  A lane keeps the leaf of its last point, tries the leaf of the last
// point of the previous round next, and otherwise locates its point (from its macro-grid
// cell's node); the
// lanes that need it descend together, so a round pays one descent's latency however
// many leaves its points span.  The round's factors exp(-kappa a delta) are multiplied in
// a fixed tree order into T, so T is the same in every lane and differs from the per-lane
// product only by rounding; T <= 1e-4 after a round gives 0 (T only falls, so this is the
// per-sample rule).
template <int ST>
__device__ __forceinline__ float warp_shadow_transmittance(const RenderArgs& A, const RayArgs& R,
                                                           const float4* s_tf, float x0,
                                                           float x1, float x2) {
  const unsigned FULL = 0xffffffffu;
  const LightRay L = light_ray(A, R, x0, x1, x2);
  const int* s_nz = tf_nonzero_prefix(A, s_tf);
  float T = 1.0f;
  int leaf = -1;                 // this lane's current leaf
  int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  BrickRef b;
  float inv_sc = 1.0f;
  bool clear = false;            // this lane's leaf is fully transparent
  int last = -1;                 // warp-uniform: the leaf of the last sample of the last round
  bool bad = false;              // malformed tree met
  for (int k0 = 0; k0 < L.n; k0 += 32) {
    const int k = k0 + (int)(threadIdx.x + blockDim.x * threadIdx.y) % 32;
    const bool valid = k < L.n;
    float P[3];
    int f[3];
    light_point(R, L, valid ? k : L.n - 1, P, f);
    bool have = valid && leaf >= 0 && f[0] >= lo[0] && f[0] < hi[0] && f[1] >= lo[1] &&
                f[1] < hi[1] && f[2] >= lo[2] && f[2] < hi[2];
    if (valid && !have) {
      int lid = -1;
      if (last >= 0) {
        const int4* w = reinterpret_cast<const int4*>(A.leaves + last);
        const int4 w1 = __ldg(w + 1), w2 = __ldg(w + 2);  // lo[3], hi[0] | hi[1], hi[2], ...
        if (f[0] >= w1.x && f[0] < w1.w && f[1] >= w1.y && f[1] < w2.x && f[2] >= w1.z &&
            f[2] < w2.y)
          lid = last;
      }
      if (lid < 0) lid = locate_cell_from(A.nodes, macro_start(R, f[0], f[1], f[2]), f[0], f[1], f[2]);
      if (lid < 0) {
        bad = true;
      } else {
        const DLeaf lf = A.leaves[lid];
        leaf = lid;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          lo[a] = lf.lo[a];
          hi[a] = lf.hi[a];
        }
        b = leaf_brick(A.patches, lf);
        inv_sc = A.lv[lf.level].inv_sc;
        clear = tf_transparent(s_nz, A.tf_n, lf.vmin, lf.vmax, A.vmin, A.inv_range);
        have = true;
      }
    }
    if (__any_sync(FULL, bad)) return T;  // malformed tree: the per-lane march stops too
    float term = 1.0f;
    if (valid && !clear) {
      const float bx = fmaf(P[0], inv_sc, 0.5f - (float)b.lo[0]);
      const float by = fmaf(P[1], inv_sc, 0.5f - (float)b.lo[1]);
      const float bz = fmaf(P[2], inv_sc, 0.5f - (float)b.lo[2]);
      if (!light_sample_transparent<ST>(A, s_nz, b, bx, by, bz)) {
        const float v = trilinear<ST>(A, b, bx, by, bz);
        const float a_tf = tf_lookup(s_tf, A.tf_n, v, A.vmin, A.inv_range).w;
        term = expf(-A.kappa * a_tf * L.delta);
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) term *= __shfl_down_sync(FULL, term, off);
    T *= __shfl_sync(FULL, term, 0);
    if (T <= 1e-4f) return 0.0f;
    last = __shfl_sync(FULL, leaf, 31);
  }
  return T;
}

// Headlight Phong factor of gradient gr (normal g / max(|g|, gamma (vmax - vmin) / h^l))
// applied to the transfer-function colour (cr, cg, cb), clamped to [0, 1].
__device__ __forceinline__ void phong(const RenderArgs& A, const DLevel& lv, const float* gr,
                                      float Lx, float Ly, float Lz, float& cr, float& cg,
                                      float& cb) {
  const float gn = sqrtf(fmaf(gr[0], gr[0], fmaf(gr[1], gr[1], gr[2] * gr[2])));
  const float gf = A.gfloor_num / lv.hmin;
  const float den = fmaxf(gn, gf);
  const float inv = den > 0.0f ? 1.0f / den : 0.0f;
  const float ndl = fabsf((gr[0] * Lx + gr[1] * Ly + gr[2] * Lz) * inv);
  const float spec = A.ks * __powf(ndl, A.shininess);
  const float diff = fmaf(A.kd, ndl, A.ka);
  cr = fminf(fmaxf(fmaf(cr, diff, spec), 0.0f), 1.0f);
  cg = fminf(fmaxf(fmaf(cg, diff, spec), 0.0f), 1.0f);
  cb = fminf(fmaxf(fmaf(cb, diff, spec), 0.0f), 1.0f);
}

// Opacity, shading and compositing of a sample whose transfer-function entry c has non-zero
// opacity (gr: its gradient, read when shading).  Returns true at early ray termination.
template <int ST, int SHADE>
__device__ __forceinline__ bool finish_sample(const RenderArgs& A, const RayArgs& R,
                                              const float4* s_tf, const SegSetup& g,
                                              const DLevel& lv, const float* beta, float4 c,
                                              const float* gr, float Lx, float Ly, float Lz,
                                              float& C0, float& C1, float& C2, float& Acc) {
  const SegState& s = g.s;
  const float alpha = -expm1f(-A.kappa * c.w * g.delta);
  float cr = c.x, cg = c.y, cb = c.z;
  if constexpr ((SHADE & 3) >= 1) phong(A, lv, gr, Lx, Ly, Lz, cr, cg, cb);
  if constexpr ((SHADE & kShadeShadow) != 0) {
    // the sample in finest-cell units: beta = X / sc - lo + 0.5
    const float sc = (float)lv.sc;
    const float T = shadow_transmittance<ST>(A, R, s_tf, (beta[0] - 0.5f + (float)s.brick.lo[0]) * sc,
                                             (beta[1] - 0.5f + (float)s.brick.lo[1]) * sc,
                                             (beta[2] - 0.5f + (float)s.brick.lo[2]) * sc);
    const float I = fmaf(1.0f - A.light_ambient, T, A.light_ambient);
    cr *= I;
    cg *= I;
    cb *= I;
  }
  const float w = (1.0f - Acc) * alpha;
  C0 = fmaf(w, cr, C0);
  C1 = fmaf(w, cg, C1);
  C2 = fmaf(w, cb, C2);
  Acc += w;
  return Acc >= A.ert_thresh;
}

// Sample k of a segment with value v at brick position beta (Sec. 3: emission-absorption
// compositing; Sec. 4: gradient shading), composited front to back into (C, Acc).
// Returns true when early ray termination stops the ray at this sample.
template <int ST, int INTERP, int SHADE>
__device__ __forceinline__ bool composite_sample(const RenderArgs& A, const RayArgs& R,
                                                 const float4* s_tf, const SegSetup& g,
                                                 const DLevel& lv, int k, const float* beta,
                                                 float v, float Lx, float Ly, float Lz,
                                                 float& C0, float& C1, float& C2, float& Acc) {
  const float4 c = tf_lookup(s_tf, A.tf_n, v, A.vmin, A.inv_range);
  if (c.w <= 0.0f) return false;
  float gr[3] = {0.0f, 0.0f, 0.0f};
  if constexpr ((SHADE & 3) >= 1) gradient<ST, INTERP, ((SHADE & 3) == 2)>(A, R, g.s, beta, k, lv, gr);
  return finish_sample<ST, SHADE>(A, R, s_tf, g, lv, beta, c, gr, Lx, Ly, Lz, C0, C1, C2, Acc);
}

template <int ST, int INTERP, int SHADE>
__device__ __forceinline__ bool sample_one(const RenderArgs& A, const RayArgs& R,
                                           const float4* s_tf, const SegSetup& g,
                                           const DLevel& lv, int k, float Lx, float Ly, float Lz,
                                           float& C0, float& C1, float& C2, float& Acc) {
  const SegState& s = g.s;
  float beta[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) beta[a] = fmaf((float)k, g.db[a], g.b0[a]);
  const float v = sample_value<ST, INTERP>(A, R, s, beta, k);
  return composite_sample<ST, INTERP, SHADE>(A, R, s_tf, g, lv, k, beta, v, Lx, Ly, Lz, C0, C1,
                                            C2, Acc);
}

// Samples of a segment whose stencil maxima are tested in groups (stencil-maximum bricks):
// the maxima of G consecutive samples are loaded together, so a run of transparent
// samples pays one load latency per group; a sample that may be opaque is then evaluated
// in full.  Every sample is counted as it is taken, in order.  Unshaded, the group's
// evaluations are unrolled; shaded (a large evaluation) they run in a rolled loop that
// rotates the loaded maxima through registers.  G = 0 (shaded): one test per sample.
#ifndef AMR_MAX_GROUP_PLAIN
#define AMR_MAX_GROUP_PLAIN 4
#endif
#ifndef AMR_MAX_GROUP_SHADED
#define AMR_MAX_GROUP_SHADED 4
#endif

// Sample k of a segment whose stencil maximum did not prove it transparent: its value
// stencil, then composite_sample.  (Reading value and gradient together from the gradient
// brick's cells for such samples measured 9 % slower on C2 at 2048^2 Phong: many of them
// still map to zero opacity, and those then load 128 bytes instead of 32.)  Returns true
// at early ray termination.
template <int ST, int SHADE>
__device__ __forceinline__ bool sample_candidate(const RenderArgs& A, const RayArgs& R,
                                                 const float4* s_tf, const SegSetup& g,
                                                 const DLevel& lv, int k, float Lx, float Ly,
                                                 float Lz, float& C0, float& C1, float& C2,
                                                 float& Acc) {
  float beta[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) beta[a] = fmaf((float)k, g.db[a], g.b0[a]);
  const Stencil<ST> st = stencil_at<ST>(g.s.brick, beta[0], beta[1], beta[2]);
  const float v = stencil_value<ST>(A, g.s.brick, st);
  return composite_sample<ST, 1, SHADE>(A, R, s_tf, g, lv, k, beta, v, Lx, Ly, Lz, C0, C1, C2,
                                        Acc);
}

template <int ST, int SHADE, int G>
__device__ __forceinline__ bool sample_segment_grouped(const RenderArgs& A, const RayArgs& R,
                                                       const float4* s_tf, const int* nz,
                                                       const SegSetup& g, const DLevel& lv,
                                                       float Lx, float Ly, float Lz, float& C0,
                                                       float& C1, float& C2, float& Acc,
                                                       unsigned& nsamp) {
  const int n = g.s.n;
  if constexpr (G == 0) {
    for (int k = 0; k < n; ++k) {
      ++nsamp;
      float beta[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) beta[a] = fmaf((float)k, g.db[a], g.b0[a]);
      const Stencil<ST> st = stencil_at<ST>(g.s.brick, beta[0], beta[1], beta[2]);
      if (stencil_transparent(A, nz, fetch_max<ST>(A, g.s.brick, st.l0))) continue;
      const float v = stencil_value<ST>(A, g.s.brick, st);
      if (composite_sample<ST, 1, SHADE>(A, R, s_tf, g, lv, k, beta, v, Lx, Ly, Lz, C0, C1, C2,
                                         Acc))
        return true;
    }
    return false;
  } else {
    for (int k0 = 0; k0 < n; k0 += G) {
      float m[G];
#pragma unroll
      for (int j = 0; j < G; ++j) {
        const int k = min(k0 + j, n - 1);
        const Stencil<ST> st = stencil_at<ST>(g.s.brick, fmaf((float)k, g.db[0], g.b0[0]),
                                              fmaf((float)k, g.db[1], g.b0[1]),
                                              fmaf((float)k, g.db[2], g.b0[2]));
        m[j] = fetch_max<ST>(A, g.s.brick, st.l0);
      }
      auto one = [&](int k, float mk) -> int {  // 1: stop (early termination)
        ++nsamp;
        if (stencil_transparent(A, nz, mk)) return 0;  // opacity zero: nothing to composite
        return sample_candidate<ST, SHADE>(A, R, s_tf, g, lv, k, Lx, Ly, Lz, C0, C1, C2, Acc)
                   ? 1 : 0;
      };
      if constexpr ((SHADE & 3) == 0) {
#pragma unroll
        for (int j = 0; j < G; ++j) {
          if (k0 + j >= n) break;
          if (one(k0 + j, m[j])) return true;
        }
      } else {
#pragma unroll 1
        for (int j = 0; j < G; ++j) {
          if (k0 + j >= n) break;
          const float mj = m[0];
#pragma unroll
          for (int q = 0; q + 1 < G; ++q) m[q] = m[q + 1];
          if (one(k0 + j, mj)) return true;
        }
      }
    }
    return false;
  }
}

// March the samples of one segment front to back.  Returns true when early ray
// termination stops the ray inside the segment.  nz: the prefix counts of the transfer
// function's non-transparent entries (read by the stencil-maximum test only).
template <int ST, int INTERP, int SHADE>
__device__ __forceinline__ bool sample_segment(const RenderArgs& A, const RayArgs& R,
                                               const float4* s_tf, const int* nz,
                                               const SegSetup& g, const DLevel& lv, float Lx,
                                               float Ly, float Lz, float& C0, float& C1, float& C2,
                                               float& Acc, unsigned& nsamp) {
  if constexpr (INTERP == 1 && (SHADE & kShadeMaxBit) != 0) {
    constexpr int G = (SHADE & 3) == 0 ? AMR_MAX_GROUP_PLAIN : AMR_MAX_GROUP_SHADED;
    return sample_segment_grouped<ST, SHADE, G>(A, R, s_tf, nz, g, lv, Lx, Ly, Lz, C0, C1, C2,
                                                Acc, nsamp);
  } else if constexpr (INTERP == 1 && SHADE == 0) {
    // software pipeline: the cells of sample k + 1 are requested before sample k is
    // composited (unshaded only: with shading the extra live registers spill, measured
    // 13 % slower on C2 at 2048^2; unshaded 2 % faster)
    Corners next = trilinear_fetch<ST>(A, g.s.brick, g.b0[0], g.b0[1], g.b0[2]);
    for (int k = 0; k < g.s.n; ++k) {
      const float v = next.value();
      float beta[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) beta[a] = fmaf((float)k, g.db[a], g.b0[a]);
      if (k + 1 < g.s.n) {
        float bn[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) bn[a] = fmaf((float)(k + 1), g.db[a], g.b0[a]);
        next = trilinear_fetch<ST>(A, g.s.brick, bn[0], bn[1], bn[2]);
      }
      ++nsamp;
      if (composite_sample<ST, INTERP, SHADE>(A, R, s_tf, g, lv, k, beta, v, Lx, Ly, Lz, C0, C1,
                                              C2, Acc))
        return true;
    }
    return false;
  } else {
    for (int k = 0; k < g.s.n; ++k) {
      ++nsamp;
      if (sample_one<ST, INTERP, SHADE>(A, R, s_tf, g, lv, k, Lx, Ly, Lz, C0, C1, C2, Acc))
        return true;
    }
    return false;
  }
}

// Resident 128-thread blocks per SM the compiler must allow for, i.e. a register budget of
// 65536 / (128 x this) per thread.  Measured on C2 at 2048^2 (Gsamples/s): Phong 3 / 4 / 5
// blocks 59.8 / 64.9 / 61.6 (cross-leaf lookups inlined); unshaded 3 / 4 / 5 / 6 blocks
// 119.3 / 119.4 / 119.7 / 126.0 (before persistent warps).
// The learned march keeps the MLP fragments live beside the ray state: 3 blocks (168
// registers) measured fastest there (coarse16@0.01 on C2 at 2048^2: 2.25x the plain march
// at 3 blocks, 1.90x at 4, 1.57x at 5).
#ifndef AMR_MIN_BLOCKS
#define AMR_MIN_BLOCKS 3
#endif
#ifndef AMR_MIN_BLOCKS_SHADED
#define AMR_MIN_BLOCKS_SHADED 4
#endif
#ifndef AMR_MIN_BLOCKS_PLAIN
#define AMR_MIN_BLOCKS_PLAIN 6
#endif
template <int SHADE>
constexpr int kMinBlocks = (SHADE & 3) == 0 ? AMR_MIN_BLOCKS_PLAIN : AMR_MIN_BLOCKS_SHADED;

// The whole march of pixel (i, j) of the view R: ray setup, kd-restart over the leaves,
// sampling and compositing.  Returns premultiplied RGBA; adds to nsamp and status.
template <int ST, int INTERP, int SHADE>
__device__ __forceinline__ float4 march_ray(const RenderArgs& A, const RayArgs& R, int i, int j,
                                            const float4* s_tf, const int* s_nz, RayF& rf,
                                            unsigned& nsamp, unsigned long long& status) {
  float C0 = 0.f, C1 = 0.f, C2 = 0.f, Acc = 0.f;
  RayX rx;
  if (make_ray(R, i, j, rx)) {
    make_frame(R, rx, rf);
    const float inv_dn = 1.0f / rf.dn;
    const float Lx = -rf.Dd[0] * (float)R.hf[0] * inv_dn;
    const float Ly = -rf.Dd[1] * (float)R.hf[1] * inv_dn;
    const float Lz = -rf.Dd[2] * (float)R.hf[2] * inv_dn;
    int pid0 = kPidIn;
    float tau0 = 0.0f, e0 = 0.0f;
    uint32_t start = 0;
    int seg = 0, prev = -1;
    while (pid0 != kPidOut) {
      if (seg >= A.max_segments) {
        status |= kStatusCapacity;
        break;
      }
      ++seg;
      int pid1 = kPidOut;
      float tau1 = rf.tau_out, e1 = exit_bound(rf);
      const int lmin = lod_min_level(R, A.lv, rf, i, j, pid0, tau0, e0);
      const int lid = next_leaf(A.nodes, A.leaves, A.face_node, A.node_box, R, i, j, rf, start, prev, pid0,
                                tau0, e0, pid1, tau1, e1, lmin);
      if (lid < 0) {
        status |= kStatusDevice;
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
      SegSetup g;
      setup_segment(A, rf, lf, lv, lid, pid0, pid1, tau0, e0, tau1, e1, n, i, j, g, lmin);
      if (sample_segment<ST, INTERP, SHADE>(A, R, s_tf, s_nz, g, lv, Lx, Ly, Lz, C0, C1, C2, Acc,
                                            nsamp))
        pid1 = kPidOut;  // early ray termination
      pid0 = pid1;
      tau0 = tau1;
      e0 = e1;
    }
  }
  return make_float4(C0, C1, C2, Acc);
}

// Stage a transfer function in shared memory with the prefix count of its non-transparent
// entries (nz[k] = entries before k with alpha != 0), for exact empty-space skipping.
__device__ __forceinline__ void stage_tf(const float4* __restrict__ tf, int n, float4* s_tf,
                                         int* s_nz, int tid, int nthreads) {
  for (int k = tid; k < n; k += nthreads) s_tf[k] = tf[k];
  __syncthreads();
  if (tid == 0) {
    int acc = 0;
    s_nz[0] = 0;
    for (int k = 0; k < n; ++k) {
      acc += s_tf[k].w != 0.0f ? 1 : 0;
      s_nz[k + 1] = acc;
    }
  }
  __syncthreads();
}

// The frame march (schedule 0): one thread per pixel, persistent warps.  Each warp takes
// 8x4-pixel tiles from a global queue (counters[kQueueCounter], zeroed before the launch)
// until none is left, so a warp that finishes its rays starts on new ones at once instead
// of idling until the slowest warp of its block is done (measured on C2 at 2048^2: Phong
// 50.0 -> 52.9 Gsamples/s against one block per 8x16 tile); the grid holds only as many
// blocks as are resident at once.  QUEUE = false: one block per 8x16 tile, each warp
// marching its own 8x4 tile once - used for the per-patch texture storage, whose fetches
// need more registers than the queue loop leaves (C2 2048^2 unshaded: 44.5 against 9.3
// Gsamples/s with the queue).
#ifndef AMR_WARP_TILE_W
#define AMR_WARP_TILE_W 8  // pixel tile of one warp: AMR_WARP_TILE_W x (32 / AMR_WARP_TILE_W)
#endif
static_assert(AMR_WARP_TILE_W == 4 || AMR_WARP_TILE_W == 8 || AMR_WARP_TILE_W == 16,
              "warp tile width");
template <int ST, int INTERP, int SHADE, bool QUEUE = true>
__global__ void __launch_bounds__(128, kMinBlocks<SHADE>)
    march_kernel(const __grid_constant__ RenderArgs A) {
  extern __shared__ float4 smem[];
  float4* s_tf = smem;
  int* s_nz = reinterpret_cast<int*>(smem + A.tf_n);
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  stage_tf(A.tf, A.tf_n, s_tf, s_nz, tid, blockDim.x * blockDim.y);
  const int lane = tid & 31;
  const RayArgs& R = A.ray;
  unsigned nsamp = 0;
  unsigned long long status = 0;
  auto march_pixel = [&](int i, int jr) {
    const int j = R.row0 + jr;
    if (i < R.width && jr < R.rows && j < R.height) {
      if constexpr ((SHADE & ~kShadeMaxBit) == 0) {
        // unshaded: the ray frame lives in shared memory (read once per segment), leaving
        // the registers to the sample loop (measured 6 % faster on C2 at 2048^2; with
        // shading the extra shared-memory reads cost more than the spills they save).  One
        // padding word keeps the odd-sized slots free of bank conflicts.
        __shared__ RayFSlot s_rf[128];
        A.out[(size_t)jr * R.width + i] =
            march_ray<ST, INTERP, SHADE>(A, R, i, j, s_tf, s_nz, s_rf[tid].f, nsamp, status);
      } else {
        RayF rf;
        A.out[(size_t)jr * R.width + i] =
            march_ray<ST, INTERP, SHADE>(A, R, i, j, s_tf, s_nz, rf, nsamp, status);
      }
    }
  };
  if constexpr (QUEUE) {
    constexpr int TW = AMR_WARP_TILE_W, TH = 32 / TW;
    const int tiles_x = (R.width + TW - 1) / TW;
    const int n_tiles = tiles_x * ((R.rows + TH - 1) / TH);
    // each pass takes one tile, and the queue hands out every tile once
    for (;;) {
      int t = 0;
      if (lane == 0) {
        const unsigned long long q = atomicAdd(A.counters + kQueueCounter, 1ull);
        t = q < (unsigned long long)n_tiles ? (int)q : n_tiles;
      }
      t = __shfl_sync(0xffffffffu, t, 0);
      if (t >= n_tiles) break;
      march_pixel((t % tiles_x) * TW + lane % TW, (t / tiles_x) * TH + lane / TW);
    }
  } else {
    march_pixel(blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y * blockDim.y + threadIdx.y);
  }
  const unsigned total = __reduce_add_sync(0xffffffffu, nsamp);
  if (lane == 0 && total) atomicAdd(A.counters, (unsigned long long)total);
  if (status) atomicOr(A.counters + 1, status);
}

}  // namespace amr
