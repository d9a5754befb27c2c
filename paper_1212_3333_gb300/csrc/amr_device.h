// Device-resident records of the raycaster and the kernel argument blocks.
//
// Layout in HBM (all arrays written once by amr_build_kdtree, read-only while rendering):
//   DNode  nodes[N]   8 B each, breadth-first order, siblings adjacent (left = c, right =
//                      c + 1), so the top of the tree is a contiguous prefix that one
//                      cache line per few nodes serves to a whole warp (Sec. 3.2 stores the
//                      second child at the next texel for the same reason).
//   int4   node_box[2N] 32 B per node slot: its box and the highest label level of
//                      a type-(a) node above it (rope restarts).
//   DLeaf  leaves[M]  96 B each, canonical (pre-order) leaf id order, with the
//                      addressing of the leaf's brick.
//   DPatch patches[P] 48 B each: where a patch's brick lives and how to address it.
//   uint32 macro[G]   per cell of a grid over the root (at most 2^21 cells): the node slot
//                      where a point location may start.
//   bricks            one brick per patch with a one- or two-cell halo (Sec. 4), x fastest,
//                      in the layout of the chosen storage strategy.
#pragma once
#include <stddef.h>
#include <stdint.h>

#include <cuda_runtime.h>

namespace amr {

constexpr int kMaxLevels = 32;
constexpr int kLeafAxis = 3;            // DNode axis value that marks a leaf
constexpr uint32_t kIndexMask = 0x3fffffffu;
constexpr int kMaxDepth = 256;          // descent bound (tree depth is checked at build)
constexpr int kMaxSamplesPerSegment = 1 << 22;
constexpr uint32_t kFaceLeaf = 0x80000000u;  // face-table entry names a leaf (id in bits 0..30)

// device counters: [0] samples, [1] status bits, [2] exact descent decisions,
// [3] exact sample counts, [4] exact neighbour / nearest positions
constexpr int kNumCounters = 8;
constexpr int kQueueCounter = 5;       // counters[5]: head of the batched work queue
constexpr int kShadeShadowBit = 4;     // kernel shading variant bit: secondary rays
constexpr int kShadeMaxBit = 8;        // kernel variant bit: stencil-maximum opacity test
constexpr int kMaxBatchViews = 128;
// status bits raised by kernels (OR-ed into counters[1])
constexpr unsigned long long kStatusCapacity = 1ull;   // segment or sample bound hit
constexpr unsigned long long kStatusDevice = 2ull;     // malformed tree reached

struct DNode {
  uint32_t meta;  // bits 31..30: split axis (3 = leaf); bits 29..0: first child or leaf id
  int32_t split;  // split plane, finest-level cell index
};

// A leaf with the addressing of its patch's brick: a segment start or a cross-leaf lookup
// reads one record instead of a leaf and then its patch (one dependent load less).
struct alignas(16) DLeaf {
  long long base;        // brick (DPatch::base), the same for every leaf of a patch
  long long gbase;       // gradient brick (DPatch::gbase)
  int32_t lo[3], hi[3];  // box, finest-level cells
  int32_t lod_anc;       // highest label level of a type-(a) node above this leaf, -1: none
  int32_t level;
  int32_t patch;
  float vmin, vmax;      // range of every value a sample of this leaf can interpolate
  int32_t faces;         // bit 2a (+1): the level cell beyond the lower (upper) face on axis
                         // a lies in the same patch and is not refined (one-cell halo), or
                         // only in leaves of this leaf's level (two-cell halo): gradient
                         // neighbours there read this leaf's brick
  int32_t sy, sz;        // brick strides (DPatch::sy, sz)
  int32_t blo[3];        // brick origin (DPatch::lo)
  int32_t dim[3];        // brick extent with halo (DPatch::dim)
};
static_assert(sizeof(DLeaf) == 96, "DLeaf is six 16-byte words");
// lo, hi and lod_anc fill the record's second and third 16-byte words (rope restarts read
// them as two int4)
static_assert(offsetof(DLeaf, lo) == 16 && offsetof(DLeaf, hi) == 28 &&
                  offsetof(DLeaf, lod_anc) == 40,
              "DLeaf box layout");

struct DPatch {
  long long base;      // pointer table: device address of the brick; linear atlas: element
                       // offset; texture table: cudaTextureObject_t; 3D atlas: unused
  long long gbase;     // the same for the gradient brick (float4 per cell), 0 if absent
  int32_t sy, sz;      // element strides of y and z (linear storages)
  int32_t lo[3];       // brick index = cell - lo + 1: the patch box lo, less one with a
                       // two-cell halo (level cells)
  int32_t dim[3];      // brick extent with halo: n + 2 (one-cell halo) or n + 4 per axis
  int32_t org[3];      // 3D atlas: texel origin of the brick
  int32_t pad[3];
};

struct DLevel {
  double h[3];       // spacing h^l
  double inv_h[3];   // 1 / h^l
  double step;       // sample step f * min_a h^l_a (world units)
  int32_t sc;        // finest cells per level-l cell, r^(L-1-l)
  float inv_sc;      // 1 / sc
  float hmin;        // min_a h^l_a as float (gradient floor, pruning filter)
  float inv_step;    // 1 / step as float
  float ginv[3];     // 0.5 / h^l_a as float (central-difference scale; exactly
                     // 0.5f * (float)inv_h[a], halving being exact)
  double hmin_d;     // min_a h^l_a (exact pruning decisions)
};

struct RayArgs {
  double eye[3], fwd[3], right[3], up[3];
  double tan_half_fov_y;
  int32_t width, height;
  int32_t row0, rows;
  double dlo[3];        // domain origin
  double hf[3];         // finest spacing h^(L-1)
  double inv_hf[3];     // 1 / hf
  double root_w[6];     // root box, world coordinates
  int32_t root_f[6];    // root box, finest cells
  unsigned long long* counters;  // [0] samples, [1] status, [2..4] exact-path counts
  // level-of-detail pruning (Sec. 3.1 type-(a) nodes): per node (breadth-first slots)
  // (pruned-leaf id << 5 | level) or -1; X(t) = lod_scale * t bounds the cell size at
  // which the descent stops; lod_scale == 0 turns pruning off
  const int32_t* lod;
  int32_t levels;       // 1 + the finest level of a type-(a) node (0: none)
  double lod_scale;
  float lod_scale_f;
  int32_t n_leaves;     // leaves of the unpruned tree (ids at or above are pruned leaves)
  // macro grid over the root (cells of macro_cell finest cells per axis, macro_dims of
  // them): per cell the slot of the deepest node holding the whole cell, where an
  // unpruned point location may start
  const uint32_t* macro;
  int32_t macro_cell;
  int32_t macro_dims[3];
};

struct RenderArgs {
  RayArgs ray;
  DLevel lv[kMaxLevels];
  const DNode* nodes;
  const DLeaf* leaves;
  const int32_t* face_node;    // per leaf, 12: per face (2a + side) the node slot holding the
                               // leaf and the cell beyond the face, then the cell alone
                               // (starts of neighbour lookups; the second half: ropes);
                               // an entry with kFaceLeaf set names a leaf id instead
  const int4* node_box;        // per node slot, 2: box lo (x, y, z, highest label level of
                               // a type-(a) node above it or -1), hi (x, y, z, 0), finest
                               // cells (rope restarts)
  const DPatch* patches;
  const void* pool;            // linear atlas base (element type of the storage)
  const float4* gpool;         // linear atlas of gradient bricks (float4 per cell)
  cudaTextureObject_t atlas;   // 3D atlas texture
  cudaTextureObject_t gatlas;  // 3D atlas of gradient bricks
  const float4* tf;            // transfer function [tf_n]
  int32_t tf_n;
  int32_t max_segments;
  int32_t skip;                // exact min/max empty-space skipping
  float kappa, ert_thresh, vmin, inv_range;
  float ka, kd, ks, shininess, gfloor_num;  // gfloor = gfloor_num / hmin_l
  float4* out;
  unsigned long long* counters;  // [0] samples, [1] status bits
  const unsigned char* mlp;      // packed learned-proposal weights (inference image)
  float tau;                     // proposal threshold on the predicted contribution
  int32_t learned;               // 0 off, 1 skip, 2 coarse (coarse_factor x step) below tau
  float inv_levels;              // 1 / (L - 1), 0 for one level
  int32_t shadow;                // secondary rays to the point light
  float light_f[3];              // light position, finest-cell units
  float light_step, light_ambient;
  int32_t samples_per_iter;      // refill schedule: samples per lane between warp steps
  int32_t coarse_factor;         // learned mode 2: step multiplier below tau
  int32_t learned_min_samples;   // learned modes: segments shorter than this skip the MLP
  long long mdelta;              // stencil-maximum brick = value brick + mdelta bytes (ptr)
};

struct TraceArgs {
  RayArgs ray;
  DLevel lv[kMaxLevels];
  const DNode* nodes;
  const DLeaf* leaves;
  const int32_t* face_node;
  const int4* node_box;
  int32_t* leaf_seq;
  double* t_seq;
  int32_t* seq_len;
  int32_t max_len;
  int32_t max_segments;
  unsigned long long* counters;
};

// One view of a batched render (kept compact: the batch travels in the parameter block).
struct BatchView {
  double eye[3], fwd[3], right[3], up[3];
  double tan_half_fov_y;
  int32_t width, height;
  int32_t item0;    // first work item (pixel tile) of the view in the batch queue
  int32_t tiles_x;  // tiles per row of the view
  int32_t tf;       // transfer-function index
  int32_t pad;
  long long out;    // float4 offset of the view's [H][W] image in the output buffer
  double lod_scale; // pruning scale of this view (0: off)
  float lod_scale_f;
};

struct BatchArgs {
  RenderArgs A;     // shared state; A.tf = n_tf tables of A.tf_n entries, A.ray = domain part
  int32_t n_views, n_items, n_tf, rays_per_thread;
  BatchView v[kMaxBatchViews];
};

}  // namespace amr
