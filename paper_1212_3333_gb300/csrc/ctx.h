// Host-side context of the raycaster: the AMR hierarchy, the kD-tree, the bricks and the
// device allocations that mirror them.
#pragma once
#include <stdint.h>

#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/amr.h"
#include "amr_device.h"

namespace amr {

// Host-side fault injection for tests of the error paths (no GPU fault is ever provoked):
// the environment variable AMR_FAULT names one failure to simulate -
//   bad_alloc     the host build runs out of memory            -> AMR_ERR_OOM
//   oom           the device upload's first allocation fails   -> AMR_ERR_OOM
//   corrupt_node  the uploaded root node names itself as a child (every index stays in
//                 range), so descents loop until their depth bound -> AMR_ERR_DEVICE
// Unset or any other value: no effect.
inline bool fault_injected(const char* what) {
  const char* v = std::getenv("AMR_FAULT");
  return v && std::strcmp(v, what) == 0;
}

struct Patch {
  int level;
  int64_t box[6];   // level-l cells
  int64_t fbox[6];  // finest cells
  int64_t n[3];     // nx, ny, nz
  std::vector<float> data;
};

// Canonical tree in pre-order (what the test hooks return and the device arrays encode).
struct Tree {
  std::vector<int32_t> axis, split, left, right, leaf;  // per node, pre-order
  std::vector<int32_t> leaf_box;                        // 6 per leaf, finest cells
  std::vector<int32_t> leaf_patch, leaf_level;
  std::vector<uint8_t> leaf_faces;  // per leaf: DLeaf::faces
  std::vector<int32_t> face_node;   // per leaf, 12: for each face (2a + side) the pre-order id
                                    // of the deepest node holding the leaf and the cell beyond
                                    // that face, then of the one holding that cell alone
  // level-of-detail: inner nodes whose box lies in one patch (Sec. 3.1 type (a)) may be
  // rendered as leaves of that patch's level; they take ids M, M+1, ... in pre-order
  std::vector<int32_t> node_lod;                        // per node, pre-order: id or -1
  std::vector<int32_t> lod_box, lod_patch, lod_level;   // per pruned leaf
  int lod_levels = 0;  // 1 + the finest level of a pruned leaf (0: none)
  int max_depth = 0;
};

struct Packing {
  int64_t dims[3] = {0, 0, 0};
  std::vector<int64_t> org;  // 3 per patch
};

struct DeviceState {
  DNode* nodes = nullptr;
  DLeaf* leaves = nullptr;
  DPatch* patches = nullptr;
  void* pool = nullptr;  // brick pool (pointer table) or linear atlas
  size_t pool_bytes = 0;
  void* gpool = nullptr; // gradient bricks, same layout, float4 per cell
  size_t gpool_bytes = 0;
  void* mpool = nullptr; // stencil-maximum bricks, same offsets as pool (ptr storage)
  std::vector<void*> garrays;                    // gradient cudaArray_t per patch
  std::vector<cudaTextureObject_t> gtexobjs;
  void* gatlas_array = nullptr;
  cudaTextureObject_t gatlas_tex = 0;
  std::vector<void*> arrays;                     // cudaArray_t per patch (texture table)
  std::vector<cudaTextureObject_t> texobjs;
  void* atlas_array = nullptr;                   // cudaArray_t of the 3D atlas
  cudaTextureObject_t atlas_tex = 0;
  unsigned long long* counters = nullptr;        // [0] samples, [1] status
  float4* tf_scratch = nullptr;                  // staging for amr_render_host
  int tf_scratch_n = 0;
  float4* img_scratch = nullptr;
  int32_t* log_counts = nullptr;                 // segment log: kept records per pixel
  unsigned long long* log_offsets = nullptr;     //   and each pixel's first record
  size_t log_pixels = 0;                         //   capacity of both, pixels
  unsigned char* proposal = nullptr;             // packed MLP weights (amr_set_proposal)
  size_t img_scratch_bytes = 0;
  int32_t* lod = nullptr;                        // per node slot: (id << 5 | level) or -1
  int32_t* face_node = nullptr;                  // per leaf and face: node slot (neighbour start)
  int4* node_box = nullptr;                      // per node slot: box lo, hi (ropes)
  uint32_t* macro = nullptr;                     // macro grid: point-location start slots
  int32_t macro_cell = 1;                        // finest cells per macro cell per axis
  int32_t macro_dims[3] = {1, 1, 1};
  int device = -1;
};

}  // namespace amr

struct amr_ctx {
  int L = 0, r = 0;
  double dlo[3] = {0, 0, 0}, h0[3] = {0, 0, 0};
  amr_dtype dtype = AMR_F32;
  std::vector<amr::Patch> patches;
  int64_t R = 1;                // r^(L-1)
  int64_t rpow[40] = {0};
  int64_t root[6] = {0, 0, 0, 0, 0, 0};
  amr::Tree tree;
  std::vector<std::vector<float>> bricks;  // per patch, with halo
  bool want_gradient = false;              // build gradient bricks too
  int halo = 1;                            // brick halo width in cells (1, or 2 with
                                           // AMR_STORE_HALO2: faces onto the same level)
  std::vector<std::vector<float4>> gbricks; // per patch: value and central differences
  bool want_max = false;                   // build stencil-maximum bricks too (ptr storage)
  std::vector<std::vector<float>> mbricks;  // per patch: max of the 8 cells of each stencil
  std::vector<float> leaf_vmin, leaf_vmax;
  amr::Packing packing;
  int storage = -1;
  unsigned long long last_counters[amr::kNumCounters] = {0};  // of the last synchronous render
  bool host_built = false;
  bool device_built = false;
  double build_seconds = 0.0;
  amr::DeviceState dev;
  amr_batch_config batch_cfg = {16, 8, 1, 0, 0};  // used when a batch call passes no config
  std::string err;
};

namespace amr {

// kdtree.cpp
amr_status validate_hierarchy(amr_ctx* c);
amr_status build_tree(amr_ctx* c);
// bricks.cpp
amr_status build_bricks(amr_ctx* c);
amr_status build_gradient_bricks(amr_ctx* c);
amr_status build_max_bricks(amr_ctx* c);
amr_status pack_atlas(amr_ctx* c);
// device.cpp
amr_status upload(amr_ctx* c, void* stream);
void release_device(amr_ctx* c);
// kernels (march.cu)
amr_status launch_render(amr_ctx* c, const RenderArgs& a, int storage, int interp, int shade,
                         int schedule, void* stream);
amr_status launch_trace(amr_ctx* c, const TraceArgs& a, void* stream);
amr_status launch_learned(amr_ctx* c, const RenderArgs& a, int storage, int shade, void* stream);
amr_status launch_batch(amr_ctx* c, const BatchArgs& b, int storage, int shade, int schedule,
                        const amr_batch_config& cfg, void* stream);
amr_status launch_log(amr_ctx* c, const RenderArgs& a, int storage, float* features,
                      float* targets, long long cap, unsigned long long* count, float keep_prob,
                      uint32_t seed, void* stream);
const char* mlp_last_error();
void fill_levels(const amr_ctx* c, DLevel* lv, double step_factor);
void fill_ray(const amr_ctx* c, const amr_camera* cam, int row0, int rows, RayArgs* ra);
double lod_scale(const amr_camera* cam, double lod_pixels);

amr_status fail(amr_ctx* c, amr_status s, const std::string& msg);

// kernel argument block of one render call (capi.cpp), and its launch
amr_status prepare_render_args(amr_ctx* c, const amr_camera* cam, int32_t tf_n,
                               const amr_render_params* p, RenderArgs* a);
amr_status launch_render_args(amr_ctx* c, const RenderArgs& a, const amr_render_params* p,
                              void* stream);
// params with AMR_SCHEDULE_AUTO replaced by the schedule a single-view call would use
amr_render_params resolve_render_schedule(const amr_camera* cam, const amr_render_params& p);

}  // namespace amr
