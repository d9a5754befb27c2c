// C ABI of the raycaster: argument checking, context lifecycle and kernel argument
// marshalling.  Declarations and contracts: include/amr.h.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <utility>

#include "ctx.h"
#include "storage16.h"

using namespace amr;

static_assert(kMaxBatchViews == AMR_MAX_BATCH_VIEWS, "batch view bound");

namespace {

thread_local std::string g_create_error;

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return fail(c, e_ == cudaErrorMemoryAllocation ? AMR_ERR_OOM : AMR_ERR_CUDA,    \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                \
  } while (0)

amr_status check_camera(amr_ctx* c, const amr_camera* cam) {
  if (!cam) return fail(c, AMR_ERR_ARG, "camera is NULL");
  if (cam->width <= 0 || cam->height <= 0 || cam->width > (1 << 16) || cam->height > (1 << 16))
    return fail(c, AMR_ERR_ARG, "image size out of range");
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(cam->eye[a]) || !std::isfinite(cam->fwd[a]) ||
        !std::isfinite(cam->right[a]) || !std::isfinite(cam->up[a]))
      return fail(c, AMR_ERR_ARG, "camera has a non-finite component");
  if (!std::isfinite(cam->tan_half_fov_y) || cam->tan_half_fov_y <= 0.0)
    return fail(c, AMR_ERR_ARG, "tan_half_fov_y must be positive");
  return AMR_OK;
}

}  // namespace

namespace amr {

void fill_ray(const amr_ctx* c, const amr_camera* cam, int row0, int rows, RayArgs* ra) {
  std::memset(ra, 0, sizeof *ra);
  for (int a = 0; a < 3; ++a) {
    ra->eye[a] = cam->eye[a];
    ra->fwd[a] = cam->fwd[a];
    ra->right[a] = cam->right[a];
    ra->up[a] = cam->up[a];
    ra->dlo[a] = c->dlo[a];
    ra->hf[a] = c->h0[a] / (double)c->R;
    ra->inv_hf[a] = 1.0 / ra->hf[a];
    ra->root_w[a] = c->dlo[a] + (double)c->root[a] * ra->hf[a];
    ra->root_w[3 + a] = c->dlo[a] + (double)c->root[3 + a] * ra->hf[a];
    ra->root_f[a] = (int32_t)c->root[a];
    ra->root_f[3 + a] = (int32_t)c->root[3 + a];
  }
  ra->n_leaves = (int32_t)c->tree.leaf_patch.size();
  ra->tan_half_fov_y = cam->tan_half_fov_y;
  ra->width = cam->width;
  ra->height = cam->height;
  ra->row0 = row0;
  ra->rows = rows;
  ra->lod = c->dev.lod;
  ra->macro = c->dev.macro;
  ra->macro_cell = c->dev.macro_cell;
  for (int a = 0; a < 3; ++a) ra->macro_dims[a] = c->dev.macro_dims[a];
  ra->levels = c->tree.lod_levels;  // levels a pruned node can have
  ra->lod_scale = 0.0;
  ra->lod_scale_f = 0.0f;
}

// pixel footprint per unit ray parameter times the pruning threshold (0: pruning off),
// in the operation order the FP64 reference uses
double lod_scale(const amr_camera* cam, double lod_pixels) {
  if (!(lod_pixels > 0.0)) return 0.0;
  return lod_pixels * ((2.0 * cam->tan_half_fov_y) / (double)cam->height);
}

void fill_levels(const amr_ctx* c, DLevel* lv, double step_factor) {
  for (int l = 0; l < c->L; ++l) {
    DLevel& d = lv[l];
    std::memset(&d, 0, sizeof d);
    double hmin = 0.0;
    for (int a = 0; a < 3; ++a) {
      d.h[a] = c->h0[a] / (double)c->rpow[l];
      d.inv_h[a] = 1.0 / d.h[a];
      if (a == 0 || d.h[a] < hmin) hmin = d.h[a];
    }
    d.step = step_factor * hmin;
    d.hmin_d = hmin;
    d.sc = (int32_t)c->rpow[c->L - 1 - l];
    d.inv_sc = 1.0f / (float)d.sc;
    d.hmin = (float)hmin;
    d.inv_step = (float)(1.0 / d.step);
    for (int a = 0; a < 3; ++a) d.ginv[a] = 0.5f * (float)d.inv_h[a];
  }
}

}  // namespace amr

extern "C" {

void amr_default_params(amr_render_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof *p);
  p->step_factor = 0.5;
  p->kappa = 8.0;
  p->ert_eps = 1e-4;
  p->vmin = 0.0;
  p->vmax = 1.0;
  p->ka = 0.3;
  p->kd = 0.6;
  p->ks = 0.3;
  p->shininess = 32.0;
  p->gamma = 1e-3;
  p->interp = AMR_INTERP_TRILINEAR;
  p->shade = 0;
  p->row0 = 0;
  p->rows = 0;
  p->skip = 0;
  p->max_segments = 0;
  p->schedule = AMR_SCHEDULE_AUTO;
  p->learned = 0;
  p->tau = 1e-3;
  p->samples_per_iter = 16;  // measured best for schedule 3 on C2 at 512^2 .. 2048^2
  p->coarse_factor = 4;
  p->light_ambient = 0.2;
  p->learned_min_samples = 1;
}

amr_status amr_create(int32_t num_levels, int32_t refine_ratio, const double domain_lo[3],
                      const double h0[3], int32_t num_patches, const int32_t* patch_level,
                      const int64_t* patch_box, const float* const* cell_data, amr_dtype dtype,
                      amr_ctx** out) {
  g_create_error.clear();
  auto bad = [](const char* m) {
    g_create_error = m;
    return AMR_ERR_ARG;
  };
  if (!out) return bad("out is NULL");
  *out = nullptr;
  if (num_levels < 1 || num_levels > kMaxLevels) return bad("num_levels out of range");
  if (refine_ratio < 2 || refine_ratio > 64) return bad("refine_ratio out of range");
  if (!domain_lo || !h0 || !patch_level || !patch_box || !cell_data) return bad("NULL array");
  if (num_patches < 1) return bad("num_patches must be positive");
  if (dtype != AMR_F32 && dtype != AMR_F16 && dtype != AMR_BF16) return bad("unknown dtype");
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(domain_lo[a]) || !std::isfinite(h0[a]) || !(h0[a] > 0.0))
      return bad("domain_lo / h0 must be finite, h0 positive");
  amr_ctx* c = new (std::nothrow) amr_ctx();
  if (!c) {
    g_create_error = "out of host memory";
    return AMR_ERR_OOM;
  }
  c->L = num_levels;
  c->r = refine_ratio;
  c->dtype = dtype;
  for (int a = 0; a < 3; ++a) {
    c->dlo[a] = domain_lo[a];
    c->h0[a] = h0[a];
  }
  c->rpow[0] = 1;
  for (int k = 1; k < 40; ++k) {
    c->rpow[k] = c->rpow[k - 1] * refine_ratio;
    if (c->rpow[k] > ((int64_t)1 << 40)) c->rpow[k] = ((int64_t)1 << 40);
  }
  if (c->rpow[num_levels - 1] >= ((int64_t)1 << 30)) {
    delete c;
    return bad("refine_ratio^(num_levels-1) too large");
  }
  c->R = c->rpow[num_levels - 1];
  try {
    c->patches.resize((size_t)num_patches);
    for (int p = 0; p < num_patches; ++p) {
      Patch& q = c->patches[p];
      q.level = patch_level[p];
      if (q.level < 0 || q.level >= num_levels) {
        delete c;
        return bad("patch level out of range");
      }
      int64_t sc = c->rpow[num_levels - 1 - q.level];
      int64_t cells = 1;
      for (int k = 0; k < 3; ++k) {
        q.box[k] = patch_box[6 * p + k];
        q.box[3 + k] = patch_box[6 * p + 3 + k];
        if (q.box[k] >= q.box[3 + k]) {
          delete c;
          return bad("patch box with lo >= hi");
        }
        if (std::llabs(q.box[k]) > ((int64_t)1 << 30) || std::llabs(q.box[3 + k]) > ((int64_t)1 << 30) ||
            std::llabs(q.box[k] * sc) >= ((int64_t)1 << 31) ||
            std::llabs(q.box[3 + k] * sc) >= ((int64_t)1 << 31)) {
          delete c;
          return bad("patch box exceeds the int32 finest index space");
        }
        q.n[k] = q.box[3 + k] - q.box[k];
        q.fbox[k] = q.box[k] * sc;
        q.fbox[3 + k] = q.box[3 + k] * sc;
        cells *= q.n[k];
      }
      if (!cell_data[p]) {
        delete c;
        return bad("cell_data entry is NULL");
      }
      q.data.assign(cell_data[p], cell_data[p] + cells);
    }
  } catch (const std::bad_alloc&) {
    delete c;
    g_create_error = "out of host memory";
    return AMR_ERR_OOM;
  }
  *out = c;
  return AMR_OK;
}

amr_status amr_build_host(amr_ctx* c, amr_storage storage_flags) {
  if (!c) return AMR_ERR_ARG;
  const int storage = (int)storage_flags & 0xff;
  const bool gradient = ((int)storage_flags & AMR_STORE_GRADIENT) != 0;
  const int halo = ((int)storage_flags & AMR_STORE_HALO2) ? 2 : 1;
  const bool maxb = ((int)storage_flags & AMR_STORE_MAXBRICK) != 0;
  if (storage < AMR_STORE_PTR || storage > AMR_STORE_ATLAS_TEX3D ||
      ((int)storage_flags & ~(0xff | AMR_STORE_GRADIENT | AMR_STORE_HALO2 | AMR_STORE_MAXBRICK)))
    return fail(c, AMR_ERR_ARG, "unknown storage");
  if (maxb && storage != AMR_STORE_PTR)
    return fail(c, AMR_ERR_ARG, "stencil-maximum bricks need the ptr storage");
  if (c->host_built && c->halo != halo) {
    // bricks, leaf ranges and face bits depend on the halo: build them again
    if (c->device_built) release_device(c);
    c->host_built = false;
    c->bricks.clear();
    c->gbricks.clear();
    c->mbricks.clear();
    c->packing = Packing();
  }
  c->halo = halo;
  if (c->dtype != AMR_F32 && storage != AMR_STORE_PTR && storage != AMR_STORE_ATLAS_LINEAR)
    return fail(c, AMR_ERR_ARG, "16-bit cells need the ptr or atlas_linear storage");
  auto t0 = std::chrono::steady_clock::now();
  try {
    if (fault_injected("bad_alloc")) throw std::bad_alloc();
    if (!c->host_built) {
      amr_status s = validate_hierarchy(c);
      if (s != AMR_OK) return s;
      s = build_tree(c);
      if (s != AMR_OK) return s;
      s = build_bricks(c);
      if (s != AMR_OK) return s;
      c->host_built = true;
    }
    if ((storage == AMR_STORE_ATLAS_LINEAR || storage == AMR_STORE_ATLAS_TEX3D) &&
        c->packing.org.empty()) {
      amr_status s = pack_atlas(c);
      if (s != AMR_OK) return s;
    }
    if (gradient && c->gbricks.empty()) {
      amr_status s = build_gradient_bricks(c);
      if (s != AMR_OK) return s;
    }
    if (maxb && c->mbricks.empty()) {
      amr_status s = build_max_bricks(c);
      if (s != AMR_OK) return s;
    }
    if (c->dtype == AMR_F16) {
      // binary16 tops out at 65504: refuse data that would be stored as infinity
      auto over = [](float v) { return std::isfinite(v) && std::isinf(storage_round(AMR_F16, v)); };
      for (const auto& b : c->bricks)
        for (float v : b)
          if (over(v)) return fail(c, AMR_ERR_ARG, "a cell value exceeds the FP16 range");
      if (gradient)
        for (const auto& g : c->gbricks)
          for (const float4& q : g)
            if (over(q.y) || over(q.z) || over(q.w))
              return fail(c, AMR_ERR_ARG, "a central difference exceeds the FP16 range");
    }
  } catch (const std::bad_alloc&) {
    return fail(c, AMR_ERR_OOM, "out of host memory during the build");
  }
  if ((c->storage != storage || c->want_gradient != gradient || c->want_max != maxb) &&
      c->device_built)
    release_device(c);
  c->storage = storage;
  c->want_gradient = gradient;
  c->want_max = maxb;
  c->build_seconds +=
      std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  c->err.clear();
  return AMR_OK;
}

amr_status amr_build_kdtree(amr_ctx* c, amr_storage storage, void* cuda_stream) {
  if (!c) return AMR_ERR_ARG;
  amr_status s = amr_build_host(c, storage);
  if (s != AMR_OK) return s;
  try {
    return upload(c, cuda_stream);
  } catch (const std::bad_alloc&) {
    return fail(c, AMR_ERR_OOM, "out of host memory during the upload");
  }
}

// AMR_SCHEDULE_AUTO: the schedule measured fastest for the call's work.  Deferred shading
// (schedule 3) wherever it applies - Phong, trilinear, no learned proposal - for images of
// fewer than kAutoDeferredPixels pixels, for batches of views and with secondary rays; the
// per-ray loop (schedule 0) otherwise.  Measured on the 5-level hierarchy (2,219 patches),
// Phong + gradient bricks, Gsamples/s per-ray / deferred: 512^2 9.5 / 29.0, 1024^2 31.1 /
// 46.0, 2048^2 65.4 / 61.1; 64 views of 256-2048 pixels: 21.6 / 30.6.  Every schedule
// gives the same image bit for bit, so the choice affects time only.
constexpr int64_t kAutoDeferredPixels = 3000000;

static const amr_render_params* resolve_schedule(const amr_render_params* p, int64_t pixels,
                                                 bool batch, amr_render_params* tmp) {
  if (!p || p->schedule != AMR_SCHEDULE_AUTO) return p;
  *tmp = *p;
  const bool deferred_applies = p->interp == AMR_INTERP_TRILINEAR && p->shade == 1 &&
                                p->learned == 0;
  // secondary rays: the deferred schedule marches each light ray with a whole warp
  tmp->schedule =
      deferred_applies && (batch || p->shadow || pixels < kAutoDeferredPixels) ? 3 : 0;
  return tmp;
}

// pixels a single-view call renders (its band), for the schedule choice
static int64_t call_pixels(const amr_camera* cam, const amr_render_params* p) {
  if (!cam || !p || cam->width <= 0 || cam->height <= 0) return 0;
  const int64_t row0 = std::max(0, std::min(p->row0, cam->height));
  const int64_t rows = p->rows <= 0 ? cam->height - row0 : std::min<int64_t>(p->rows, cam->height - row0);
  return (int64_t)cam->width * std::max<int64_t>(rows, 0);
}

static amr_status prepare_render(amr_ctx* c, const amr_camera* cam, int32_t tf_n,
                                 const amr_render_params* p, RenderArgs* a) {
  if (!c) return AMR_ERR_ARG;
  if (!c->device_built) return fail(c, AMR_ERR_STATE, "render before amr_build_kdtree");
  amr_status s = check_camera(c, cam);
  if (s != AMR_OK) return s;
  if (!p) return fail(c, AMR_ERR_ARG, "params is NULL");
  if (tf_n < 2 || tf_n > 2048) return fail(c, AMR_ERR_ARG, "tf_n must be in [2, 2048]");
  if (!(p->vmax > p->vmin)) return fail(c, AMR_ERR_ARG, "vmax must exceed vmin");
  if (!(p->step_factor > 0.0) || !std::isfinite(p->step_factor))
    return fail(c, AMR_ERR_ARG, "step_factor must be positive");
  if (!(p->kappa >= 0.0)) return fail(c, AMR_ERR_ARG, "kappa must be non-negative");
  if (p->interp != 0 && p->interp != 1) return fail(c, AMR_ERR_ARG, "unknown interp");
  if (p->shade != 0 && p->shade != 1) return fail(c, AMR_ERR_ARG, "unknown shade");
  if (p->schedule < 0 || p->schedule > 3)
    return fail(c, AMR_ERR_ARG, "unknown schedule (AMR_SCHEDULE_AUTO is resolved before this)");
  if (p->schedule == 3 && (p->interp != AMR_INTERP_TRILINEAR || p->shade != 1 || p->learned != 0))
    return fail(c, AMR_ERR_ARG, "deferred shading renders trilinear with shade = 1, no proposal");
  if (p->schedule >= 2 && (p->samples_per_iter < 1 || p->samples_per_iter > 64))
    return fail(c, AMR_ERR_ARG, "samples_per_iter must be in [1, 64]");
  if (p->schedule == 2 && p->interp != AMR_INTERP_TRILINEAR)
    return fail(c, AMR_ERR_ARG, "the refill schedule renders trilinear");
  if (!(p->lod_pixels >= 0.0) || !std::isfinite(p->lod_pixels))
    return fail(c, AMR_ERR_ARG, "lod_pixels must be finite and non-negative");
  if (p->lod_pixels > 0.0 && (p->schedule == 1 || p->learned != 0))
    return fail(c, AMR_ERR_ARG,
                "level-of-detail pruning needs schedule 0, 2 or 3 without the proposal");
  if (p->shadow != 0 && p->shadow != 1) return fail(c, AMR_ERR_ARG, "shadow must be 0 or 1");
  if (p->shadow) {
    for (int a = 0; a < 3; ++a)
      if (!std::isfinite(p->light[a])) return fail(c, AMR_ERR_ARG, "light must be finite");
    if (!(p->light_step > 0.0) || !std::isfinite(p->light_step))
      return fail(c, AMR_ERR_ARG, "light_step must be positive");
    if (!(p->light_ambient >= 0.0 && p->light_ambient <= 1.0))
      return fail(c, AMR_ERR_ARG, "light_ambient must be in [0, 1]");
    if (p->interp != AMR_INTERP_TRILINEAR || (p->schedule != 0 && p->schedule != 3) ||
        p->learned != 0)
      return fail(c, AMR_ERR_ARG,
                  "secondary rays need trilinear sampling, schedule 0 or 3, no proposal");
  }
  if (p->row0 < 0 || p->row0 >= cam->height) return fail(c, AMR_ERR_ARG, "row0 out of range");
  int rows = p->rows <= 0 ? cam->height - p->row0 : std::min(p->rows, cam->height - p->row0);
  std::memset(a, 0, sizeof *a);
  fill_ray(c, cam, p->row0, rows, &a->ray);
  a->ray.lod_scale = lod_scale(cam, p->lod_pixels);
  a->ray.lod_scale_f = (float)a->ray.lod_scale;
  fill_levels(c, a->lv, p->step_factor);
  a->nodes = c->dev.nodes;
  a->leaves = c->dev.leaves;
  a->face_node = c->dev.face_node;
  a->node_box = c->dev.node_box;
  a->patches = c->dev.patches;
  a->pool = c->dev.pool;
  a->gpool = (const float4*)c->dev.gpool;
  a->atlas = c->dev.atlas_tex;
  a->gatlas = c->dev.gatlas_tex;
  a->tf_n = tf_n;
  int64_t ms = p->max_segments > 0 ? p->max_segments : 4 * (int64_t)c->tree.axis.size() + 64;
  a->max_segments = (int32_t)std::min<int64_t>(ms, INT32_MAX);
  a->skip = p->skip ? 1 : 0;
  a->kappa = (float)p->kappa;
  a->ert_thresh = p->ert_eps > 0.0 ? (float)(1.0 - p->ert_eps) : 2.0f;
  a->vmin = (float)p->vmin;
  a->inv_range = (float)(1.0 / (p->vmax - p->vmin));
  a->ka = (float)p->ka;
  a->kd = (float)p->kd;
  a->ks = (float)p->ks;
  a->shininess = (float)p->shininess;
  a->gfloor_num = (float)(p->gamma * (p->vmax - p->vmin));
  a->counters = c->dev.counters;
  a->ray.counters = c->dev.counters;
  a->mlp = c->dev.proposal;
  a->tau = (float)p->tau;
  a->learned = p->learned;
  a->inv_levels = c->L > 1 ? 1.0f / (float)(c->L - 1) : 0.0f;
  a->samples_per_iter = p->samples_per_iter;
  a->shadow = p->shadow;
  for (int q = 0; q < 3; ++q)
    a->light_f[q] = (float)((p->light[q] - c->dlo[q]) * a->ray.inv_hf[q]);
  a->light_step = (float)p->light_step;
  a->light_ambient = (float)p->light_ambient;
  a->coarse_factor = p->coarse_factor;
  a->learned_min_samples = p->learned_min_samples;
  a->mdelta = c->dev.mpool ? (long long)((char*)c->dev.mpool - (char*)c->dev.pool) : 0;
  if (c->dtype != AMR_F32 && (p->interp != AMR_INTERP_TRILINEAR || p->schedule == 1))
    return fail(c, AMR_ERR_ARG, "16-bit cells render trilinear with schedule 0, 2 or 3");
  if (p->learned != 0) {
    if (p->learned != 1 && p->learned != 2) return fail(c, AMR_ERR_ARG, "unknown learned mode");
    if (p->learned == 2 && (p->coarse_factor < 2 || p->coarse_factor > 64))
      return fail(c, AMR_ERR_ARG, "coarse_factor must be in [2, 64]");
    if (p->learned_min_samples < 1 || p->learned_min_samples > kMaxSamplesPerSegment)
      return fail(c, AMR_ERR_ARG, "learned_min_samples must be in [1, 2^22]");
    if (c->dtype != AMR_F32) return fail(c, AMR_ERR_ARG, "the learned proposal needs FP32 cells");
    if (!c->dev.proposal) return fail(c, AMR_ERR_STATE, "learned render before amr_set_proposal");
    if (p->interp != AMR_INTERP_TRILINEAR)
      return fail(c, AMR_ERR_ARG, "the learned proposal renders with trilinear sampling");
  }
  return AMR_OK;
}

// kernel storage id: the strategy, or its 16-bit-cell variant (ids 4..7)
static int kernel_storage(const amr_ctx* c) {
  if (c->dtype == AMR_F32) return c->storage;
  return c->storage + (c->dtype == AMR_F16 ? 4 : 5);
}

// shading variant: 2 = Phong reading the gradient bricks (trilinear only), when built;
// plus the stencil-maximum opacity test (trilinear, per-ray or deferred schedule, no
// secondary rays or proposal), when those bricks were built
static int kernel_shade(const amr_ctx* c, const amr_render_params* p) {
  int sh = p->shade;
  if (p->shade && p->interp == AMR_INTERP_TRILINEAR && c->want_gradient && c->dev.gpool_bytes)
    sh = 2;
  if (c->dev.mpool && p->interp == AMR_INTERP_TRILINEAR && !p->shadow &&
      (p->learned || p->schedule == 0 || p->schedule == 3))
    sh |= kShadeMaxBit;
  return sh | (p->shadow ? kShadeShadowBit : 0);
}

static amr_status finish_render(amr_ctx* c, cudaStream_t st, uint64_t* samples_out) {
  if (!samples_out) return AMR_OK;
  unsigned long long h[kNumCounters] = {0};
  CK(cudaMemcpyAsync(h, c->dev.counters, sizeof h, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  std::memcpy(c->last_counters, h, sizeof h);
  *samples_out = h[0];
  if (h[1] & kStatusDevice) return fail(c, AMR_ERR_DEVICE, "device reported a malformed tree");
  if (h[1] & kStatusCapacity)
    return fail(c, AMR_ERR_CAPACITY, "a ray exceeded the segment or sample bound");
  return AMR_OK;
}

}  // extern "C"

namespace amr {
amr_status prepare_render_args(amr_ctx* c, const amr_camera* cam, int32_t tf_n,
                               const amr_render_params* p, RenderArgs* a) {
  return prepare_render(c, cam, tf_n, p, a);
}
amr_render_params resolve_render_schedule(const amr_camera* cam, const amr_render_params& p) {
  amr_render_params tmp;
  return *resolve_schedule(&p, call_pixels(cam, &p), false, &tmp);
}
amr_status launch_render_args(amr_ctx* c, const RenderArgs& a, const amr_render_params* p,
                              void* stream) {
  if (p->learned) return launch_learned(c, a, c->storage, kernel_shade(c, p), stream);
  return launch_render(c, a, kernel_storage(c), p->interp, kernel_shade(c, p), p->schedule, stream);
}
}  // namespace amr

extern "C" {

amr_status amr_render(amr_ctx* c, const amr_camera* cam, const float* tf_rgba_dev, int32_t tf_n,
                      const amr_render_params* params_in, float* out_rgba_dev, void* cuda_stream,
                      uint64_t* samples_out) {
  amr_render_params tmp;
  const amr_render_params* params =
      resolve_schedule(params_in, call_pixels(cam, params_in), false, &tmp);
  RenderArgs a;
  amr_status s = prepare_render(c, cam, tf_n, params, &a);
  if (s != AMR_OK) return s;
  if (!tf_rgba_dev || !out_rgba_dev) return fail(c, AMR_ERR_ARG, "NULL device buffer");
  if (((uintptr_t)tf_rgba_dev | (uintptr_t)out_rgba_dev) & 15)
    return fail(c, AMR_ERR_ARG, "device buffers must be 16-byte aligned");
  a.tf = reinterpret_cast<const float4*>(tf_rgba_dev);
  a.out = reinterpret_cast<float4*>(out_rgba_dev);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  CK(cudaMemsetAsync(c->dev.counters, 0, kNumCounters * sizeof(unsigned long long), st));
  s = launch_render_args(c, a, params, cuda_stream);
  if (s != AMR_OK) return s;
  return finish_render(c, st, samples_out);
}

amr_status amr_render_host(amr_ctx* c, const amr_camera* cam, const float* tf_rgba_host,
                           int32_t tf_n, const amr_render_params* params_in, float* out_rgba_host,
                           void* cuda_stream, uint64_t* samples_out) {
  amr_render_params tmp;
  const amr_render_params* params =
      resolve_schedule(params_in, call_pixels(cam, params_in), false, &tmp);
  RenderArgs a;
  amr_status s = prepare_render(c, cam, tf_n, params, &a);
  if (s != AMR_OK) return s;
  if (!tf_rgba_host || !out_rgba_host) return fail(c, AMR_ERR_ARG, "NULL host buffer");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  DeviceState& d = c->dev;
  if (d.tf_scratch_n < tf_n) {
    cudaFree(d.tf_scratch);
    d.tf_scratch = nullptr;
    d.tf_scratch_n = 0;
    CK(cudaMalloc(&d.tf_scratch, (size_t)tf_n * sizeof(float4)));
    d.tf_scratch_n = tf_n;
  }
  const size_t img_bytes = (size_t)a.ray.rows * a.ray.width * sizeof(float4);
  if (d.img_scratch_bytes < img_bytes) {
    cudaFree(d.img_scratch);
    d.img_scratch = nullptr;
    d.img_scratch_bytes = 0;
    CK(cudaMalloc(&d.img_scratch, img_bytes));
    d.img_scratch_bytes = img_bytes;
  }
  CK(cudaMemcpyAsync(d.tf_scratch, tf_rgba_host, (size_t)tf_n * sizeof(float4),
                     cudaMemcpyHostToDevice, st));
  a.tf = d.tf_scratch;
  a.out = d.img_scratch;
  CK(cudaMemsetAsync(d.counters, 0, kNumCounters * sizeof(unsigned long long), st));
  s = launch_render_args(c, a, params, cuda_stream);
  if (s != AMR_OK) return s;
  CK(cudaMemcpyAsync(out_rgba_host, d.img_scratch, img_bytes, cudaMemcpyDeviceToHost, st));
  if (samples_out) return finish_render(c, st, samples_out);
  CK(cudaStreamSynchronize(st));
  return AMR_OK;
}

}  // extern "C"

namespace {

// Kernel arguments of one batched render: the shared render state from the first view,
// then the view table (tiles in view order) and its checks.
amr_status prepare_batch(amr_ctx* c, const amr_view* views, int32_t n_views, const float* tfs_dev,
                         int32_t n_tf, int32_t tf_n, const amr_render_params* p, float* out_dev,
                         int64_t out_floats, const amr_batch_config& cfg, BatchArgs* b) {
  if (!c) return AMR_ERR_ARG;
  if (!views || n_views < 1 || n_views > kMaxBatchViews)
    return fail(c, AMR_ERR_ARG, "n_views must be in [1, AMR_MAX_BATCH_VIEWS]");
  if (!p) return fail(c, AMR_ERR_ARG, "params is NULL");
  if (n_tf < 1 || n_tf > 8 || (int64_t)n_tf * tf_n > 2048)
    return fail(c, AMR_ERR_ARG, "need 1 <= n_tf <= 8 and n_tf * tf_n <= 2048");
  if (p->row0 != 0 || p->rows > 0)
    return fail(c, AMR_ERR_ARG, "batched views render whole images (row0 = 0, rows <= 0)");
  if (p->interp != AMR_INTERP_TRILINEAR || (p->schedule != 0 && p->schedule != 3) ||
      p->learned != 0 || p->shadow)
    return fail(c, AMR_ERR_ARG,
                "batched rendering is trilinear, schedule 0 or 3, without the proposal or "
                "secondary rays");
  if (cfg.rays_per_thread < 1 || cfg.rays_per_thread > 8 || cfg.blocks_per_sm < 0)
    return fail(c, AMR_ERR_ARG, "batch config: rays_per_thread in [1, 8], blocks_per_sm >= 0");
  if (cfg.samples_per_iter < 0 || cfg.samples_per_iter > 64)
    return fail(c, AMR_ERR_ARG, "batch config: samples_per_iter in [0, 64]");
  if (!((cfg.tile_w == 8 && cfg.tile_h == 8) || (cfg.tile_w == 16 && cfg.tile_h == 8) ||
        (cfg.tile_w == 16 && cfg.tile_h == 16)))
    return fail(c, AMR_ERR_ARG, "batch tile must be 8x8, 16x8 or 16x16");
  amr_status s = prepare_render(c, &views[0].cam, tf_n, p, &b->A);
  if (s != AMR_OK) return s;
  if (kernel_storage(c) != AMR_STORE_PTR)
    return fail(c, AMR_ERR_ARG, "batched rendering needs the ptr storage with FP32 cells");
  if (!tfs_dev || !out_dev) return fail(c, AMR_ERR_ARG, "NULL device buffer");
  if (((uintptr_t)tfs_dev | (uintptr_t)out_dev) & 15)
    return fail(c, AMR_ERR_ARG, "device buffers must be 16-byte aligned");
  std::vector<std::pair<int64_t, int64_t>> ranges;
  int64_t items = 0;
  const int64_t tile_rows = (int64_t)cfg.tile_h * cfg.rays_per_thread;
  for (int v = 0; v < n_views; ++v) {
    const amr_view& in = views[v];
    s = check_camera(c, &in.cam);
    if (s != AMR_OK) return s;
    if (in.tf_index < 0 || in.tf_index >= n_tf) return fail(c, AMR_ERR_ARG, "tf_index out of range");
    const int64_t n = 4 * (int64_t)in.cam.width * in.cam.height;
    if (in.out_offset < 0 || (in.out_offset & 3) || in.out_offset + n > out_floats)
      return fail(c, AMR_ERR_ARG, "view image outside the output buffer or not 16-byte aligned");
    ranges.push_back({in.out_offset, in.out_offset + n});
    BatchView& bv = b->v[v];
    std::memset(&bv, 0, sizeof bv);
    for (int a = 0; a < 3; ++a) {
      bv.eye[a] = in.cam.eye[a];
      bv.fwd[a] = in.cam.fwd[a];
      bv.right[a] = in.cam.right[a];
      bv.up[a] = in.cam.up[a];
    }
    bv.tan_half_fov_y = in.cam.tan_half_fov_y;
    bv.width = in.cam.width;
    bv.height = in.cam.height;
    bv.tiles_x = (int32_t)((in.cam.width + cfg.tile_w - 1) / cfg.tile_w);
    bv.item0 = (int32_t)items;
    bv.tf = in.tf_index;
    bv.out = in.out_offset / 4;
    bv.lod_scale = lod_scale(&in.cam, p->lod_pixels);
    bv.lod_scale_f = (float)bv.lod_scale;
    items += (int64_t)bv.tiles_x * ((in.cam.height + tile_rows - 1) / tile_rows);
    if (items >= ((int64_t)1 << 31)) return fail(c, AMR_ERR_ARG, "too many pixel tiles");
  }
  std::sort(ranges.begin(), ranges.end());
  for (size_t k = 1; k < ranges.size(); ++k)
    if (ranges[k].first < ranges[k - 1].second)
      return fail(c, AMR_ERR_ARG, "view images overlap in the output buffer");
  b->n_views = n_views;
  b->n_items = (int32_t)items;
  b->n_tf = n_tf;
  b->rays_per_thread = cfg.rays_per_thread;
  b->A.tf = reinterpret_cast<const float4*>(tfs_dev);
  b->A.out = reinterpret_cast<float4*>(out_dev);
  if (cfg.samples_per_iter > 0) b->A.samples_per_iter = cfg.samples_per_iter;
  return AMR_OK;
}

}  // namespace

extern "C" {

amr_status amr_render_batch(amr_ctx* c, const amr_view* views, int32_t n_views,
                            const float* tfs_rgba_dev, int32_t n_tf, int32_t tf_n,
                            const amr_render_params* params_in, float* out_rgba_dev,
                            int64_t out_floats, const amr_batch_config* config, void* cuda_stream,
                            uint64_t* samples_out) {
  if (!c) return AMR_ERR_ARG;
  amr_render_params tmp;
  const amr_render_params* params = resolve_schedule(params_in, 0, true, &tmp);
  const amr_batch_config cfg = config ? *config : c->batch_cfg;
  std::unique_ptr<BatchArgs> b(new (std::nothrow) BatchArgs());
  if (!b) return fail(c, AMR_ERR_OOM, "out of host memory");
  amr_status s = prepare_batch(c, views, n_views, tfs_rgba_dev, n_tf, tf_n, params, out_rgba_dev,
                               out_floats, cfg, b.get());
  if (s != AMR_OK) return s;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  CK(cudaMemsetAsync(c->dev.counters, 0, kNumCounters * sizeof(unsigned long long), st));
  s = launch_batch(c, *b, kernel_storage(c), kernel_shade(c, params), params->schedule, cfg,
                   cuda_stream);
  if (s != AMR_OK) return s;
  return finish_render(c, st, samples_out);
}

amr_status amr_batch_autotune(amr_ctx* c, const amr_view* views, int32_t n_views,
                              const float* tfs_rgba_dev, int32_t n_tf, int32_t tf_n,
                              const amr_render_params* params_in, float* out_rgba_dev,
                              int64_t out_floats, int32_t reps, void* cuda_stream,
                              amr_batch_config* best_out, float* ms_out) {
  if (!c) return AMR_ERR_ARG;
  amr_render_params tmp;
  const amr_render_params* params = resolve_schedule(params_in, 0, true, &tmp);
  if (reps < 1 || reps > 1000) return fail(c, AMR_ERR_ARG, "reps must be in [1, 1000]");
  static const int shapes[3][2] = {{8, 8}, {16, 8}, {16, 16}};
  static const int rpts[3] = {1, 2, 4};
  cudaStream_t st = (cudaStream_t)cuda_stream;
  std::unique_ptr<BatchArgs> b(new (std::nothrow) BatchArgs());
  if (!b) return fail(c, AMR_ERR_OOM, "out of host memory");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  auto done = [&](amr_status r) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return r;
  };
  float best_ms = -1.0f;
  amr_batch_config best = c->batch_cfg;
  // candidates 0..8: tile shape x rays per thread; 9..12: the best of those with 4, 8, 16
  // and 32 samples per iteration (deferred shading only)
  static const int spis[4] = {4, 8, 16, 32};
  const int shade = kernel_shade(c, params);
  for (int k = 0; k < AMR_BATCH_CANDIDATES; ++k) {
    amr_batch_config cfg = {shapes[k / 3][0], shapes[k / 3][1], rpts[k % 3], 0, 0};
    if (k >= 9) {
      if (params->schedule != 3) {
        if (ms_out) ms_out[k] = -1.0f;
        continue;
      }
      cfg = best;
      cfg.samples_per_iter = spis[k - 9];
    }
    amr_status s = prepare_batch(c, views, n_views, tfs_rgba_dev, n_tf, tf_n, params,
                                 out_rgba_dev, out_floats, cfg, b.get());
    if (s != AMR_OK) return done(s);
    float ms = 0.0f;
    for (int r = -1; r < reps; ++r) {  // one untimed warm-up
      if (r == 0 && cudaEventRecord(e0, st) != cudaSuccess) return done(fail(c, AMR_ERR_CUDA, "event"));
      if (cudaMemsetAsync(c->dev.counters, 0, kNumCounters * sizeof(unsigned long long), st) !=
          cudaSuccess)
        return done(fail(c, AMR_ERR_CUDA, "cudaMemsetAsync"));
      s = launch_batch(c, *b, kernel_storage(c), shade, params->schedule, cfg, cuda_stream);
      if (s != AMR_OK) return done(s);
    }
    if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
      return done(fail(c, AMR_ERR_CUDA, "batch autotune timing failed"));
    uint64_t n = 0;
    s = finish_render(c, st, &n);  // surfaces device status of the last run
    if (s != AMR_OK) return done(s);
    ms /= (float)reps;
    if (ms_out) ms_out[k] = ms;
    if (best_ms < 0.0f || ms < best_ms) {
      best_ms = ms;
      best = cfg;
    }
  }
  c->batch_cfg = best;
  if (best_out) *best_out = best;
  return done(AMR_OK);
}

amr_status amr_set_proposal(amr_ctx* c, const void* packed_dev, void* cuda_stream) {
  if (!c) return AMR_ERR_ARG;
  if (!c->device_built) return fail(c, AMR_ERR_STATE, "amr_set_proposal before amr_build_kdtree");
  if (!packed_dev) return fail(c, AMR_ERR_ARG, "packed weights are NULL");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (!c->dev.proposal) CK(cudaMalloc(&c->dev.proposal, AMR_MLP_PACKED_BYTES));
  CK(cudaMemcpyAsync(c->dev.proposal, packed_dev, AMR_MLP_PACKED_BYTES, cudaMemcpyDeviceToDevice, st));
  CK(cudaStreamSynchronize(st));
  return AMR_OK;
}

amr_status amr_log_segments(amr_ctx* c, const amr_camera* cam, const float* tf_rgba_dev,
                            int32_t tf_n, const amr_render_params* params, float* features_dev,
                            float* targets_dev, int64_t capacity, unsigned long long* count_dev,
                            float keep_prob, uint32_t seed, void* cuda_stream) {
  if (!params) return fail(c, AMR_ERR_ARG, "params is NULL");
  if (c && c->dtype != AMR_F32) return fail(c, AMR_ERR_ARG, "segment logging needs FP32 cells");
  amr_render_params p = *params;
  p.schedule = 0;   // the logging kernel runs the per-ray loop
  p.ert_eps = 0.0;  // log every segment of the ray
  p.learned = 0;
  p.interp = AMR_INTERP_TRILINEAR;
  RenderArgs a;
  amr_status s = prepare_render(c, cam, tf_n, &p, &a);
  if (s != AMR_OK) return s;
  if (!tf_rgba_dev || !features_dev || !targets_dev || !count_dev || capacity < 0)
    return fail(c, AMR_ERR_ARG, "bad segment-log buffers");
  if (!(keep_prob >= 0.0f && keep_prob <= 1.0f))
    return fail(c, AMR_ERR_ARG, "keep_prob must be in [0, 1]");
  a.tf = reinterpret_cast<const float4*>(tf_rgba_dev);
  return launch_log(c, a, c->storage, features_dev, targets_dev, capacity, count_dev, keep_prob,
                    seed, cuda_stream);
}

amr_status amr_destroy(amr_ctx* c) {
  if (!c) return AMR_OK;
  release_device(c);
  delete c;
  return AMR_OK;
}

const char* amr_last_error(const amr_ctx* c) {
  if (c) return c->err.c_str();
  return g_create_error.empty() ? amr::mlp_last_error() : g_create_error.c_str();
}

amr_status amr_get_stats(const amr_ctx* c, amr_stats* out) {
  if (!c || !out) return AMR_ERR_ARG;
  std::memset(out, 0, sizeof *out);
  out->num_patches = (int64_t)c->patches.size();
  for (const Patch& p : c->patches) out->num_cells += p.n[0] * p.n[1] * p.n[2];
  out->storage = c->storage;
  out->build_seconds = c->build_seconds;
  for (int k = 0; k < 3; ++k) out->exact_paths[k] = (int64_t)c->last_counters[2 + k];
  if (!c->host_built) return AMR_OK;
  out->num_nodes = (int64_t)c->tree.axis.size();
  out->num_leaves = (int64_t)c->tree.leaf_patch.size();
  out->max_depth = c->tree.max_depth;
  int64_t brick = 0;
  for (const auto& b : c->bricks) brick += (int64_t)b.size();
  out->brick_bytes = c->device_built ? (int64_t)c->dev.pool_bytes : brick * 4;
  out->tree_bytes = out->num_nodes * (int64_t)sizeof(DNode) +
                    out->num_leaves * (int64_t)sizeof(DLeaf) +
                    out->num_patches * (int64_t)sizeof(DPatch);
  if (!c->packing.org.empty()) {
    double vol = 1.0;
    for (int a = 0; a < 3; ++a) {
      out->atlas_dims[a] = (int32_t)c->packing.dims[a];
      vol *= (double)c->packing.dims[a];
    }
    out->atlas_efficiency = (double)out->num_cells / vol;
    out->atlas_efficiency_halo = (double)brick / vol;
  }
  return AMR_OK;
}

amr_status amr_get_leaves(const amr_ctx* c, int32_t* box6, int32_t* patch, int32_t* level,
                          int64_t cap, int64_t* n) {
  if (!c || !n) return AMR_ERR_ARG;
  if (!c->host_built) return AMR_ERR_STATE;
  const int64_t m = (int64_t)c->tree.leaf_patch.size();
  *n = m;
  if (cap < m) return AMR_ERR_CAPACITY;
  if (!box6 || !patch || !level) return AMR_ERR_ARG;
  std::memcpy(box6, c->tree.leaf_box.data(), sizeof(int32_t) * 6 * (size_t)m);
  std::memcpy(patch, c->tree.leaf_patch.data(), sizeof(int32_t) * (size_t)m);
  std::memcpy(level, c->tree.leaf_level.data(), sizeof(int32_t) * (size_t)m);
  return AMR_OK;
}

amr_status amr_get_nodes(const amr_ctx* c, int32_t* axis, int32_t* split, int32_t* left,
                         int32_t* right, int32_t* leaf, int64_t cap, int64_t* n) {
  if (!c || !n) return AMR_ERR_ARG;
  if (!c->host_built) return AMR_ERR_STATE;
  const int64_t m = (int64_t)c->tree.axis.size();
  *n = m;
  if (cap < m) return AMR_ERR_CAPACITY;
  if (!axis || !split || !left || !right || !leaf) return AMR_ERR_ARG;
  const size_t b = sizeof(int32_t) * (size_t)m;
  std::memcpy(axis, c->tree.axis.data(), b);
  std::memcpy(split, c->tree.split.data(), b);
  std::memcpy(left, c->tree.left.data(), b);
  std::memcpy(right, c->tree.right.data(), b);
  std::memcpy(leaf, c->tree.leaf.data(), b);
  return AMR_OK;
}

amr_status amr_get_lod_leaves(const amr_ctx* c, int32_t* box6, int32_t* patch, int32_t* level,
                              int32_t* node, int64_t cap, int64_t* n) {
  if (!c || !n) return AMR_ERR_ARG;
  if (!c->host_built) return AMR_ERR_STATE;
  const Tree& t = c->tree;
  const int64_t m = (int64_t)t.lod_patch.size();
  *n = m;
  if (cap < m) return AMR_ERR_CAPACITY;
  if (m && (!box6 || !patch || !level || !node)) return AMR_ERR_ARG;
  std::memcpy(box6, t.lod_box.data(), sizeof(int32_t) * 6 * (size_t)m);
  std::memcpy(patch, t.lod_patch.data(), sizeof(int32_t) * (size_t)m);
  std::memcpy(level, t.lod_level.data(), sizeof(int32_t) * (size_t)m);
  const int32_t M = (int32_t)t.leaf_patch.size();
  for (size_t k = 0; k < t.node_lod.size(); ++k)
    if (t.node_lod[k] >= 0) node[t.node_lod[k] - M] = (int32_t)k;
  return AMR_OK;
}

amr_status amr_get_leaf_faces(const amr_ctx* c, int32_t* faces, int32_t* face_node, int64_t cap,
                              int64_t* n) {
  if (!c || !n) return AMR_ERR_ARG;
  if (!c->host_built) return AMR_ERR_STATE;
  const Tree& t = c->tree;
  const int64_t m = (int64_t)t.leaf_patch.size();
  *n = m;
  if (cap < m) return AMR_ERR_CAPACITY;
  if (!faces || !face_node) return AMR_ERR_ARG;
  for (int64_t k = 0; k < m; ++k) faces[k] = t.leaf_faces[(size_t)k];
  std::memcpy(face_node, t.face_node.data(), sizeof(int32_t) * 12 * (size_t)m);
  return AMR_OK;
}

amr_status amr_get_brick(const amr_ctx* c, int32_t patch, float* out, int64_t cap, int64_t* n) {
  if (!c || !n) return AMR_ERR_ARG;
  if (!c->host_built) return AMR_ERR_STATE;
  if (patch < 0 || patch >= (int32_t)c->patches.size()) return AMR_ERR_ARG;
  const std::vector<float>& b = c->bricks[(size_t)patch];
  *n = (int64_t)b.size();
  if (cap < *n) return AMR_ERR_CAPACITY;
  if (!out) return AMR_ERR_ARG;
  for (size_t i = 0; i < b.size(); ++i) out[i] = storage_round(c->dtype, b[i]);
  return AMR_OK;
}

amr_status amr_trace(amr_ctx* c, const amr_camera* cam, double lod_pixels, int32_t* leaf_seq_dev,
                     double* t_seq_dev, int32_t* seq_len_dev, int32_t max_len, void* cuda_stream) {
  if (!c) return AMR_ERR_ARG;
  if (!c->device_built) return fail(c, AMR_ERR_STATE, "trace before amr_build_kdtree");
  amr_status s = check_camera(c, cam);
  if (s != AMR_OK) return s;
  if (!leaf_seq_dev || !seq_len_dev || max_len < 1)
    return fail(c, AMR_ERR_ARG, "bad trace buffers");
  if (!(lod_pixels >= 0.0) || !std::isfinite(lod_pixels))
    return fail(c, AMR_ERR_ARG, "lod_pixels must be finite and non-negative");
  std::unique_ptr<TraceArgs> ap(new (std::nothrow) TraceArgs());
  if (!ap) return fail(c, AMR_ERR_OOM, "out of host memory");
  TraceArgs& a = *ap;
  std::memset(&a, 0, sizeof a);
  fill_ray(c, cam, 0, cam->height, &a.ray);
  fill_levels(c, a.lv, 0.5);
  a.ray.lod_scale = lod_scale(cam, lod_pixels);
  a.ray.lod_scale_f = (float)a.ray.lod_scale;
  a.nodes = c->dev.nodes;
  a.leaves = c->dev.leaves;
  a.face_node = c->dev.face_node;
  a.node_box = c->dev.node_box;
  a.leaf_seq = leaf_seq_dev;
  a.t_seq = t_seq_dev;
  a.seq_len = seq_len_dev;
  a.max_len = max_len;
  a.max_segments = (int32_t)std::min<int64_t>(4 * (int64_t)c->tree.axis.size() + 64, INT32_MAX);
  a.counters = c->dev.counters;
  a.ray.counters = c->dev.counters;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  CK(cudaMemsetAsync(c->dev.counters, 0, kNumCounters * sizeof(unsigned long long), st));
  s = launch_trace(c, a, cuda_stream);
  if (s != AMR_OK) return s;
  unsigned long long h[2] = {0, 0};
  CK(cudaMemcpyAsync(h, c->dev.counters, sizeof h, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (h[1] & kStatusDevice) return fail(c, AMR_ERR_DEVICE, "device reported a malformed tree");
  if (h[1] & kStatusCapacity) return fail(c, AMR_ERR_CAPACITY, "segment bound exceeded");
  return AMR_OK;
}

}  // extern "C"
