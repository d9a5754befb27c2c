/*
 * amr.h - C ABI of the GB300 single-pass raycaster for structured AMR data.
 *
 * Method: Kaehler & Abel, "Single-Pass GPU-Raycasting for Structured Adaptive Mesh
 * Refinement Data" (arXiv 1212.3333).  The library partitions overlapping AMR patches
 * into a kD-tree of non-overlapping, single-level leaves (Sec. 3.1), stores one brick per
 * patch (Sec. 4), and marches every pixel's ray front to back through the leaves with
 * kd-restart (Sec. 3.3), sampling each leaf at a step proportional to its level's cell
 * size, with trilinear interpolation, optional gradient Phong shading across block
 * boundaries (Sec. 4, Fig. 6) and emission-absorption compositing (Sec. 3, Sec. 5).
 *
 * Conventions
 *   - Every call returns an amr_status; nothing aborts or exits.  amr_last_error() gives
 *     a message for the last failing call on a context (per context, not thread-safe:
 *     use one context per thread at a time).
 *   - Every device loop is bounded; a kernel that meets a bound (segments per ray, samples
 *     per segment, descent depth) sets a status word instead of trapping, and the call
 *     that synchronises reports AMR_ERR_CAPACITY or AMR_ERR_DEVICE.
 *   - Fault injection for tests (host side only): the environment variable AMR_FAULT =
 *     bad_alloc makes the host build fail with AMR_ERR_OOM, oom the device upload's first
 *     allocation (AMR_ERR_OOM), corrupt_node uploads a root node that names itself as a
 *     child (indices stay in range; renders report AMR_ERR_DEVICE).  Unset: no effect.
 *   - Level l has spacing h^l = h^0 / r^l per axis (Sec. 2).  Patch boxes are int64[6]
 *     {lo_x, lo_y, lo_z, hi_x, hi_y, hi_z}, half-open, in level-l cell indices.  Level 0
 *     must tile its bounding box (the kD root, Sec. 3.1); same-level patches must be
 *     disjoint; every patch must lie inside the root.
 *   - Cell data is one float32 per cell, x fastest: index i + nx*(j + ny*k).
 *   - Tree coordinates are int32 cells of the finest level (L-1).
 *   - Device pointers are plain CUDA device addresses (e.g. torch tensor data_ptr());
 *     streams are cudaStream_t passed as void* (NULL = legacy default stream).
 *   - The context owns every device allocation it makes; outputs and streams belong to
 *     the caller.  Rendering is asynchronous on the given stream.
 */
#ifndef AMR_H
#define AMR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct amr_ctx amr_ctx; /* opaque; owned by the library */

typedef enum {
  AMR_OK = 0,
  AMR_ERR_ARG = 1,        /* invalid argument (null pointer, bad size, bad box, bad enum) */
  AMR_ERR_OVERLAP = 2,    /* two patches of one level overlap */
  AMR_ERR_NOT_TILED = 3,  /* level 0 does not tile its bounding box */
  AMR_ERR_STATE = 4,      /* call out of order (e.g. render before build) */
  AMR_ERR_OOM = 5,        /* host or device allocation failed */
  AMR_ERR_CUDA = 6,       /* a CUDA runtime call failed */
  AMR_ERR_CAPACITY = 7,   /* a bounded device loop hit its limit (segments, samples) */
  AMR_ERR_DEVICE = 8      /* the device reported an inconsistent structure */
} amr_status;

/* Device storage type of the brick cells.  AMR_F16 (IEEE binary16) and AMR_BF16 (bfloat16)
 * halve the brick bytes; cells are rounded to nearest-even once at upload and widened to
 * FP32 before interpolation, so gradients, transfer function and compositing stay FP32,
 * and ray/leaf entry and exit stay FP64-exact.  The paper stores FP32 cells; the 16-bit
 * forms trade accuracy for bandwidth on its bandwidth-bound march (Sec. 5). */
typedef enum { AMR_F32 = 0, AMR_F16 = 1, AMR_BF16 = 2 } amr_dtype;

/* Brick storage strategies (Sec. 4).  The paper's GL designs are a packed memory-pool
 * texture (Sec. 4.1) and bindless texture handles (Sec. 4.2); these are their CUDA
 * counterparts. */
typedef enum {
  AMR_STORE_PTR = 0,          /* per-patch table of device pointers into one brick pool */
  AMR_STORE_TEXOBJ = 1,       /* per-patch table of cudaTextureObject_t, one 3D array each */
  AMR_STORE_ATLAS_LINEAR = 2, /* NFDH-packed atlas (Sec. 4.1) in linear device memory */
  AMR_STORE_ATLAS_TEX3D = 3,  /* NFDH-packed atlas in one 3D cudaArray, read as a texture */
  /* flag, OR-ed with a strategy: also build gradient bricks (float4 per cell: value and the
   * three central differences of the cell values, 4x the brick bytes).  Shaded trilinear
   * renders then read one float4 stencil per opaque sample instead of 32 cells whenever
   * all six gradient neighbours lie in the sample's leaf; results are unchanged. */
  AMR_STORE_GRADIENT = 0x100,
  /* flag: bricks carry a two-cell halo (the paper's bricks, Sec. 4, need one), and a leaf
   * face whose far side - the slab of one cell of the leaf's level - lies only in leaves
   * of that same level (any patch) lets the gradient neighbours there read the leaf's own
   * brick, as a face onto the same unrefined patch does with one cell.  The halo cells
   * hold V_l like the first layer.  Not in the paper; results agree with the one-cell
   * layout to FP32 rounding. */
  AMR_STORE_HALO2 = 0x200,
  /* flag (AMR_STORE_PTR only): also build stencil-maximum bricks - per cell the largest of
   * the eight cells of the trilinear stencil it starts, in the cell type.  A trilinear
   * value never exceeds its stencil's maximum and the transfer function's lookup is
   * monotone, so a sample whose stencil maximum maps to zero opacity (with one table entry
   * of margin for rounding) is transparent; the per-ray and deferred marches decide such
   * samples with one load instead of eight.  Images and sample counts are unchanged (each
   * sample is still taken); not in the paper. */
  AMR_STORE_MAXBRICK = 0x400
} amr_storage;

/* Pinhole camera.  Pixel (i, j), row 0 at the top, has the ray o = eye,
 * d = fwd + u*right + v*up with u = (2(i+0.5)/W - 1) * tan_half_fov_y * W/H and
 * v = (1 - 2(j+0.5)/H) * tan_half_fov_y (d is not normalised). */
typedef struct {
  double eye[3], fwd[3], right[3], up[3];
  double tan_half_fov_y;
  int32_t width, height;
} amr_camera;

typedef enum { AMR_INTERP_NEAREST = 0, AMR_INTERP_TRILINEAR = 1 } amr_interp;

/* amr_render_params.schedule value that lets the library choose (the default): deferred
 * shading (3) where it applies (Phong, trilinear, no learned proposal) for images of fewer
 * than 3,000,000 pixels, for batches of views and with secondary rays; the per-ray loop
 * (0) otherwise.  Not in the paper; every schedule renders the same image bit for bit
 * (with secondary rays: to rounding, see shadow). */
#define AMR_SCHEDULE_AUTO (-1)

typedef struct {
  double step_factor; /* sample step = step_factor * h^l of the leaf's level (Sec. 3.3) */
  double kappa;       /* extinction scale: sigma = kappa * alpha_TF (world^-1) */
  double ert_eps;     /* early ray termination once A >= 1 - ert_eps; <= 0 disables */
  double vmin, vmax;  /* value range mapped onto the transfer function */
  double ka, kd, ks, shininess; /* headlight Phong constants (shade = 1) */
  double gamma;       /* gradient floor: n = g / max(|g|, gamma (vmax-vmin) / h^l) */
  int32_t interp;     /* amr_interp */
  int32_t shade;      /* 0: unshaded, 1: central-difference gradient Phong (Sec. 4, Fig. 6) */
  int32_t row0;       /* first image row to render (band partitioning); 0 for all */
  int32_t rows;       /* number of rows; <= 0: all rows from row0 */
  int32_t skip;       /* 0: none; 1: exact leaf min/max empty-space skipping */
  int32_t max_segments; /* per-ray segment bound; <= 0: 4 * nodes + 64 */
  int32_t schedule;   /* 0: one loop per ray; 1: warp wavefront (the samples of a warp's
                         current segments spread over its lanes, shading on the compacted
                         opaque samples); 2: persistent warps that refill finished lanes
                         with new rays and fetch segments in batches (trilinear only);
                         3: warps march their rays in step and shade the opaque samples
                         32 at a time (trilinear, shade = 1 only).  All give the same
                         image.  AMR_SCHEDULE_AUTO (-1, the default) picks one per call. */
  int32_t learned;    /* learned segment proposal (needs amr_set_proposal; trilinear; ptr or
                         atlas_linear storage, FP32 cells): 0 off; 1 skip segments whose predicted
                         contribution is below tau; 2 sample them with a coarse_factor times
                         coarser step */
  double tau;         /* proposal threshold (default 1e-3) */
  int32_t samples_per_iter; /* schedules 2 and 3: samples a lane takes between warp steps,
                               1..64 (default 16) */
  int32_t coarse_factor;    /* learned mode 2: a segment predicted below tau takes
                               ceil(n / coarse_factor) samples, 2..64 (default 4) */
  double lod_pixels;        /* level-of-detail pruning (Sec. 3.1 type-(a) nodes, Sec. 3.3):
                               > 0 stops the descent at an inner node lying in one patch of
                               level l once min_a h^l_a <= lod_pixels * (2 tan_half_fov_y / H)
                               * t0 (t0 the segment's entry parameter, a unit fwd assumed),
                               and samples it at level l; gradients then read the same pruned
                               tree.  0 (default) renders every level.  Schedules 0, 2 and
                               3, no learned proposal. */
  int32_t shadow;           /* 1: secondary rays to a point light (the global-illumination
                               example of Sec. 5): an opaque sample at x is lit by
                               I = light_ambient + (1 - light_ambient) T, T the transmittance
                               of the part of x -> light inside the root box, marched with
                               n = max(1, ceil(len / light_step)) midpoint samples of the AMR
                               field (T = prod exp(-kappa a_TF len / n), 0 once <= 1e-4);
                               its colour is multiplied by I.  Trilinear; schedule 0 (each
                               lane marches its samples' light rays) or 3 with shade = 1
                               (a warp marches each light ray 32 samples at a time; T then
                               differs from schedule 0's by rounding only). */
  double light[3];          /* light position (world) */
  double light_step;        /* world step along secondary rays (> 0 with shadow) */
  double light_ambient;     /* in [0, 1] (default 0.2) */
  int32_t learned_min_samples; /* learned modes: the proposal is consulted only for segments
                                  of at least this many samples (shorter ones are sampled as
                                  the plain march samples them), 1..2^22 (default 1: every
                                  segment; skipping short segments is where the proposal
                                  saves most, measured on the 5-level hierarchy) */
  int32_t reserved;
} amr_render_params;

/* Fills p with the defaults: step 0.5, kappa 8, ert_eps 1e-4, vmin 0, vmax 1, ka 0.3,
 * kd 0.6, ks 0.3, shininess 32, gamma 1e-3, trilinear, unshaded, all rows, no skip,
 * schedule AMR_SCHEDULE_AUTO, samples_per_iter 16. */
void amr_default_params(amr_render_params* p);

/* Create a context from an AMR hierarchy (Sec. 2: h^l = h^0 / r^l, patches Gamma^l_m).
 *   num_levels    L >= 1;  refine_ratio r >= 2 (constant, as in the paper's notation)
 *   domain_lo[3]  world position of level-0 cell index 0;  h0[3] level-0 spacing
 *   num_patches   P >= 1;  patch_level[P] in [0, L);  patch_box[6P] as above
 *   cell_data[P]  host pointers, float32, x fastest; copied (the caller keeps ownership)
 *   dtype         device storage type of the brick cells (amr_dtype; input is always FP32)
 * Returns AMR_ERR_ARG for malformed input; tiling and overlaps are checked at build. */
amr_status amr_create(int32_t num_levels, int32_t refine_ratio, const double domain_lo[3],
                      const double h0[3], int32_t num_patches, const int32_t* patch_level,
                      const int64_t* patch_box, const float* const* cell_data,
                      amr_dtype dtype, amr_ctx** out);

/* Build the kD-tree (Sec. 3.1: min-crossing planes, balanced tie-break, level-by-level
 * refinement), the per-patch bricks with a one-cell halo (Sec. 4: one brick per subgrid),
 * the chosen storage (Sec. 4.1 packing / 4.2 handle table) and upload everything on
 * `cuda_stream`.  `storage` is an amr_storage strategy, optionally OR AMR_STORE_GRADIENT
 * and / or AMR_STORE_HALO2 (a different halo than the context's first build rebuilds the
 * host data).
 * The call returns after the uploads complete.  With AMR_F16 / AMR_BF16 cells: only
 * AMR_STORE_PTR and AMR_STORE_ATLAS_LINEAR (else AMR_ERR_ARG); gradient bricks hold the
 * value and the FP32 central differences, each rounded to the 16-bit type; AMR_F16 returns
 * AMR_ERR_ARG if a finite cell value (or, with gradient bricks, a central difference)
 * would round to infinity (|x| >= 65520).  Device leaf min/max ranges are those of the
 * rounded cells, so exact skipping stays exact. */
amr_status amr_build_kdtree(amr_ctx* ctx, amr_storage storage, void* cuda_stream);

/* Host-only part of amr_build_kdtree (tree, bricks, packing), for inspecting the tree
 * without a GPU.  amr_build_kdtree may follow it (it then only uploads). */
amr_status amr_build_host(amr_ctx* ctx, amr_storage storage);

/* Render one image (Sec. 3.3 ray traversal, Sec. 3 compositing) into out_rgba_dev:
 * caller-owned device float32 [rows][W][4], premultiplied RGBA, row 0 = image row row0.
 * tf_rgba_dev: device float32 [tf_n][4] (2 <= tf_n <= 2048), linear between entries over
 * [vmin, vmax].  Both device buffers must be 16-byte aligned.  Asynchronous on cuda_stream.  samples_out (nullable, host): when given,
 * the call synchronises the stream, checks the device status word and stores the exact
 * number of samples taken (sum over segments of the per-segment sample count).
 * 16-bit cells render trilinear with the per-ray schedule (else AMR_ERR_ARG). */
amr_status amr_render(amr_ctx* ctx, const amr_camera* cam, const float* tf_rgba_dev,
                      int32_t tf_n, const amr_render_params* params, float* out_rgba_dev,
                      void* cuda_stream, uint64_t* samples_out);

/* amr_render with host buffers: copies tf_rgba_host to the device, renders, copies the
 * image back to out_rgba_host ([rows][W][4] float32) and synchronises.  Page-locked host
 * buffers make the copies asynchronous with respect to other streams. */
amr_status amr_render_host(amr_ctx* ctx, const amr_camera* cam, const float* tf_rgba_host,
                           int32_t tf_n, const amr_render_params* params, float* out_rgba_host,
                           void* cuda_stream, uint64_t* samples_out);

/* amr_render_host for callers that must not allocate device memory during rendering (a
 * host application whose device memory another allocator owns and caps, or a process
 * whose device footprint must not grow after start-up).  The paper has no counterpart.
 * It calls no cudaMalloc / cudaFree: counters, the transfer function and the image are
 * staged in one fixed 4 MiB + 32 KiB + 64 B array that is part of the library (every GPU
 * that loads the library holds it until the process exits).  The frame is rendered in
 * 16-row bands that fit the array and copied band by band into out_rgba_host, so results
 * equal amr_render_host's; limits: 2 <= tf_n <= 2048, image width <= 16384
 * (AMR_ERR_ARG beyond them).  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) for that device; make that first call before any stream
 * capture.  Under CUDA's lazy module loading that first call is also when the array is
 * committed on the device, so a caller whose footprint must be fixed before rendering
 * makes one call at start-up.  The current device must be the one the context was built
 * on (else AMR_ERR_STATE).  Every call reuses the array (the counters are cleared per
 * call); calls that overlap on the GPU race, so serialise them.  Synchronises the stream
 * before returning, on errors too once work was queued; samples_out (nullable) receives
 * the sample count. */
amr_status amr_render_host_noalloc(amr_ctx* ctx, const amr_camera* cam,
                                   const float* tf_rgba_host, int32_t tf_n,
                                   const amr_render_params* params, float* out_rgba_host,
                                   void* cuda_stream, uint64_t* samples_out);

/* ---------------------------------------------------------------------------------- */
/* batched multi-view rendering (not in the paper, which renders one view per pass)      */
/* ---------------------------------------------------------------------------------- */

#define AMR_MAX_BATCH_VIEWS 128
#define AMR_BATCH_CANDIDATES 13  /* tiles 8x8, 16x8, 16x16  x  rays per thread 1, 2, 4;
                                    then samples per iteration 4, 8, 16, 32 */

/* One view of a batch: its camera, which transfer function it uses, and where its image
 * starts in the shared output buffer (in floats; a multiple of 4). */
typedef struct {
  amr_camera cam;
  int32_t tf_index;
  int32_t reserved;
  int64_t out_offset;
} amr_view;

/* Work decomposition of a batched render: pixel tiles of tile_w x tile_h threads (8x8,
 * 16x8 or 16x16), each thread marching rays_per_thread (1..8) pixels of a column of its
 * tile, so a queue item covers tile_w x (tile_h * rays_per_thread) pixels; blocks_per_sm
 * caps the persistent grid per SM (0: as many as fit); samples_per_iter (0: the params'
 * value, else 1..64) is the deferred schedule's samples per lane between warp steps. */
typedef struct {
  int32_t tile_w, tile_h, rays_per_thread, blocks_per_sm;
  int32_t samples_per_iter;
} amr_batch_config;

/* Render n_views (1..AMR_MAX_BATCH_VIEWS) views of the context's dataset in one persistent
 * launch: the pixel tiles of all views form one work queue that resident blocks drain.
 * Every view's image equals, bit for bit, amr_render of that view alone with the same
 * params and its transfer function.
 *   views          host array [n_views]; whole images (params->row0 = 0, rows <= 0)
 *   tfs_rgba_dev   device float32 [n_tf][tf_n][4], 1 <= n_tf <= 8, n_tf * tf_n <= 2048
 *   out_rgba_dev   device float32 [out_floats]; view v writes [H][W][4] at out_offset;
 *                  images must not overlap; buffers 16-byte aligned
 *   config         NULL: the context's last autotuned configuration (initially 16x8, 1,
 *                  the params' samples_per_iter)
 * Needs the ptr storage with FP32 cells, trilinear sampling, schedule 0 (per-ray loop) or
 * 3 (deferred shading, shade = 1), no learned proposal and no secondary rays (else
 * AMR_ERR_ARG).  Issues one cudaMemsetAsync and one kernel launch
 * on cuda_stream and allocates nothing, so with samples_out NULL the call can be captured
 * in a CUDA graph; samples_out (nullable, host) synchronises and returns the total sample
 * count of all views (plus the device status check, as amr_render). */
amr_status amr_render_batch(amr_ctx* ctx, const amr_view* views, int32_t n_views,
                            const float* tfs_rgba_dev, int32_t n_tf, int32_t tf_n,
                            const amr_render_params* params, float* out_rgba_dev,
                            int64_t out_floats, const amr_batch_config* config,
                            void* cuda_stream, uint64_t* samples_out);

/* Time candidate configurations on this batch, one warm-up and `reps` (1..1000) timed
 * renders each, CUDA events on cuda_stream: first the 9 tiles 8x8 / 16x8 / 16x16 x rays
 * per thread 1 / 2 / 4 (blocks_per_sm 0, the params' samples_per_iter), then - for deferred
 * shading (schedule 3, also as AMR_SCHEDULE_AUTO picks it for batches) - the best of those
 * with samples_per_iter 4, 8, 16 and 32.  ms_out (nullable) receives the mean milliseconds
 * of the AMR_BATCH_CANDIDATES candidates in that order (tile-major; -1 for the last four
 * under the per-ray schedule, which has no samples-per-iteration knob); best_out
 * (nullable) the fastest, which the context also keeps for amr_render_batch calls without
 * a config.  Synchronises; arguments as amr_render_batch. */
amr_status amr_batch_autotune(amr_ctx* ctx, const amr_view* views, int32_t n_views,
                              const float* tfs_rgba_dev, int32_t n_tf, int32_t tf_n,
                              const amr_render_params* params, float* out_rgba_dev,
                              int64_t out_floats, int32_t reps, void* cuda_stream,
                              amr_batch_config* best_out, float* ms_out);

/* ---------------------------------------------------------------------------------- */
/* learned segment proposal (not in the paper): a 12-64-64-64-1 MLP, ReLU hidden layers,  */
/* sigmoid output, predicting a segment's opacity contribution A_out - A_in from 12       */
/* features: entry xyz, exit xyz (root-box units), level / (L-1), leaf value min and max  */
/* through the TF domain, accumulated opacity, octahedral ray direction.                  */
/* ---------------------------------------------------------------------------------- */

#define AMR_MLP_FEATURES 12
#define AMR_MLP_PARAMS 9217      /* W1[64][12] b1[64] W2[64][64] b2[64] W3[64][64] b3[64]
                                    W4[1][64] b4[1], FP32, W[out][in] row-major */
#define AMR_MLP_PACKED_BYTES 23440 /* inference image: BF16 weights, padded rows, FP32 biases */
#define AMR_MLP_GRAD_BLOCKS 152    /* blocks of the gradient pass (at most) */
#define AMR_MLP_GRAD_SCRATCH (AMR_MLP_GRAD_BLOCKS * (AMR_MLP_PARAMS + 1)) /* floats */

/* Record training data: the plain march of one view (no early termination) writes, for each
 * segment a seeded hash keeps with probability keep_prob, its 12 features to
 * features_dev[k*12 ..] and its contribution A_out - A_in to targets_dev[k].  Records follow
 * pixel order (row-major within the view's rows), then segment order along the ray, and k
 * continues from *count_dev, which grows by the view's record count (the caller zeroes it
 * before the first view; records with k >= capacity are dropped but still counted): the
 * same views give the same records in the same places.  A first pass counts each pixel's
 * records into per-pixel buffers the context keeps (allocated on first use, grown for
 * larger views); calls on one context must therefore be ordered (one stream).  Storage must
 * be ptr or atlas_linear with FP32 cells.  Asynchronous.  Errors: AMR_ERR_ARG, AMR_ERR_OOM,
 * AMR_ERR_CUDA. */
amr_status amr_log_segments(amr_ctx* ctx, const amr_camera* cam, const float* tf_rgba_dev,
                            int32_t tf_n, const amr_render_params* params, float* features_dev,
                            float* targets_dev, int64_t capacity, unsigned long long* count_dev,
                            float keep_prob, uint32_t seed, void* cuda_stream);

/* FP32 parameters (AMR_MLP_PARAMS, device) -> packed inference image (AMR_MLP_PACKED_BYTES,
 * device, 16-byte aligned): BF16 weights as the tensor-core kernels read them. */
amr_status amr_mlp_pack(const float* params_dev, void* packed_dev, void* cuda_stream);

/* Inference through the same mma.sync BF16 warp routine the learned march uses:
 * y_dev[r] = sigmoid(MLP(x_dev[r*12 ..])) for r < n (FP32 accumulation, activations rounded
 * to BF16 between layers).  Asynchronous.  Errors: amr_last_error(NULL). */
amr_status amr_mlp_forward(const void* packed_dev, const float* x_dev, int64_t n, float* y_dev,
                           void* cuda_stream);

/* Mean binary cross-entropy of sigmoid(MLP(x)) against targets t in [0,1] over a batch of n
 * rows and its gradient with respect to all AMR_MLP_PARAMS parameters.  Batch row r is
 * dataset row (perm_a * (first + r) + perm_b) mod n_total of x_dev[n_total][12] and
 * t_dev[n_total]; with perm_a coprime to n_total, consecutive batches walk a pseudo-random
 * permutation (perm_a = 1, perm_b = 0: rows first .. first + n - 1).  The forward rounds
 * weights and activations to BF16 as inference does; the backward is FP32.  Overwrites
 * grad_dev and loss_dev[0].  scratch_dev: caller-owned device buffer of AMR_MLP_GRAD_SCRATCH
 * floats (no contents expected; overwritten) holding each block's partial sums, which a
 * second kernel adds in a fixed order: the same inputs give the same gradient and loss bit
 * for bit.  A scratch buffer must not be shared by calls in flight on different streams.
 * Asynchronous.  Limits: n_total, perm_a < 2^31.  Errors: AMR_ERR_ARG (a null pointer, n or
 * n_total not positive, limits), AMR_ERR_CUDA; amr_last_error(NULL). */
amr_status amr_mlp_loss_grad(const float* params_dev, const float* x_dev, const float* t_dev,
                             int64_t n_total, int64_t first, int64_t n, int64_t perm_a,
                             int64_t perm_b, float* grad_dev, float* loss_dev, float* scratch_dev,
                             void* cuda_stream);

/* One Adam step (bias-corrected, step >= 1) on the AMR_MLP_PARAMS FP32 parameters. */
amr_status amr_mlp_adam(float* params_dev, const float* grad_dev, float* m_dev, float* v_dev,
                        float lr, float beta1, float beta2, float eps, int32_t step,
                        void* cuda_stream);

/* Install packed proposal weights (device, AMR_MLP_PACKED_BYTES) in the context for renders
 * with params->learned != 0.  Copies them; synchronises the stream. */
amr_status amr_set_proposal(amr_ctx* ctx, const void* packed_dev, void* cuda_stream);

/* Release the context and every device allocation it owns (NULL-safe). */
amr_status amr_destroy(amr_ctx* ctx);

/* Message of the last failing call on ctx ("" if none; ctx may be NULL for a failed
 * amr_create, which reports through a process-wide slot). */
const char* amr_last_error(const amr_ctx* ctx);

/* ---------------------------------------------------------------------------------- */
/* inspection and test hooks                                                            */
/* ---------------------------------------------------------------------------------- */

typedef struct {
  int64_t num_nodes, num_leaves, num_patches, num_cells;
  int64_t brick_bytes;      /* device bytes of cell data incl. halos (all storages) */
  int64_t tree_bytes;       /* device bytes of nodes + leaves + patch table */
  int32_t atlas_dims[3];    /* atlas extent in texels (atlas storages), else 0 */
  double atlas_efficiency;  /* cells / atlas texels (halos excluded), atlas storages */
  double atlas_efficiency_halo; /* brick texels incl. halos / atlas texels */
  double build_seconds;     /* host build time (tree + bricks + packing) */
  int32_t max_depth;        /* deepest leaf (root = 0) */
  int32_t storage;          /* amr_storage in use, -1 before build */
  int64_t exact_paths[3];   /* last render with samples_out: FP64 recomputations of descent
                               decisions, sample counts, and sample / neighbour positions */
} amr_stats;

amr_status amr_get_stats(const amr_ctx* ctx, amr_stats* out);

/* Leaves in canonical order (pre-order over the tree): box int32[6*n] in finest cells,
 * patch id, level.  cap = capacity in leaves; *n receives the leaf count (also when cap
 * is too small, which returns AMR_ERR_CAPACITY). */
amr_status amr_get_leaves(const amr_ctx* ctx, int32_t* box6, int32_t* patch, int32_t* level,
                          int64_t cap, int64_t* n);

/* Nodes in pre-order: axis (-1 for a leaf), split plane (finest cells), pre-order ids of
 * the two children (-1 for a leaf), leaf id (-1 for an internal node). */
amr_status amr_get_nodes(const amr_ctx* ctx, int32_t* axis, int32_t* split, int32_t* left,
                         int32_t* right, int32_t* leaf, int64_t cap, int64_t* n);

/* Type-(a) nodes (Sec. 3.1) in the order of their pruned-leaf ids M, M+1, ...: box
 * (finest cells, 6 per node), the patch of that level holding the box, its level, and the
 * node's pre-order id.  cap in nodes; *n receives their count. */
amr_status amr_get_lod_leaves(const amr_ctx* ctx, int32_t* box6, int32_t* patch, int32_t* level,
                              int32_t* node, int64_t cap, int64_t* n);

/* Per leaf (canonical order): faces, bit 2a (+1) set when the level cell beyond the lower
 * (upper) face on axis a lies in the leaf's patch and overlaps only leaves of that patch;
 * face_node [12 per leaf]: for each face 2a + side the pre-order id of the deepest node
 * holding the leaf and that cell (clipped to the root), then of the one holding the cell
 * alone (the root when the cell lies outside it).  These drive the kernels' gradient
 * neighbour lookups.  cap in leaves; *n receives the leaf count. */
amr_status amr_get_leaf_faces(const amr_ctx* ctx, int32_t* faces, int32_t* face_node, int64_t cap,
                              int64_t* n);

/* The host brick of patch p with its one-cell halo: float32 [(nz+2)][(ny+2)][(nx+2)],
 * brick index b = level cell c - lo + 1.  cap in floats; *n receives the brick size.
 * With 16-bit cells the values are the rounded ones the device holds. */
amr_status amr_get_brick(const amr_ctx* ctx, int32_t patch, float* out, int64_t cap,
                         int64_t* n);

/* Per-pixel traversal (Sec. 3.3 kd-restart) on the device: for pixel (i, j) with
 * p = j*W + i, leaf_seq_dev[p*max_len + k] is the k-th leaf id, t_seq_dev (nullable)
 * [p*max_len + k][2] its entry/exit ray parameters (float64), seq_len_dev[p] the number
 * of segments (0 for a miss, -1 when more than max_len).  All device buffers.
 * lod_pixels > 0 prunes the descent as amr_render_params.lod_pixels does; pruned inner
 * nodes report ids after the M leaves (M + k for the k-th such node in pre-order). */
amr_status amr_trace(amr_ctx* ctx, const amr_camera* cam, double lod_pixels,
                     int32_t* leaf_seq_dev, double* t_seq_dev, int32_t* seq_len_dev,
                     int32_t max_len, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* AMR_H */
