/*
 * FP64 CPU oracle for single-pass kD-tree raycasting of structured AMR (SAMR) data,
 * after Kaehler & Abel, "Single-Pass GPU-Raycasting for Structured Adaptive Mesh
 * Refinement Data" (arXiv 1212.3333).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference the CUDA path is
 * checked against.  It shares no code, header, table or helper with the product library
 * and is loaded only by the tests, the smoke check and the CPU-baseline leg of the bench.
 * Every quantity is computed in double precision, in the order the definitions below
 * state them.  Build with -ffp-contract=off: the traversal decisions are compared bit for
 * bit with the GPU, so no multiply-add may be fused.
 *
 * Contents (paper section in brackets):
 *   kD-tree build by brute-force plane sweep          [Sec. 3.1 "kD-tree construction"]
 *   level value V_l, trilinear S_l, AMR field F        [Sec. 2 (SAMR), Sec. 4 interpolation]
 *   ray generation, root slab test, kd-restart         [Sec. 3.3 "Ray traversal"]
 *   level-proportional midpoint sampling               [Sec. 3.3, sampling rate vs cell size]
 *   transfer function, emission-absorption compositing [Sec. 3 outline, Sec. 5]
 *   central-difference gradients + headlight Phong     [Sec. 4, Fig. 6, Sec. 5]
 *   12-64-64-64-1 MLP forward/backward (learned segment proposal; not in the paper)
 *
 * Readings where the paper is silent (all fixed here and mirrored by the CUDA path):
 *   - boxes are half-open [lo,hi) in level-l cells; tree coordinates are integers in the
 *     finest level's index space; level 0 must tile its bounding box (the root).
 *   - split choice: fewest piece crossings, then smallest |V_left - V_right| (geometric
 *     volume of the node on each side), then smallest axis, then smallest plane;
 *     candidate planes are the level-l cell faces strictly inside the node.
 *   - a leaf fully covered by a level-l piece is relabelled to that patch at level l;
 *     a leaf no level-l patch touches keeps its label.
 *   - V_l(c): clamp c into the domain; the level-l patch value if one holds c, else
 *     S_l'(centre of c) at the finest coarser level l' whose patch holds that centre.
 *   - kd-restart near child = the side the ray enters first (d_a > 0: lower); t_s >= t1
 *     -> near only, t_s <= t0 -> far only, else near with t1 = t_s; d_a == 0 -> the side
 *     holding the origin (lower iff o_a < plane).
 *   - n = max(1, ceil(len / (f * h^l))) equal sub-steps per segment, samples at the
 *     sub-step midpoints; the sample value is S_l of the segment's leaf level.
 *   - alpha = 1 - exp(-kappa * a_TF * delta); C += (1-A) alpha rgb; A += (1-A) alpha;
 *     stop once A >= 1 - eps_ert (eps_ert <= 0: never).
 *   - level of detail (Sec. 3.1 type-(a) nodes, Sec. 3.3 pruning): an inner node whose box
 *     lies in one patch of level l (its label) may stand in for its subtree.  With
 *     lod_pixels > 0 the segment starting at t0 stops the descent at the first such node
 *     with hmin^l <= X = lod_pixels * (2 tan_half_fov_y / H) * t0 (the level's cells cover
 *     at most lod_pixels pixels at parameter t0, t in units of a unit fwd vector) and is
 *     sampled at level l from that patch; F_X, the field of that pruned tree, replaces F
 *     in the segment's gradients.  Pruned nodes take leaf ids after the leaves, in
 *     pre-order.
 *   - secondary rays to a point light (the global-illumination example of Sec. 5 and its
 *     figure; the paper gives no formula): an opaque sample at x is lit by
 *     I = ambient + (1 - ambient) T, T = prod_k (1 - alpha_k) over n = max(1, ceil(len /
 *     step)) midpoint samples of F on the part of the segment from x to the light inside
 *     the root box (len its world length, alpha_k = 1 - exp(-kappa a_TF(F) len / n)), the
 *     march stopping with T = 0 once T <= 1e-4; the sample's colour is multiplied by I.
 *   - gradient g_a = (F(x + h^l e_a) - F(x - h^l e_a)) / (2 h^l_a);
 *     n = g / max(|g|, gamma (vmax - vmin) / h^l); headlight L = V = H = -d/|d|;
 *     rgb' = clamp(rgb (ka + kd |n.L|) + ks |n.L|^shininess, 0, 1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef long long i64;

enum { ORC_OK = 0, ORC_ERR_ARG = -1, ORC_ERR_OVERLAP = -2, ORC_ERR_NOT_TILED = -3,
       ORC_ERR_STATE = -4, ORC_ERR_OOM = -5, ORC_ERR_CAPACITY = -6 };

typedef struct {
  int level;
  i64 box[6];   /* level-l cells */
  i64 fbox[6];  /* finest-level cells */
  float* data;  /* own copy, x fastest */
  i64 nx, ny, nz;
} opatch;

typedef struct {
  int axis;     /* -1: leaf */
  i64 split;    /* finest coordinate of the plane */
  int left, right;
  i64 box[6];   /* finest coordinates */
  int patch, level;
} onode;

typedef struct orc_hier {
  int L, r, P;
  double dlo[3], h0[3];
  i64 R;           /* r^(L-1) */
  i64 rpow[64];    /* r^k */
  opatch* patches;
  int* by_level;   /* patch ids grouped by level */
  int lev_start[65];
  i64 root[6];     /* finest */
  /* tree */
  onode* nodes;
  int nn, cap;
  int* pre2node;   /* pre-order id -> node index */
  int* leaf2node;  /* leaf id -> node index */
  int* node2leaf;  /* node index -> leaf id (-1 internal) */
  int* node2lod;   /* node index -> id of the node as a pruned leaf (-1: not a type-(a) node) */
  int nleaves, nlod;
  int built;
} orc_hier;

typedef struct {
  double eye[3], fwd[3], right[3], up[3];
  double tan_half_fov_y;
  int width, height;
} orc_camera;

typedef struct {
  double step_factor, kappa, ert_eps, vmin, vmax;
  double ka, kd, ks, shininess, gamma;
  double world_step;  /* > 0: one world-space step for every level */
  int interp;         /* 0 nearest, 1 trilinear */
  int shade;          /* 0 none, 1 gradient Phong */
  int lookup;         /* F's finest-level search: 0 kD-tree descent, 1 scan of all patches */
  int max_segments;   /* per ray; exceeding it is a capacity error */
  double lod_pixels;  /* > 0: level-of-detail pruning threshold in pixels */
  int shadow;         /* 1: secondary rays to the point light */
  double light[3];    /* light position (world) */
  double light_step;  /* world step along secondary rays */
  double light_ambient;
} orc_params;

/* ------------------------------------------------------------------------------------ */
/* small integer helpers                                                                */
/* ------------------------------------------------------------------------------------ */

static i64 floordiv(i64 a, i64 b) { /* b > 0 */
  i64 q = a / b;
  if ((a % b != 0) && (a < 0)) q -= 1;
  return q;
}

static i64 vol6(const i64* b) { return (b[3] - b[0]) * (b[4] - b[1]) * (b[5] - b[2]); }

static int box_contains_cell(const i64* b, i64 i, i64 j, i64 k) {
  return b[0] <= i && i < b[3] && b[1] <= j && j < b[4] && b[2] <= k && k < b[5];
}

/* intersection of two half-open boxes into out; returns 1 if it has positive volume */
static int box_and(const i64* a, const i64* b, i64* out) {
  for (int k = 0; k < 3; ++k) {
    out[k] = a[k] > b[k] ? a[k] : b[k];
    out[3 + k] = a[3 + k] < b[3 + k] ? a[3 + k] : b[3 + k];
    if (out[k] >= out[3 + k]) return 0;
  }
  return 1;
}

/* ------------------------------------------------------------------------------------ */
/* hierarchy                                                                            */
/* ------------------------------------------------------------------------------------ */

void orc_destroy(orc_hier* h) {
  if (!h) return;
  if (h->patches) {
    for (int p = 0; p < h->P; ++p) free(h->patches[p].data);
    free(h->patches);
  }
  free(h->by_level);
  free(h->nodes);
  free(h->pre2node);
  free(h->leaf2node);
  free(h->node2leaf);
  free(h->node2lod);
  free(h);
}

/* Copies boxes and data.  Validation (tiling, overlaps) happens in orc_build. */
orc_hier* orc_create(int L, int r, const double* dlo, const double* h0, int P,
                     const int* level, const i64* box, const float* const* data) {
  if (L < 1 || L > 30 || r < 2 || P < 1) return NULL;
  orc_hier* h = (orc_hier*)calloc(1, sizeof(orc_hier));
  if (!h) return NULL;
  h->L = L; h->r = r; h->P = P;
  for (int k = 0; k < 3; ++k) { h->dlo[k] = dlo[k]; h->h0[k] = h0[k]; }
  h->rpow[0] = 1;
  for (int k = 1; k < 64; ++k) h->rpow[k] = (k < 40) ? h->rpow[k - 1] * r : 0;
  h->R = h->rpow[L - 1];
  h->patches = (opatch*)calloc((size_t)P, sizeof(opatch));
  h->by_level = (int*)calloc((size_t)P, sizeof(int));
  if (!h->patches || !h->by_level) { orc_destroy(h); return NULL; }
  for (int p = 0; p < P; ++p) {
    opatch* q = &h->patches[p];
    q->level = level[p];
    if (q->level < 0 || q->level >= L) { orc_destroy(h); return NULL; }
    for (int k = 0; k < 6; ++k) q->box[k] = box[6 * p + k];
    for (int k = 0; k < 3; ++k)
      if (q->box[k] >= q->box[3 + k]) { orc_destroy(h); return NULL; }
    i64 sc = h->rpow[L - 1 - q->level];
    for (int k = 0; k < 6; ++k) q->fbox[k] = q->box[k] * sc;
    q->nx = q->box[3] - q->box[0];
    q->ny = q->box[4] - q->box[1];
    q->nz = q->box[5] - q->box[2];
    size_t n = (size_t)(q->nx * q->ny * q->nz);
    q->data = (float*)malloc(n * sizeof(float));
    if (!q->data) { orc_destroy(h); return NULL; }
    memcpy(q->data, data[p], n * sizeof(float));
  }
  int c = 0;
  for (int l = 0; l < L; ++l) {
    h->lev_start[l] = c;
    for (int p = 0; p < P; ++p)
      if (h->patches[p].level == l) h->by_level[c++] = p;
  }
  h->lev_start[L] = c;
  return h;
}

/* ------------------------------------------------------------------------------------ */
/* kD-tree build (Sec. 3.1), brute force over every candidate plane                     */
/* ------------------------------------------------------------------------------------ */

typedef struct { i64 b[6]; int patch; } opiece;

static int new_node(orc_hier* h, const i64* box, int patch, int level) {
  if (h->nn == h->cap) {
    int nc = h->cap ? 2 * h->cap : 1024;
    onode* nb = (onode*)realloc(h->nodes, (size_t)nc * sizeof(onode));
    if (!nb) return -1;
    h->nodes = nb;
    h->cap = nc;
  }
  onode* n = &h->nodes[h->nn];
  n->axis = -1; n->split = 0; n->left = n->right = -1;
  for (int k = 0; k < 6; ++k) n->box[k] = box[k];
  n->patch = patch; n->level = level;
  return h->nn++;
}

/* Split `node` until every leaf lies inside one piece or touches none (pieces are the
 * level-l patch boxes intersected with the node, finest coordinates). */
static int refine(orc_hier* h, int node, const opiece* pc, int np, int l) {
  if (np == 0) return ORC_OK;
  i64 nb[6];
  memcpy(nb, h->nodes[node].box, sizeof nb);
  for (int q = 0; q < np; ++q) {
    if (memcmp(pc[q].b, nb, sizeof nb) == 0) { /* piece covers the node */
      h->nodes[node].patch = pc[q].patch;
      h->nodes[node].level = l;
      return ORC_OK;
    }
  }
  i64 step = h->rpow[h->L - 1 - l];
  int best_a = -1;
  i64 best_s = 0, best_cost = 0, best_bal = 0;
  for (int a = 0; a < 3; ++a) {
    i64 area = 1;
    for (int k = 0; k < 3; ++k)
      if (k != a) area *= nb[3 + k] - nb[k];
    for (i64 s = nb[a] + step; s < nb[3 + a]; s += step) {
      i64 cost = 0;
      for (int q = 0; q < np; ++q)
        if (pc[q].b[a] < s && s < pc[q].b[3 + a]) cost++;
      i64 d = (s - nb[a]) - (nb[3 + a] - s);
      i64 bal = (d < 0 ? -d : d) * area;
      if (best_a < 0 || cost < best_cost || (cost == best_cost && bal < best_bal)) {
        best_a = a; best_s = s; best_cost = cost; best_bal = bal;
      }
    }
  }
  if (best_a < 0) return ORC_ERR_STATE; /* cannot happen for level-aligned pieces */
  i64 lb[6], rb[6];
  memcpy(lb, nb, sizeof lb);
  memcpy(rb, nb, sizeof rb);
  lb[3 + best_a] = best_s;
  rb[best_a] = best_s;
  int lab_p = h->nodes[node].patch, lab_l = h->nodes[node].level;
  int li = new_node(h, lb, lab_p, lab_l);
  int ri = new_node(h, rb, lab_p, lab_l);
  if (li < 0 || ri < 0) return ORC_ERR_OOM;
  h->nodes[node].axis = best_a;
  h->nodes[node].split = best_s;
  h->nodes[node].left = li;
  h->nodes[node].right = ri;
  opiece* lp = (opiece*)malloc((size_t)np * sizeof(opiece));
  opiece* rp = (opiece*)malloc((size_t)np * sizeof(opiece));
  if (!lp || !rp) { free(lp); free(rp); return ORC_ERR_OOM; }
  int nl = 0, nr = 0;
  for (int q = 0; q < np; ++q) {
    if (box_and(pc[q].b, lb, lp[nl].b)) lp[nl++].patch = pc[q].patch;
    if (box_and(pc[q].b, rb, rp[nr].b)) rp[nr++].patch = pc[q].patch;
  }
  int rc = refine(h, li, lp, nl, l);
  if (rc == ORC_OK) rc = refine(h, ri, rp, nr, l);
  free(lp);
  free(rp);
  return rc;
}

static int validate(orc_hier* h) {
  /* root = bounding box of the level-0 patches, which must tile it */
  int s0 = h->lev_start[0], e0 = h->lev_start[1];
  if (e0 == s0) return ORC_ERR_NOT_TILED;
  for (int k = 0; k < 3; ++k) { h->root[k] = INT64_MAX; h->root[3 + k] = INT64_MIN; }
  for (int c = s0; c < e0; ++c) {
    const i64* b = h->patches[h->by_level[c]].fbox;
    for (int k = 0; k < 3; ++k) {
      if (b[k] < h->root[k]) h->root[k] = b[k];
      if (b[3 + k] > h->root[3 + k]) h->root[3 + k] = b[3 + k];
    }
  }
  /* same-level patches must be disjoint */
  for (int l = 0; l < h->L; ++l) {
    for (int c = h->lev_start[l]; c < h->lev_start[l + 1]; ++c)
      for (int d = c + 1; d < h->lev_start[l + 1]; ++d) {
        i64 tmp[6];
        if (box_and(h->patches[h->by_level[c]].box, h->patches[h->by_level[d]].box, tmp))
          return ORC_ERR_OVERLAP;
      }
  }
  i64 sum = 0;
  for (int c = s0; c < e0; ++c) sum += vol6(h->patches[h->by_level[c]].fbox);
  if (sum != vol6(h->root)) return ORC_ERR_NOT_TILED;
  /* every patch must lie inside the root */
  for (int p = 0; p < h->P; ++p)
    for (int k = 0; k < 3; ++k)
      if (h->patches[p].fbox[k] < h->root[k] || h->patches[p].fbox[3 + k] > h->root[3 + k])
        return ORC_ERR_ARG;
  return ORC_OK;
}

int orc_build(orc_hier* h) {
  if (!h) return ORC_ERR_ARG;
  if (h->built) return ORC_ERR_STATE;
  int rc = validate(h);
  if (rc != ORC_OK) return rc;
  int root = new_node(h, h->root, -1, -1);
  if (root < 0) return ORC_ERR_OOM;
  /* level 0: the pieces are the level-0 patches themselves */
  int n0 = h->lev_start[1] - h->lev_start[0];
  opiece* pc = (opiece*)malloc((size_t)(n0 > 1 ? n0 : 1) * sizeof(opiece));
  if (!pc) return ORC_ERR_OOM;
  for (int c = 0; c < n0; ++c) {
    int p = h->by_level[h->lev_start[0] + c];
    memcpy(pc[c].b, h->patches[p].fbox, sizeof pc[c].b);
    pc[c].patch = p;
  }
  rc = refine(h, root, pc, n0, 0);
  free(pc);
  if (rc != ORC_OK) return rc;
  /* levels 1..L-1: re-split every current leaf on its (patch & leaf) pieces */
  for (int l = 1; l < h->L && rc == ORC_OK; ++l) {
    int nl = h->lev_start[l + 1] - h->lev_start[l];
    if (nl == 0) continue;
    int cur = h->nn;
    int* leaves = (int*)malloc((size_t)cur * sizeof(int));
    pc = (opiece*)malloc((size_t)nl * sizeof(opiece));
    if (!leaves || !pc) { free(leaves); free(pc); return ORC_ERR_OOM; }
    int m = 0;
    for (int i = 0; i < cur; ++i)
      if (h->nodes[i].axis < 0) leaves[m++] = i;
    for (int i = 0; i < m && rc == ORC_OK; ++i) {
      int np = 0;
      i64 lb[6];
      memcpy(lb, h->nodes[leaves[i]].box, sizeof lb);
      for (int c = 0; c < nl; ++c) {
        int p = h->by_level[h->lev_start[l] + c];
        if (box_and(h->patches[p].fbox, lb, pc[np].b)) pc[np++].patch = p;
      }
      rc = refine(h, leaves[i], pc, np, l);
    }
    free(leaves);
    free(pc);
  }
  if (rc != ORC_OK) return rc;
  /* canonical ids: pre-order over the final tree */
  h->pre2node = (int*)malloc((size_t)h->nn * sizeof(int));
  h->node2leaf = (int*)malloc((size_t)h->nn * sizeof(int));
  h->leaf2node = (int*)malloc((size_t)h->nn * sizeof(int));
  h->node2lod = (int*)malloc((size_t)h->nn * sizeof(int));
  int* stack = (int*)malloc((size_t)h->nn * sizeof(int));
  if (!h->pre2node || !h->node2leaf || !h->leaf2node || !h->node2lod || !stack) {
    free(stack);
    return ORC_ERR_OOM;
  }
  int sp = 0, k = 0;
  h->nleaves = 0;
  stack[sp++] = 0;
  while (sp) {
    int i = stack[--sp];
    h->pre2node[k++] = i;
    if (h->nodes[i].axis < 0) {
      h->node2leaf[i] = h->nleaves;
      h->leaf2node[h->nleaves++] = i;
    } else {
      h->node2leaf[i] = -1;
      stack[sp++] = h->nodes[i].right;
      stack[sp++] = h->nodes[i].left;
    }
  }
  free(stack);
  /* type-(a) nodes, numbered after the leaves in pre-order */
  h->nlod = 0;
  for (int q = 0; q < h->nn; ++q) {
    int i = h->pre2node[q];
    h->node2lod[i] = (h->nodes[i].axis >= 0 && h->nodes[i].patch >= 0) ? h->nleaves + h->nlod++ : -1;
  }
  h->built = 1;
  return ORC_OK;
}

int orc_num_nodes(const orc_hier* h) { return h && h->built ? h->nn : -1; }
int orc_num_leaves(const orc_hier* h) { return h && h->built ? h->nleaves : -1; }

/* Leaves in canonical order: box (finest coordinates) int64[6], patch id, level. */
int orc_get_leaves(const orc_hier* h, i64* box6, int* patch, int* level) {
  if (!h || !h->built) return ORC_ERR_STATE;
  for (int i = 0; i < h->nleaves; ++i) {
    const onode* n = &h->nodes[h->leaf2node[i]];
    for (int k = 0; k < 6; ++k) box6[6 * i + k] = n->box[k];
    patch[i] = n->patch;
    level[i] = n->level;
  }
  return h->nleaves;
}

/* Nodes in pre-order: axis (-1 leaf), split, pre-order ids of both children (-1), leaf id. */
int orc_get_nodes(const orc_hier* h, int* axis, i64* split, int* left, int* right, int* leaf) {
  if (!h || !h->built) return ORC_ERR_STATE;
  int* node2pre = (int*)malloc((size_t)h->nn * sizeof(int));
  if (!node2pre) return ORC_ERR_OOM;
  for (int k = 0; k < h->nn; ++k) node2pre[h->pre2node[k]] = k;
  for (int k = 0; k < h->nn; ++k) {
    const onode* n = &h->nodes[h->pre2node[k]];
    axis[k] = n->axis;
    split[k] = n->axis < 0 ? 0 : n->split;
    left[k] = n->axis < 0 ? -1 : node2pre[n->left];
    right[k] = n->axis < 0 ? -1 : node2pre[n->right];
    leaf[k] = h->node2leaf[h->pre2node[k]];
  }
  free(node2pre);
  return h->nn;
}

/* Labels in pre-order: patch and level of every node (for an inner node: the patch of
 * that level holding its whole box, or -1), and its pruned-leaf id (-1 if none). */
int orc_get_node_labels(const orc_hier* h, int* patch, int* level, int* lod) {
  if (!h || !h->built) return ORC_ERR_STATE;
  for (int k = 0; k < h->nn; ++k) {
    const onode* n = &h->nodes[h->pre2node[k]];
    patch[k] = n->patch;
    level[k] = n->level;
    lod[k] = h->node2lod[h->pre2node[k]];
  }
  return h->nlod;
}

/* ------------------------------------------------------------------------------------ */
/* field: V_l, S_l, F (Sec. 2 and Sec. 4)                                               */
/* ------------------------------------------------------------------------------------ */

static double hl(const orc_hier* h, int l, int a) { return h->h0[a] / (double)h->rpow[l]; }

/* level-l patch holding cell c, or -1 (same-level patches are disjoint) */
static int patch_at(const orc_hier* h, int l, i64 i, i64 j, i64 k, int hint) {
  if (hint >= 0 && h->patches[hint].level == l && box_contains_cell(h->patches[hint].box, i, j, k))
    return hint;
  for (int c = h->lev_start[l]; c < h->lev_start[l + 1]; ++c) {
    int p = h->by_level[c];
    if (box_contains_cell(h->patches[p].box, i, j, k)) return p;
  }
  return -1;
}

static double cell_value(const opatch* q, i64 i, i64 j, i64 k) {
  i64 ii = i - q->box[0], jj = j - q->box[1], kk = k - q->box[2];
  return (double)q->data[ii + q->nx * (jj + q->ny * kk)];
}

static double S_level(const orc_hier* h, int l, const double* x, int hint);

/* V_l(c): the value the level-l grid holds at cell c (clamped into the domain). */
static double V_level(const orc_hier* h, int l, i64 c0, i64 c1, i64 c2, int hint) {
  i64 c[3] = {c0, c1, c2};
  i64 sc = h->rpow[h->L - 1 - l];
  for (int a = 0; a < 3; ++a) {
    i64 lo = h->root[a] / sc, hi = h->root[3 + a] / sc; /* root is level-0 aligned */
    if (c[a] < lo) c[a] = lo;
    if (c[a] > hi - 1) c[a] = hi - 1;
  }
  int p = patch_at(h, l, c[0], c[1], c[2], hint);
  if (p >= 0) return cell_value(&h->patches[p], c[0], c[1], c[2]);
  for (int lc = l - 1; lc >= 0; --lc) {
    i64 f = h->rpow[l - lc];
    int pc = patch_at(h, lc, floordiv(c[0], f), floordiv(c[1], f), floordiv(c[2], f), -1);
    if (pc >= 0) {
      double xc[3];
      for (int a = 0; a < 3; ++a) xc[a] = h->dlo[a] + ((double)c[a] + 0.5) * hl(h, l, a);
      return S_level(h, lc, xc, pc);
    }
  }
  return NAN; /* unreachable once level 0 tiles the root */
}

/* S_l(x): trilinear interpolation of V_l at point x (cell-centred samples). */
static double S_level(const orc_hier* h, int l, const double* x, int hint) {
  i64 i0[3];
  double w[3];
  for (int a = 0; a < 3; ++a) {
    double xi = (x[a] - h->dlo[a]) / hl(h, l, a) - 0.5;
    double f = floor(xi);
    i0[a] = (i64)f;
    w[a] = xi - f;
  }
  double v[2][2][2];
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx)
        v[dz][dy][dx] = V_level(h, l, i0[0] + dx, i0[1] + dy, i0[2] + dz, hint);
  double c00 = v[0][0][0] * (1.0 - w[0]) + v[0][0][1] * w[0];
  double c10 = v[0][1][0] * (1.0 - w[0]) + v[0][1][1] * w[0];
  double c01 = v[1][0][0] * (1.0 - w[0]) + v[1][0][1] * w[0];
  double c11 = v[1][1][0] * (1.0 - w[0]) + v[1][1][1] * w[0];
  double c0 = c00 * (1.0 - w[1]) + c10 * w[1];
  double c1 = c01 * (1.0 - w[1]) + c11 * w[1];
  return c0 * (1.0 - w[2]) + c1 * w[2];
}

/* nearest: value of the level-l cell that contains x */
static double N_level(const orc_hier* h, int l, const double* x, int hint) {
  i64 c[3];
  for (int a = 0; a < 3; ++a) c[a] = (i64)floor((x[a] - h->dlo[a]) / hl(h, l, a));
  return V_level(h, l, c[0], c[1], c[2], hint);
}

static double sample_level(const orc_hier* h, int l, const double* x, int hint, int interp) {
  return interp ? S_level(h, l, x, hint) : N_level(h, l, x, hint);
}

/* finest-level cell holding x, clamped into the root */
static void finest_cell(const orc_hier* h, const double* x, i64* f) {
  for (int a = 0; a < 3; ++a) {
    double hf = h->h0[a] / (double)h->R;
    double q = floor((x[a] - h->dlo[a]) / hf);
    i64 c;
    if (q < (double)h->root[a]) c = h->root[a];
    else if (q > (double)(h->root[3 + a] - 1)) c = h->root[3 + a] - 1;
    else c = (i64)q;
    f[a] = c;
  }
}

/* finest level (and its patch) holding finest cell f, by scanning every patch */
static int scan_finest(const orc_hier* h, const i64* f, int* patch) {
  for (int l = h->L - 1; l >= 0; --l) {
    i64 sc = h->rpow[h->L - 1 - l];
    int p = patch_at(h, l, floordiv(f[0], sc), floordiv(f[1], sc), floordiv(f[2], sc), -1);
    if (p >= 0) { *patch = p; return l; }
  }
  *patch = -1;
  return -1;
}

/* smallest spacing of level l */
static double hmin_level(const orc_hier* h, int l) {
  double m = hl(h, l, 0);
  if (hl(h, l, 1) < m) m = hl(h, l, 1);
  if (hl(h, l, 2) < m) m = hl(h, l, 2);
  return m;
}

/* level-of-detail stop: an inner node lying in one patch of level l whose cells are at
 * most X wide (X <= 0: pruning off) */
static int lod_stop(const orc_hier* h, const onode* n, double X) {
  return X > 0.0 && n->axis >= 0 && n->patch >= 0 && hmin_level(h, n->level) <= X;
}

/* leaf (or pruned node) holding finest cell f, by descending the kD-tree (left iff
 * f_a < split) */
static int kd_leaf(const orc_hier* h, const i64* f, double X) {
  int i = 0;
  while (h->nodes[i].axis >= 0) {
    const onode* n = &h->nodes[i];
    if (lod_stop(h, n, X)) return i;
    i = (f[n->axis] < n->split) ? n->left : n->right;
  }
  return i;
}

/* F(x): sample at the finest level whose patch holds (the clamped) x; with pruning bound
 * X > 0, F_X(x): sample at the level of the kD node the pruned descent stops at */
static double F_field(const orc_hier* h, const double* x, int interp, int lookup, double X) {
  i64 f[3];
  finest_cell(h, x, f);
  int l, p;
  if (lookup == 1 && X <= 0.0) {
    l = scan_finest(h, f, &p);
  } else {
    const onode* n = &h->nodes[kd_leaf(h, f, X)];
    l = n->level;
    p = n->patch;
  }
  return sample_level(h, l, x, p, interp);
}

double orc_V(const orc_hier* h, int l, i64 i, i64 j, i64 k) {
  if (!h || !h->built || l < 0 || l >= h->L) return NAN;
  return V_level(h, l, i, j, k, -1);
}
double orc_S(const orc_hier* h, int l, const double* x) {
  if (!h || !h->built || l < 0 || l >= h->L) return NAN;
  return S_level(h, l, x, -1);
}
double orc_F(const orc_hier* h, const double* x, int interp, int lookup) {
  if (!h || !h->built) return NAN;
  return F_field(h, x, interp, lookup, 0.0);
}
/* finest covering level of x by scan; *patch receives the patch */
int orc_lookup_scan(const orc_hier* h, const double* x, int* patch) {
  if (!h || !h->built) return ORC_ERR_STATE;
  i64 f[3];
  finest_cell(h, x, f);
  return scan_finest(h, f, patch);
}
/* leaf id holding x by kD descent */
int orc_lookup_leaf(const orc_hier* h, const double* x) {
  if (!h || !h->built) return ORC_ERR_STATE;
  i64 f[3];
  finest_cell(h, x, f);
  return h->node2leaf[kd_leaf(h, f, 0.0)];
}

/* ------------------------------------------------------------------------------------ */
/* rays and kd-restart (Sec. 3.3)                                                       */
/* ------------------------------------------------------------------------------------ */

typedef struct {
  double o[3], d[3], inv[3];
  double t_in, t_out;
  int hit;
} oray;

static double plane_world(const orc_hier* h, int a, i64 s) {
  return h->dlo[a] + (double)s * (h->h0[a] / (double)h->R);
}

static void make_ray(const orc_hier* h, const orc_camera* cam, int i, int j, oray* ry) {
  double W = (double)cam->width, H = (double)cam->height;
  double aspect = W / H;
  double u = ((2.0 * ((double)i + 0.5)) / W - 1.0) * cam->tan_half_fov_y * aspect;
  double v = (1.0 - (2.0 * ((double)j + 0.5)) / H) * cam->tan_half_fov_y;
  for (int a = 0; a < 3; ++a) {
    ry->o[a] = cam->eye[a];
    ry->d[a] = (cam->fwd[a] + u * cam->right[a]) + v * cam->up[a];
    ry->inv[a] = ry->d[a] != 0.0 ? 1.0 / ry->d[a] : 0.0;
  }
  double t_in = 0.0, t_out = INFINITY;
  ry->hit = 1;
  for (int a = 0; a < 3; ++a) {
    double lo = plane_world(h, a, h->root[a]);
    double hi = plane_world(h, a, h->root[3 + a]);
    if (ry->d[a] != 0.0) {
      double ta = (lo - ry->o[a]) * ry->inv[a];
      double tb = (hi - ry->o[a]) * ry->inv[a];
      double tn = ta < tb ? ta : tb;
      double tf = ta < tb ? tb : ta;
      if (tn > t_in) t_in = tn;
      if (tf < t_out) t_out = tf;
    } else if (ry->o[a] < lo || ry->o[a] >= hi) {
      ry->hit = 0;
    }
  }
  if (!(t_in < t_out)) ry->hit = 0;
  ry->t_in = t_in;
  ry->t_out = t_out;
}

/* descend from the root for the segment starting at t0; returns the leaf node index (or
 * the pruned inner node, for pruning bound X > 0) and narrows *t1 (entering with the
 * ray's exit parameter) */
static int restart_descend(const orc_hier* h, const oray* ry, double t0, double* t1,
                           double X) {
  int i = 0;
  while (h->nodes[i].axis >= 0) {
    const onode* n = &h->nodes[i];
    if (lod_stop(h, n, X)) return i;
    int a = n->axis;
    double sw = plane_world(h, a, n->split);
    if (ry->d[a] == 0.0) {
      i = (ry->o[a] < sw) ? n->left : n->right;
      continue;
    }
    double ts = (sw - ry->o[a]) * ry->inv[a];
    int near_c = ry->d[a] > 0.0 ? n->left : n->right;
    int far_c = ry->d[a] > 0.0 ? n->right : n->left;
    if (ts >= *t1) {
      i = near_c;
    } else if (ts <= t0) {
      i = far_c;
    } else {
      i = near_c;
      *t1 = ts;
    }
  }
  return i;
}

/* pixel footprint per unit ray parameter times the pruning threshold (0: pruning off) */
static double lod_scale(const orc_camera* cam, double lod_pixels) {
  if (!(lod_pixels > 0.0)) return 0.0;
  return lod_pixels * ((2.0 * cam->tan_half_fov_y) / (double)cam->height);
}

/* Per-pixel traversal sequence: leaf ids and segment parameters.  Returns the number of
 * segments (0: the ray misses the root), or ORC_ERR_CAPACITY when `cap` is too small.
 * lod_pixels > 0 prunes the descent (pruned nodes report their ids after the leaves). */
int orc_trace_lod(const orc_hier* h, const orc_camera* cam, int i, int j, double lod_pixels,
                  int* leaf, double* t0s, double* t1s, int cap) {
  if (!h || !h->built) return ORC_ERR_STATE;
  oray ry;
  make_ray(h, cam, i, j, &ry);
  if (!ry.hit) return 0;
  const double ls = lod_scale(cam, lod_pixels);
  int n = 0;
  double t0 = ry.t_in;
  while (t0 < ry.t_out) {
    double t1 = ry.t_out;
    int nd = restart_descend(h, &ry, t0, &t1, ls > 0.0 ? ls * t0 : 0.0);
    if (n >= cap) return ORC_ERR_CAPACITY;
    leaf[n] = h->nodes[nd].axis < 0 ? h->node2leaf[nd] : h->node2lod[nd];
    t0s[n] = t0;
    t1s[n] = t1;
    n++;
    t0 = t1;
  }
  return n;
}

int orc_trace(const orc_hier* h, const orc_camera* cam, int i, int j, int* leaf,
              double* t0s, double* t1s, int cap) {
  return orc_trace_lod(h, cam, i, j, 0.0, leaf, t0s, t1s, cap);
}

/* ------------------------------------------------------------------------------------ */
/* shading and compositing                                                              */
/* ------------------------------------------------------------------------------------ */

static void tf_lookup(const float* tf, int n, double vmin, double vmax, double v, double* rgba) {
  double u = (v - vmin) / (vmax - vmin);
  if (u < 0.0) u = 0.0;
  if (u > 1.0) u = 1.0;
  u = u * (double)(n - 1);
  int i = (int)floor(u);
  if (i > n - 2) i = n - 2;
  double w = u - (double)i;
  for (int c = 0; c < 4; ++c)
    rgba[c] = (1.0 - w) * (double)tf[4 * i + c] + w * (double)tf[4 * (i + 1) + c];
}

static double clamp01(double x) { return x < 0.0 ? 0.0 : (x > 1.0 ? 1.0 : x); }

/* Transmittance from world point x to the light: the part of the segment x -> light inside
 * the root box, n = max(1, ceil(len / step)) midpoint samples of F (trilinear, finest
 * level), T = prod (1 - alpha_k); stops with T = 0 once T <= 1e-4. */
static double shadow_T(const orc_hier* h, const float* tf, int tfn, const orc_params* pr,
                       const double* x) {
  double D[3], s_out = 1.0;
  for (int a = 0; a < 3; ++a) {
    D[a] = pr->light[a] - x[a];
    if (D[a] != 0.0) {
      double bound = D[a] > 0.0 ? plane_world(h, a, h->root[3 + a]) : plane_world(h, a, h->root[a]);
      double sa = (bound - x[a]) / D[a];
      if (sa < s_out) s_out = sa;
    }
  }
  if (s_out < 0.0) s_out = 0.0;
  double dl = sqrt((D[0] * D[0] + D[1] * D[1]) + D[2] * D[2]);
  double len = s_out * dl;
  double nf = ceil(len / pr->light_step);
  i64 n = nf < 1.0 ? 1 : (i64)nf;
  double delta = len / (double)n;
  double T = 1.0;
  for (i64 k = 0; k < n; ++k) {
    double s = ((double)k + 0.5) / (double)n * s_out;
    double p[3];
    for (int a = 0; a < 3; ++a) p[a] = x[a] + s * D[a];
    double v = F_field(h, p, 1, 0, 0.0);
    double rgba[4];
    tf_lookup(tf, tfn, pr->vmin, pr->vmax, v, rgba);
    T *= exp(-pr->kappa * rgba[3] * delta);
    if (T <= 1e-4) return 0.0;
  }
  return T;
}

double orc_shadow_T(const orc_hier* h, const float* tf, int tfn, const orc_params* pr,
                    const double* x) {
  if (!h || !h->built || !tf || tfn < 2 || !pr || !x || !(pr->light_step > 0.0)) return NAN;
  return shadow_T(h, tf, tfn, pr, x);
}

typedef struct {
  double rgba[4];
  unsigned long long samples;
  int segments;
  int status;
} opixel;

static void render_pixel(const orc_hier* h, const orc_camera* cam, const float* tf, int tfn,
                         const orc_params* pr, int i, int j, opixel* out) {
  memset(out, 0, sizeof *out);
  oray ry;
  make_ray(h, cam, i, j, &ry);
  if (!ry.hit) return;
  double dn = sqrt((ry.d[0] * ry.d[0] + ry.d[1] * ry.d[1]) + ry.d[2] * ry.d[2]);
  double Lv[3] = {-ry.d[0] / dn, -ry.d[1] / dn, -ry.d[2] / dn};
  double C[3] = {0.0, 0.0, 0.0}, A = 0.0;
  const double ls = lod_scale(cam, pr->lod_pixels);
  double t0 = ry.t_in;
  int done = 0;
  while (t0 < ry.t_out && !done) {
    double t1 = ry.t_out;
    const double X = ls > 0.0 ? ls * t0 : 0.0;  /* pruning bound of this segment */
    int nd = restart_descend(h, &ry, t0, &t1, X);
    if (pr->max_segments > 0 && out->segments >= pr->max_segments) { out->status = 1; break; }
    out->segments++;
    const onode* leaf = &h->nodes[nd];
    int l = leaf->level, p = leaf->patch;
    double hmin = hl(h, l, 0);
    if (hl(h, l, 1) < hmin) hmin = hl(h, l, 1);
    if (hl(h, l, 2) < hmin) hmin = hl(h, l, 2);
    double step = pr->world_step > 0.0 ? pr->world_step : pr->step_factor * hmin;
    double len = (t1 - t0) * dn;
    double nf = ceil(len / step);
    i64 n = nf < 1.0 ? 1 : (i64)nf;
    double dt = (t1 - t0) / (double)n;
    double delta = len / (double)n;
    for (i64 k = 0; k < n; ++k) {
      double t = t0 + ((double)k + 0.5) * dt;
      double x[3];
      for (int a = 0; a < 3; ++a) x[a] = ry.o[a] + t * ry.d[a];
      double v = sample_level(h, l, x, p, pr->interp);
      double rgba[4];
      tf_lookup(tf, tfn, pr->vmin, pr->vmax, v, rgba);
      out->samples++;
      if (rgba[3] == 0.0) continue; /* contributes nothing */
      double alpha = 1.0 - exp(-pr->kappa * rgba[3] * delta);
      double rgb[3] = {rgba[0], rgba[1], rgba[2]};
      if (pr->shade) {
        double g[3];
        for (int a = 0; a < 3; ++a) {
          double xp[3] = {x[0], x[1], x[2]}, xm[3] = {x[0], x[1], x[2]};
          double ha = hl(h, l, a);
          xp[a] = x[a] + ha;
          xm[a] = x[a] - ha;
          g[a] = (F_field(h, xp, pr->interp, pr->lookup, X) -
                  F_field(h, xm, pr->interp, pr->lookup, X)) /
                 (2.0 * ha);
        }
        double gn = sqrt((g[0] * g[0] + g[1] * g[1]) + g[2] * g[2]);
        double gf = pr->gamma * (pr->vmax - pr->vmin) / hmin;
        double den = gn > gf ? gn : gf;
        double nv[3] = {0.0, 0.0, 0.0};
        if (den > 0.0)
          for (int a = 0; a < 3; ++a) nv[a] = g[a] / den;
        double ndl = fabs((nv[0] * Lv[0] + nv[1] * Lv[1]) + nv[2] * Lv[2]);
        double spec = pr->ks * pow(ndl, pr->shininess);
        for (int c = 0; c < 3; ++c) rgb[c] = clamp01(rgb[c] * (pr->ka + pr->kd * ndl) + spec);
      }
      if (pr->shadow) {
        double T = shadow_T(h, tf, tfn, pr, x);
        double I = pr->light_ambient + (1.0 - pr->light_ambient) * T;
        for (int c = 0; c < 3; ++c) rgb[c] *= I;
      }
      double wgt = (1.0 - A) * alpha;
      for (int c = 0; c < 3; ++c) C[c] += wgt * rgb[c];
      A += wgt;
      if (pr->ert_eps > 0.0 && A >= 1.0 - pr->ert_eps) { done = 1; break; }
    }
    t0 = t1;
  }
  out->rgba[0] = C[0];
  out->rgba[1] = C[1];
  out->rgba[2] = C[2];
  out->rgba[3] = A;
}

/* Render the listed pixels (px[k], py[k]) into out_rgba[4k..4k+3].  samples_out[k] (nullable)
 * receives the number of samples taken.  Returns the number of pixels that hit the
 * segment cap (0 when all completed), or a negative error. */
int orc_render_pixels(const orc_hier* h, const orc_camera* cam, const float* tf, int tfn,
                      const orc_params* pr, int npix, const int* px, const int* py,
                      double* out_rgba, unsigned long long* samples_out, int nthreads) {
  if (!h || !h->built) return ORC_ERR_STATE;
  if (!cam || !tf || tfn < 2 || !pr || npix < 0 || (npix && (!px || !py || !out_rgba)))
    return ORC_ERR_ARG;
  int capped = 0;
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 8) num_threads(nthreads) reduction(+ : capped)
#endif
  for (int k = 0; k < npix; ++k) {
    opixel o;
    render_pixel(h, cam, tf, tfn, pr, px[k], py[k], &o);
    for (int c = 0; c < 4; ++c) out_rgba[4 * k + c] = o.rgba[c];
    if (samples_out) samples_out[k] = o.samples;
    capped += o.status;
  }
  (void)nthreads;
  return capped;
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------------------ */
/* MLP 12-64-64-64-1 with ReLU hidden layers and a sigmoid output (learned proposal).   */
/* Weights W_k are [out][in] row-major, biases b_k [out].  x: [n][12].                    */
/* ------------------------------------------------------------------------------------ */

#define MLP_IN 12
#define MLP_H 64

static void mlp_one(const double* W1, const double* b1, const double* W2, const double* b2,
                    const double* W3, const double* b3, const double* W4, const double* b4,
                    const double* x, double* z1, double* a1, double* z2, double* a2,
                    double* z3, double* a3, double* z4, double* y) {
  for (int o = 0; o < MLP_H; ++o) {
    double s = b1[o];
    for (int i = 0; i < MLP_IN; ++i) s += W1[o * MLP_IN + i] * x[i];
    z1[o] = s;
    a1[o] = s > 0.0 ? s : 0.0;
  }
  for (int o = 0; o < MLP_H; ++o) {
    double s = b2[o];
    for (int i = 0; i < MLP_H; ++i) s += W2[o * MLP_H + i] * a1[i];
    z2[o] = s;
    a2[o] = s > 0.0 ? s : 0.0;
  }
  for (int o = 0; o < MLP_H; ++o) {
    double s = b3[o];
    for (int i = 0; i < MLP_H; ++i) s += W3[o * MLP_H + i] * a2[i];
    z3[o] = s;
    a3[o] = s > 0.0 ? s : 0.0;
  }
  double s = b4[0];
  for (int i = 0; i < MLP_H; ++i) s += W4[i] * a3[i];
  *z4 = s;
  *y = 1.0 / (1.0 + exp(-s));
}

/* Forward pass: y[n] = sigmoid(MLP(x)). */
void orc_mlp_forward(const double* W1, const double* b1, const double* W2, const double* b2,
                     const double* W3, const double* b3, const double* W4, const double* b4,
                     int n, const double* x, double* y) {
  for (int k = 0; k < n; ++k) {
    double z1[MLP_H], a1[MLP_H], z2[MLP_H], a2[MLP_H], z3[MLP_H], a3[MLP_H], z4;
    mlp_one(W1, b1, W2, b2, W3, b3, W4, b4, x + MLP_IN * k, z1, a1, z2, a2, z3, a3, &z4, y + k);
  }
}

/* Mean binary cross-entropy over n rows, loss = -mean(t log y + (1-t) log(1-y)), and its
 * gradient with respect to every weight and bias (same shapes as the parameters). */
double orc_mlp_loss_grad(const double* W1, const double* b1, const double* W2, const double* b2,
                         const double* W3, const double* b3, const double* W4, const double* b4,
                         int n, const double* x, const double* t,
                         double* gW1, double* gb1, double* gW2, double* gb2,
                         double* gW3, double* gb3, double* gW4, double* gb4) {
  memset(gW1, 0, sizeof(double) * MLP_H * MLP_IN);
  memset(gb1, 0, sizeof(double) * MLP_H);
  memset(gW2, 0, sizeof(double) * MLP_H * MLP_H);
  memset(gb2, 0, sizeof(double) * MLP_H);
  memset(gW3, 0, sizeof(double) * MLP_H * MLP_H);
  memset(gb3, 0, sizeof(double) * MLP_H);
  memset(gW4, 0, sizeof(double) * MLP_H);
  gb4[0] = 0.0;
  double loss = 0.0;
  for (int k = 0; k < n; ++k) {
    const double* xk = x + MLP_IN * k;
    double z1[MLP_H], a1[MLP_H], z2[MLP_H], a2[MLP_H], z3[MLP_H], a3[MLP_H], z4, y;
    mlp_one(W1, b1, W2, b2, W3, b3, W4, b4, xk, z1, a1, z2, a2, z3, a3, &z4, &y);
    /* BCE through the sigmoid, written on the logit for stability:
       l = softplus(z) - t z, dl/dz = sigmoid(z) - t */
    double sp = z4 > 0.0 ? z4 + log1p(exp(-z4)) : log1p(exp(z4));
    loss += sp - t[k] * z4;
    double dz4 = (y - t[k]) / (double)n;
    double d3[MLP_H], d2[MLP_H], d1[MLP_H];
    gb4[0] += dz4;
    for (int i = 0; i < MLP_H; ++i) {
      gW4[i] += dz4 * a3[i];
      d3[i] = z3[i] > 0.0 ? dz4 * W4[i] : 0.0;
    }
    for (int o = 0; o < MLP_H; ++o) {
      gb3[o] += d3[o];
      for (int i = 0; i < MLP_H; ++i) gW3[o * MLP_H + i] += d3[o] * a2[i];
    }
    for (int i = 0; i < MLP_H; ++i) {
      double s = 0.0;
      for (int o = 0; o < MLP_H; ++o) s += W3[o * MLP_H + i] * d3[o];
      d2[i] = z2[i] > 0.0 ? s : 0.0;
    }
    for (int o = 0; o < MLP_H; ++o) {
      gb2[o] += d2[o];
      for (int i = 0; i < MLP_H; ++i) gW2[o * MLP_H + i] += d2[o] * a1[i];
    }
    for (int i = 0; i < MLP_H; ++i) {
      double s = 0.0;
      for (int o = 0; o < MLP_H; ++o) s += W2[o * MLP_H + i] * d2[o];
      d1[i] = z1[i] > 0.0 ? s : 0.0;
    }
    for (int o = 0; o < MLP_H; ++o) {
      gb1[o] += d1[o];
      for (int i = 0; i < MLP_IN; ++i) gW1[o * MLP_IN + i] += d1[o] * xk[i];
    }
  }
  return loss / (double)n;
}
