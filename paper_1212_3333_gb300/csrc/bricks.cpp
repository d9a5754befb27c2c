// Bricks, halos and the packed atlas (Sec. 4 of Kaehler & Abel).
//
// One brick per patch (Sec. 4: fewer interfaces and less fragmentation than one brick per
// kD node), holding the patch cells plus a halo of H = c->halo cells (one, or two so that
// gradient neighbours up to one cell beyond a leaf face onto the same level also read the
// brick) so that trilinear interpolation anywhere inside the patch box reads only its own
// brick.  Brick index = cell - patch lo + H.  A halo cell c of a level-l
// patch holds the level-l value V_l(c): c is first clamped into the domain; if some
// level-l patch holds c, its stored value; otherwise the trilinear value, at the centre
// of c, of the finest coarser level whose patch holds that centre.  This is the
// cell-centred counterpart of the paper's replacement of dangling values by interpolated
// coarse values (Sec. 4).  Levels are filled coarse to fine, so a coarser brick is
// complete (halo included) when a finer halo reads it.
//
// The atlas (Sec. 4.1) packs the bricks into one 3D block with next-fit-decreasing-height:
// bricks sorted by decreasing z, y, x extent fill rows along x, rows along y, then layers
// along z; square bases of several widths are tried and the smallest volume is kept.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <unordered_map>

#include "ctx.h"

namespace amr {

namespace {

inline int64_t floor_div(int64_t a, int64_t b) {
  int64_t q = a / b;
  return (a % b != 0 && ((a < 0) != (b < 0))) ? q - 1 : q;
}

// patches of one level bucketed by 16^3-cell blocks of that level's index space
class LevelIndex {
 public:
  void add(int p, const int64_t* box) {
    for (int64_t bz = floor_div(box[2], kB); bz <= floor_div(box[5] - 1, kB); ++bz)
      for (int64_t by = floor_div(box[1], kB); by <= floor_div(box[4] - 1, kB); ++by)
        for (int64_t bx = floor_div(box[0], kB); bx <= floor_div(box[3] - 1, kB); ++bx)
          map_[key(bx, by, bz)].push_back(p);
  }
  int find(const std::vector<Patch>& ps, int64_t i, int64_t j, int64_t k) const {
    auto it = map_.find(key(floor_div(i, kB), floor_div(j, kB), floor_div(k, kB)));
    if (it == map_.end()) return -1;
    for (int p : it->second) {
      const int64_t* b = ps[p].box;
      if (b[0] <= i && i < b[3] && b[1] <= j && j < b[4] && b[2] <= k && k < b[5]) return p;
    }
    return -1;
  }

 private:
  static constexpr int64_t kB = 16;
  static uint64_t key(int64_t x, int64_t y, int64_t z) {
    const uint64_t o = (uint64_t)1 << 20;
    return (((uint64_t)(x + o)) << 42) ^ (((uint64_t)(y + o)) << 21) ^ (uint64_t)(z + o);
  }
  std::unordered_map<uint64_t, std::vector<int>> map_;
};

struct BrickView {
  const float* v;
  int64_t d[3];
  int64_t lo[3];
  float at(int64_t bi, int64_t bj, int64_t bk) const { return v[bi + d[0] * (bj + d[1] * bk)]; }
};

}  // namespace

amr_status build_bricks(amr_ctx* c) {
  const int L = c->L;
  const size_t P = c->patches.size();
  std::vector<LevelIndex> index(L);
  for (size_t p = 0; p < P; ++p) index[c->patches[p].level].add((int)p, c->patches[p].box);
  c->bricks.assign(P, {});
  std::vector<int> order(P);
  for (size_t p = 0; p < P; ++p) order[p] = (int)p;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return c->patches[a].level < c->patches[b].level; });
  auto view = [&](int p) {
    BrickView bv;
    bv.v = c->bricks[p].data();
    for (int k = 0; k < 3; ++k) {
      bv.d[k] = c->patches[p].n[k] + 2 * c->halo;
      bv.lo[k] = c->patches[p].box[k];
    }
    return bv;
  };
  // trilinear value of level lc at world point x from patch q's completed brick
  auto coarse_value = [&](int q, int lc, const double* x) {
    BrickView bv = view(q);
    double w[3];
    int64_t i0[3];
    for (int a = 0; a < 3; ++a) {
      double hl = c->h0[a] / (double)c->rpow[lc];
      double beta = (x[a] - c->dlo[a]) / hl - 0.5 - (double)bv.lo[a] + (double)c->halo;
      double f = std::floor(beta);
      int64_t i = (int64_t)f;
      double wa = beta - f;
      if (i < 0) { i = 0; wa = 0.0; }
      if (i > bv.d[a] - 2) { i = bv.d[a] - 2; wa = 1.0; }
      i0[a] = i;
      w[a] = wa;
    }
    double v[2][2][2];
    for (int dz = 0; dz < 2; ++dz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx)
          v[dz][dy][dx] = bv.at(i0[0] + dx, i0[1] + dy, i0[2] + dz);
    double c00 = v[0][0][0] * (1.0 - w[0]) + v[0][0][1] * w[0];
    double c10 = v[0][1][0] * (1.0 - w[0]) + v[0][1][1] * w[0];
    double c01 = v[1][0][0] * (1.0 - w[0]) + v[1][0][1] * w[0];
    double c11 = v[1][1][0] * (1.0 - w[0]) + v[1][1][1] * w[0];
    double c0 = c00 * (1.0 - w[1]) + c10 * w[1];
    double c1 = c01 * (1.0 - w[1]) + c11 * w[1];
    return c0 * (1.0 - w[2]) + c1 * w[2];
  };
  // levels in turn (a halo reads only coarser, completed bricks); patches of one level in
  // parallel
  bool uncovered = false;
  size_t first = 0;
  while (first < P) {
    size_t last = first;
    while (last < P && c->patches[order[last]].level == c->patches[order[first]].level) ++last;
#pragma omp parallel for schedule(dynamic, 4)
  for (long long oi = (long long)first; oi < (long long)last; ++oi) {
    const int p = order[(size_t)oi];
    const Patch& pt = c->patches[p];
    const int l = pt.level;
    const int64_t sc = c->rpow[L - 1 - l];
    const int64_t H = c->halo;
    const int64_t d0 = pt.n[0] + 2 * H, d1 = pt.n[1] + 2 * H, d2 = pt.n[2] + 2 * H;
    std::vector<float>& br = c->bricks[p];
    br.assign((size_t)(d0 * d1 * d2), 0.0f);
    int64_t rlo[3], rhi[3];
    for (int a = 0; a < 3; ++a) {
      rlo[a] = c->root[a] / sc;
      rhi[a] = c->root[3 + a] / sc;
    }
    // V_l at a cell outside the patch (halo): clamp, same-level patch, else coarse value
    auto halo_value = [&](int64_t bi, int64_t bj, int64_t bk, float* out) -> bool {
      int64_t cc[3] = {pt.box[0] + bi - H, pt.box[1] + bj - H, pt.box[2] + bk - H};
      for (int a = 0; a < 3; ++a) cc[a] = std::min(std::max(cc[a], rlo[a]), rhi[a] - 1);
      int q = index[l].find(c->patches, cc[0], cc[1], cc[2]);
      if (q >= 0) {
        const Patch& o = c->patches[q];
        *out = o.data[(size_t)((cc[0] - o.box[0]) +
                               o.n[0] * ((cc[1] - o.box[1]) + o.n[1] * (cc[2] - o.box[2])))];
        return true;
      }
      for (int lc = l - 1; lc >= 0; --lc) {
        int64_t f = c->rpow[l - lc];
        int qc = index[lc].find(c->patches, floor_div(cc[0], f), floor_div(cc[1], f),
                                floor_div(cc[2], f));
        if (qc >= 0) {
          double x[3];
          for (int a = 0; a < 3; ++a)
            x[a] = c->dlo[a] + ((double)cc[a] + 0.5) * (c->h0[a] / (double)c->rpow[l]);
          *out = (float)coarse_value(qc, lc, x);
          return true;
        }
      }
      return false;
    };
    for (int64_t bk = 0; bk < d2; ++bk)
      for (int64_t bj = 0; bj < d1; ++bj) {
        float* row = br.data() + (size_t)(d0 * (bj + d1 * bk));
        bool interior_row = bj >= H && bj < pt.n[1] + H && bk >= H && bk < pt.n[2] + H;
        if (interior_row) {
          std::memcpy(row + H, pt.data.data() + (size_t)(pt.n[0] * ((bj - H) + pt.n[1] * (bk - H))),
                      sizeof(float) * (size_t)pt.n[0]);
          for (int64_t e = 0; e < H; ++e)
            if (!halo_value(e, bj, bk, row + e) || !halo_value(d0 - 1 - e, bj, bk, row + d0 - 1 - e)) {
#pragma omp atomic write
              uncovered = true;
            }
        } else {
          for (int64_t bi = 0; bi < d0; ++bi)
            if (!halo_value(bi, bj, bk, row + bi)) {
#pragma omp atomic write
              uncovered = true;
            }
        }
      }
  }
    first = last;
  }
  if (uncovered) return fail(c, AMR_ERR_DEVICE, "halo cell not covered by any coarser level");
  // value range every sample of a leaf can reach: the brick cells under the trilinear
  // stencils of all points of the leaf box
  // (leaves first, then the pruned inner nodes of level-of-detail rendering)
  const Tree& t = c->tree;
  const size_t M = t.leaf_patch.size(), ML = t.lod_patch.size();
  c->leaf_vmin.assign(M + ML, 0.0f);
  c->leaf_vmax.assign(M + ML, 0.0f);
#pragma omp parallel for schedule(dynamic, 64)
  for (long long mi = 0; mi < (long long)(M + ML); ++mi) {
    const size_t m = (size_t)mi;
    const bool lod = m >= M;
    const int p = lod ? t.lod_patch[m - M] : t.leaf_patch[m];
    const int32_t* box = lod ? &t.lod_box[6 * (m - M)] : &t.leaf_box[6 * m];
    const Patch& pt = c->patches[p];
    const int64_t sc = c->rpow[L - 1 - pt.level];
    BrickView bv = view(p);
    int64_t lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
      // leaf extent in brick coordinates: beta = X - lo + H - 0.5 with X = finest / sc
      const double sh = (double)c->halo - 0.5;
      double bmin = (double)box[a] / (double)sc - (double)pt.box[a] + sh;
      double bmax = (double)box[3 + a] / (double)sc - (double)pt.box[a] + sh;
      lo[a] = std::max<int64_t>(0, (int64_t)std::floor(bmin));
      hi[a] = std::min<int64_t>(bv.d[a] - 1, (int64_t)std::floor(bmax) + 1);
    }
    float mn = INFINITY, mx = -INFINITY;
    for (int64_t k = lo[2]; k <= hi[2]; ++k)
      for (int64_t j = lo[1]; j <= hi[1]; ++j)
        for (int64_t i = lo[0]; i <= hi[0]; ++i) {
          float v = bv.at(i, j, k);
          mn = std::min(mn, v);
          mx = std::max(mx, v);
        }
    c->leaf_vmin[m] = mn;
    c->leaf_vmax[m] = mx;
  }
  return AMR_OK;
}

// Gradient bricks: per cell (V, V(c+x) - V(c-x), V(c+y) - V(c-y), V(c+z) - V(c-z)).  A one-cell
// shift commutes with trilinear interpolation, so interpolating these differences at beta
// gives exactly the central difference S(beta + e_a) - S(beta - e_a) of the trilinear
// field whenever both neighbours read this brick.  Outer-layer cells (no neighbour on one
// side) hold zero differences; the kernels use the gradient brick only away from them.
amr_status build_gradient_bricks(amr_ctx* c) {
  const size_t P = c->patches.size();
  c->gbricks.assign(P, {});
#pragma omp parallel for schedule(dynamic, 4)
  for (long long pi = 0; pi < (long long)P; ++pi) {
    const size_t p = (size_t)pi;
    const int64_t H = c->halo;
    const int64_t d0 = c->patches[p].n[0] + 2 * H, d1 = c->patches[p].n[1] + 2 * H,
                  d2 = c->patches[p].n[2] + 2 * H;
    const std::vector<float>& v = c->bricks[p];
    std::vector<float4>& g = c->gbricks[p];
    g.resize(v.size());
    auto at = [&](int64_t i, int64_t j, int64_t k) { return v[(size_t)(i + d0 * (j + d1 * k))]; };
    for (int64_t k = 0; k < d2; ++k)
      for (int64_t j = 0; j < d1; ++j)
        for (int64_t i = 0; i < d0; ++i) {
          float4 q;
          q.x = at(i, j, k);
          q.y = (i > 0 && i < d0 - 1) ? at(i + 1, j, k) - at(i - 1, j, k) : 0.0f;
          q.z = (j > 0 && j < d1 - 1) ? at(i, j + 1, k) - at(i, j - 1, k) : 0.0f;
          q.w = (k > 0 && k < d2 - 1) ? at(i, j, k + 1) - at(i, j, k - 1) : 0.0f;
          g[(size_t)(i + d0 * (j + d1 * k))] = q;
        }
  }
  return AMR_OK;
}

// Stencil-maximum bricks: per cell c the largest of the eight cells c + {0, 1}^3 - the
// cells of the trilinear stencil whose lower corner is c - and +infinity in the outer
// layer, which no stencil starts at.  A trilinear value never exceeds its corners'
// maximum, so a sample whose stencil maximum the transfer function maps to zero opacity
// is transparent; the kernels test that with one load instead of eight.
amr_status build_max_bricks(amr_ctx* c) {
  const size_t P = c->patches.size();
  c->mbricks.assign(P, {});
#pragma omp parallel for schedule(dynamic, 4)
  for (long long pi = 0; pi < (long long)P; ++pi) {
    const size_t p = (size_t)pi;
    const int64_t H = c->halo;
    const int64_t d0 = c->patches[p].n[0] + 2 * H, d1 = c->patches[p].n[1] + 2 * H,
                  d2 = c->patches[p].n[2] + 2 * H;
    const std::vector<float>& v = c->bricks[p];
    std::vector<float>& m = c->mbricks[p];
    m.assign(v.size(), INFINITY);
    auto at = [&](int64_t i, int64_t j, int64_t k) { return v[(size_t)(i + d0 * (j + d1 * k))]; };
    for (int64_t k = 0; k + 1 < d2; ++k)
      for (int64_t j = 0; j + 1 < d1; ++j)
        for (int64_t i = 0; i + 1 < d0; ++i) {
          float mx = at(i, j, k);
          for (int dz = 0; dz < 2; ++dz)
            for (int dy = 0; dy < 2; ++dy)
              for (int dx = 0; dx < 2; ++dx) mx = std::max(mx, at(i + dx, j + dy, k + dz));
          m[(size_t)(i + d0 * (j + d1 * k))] = mx;
        }
  }
  return AMR_OK;
}

// Next-fit decreasing height in 3D over square bases; returns the container height.
static int64_t nfdh(const std::vector<std::array<int64_t, 3>>& ext, const std::vector<int>& order,
                    int64_t W, std::vector<int64_t>& org) {
  int64_t x = 0, y = 0, z = 0, row_h = 0, layer_h = 0;
  org.assign(ext.size() * 3, 0);
  for (int p : order) {
    const auto& e = ext[p];
    if (x + e[0] > W) {  // next row
      x = 0;
      y += row_h;
      row_h = 0;
    }
    if (y + e[1] > W) {  // next layer
      x = 0;
      y = 0;
      row_h = 0;
      z += layer_h;
      layer_h = 0;
    }
    org[3 * p] = x;
    org[3 * p + 1] = y;
    org[3 * p + 2] = z;
    x += e[0];
    row_h = std::max(row_h, e[1]);
    layer_h = std::max(layer_h, e[2]);
  }
  return z + layer_h;
}

amr_status pack_atlas(amr_ctx* c) {
  const size_t P = c->patches.size();
  std::vector<std::array<int64_t, 3>> ext(P);
  int64_t mx = 0;
  for (size_t p = 0; p < P; ++p) {
    for (int a = 0; a < 3; ++a) ext[p][a] = c->patches[p].n[a] + 2 * c->halo;
    mx = std::max(mx, std::max(ext[p][0], ext[p][1]));
  }
  std::vector<int> order(P);
  for (size_t p = 0; p < P; ++p) order[p] = (int)p;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    if (ext[a][2] != ext[b][2]) return ext[a][2] > ext[b][2];
    if (ext[a][1] != ext[b][1]) return ext[a][1] > ext[b][1];
    return ext[a][0] > ext[b][0];
  });
  int64_t best_vol = -1, best_w = 0, best_h = 0;
  std::vector<int64_t> org, best_org;
  int64_t w0 = ((mx + 15) / 16) * 16;
  for (int64_t W = w0; W <= std::max<int64_t>(w0, 4096); W += 16) {
    int64_t H = nfdh(ext, order, W, org);
    int64_t vol = W * W * H;
    if (best_vol < 0 || vol < best_vol) {
      best_vol = vol;
      best_w = W;
      best_h = H;
      best_org = org;
    }
  }
  c->packing.dims[0] = best_w;
  c->packing.dims[1] = best_w;
  c->packing.dims[2] = best_h;
  c->packing.org = best_org;
  return AMR_OK;
}

}  // namespace amr
