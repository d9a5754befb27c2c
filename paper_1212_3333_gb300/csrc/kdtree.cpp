// kD-tree construction for SAMR hierarchies (Sec. 3.1 of Kaehler & Abel).
//
// The root is the bounding box of the level-0 patches.  Each node is split by the
// axis-aligned plane that crosses the fewest patch pieces and leaves at least one cell
// slab on each side; ties go to the plane whose two sides hold the most equal volume
// (then the smaller axis, then the smaller plane).  A node stops splitting once it lies in
// one piece or touches none.  Levels 1..L-1 are processed in turn: every current leaf is
// re-split on the intersections of the level-l patches with it, which are found by a
// top-down descent from the root visiting only nodes that overlap the patch.
//
// Plane choice is a sweep over the sorted piece faces on each axis: the crossing count is
// constant between consecutive faces, so each open interval contributes one candidate
// (its grid plane closest to the node centre) and each face one more.  All coordinates
// are integers of the finest level.
#include <algorithm>
#include <chrono>
#include <cstring>

#include "ctx.h"

namespace amr {

amr_status fail(amr_ctx* c, amr_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

namespace {

inline bool intersect(const int64_t* a, const int64_t* b, int64_t* out) {
  for (int k = 0; k < 3; ++k) {
    int64_t lo = std::max(a[k], b[k]);
    int64_t hi = std::min(a[3 + k], b[3 + k]);
    if (lo >= hi) return false;
    if (out) {
      out[k] = lo;
      out[3 + k] = hi;
    }
  }
  return true;
}

inline int64_t floor_div(int64_t a, int64_t b) {
  int64_t q = a / b;
  return (a % b != 0 && ((a < 0) != (b < 0))) ? q - 1 : q;
}

struct Piece {
  int64_t b[6];
  int patch;
};

struct BNode {
  int64_t box[6];
  int axis;  // -1 leaf
  int64_t split;
  int left, right;
  int patch, level;
};

struct Candidate {
  bool valid = false;
  int64_t cost = 0, bal = 0;
  int axis = 0;
  int64_t s = 0;
};

class Builder {
 public:
  explicit Builder(amr_ctx* c) : c_(c) {}

  amr_status run() {
    nodes_.reserve(1024);
    new_node(c_->root, -1, -1);
    std::vector<Piece> pcs;
    for (size_t p = 0; p < c_->patches.size(); ++p) {
      if (c_->patches[p].level != 0) continue;
      Piece q;
      std::memcpy(q.b, c_->patches[p].fbox, sizeof q.b);
      q.patch = (int)p;
      pcs.push_back(q);
    }
    refine(0, pcs, 0);
    for (int l = 1; l < c_->L; ++l) {
      std::vector<int> slot(nodes_.size(), -1);
      std::vector<std::vector<Piece>> lists;
      std::vector<int> owners;
      for (size_t p = 0; p < c_->patches.size(); ++p) {
        if (c_->patches[p].level != l) continue;
        collect(0, c_->patches[p].fbox, (int)p, slot, lists, owners);
      }
      for (size_t k = 0; k < owners.size(); ++k) refine(owners[k], lists[k], l);
    }
    return finish();
  }

 private:
  amr_ctx* c_;
  std::vector<BNode> nodes_;

  int new_node(const int64_t* box, int patch, int level) {
    BNode n;
    std::memcpy(n.box, box, sizeof n.box);
    n.axis = -1;
    n.split = 0;
    n.left = n.right = -1;
    n.patch = patch;
    n.level = level;
    nodes_.push_back(n);
    return (int)nodes_.size() - 1;
  }

  // leaves of the current tree overlapping patch box q receive the piece q & leaf
  void collect(int i, const int64_t* q, int patch, std::vector<int>& slot,
               std::vector<std::vector<Piece>>& lists, std::vector<int>& owners) {
    int64_t cut[6];
    if (!intersect(nodes_[i].box, q, cut)) return;
    if (nodes_[i].axis < 0) {
      if (slot[i] < 0) {
        slot[i] = (int)lists.size();
        lists.emplace_back();
        owners.push_back(i);
      }
      Piece pc;
      std::memcpy(pc.b, cut, sizeof pc.b);
      pc.patch = patch;
      lists[slot[i]].push_back(pc);
      return;
    }
    int a = nodes_[i].axis;
    int64_t s = nodes_[i].split;
    if (q[a] < s) collect(nodes_[i].left, q, patch, slot, lists, owners);
    if (q[3 + a] > s) collect(nodes_[i].right, q, patch, slot, lists, owners);
  }

  // every leaf overlapping box q belongs to patch p
  bool same_patch(int i, const int64_t* q, int p) const {
    if (!intersect(nodes_[i].box, q, nullptr)) return true;
    if (nodes_[i].axis < 0) return nodes_[i].patch == p;
    return same_patch(nodes_[i].left, q, p) && same_patch(nodes_[i].right, q, p);
  }
  // every leaf overlapping box q is of level l
  bool same_level(int i, const int64_t* q, int l) const {
    if (!intersect(nodes_[i].box, q, nullptr)) return true;
    if (nodes_[i].axis < 0) return nodes_[i].level == l;
    return same_level(nodes_[i].left, q, l) && same_level(nodes_[i].right, q, l);
  }

  static void offer(Candidate& best, int64_t cost, int64_t bal, int axis, int64_t s) {
    if (!best.valid || cost < best.cost || (cost == best.cost && bal < best.bal)) {
      best.valid = true;
      best.cost = cost;
      best.bal = bal;
      best.axis = axis;
      best.s = s;
    }
  }

  Candidate choose(const int64_t* box, const std::vector<Piece>& pcs, int64_t step) const {
    Candidate best;
    std::vector<int64_t> los(pcs.size()), his(pcs.size()), pos;
    for (int a = 0; a < 3; ++a) {
      const int64_t lo = box[a], hi = box[3 + a];
      int64_t area = 1;
      for (int k = 0; k < 3; ++k)
        if (k != a) area *= box[3 + k] - box[k];
      const int64_t c2 = lo + hi;  // twice the node centre
      for (size_t q = 0; q < pcs.size(); ++q) {
        los[q] = pcs[q].b[a];
        his[q] = pcs[q].b[3 + a];
      }
      std::sort(los.begin(), los.end());
      std::sort(his.begin(), his.end());
      pos.assign(los.begin(), los.end());
      pos.insert(pos.end(), his.begin(), his.end());
      pos.push_back(lo);
      pos.push_back(hi);
      std::sort(pos.begin(), pos.end());
      pos.erase(std::unique(pos.begin(), pos.end()), pos.end());
      auto count_le = [](const std::vector<int64_t>& v, int64_t x) {
        return (int64_t)(std::upper_bound(v.begin(), v.end(), x) - v.begin());
      };
      auto count_lt = [](const std::vector<int64_t>& v, int64_t x) {
        return (int64_t)(std::lower_bound(v.begin(), v.end(), x) - v.begin());
      };
      for (size_t i = 0; i < pos.size(); ++i) {
        const int64_t x = pos[i];
        if (i > 0) {
          // open interval (pos[i-1], x): pieces spanning it all started at or before its
          // left end and had not ended there
          const int64_t xa = pos[i - 1];
          const int64_t first = xa + step, last = x - step;
          if (first <= last) {
            int64_t cost = count_le(los, xa) - count_le(his, xa);
            int64_t g = lo + floor_div(c2 - 2 * lo, 2 * step) * step;  // largest grid g, 2g <= c2
            int64_t g1 = std::min(std::max(g, first), last);
            int64_t g2 = std::min(std::max(g + step, first), last);
            int64_t b1 = std::abs(2 * g1 - c2), b2 = std::abs(2 * g2 - c2);
            int64_t gs = (b2 < b1 || (b2 == b1 && g2 < g1)) ? g2 : g1;
            offer(best, cost, std::abs(2 * gs - c2) * area, a, gs);
          }
        }
        if (lo < x && x < hi) {
          int64_t cost = count_lt(los, x) - count_le(his, x);
          offer(best, cost, std::abs(2 * x - c2) * area, a, x);
        }
      }
    }
    return best;
  }

  void refine(int i, std::vector<Piece>& pcs, int l) {
    if (pcs.empty()) return;
    for (const Piece& q : pcs) {
      if (std::memcmp(q.b, nodes_[i].box, sizeof q.b) == 0) {
        nodes_[i].patch = q.patch;
        nodes_[i].level = l;
        return;
      }
    }
    int64_t box[6];
    std::memcpy(box, nodes_[i].box, sizeof box);
    Candidate cd = choose(box, pcs, c_->rpow[c_->L - 1 - l]);
    // a node that is not covered by one piece always has a piece face strictly inside
    int64_t lb[6], rb[6];
    std::memcpy(lb, box, sizeof lb);
    std::memcpy(rb, box, sizeof rb);
    lb[3 + cd.axis] = cd.s;
    rb[cd.axis] = cd.s;
    int lp = nodes_[i].patch, ll = nodes_[i].level;
    int li = new_node(lb, lp, ll);
    int ri = new_node(rb, lp, ll);
    nodes_[i].axis = cd.axis;
    nodes_[i].split = cd.s;
    nodes_[i].left = li;
    nodes_[i].right = ri;
    std::vector<Piece> left, right;
    for (const Piece& q : pcs) {
      Piece t;
      t.patch = q.patch;
      if (intersect(q.b, lb, t.b)) left.push_back(t);
      if (intersect(q.b, rb, t.b)) right.push_back(t);
    }
    pcs.clear();
    pcs.shrink_to_fit();
    refine(li, left, l);
    refine(ri, right, l);
  }

  amr_status finish() {
    Tree& t = c_->tree;
    const size_t n = nodes_.size();
    t.axis.assign(n, -1);
    t.split.assign(n, 0);
    t.left.assign(n, -1);
    t.right.assign(n, -1);
    t.leaf.assign(n, -1);
    t.leaf_box.clear();
    t.leaf_patch.clear();
    t.leaf_level.clear();
    t.max_depth = 0;
    std::vector<int> pre(n, -1);
    // pre-order ids
    std::vector<std::pair<int, int>> stack;
    stack.push_back({0, 0});
    int next = 0;
    std::vector<int> order;
    order.reserve(n);
    std::vector<int> depth(n, 0);
    while (!stack.empty()) {
      auto [i, d] = stack.back();
      stack.pop_back();
      pre[i] = next++;
      order.push_back(i);
      depth[i] = d;
      t.max_depth = std::max(t.max_depth, d);
      if (nodes_[i].axis >= 0) {
        stack.push_back({nodes_[i].right, d + 1});
        stack.push_back({nodes_[i].left, d + 1});
      }
    }
    for (size_t k = 0; k < n; ++k) {
      const BNode& b = nodes_[order[k]];
      if (b.axis < 0) {
        if (b.patch < 0) return fail(c_, AMR_ERR_DEVICE, "kD build left an unlabelled leaf");
        t.leaf[k] = (int32_t)t.leaf_patch.size();
        for (int q = 0; q < 6; ++q) t.leaf_box.push_back((int32_t)b.box[q]);
        t.leaf_patch.push_back(b.patch);
        t.leaf_level.push_back(b.level);
      } else {
        t.axis[k] = b.axis;
        t.split[k] = (int32_t)b.split;
        t.left[k] = pre[b.left];
        t.right[k] = pre[b.right];
      }
    }
    // face bits: the slab of one level cell beyond a leaf face lies inside the leaf's patch
    // and overlaps only leaves of that patch (one-cell halo), or overlaps only leaves of the
    // leaf's level (two-cell halo), so gradient neighbours there read the leaf's own brick
    t.leaf_faces.assign(t.leaf_patch.size(), 0);
    t.face_node.assign(12 * t.leaf_patch.size(), 0);
    std::vector<int> node2pre(n);
    for (size_t k = 0; k < n; ++k) node2pre[order[k]] = (int)k;
#pragma omp parallel for schedule(dynamic, 256)
    for (long long kk = 0; kk < (long long)n; ++kk) {
      const size_t k = (size_t)kk;
      const BNode& b = nodes_[order[k]];
      if (b.axis >= 0) continue;
      const Patch& pt = c_->patches[b.patch];
      const int64_t sc = c_->rpow[c_->L - 1 - b.level];
      uint8_t f = 0;
      for (int a = 0; a < 3; ++a)
        for (int side = 0; side < 2; ++side) {
          int64_t q[6];
          std::memcpy(q, b.box, sizeof q);
          if (side == 0) {
            q[3 + a] = b.box[a];
            q[a] = b.box[a] - sc;
          } else {
            q[a] = b.box[3 + a];
            q[3 + a] = b.box[3 + a] + sc;
          }
          // deepest node holding the leaf and the slab (clipped to the root: points beyond
          // it descend like their clamped positions); a neighbour lookup may also land in
          // the leaf itself, near its boundary
          // (second: the slab alone, for a neighbour known to lie beyond the face)
          for (int only_slab = 0; only_slab < 2; ++only_slab) {
            int64_t qc[6];
            for (int r = 0; r < 3; ++r) {
              const int64_t lo = only_slab ? q[r] : std::min(q[r], b.box[r]);
              const int64_t hi = only_slab ? q[3 + r] : std::max(q[3 + r], b.box[3 + r]);
              qc[r] = std::max(lo, c_->root[r]);
              qc[3 + r] = std::min(hi, c_->root[3 + r]);
            }
            int i = 0;
            if (qc[a] < qc[3 + a]) {
              while (nodes_[i].axis >= 0) {
                const int ax = nodes_[i].axis;
                const int64_t sp = nodes_[i].split;
                if (qc[3 + ax] <= sp) i = nodes_[i].left;
                else if (qc[ax] >= sp) i = nodes_[i].right;
                else break;
              }
            }
            t.face_node[12 * (size_t)t.leaf[k] + 6 * only_slab + 2 * a + side] = node2pre[i];
          }
          if (c_->halo >= 2) {
            // two-cell halo: the slab may lie in any patch of the leaf's level (the brick's
            // halo holds V_l there, and the stencils of points up to one cell beyond the
            // face reach two cells beyond it); it must lie inside the root
            if ((side == 0 && q[a] < c_->root[a]) || (side == 1 && q[3 + a] > c_->root[3 + a]))
              continue;
            if (same_level(0, q, b.level)) f |= (uint8_t)(1u << (2 * a + side));
            continue;
          }
          if ((side == 0 && q[a] < pt.fbox[a]) || (side == 1 && q[3 + a] > pt.fbox[3 + a]))
            continue;
          if (same_patch(0, q, b.patch)) f |= (uint8_t)(1u << (2 * a + side));
        }
      t.leaf_faces[(size_t)t.leaf[k]] = f;
    }
    // inner nodes lying in one patch (labelled when they were still leaves) can stand in
    // for their subtree at that patch's level: ids after the leaves, in pre-order
    t.node_lod.assign(n, -1);
    t.lod_box.clear();
    t.lod_patch.clear();
    t.lod_level.clear();
    t.lod_levels = 0;
    const int32_t M = (int32_t)t.leaf_patch.size();
    for (size_t k = 0; k < n; ++k) {
      const BNode& b = nodes_[order[k]];
      if (b.axis < 0 || b.patch < 0) continue;
      t.node_lod[k] = M + (int32_t)t.lod_patch.size();
      for (int q = 0; q < 6; ++q) t.lod_box.push_back((int32_t)b.box[q]);
      t.lod_patch.push_back(b.patch);
      t.lod_level.push_back(b.level);
      t.lod_levels = std::max(t.lod_levels, b.level + 1);
    }
    if (t.max_depth >= kMaxDepth)
      return fail(c_, AMR_ERR_CAPACITY, "kD-tree deeper than the device descent bound");
    return AMR_OK;
  }
};

}  // namespace

amr_status validate_hierarchy(amr_ctx* c) {
  const int64_t big = (int64_t)1 << 62;
  int64_t root[6] = {big, big, big, -big, -big, -big};
  bool any0 = false;
  for (const Patch& p : c->patches) {
    if (p.level != 0) continue;
    any0 = true;
    for (int k = 0; k < 3; ++k) {
      root[k] = std::min(root[k], p.fbox[k]);
      root[3 + k] = std::max(root[3 + k], p.fbox[3 + k]);
    }
  }
  if (!any0) return fail(c, AMR_ERR_NOT_TILED, "no level-0 patch");
  // same-level disjointness: sweep along x within each level
  for (int l = 0; l < c->L; ++l) {
    std::vector<int> ids;
    for (size_t p = 0; p < c->patches.size(); ++p)
      if (c->patches[p].level == l) ids.push_back((int)p);
    std::sort(ids.begin(), ids.end(),
              [&](int a, int b) { return c->patches[a].box[0] < c->patches[b].box[0]; });
    for (size_t i = 0; i < ids.size(); ++i) {
      const int64_t* a = c->patches[ids[i]].box;
      for (size_t j = i + 1; j < ids.size() && c->patches[ids[j]].box[0] < a[3]; ++j) {
        if (intersect(a, c->patches[ids[j]].box, nullptr))
          return fail(c, AMR_ERR_OVERLAP,
                      "patches " + std::to_string(ids[i]) + " and " + std::to_string(ids[j]) +
                          " of level " + std::to_string(l) + " overlap");
      }
    }
  }
  int64_t vol = 0;
  for (const Patch& p : c->patches)
    if (p.level == 0)
      vol += (p.fbox[3] - p.fbox[0]) * (p.fbox[4] - p.fbox[1]) * (p.fbox[5] - p.fbox[2]);
  if (vol != (root[3] - root[0]) * (root[4] - root[1]) * (root[5] - root[2]))
    return fail(c, AMR_ERR_NOT_TILED, "level 0 does not tile its bounding box");
  for (size_t p = 0; p < c->patches.size(); ++p)
    for (int k = 0; k < 3; ++k)
      if (c->patches[p].fbox[k] < root[k] || c->patches[p].fbox[3 + k] > root[3 + k])
        return fail(c, AMR_ERR_ARG, "patch " + std::to_string(p) + " extends outside the root");
  for (int k = 0; k < 6; ++k) {
    if (root[k] > INT32_MAX || root[k] < INT32_MIN)
      return fail(c, AMR_ERR_CAPACITY, "finest index space exceeds int32");
    c->root[k] = root[k];
  }
  return AMR_OK;
}

amr_status build_tree(amr_ctx* c) {
  Builder b(c);
  return b.run();
}

}  // namespace amr
