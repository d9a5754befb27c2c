// Upload of the tree, leaves, patch table and bricks to the device, in one of the four
// brick storage strategies (Sec. 4.1 packed pool, Sec. 4.2 handle table, rebuilt for CUDA).
#include <algorithm>
#include <cstring>
#include <deque>

#include "ctx.h"
#include "storage16.h"

namespace amr {

namespace {

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return fail(c, e_ == cudaErrorMemoryAllocation ? AMR_ERR_OOM : AMR_ERR_CUDA,    \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                \
  } while (0)

// breadth-first re-layout: children of a node are adjacent, the top levels contiguous;
// lod receives each slot's pruned-leaf entry (id << 5 | level) or -1, box each slot's box
// (lo, hi as two int4, finest cells) starting from the root box with the highest label
// level of a type-(a) node above the slot in lo.w, leaf_anc that level per leaf
std::vector<DNode> layout_nodes(const Tree& t, const int64_t* root, std::vector<int32_t>& lod,
                                std::vector<int32_t>& slot_of, std::vector<int4>& box,
                                std::vector<int32_t>& leaf_anc) {
  const size_t n = t.axis.size();
  std::vector<DNode> out(n);
  lod.assign(n, -1);
  slot_of.assign(n, 0);
  box.assign(2 * std::max<size_t>(n, 1), make_int4(0, 0, 0, 0));
  leaf_anc.assign(t.leaf_patch.size(), -1);
  struct Item {
    int pre, slot;
    int32_t b[6];
    int32_t anc;  // highest label level of a type-(a) node above this one, -1: none
  };
  std::deque<Item> q;
  Item r{0, 0, {}, -1};
  for (int k = 0; k < 6; ++k) r.b[k] = (int32_t)root[k];
  q.push_back(r);
  int next = 1;
  while (!q.empty()) {
    const Item it = q.front();
    q.pop_front();
    const int pre = it.pre, slot = it.slot;
    slot_of[pre] = slot;
    box[2 * (size_t)slot] = make_int4(it.b[0], it.b[1], it.b[2], it.anc);
    box[2 * (size_t)slot + 1] = make_int4(it.b[3], it.b[4], it.b[5], 0);
    const int32_t lq = t.node_lod.empty() ? -1 : t.node_lod[pre];
    const int32_t lvl = lq >= 0 ? t.lod_level[(size_t)lq - t.leaf_patch.size()] : -1;
    if (lq >= 0) lod[slot] = (lq << 5) | lvl;
    DNode d;
    if (t.axis[pre] < 0) {
      d.meta = ((uint32_t)kLeafAxis << 30) | ((uint32_t)t.leaf[pre] & kIndexMask);
      d.split = 0;
      leaf_anc[(size_t)t.leaf[pre]] = it.anc;
    } else {
      int first = next;
      next += 2;
      const int ax = t.axis[pre];
      d.meta = ((uint32_t)ax << 30) | ((uint32_t)first & kIndexMask);
      d.split = t.split[pre];
      const int32_t anc = std::max(it.anc, lvl);
      Item lc{t.left[pre], first, {}, anc}, rc{t.right[pre], first + 1, {}, anc};
      std::memcpy(lc.b, it.b, sizeof lc.b);
      std::memcpy(rc.b, it.b, sizeof rc.b);
      lc.b[3 + ax] = t.split[pre];
      rc.b[ax] = t.split[pre];
      q.push_back(lc);
      q.push_back(rc);
    }
    out[slot] = d;
  }
  return out;
}

// Macro grid over the root for point location: cells of G finest cells per axis (G = the
// finest cells of one level-0 cell, doubled until the grid has at most 2^21 cells), each
// holding the slot of the deepest node whose box contains the whole cell.  A point lies
// in its cell, so a descent from that node reaches the same leaf as one from the root.
std::vector<uint32_t> macro_grid(const std::vector<DNode>& nodes, const int64_t* root, int64_t R,
                                 int32_t* cell, int32_t* dims) {
  int64_t G = std::max<int64_t>(R, 1), ext[3], n[3];
  for (int a = 0; a < 3; ++a) ext[a] = root[3 + a] - root[a];
  for (;;) {
    for (int a = 0; a < 3; ++a) n[a] = (ext[a] + G - 1) / G;
    if (n[0] * n[1] * n[2] <= ((int64_t)1 << 21)) break;
    G *= 2;
  }
  *cell = (int32_t)G;
  for (int a = 0; a < 3; ++a) dims[a] = (int32_t)n[a];
  std::vector<uint32_t> out((size_t)(n[0] * n[1] * n[2]), 0u);
#pragma omp parallel for schedule(static)
  for (long long gi = 0; gi < (long long)out.size(); ++gi) {
    const int64_t g[3] = {gi % n[0], (gi / n[0]) % n[1], gi / (n[0] * n[1])};
    int64_t lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
      lo[a] = root[a] + g[a] * G;
      hi[a] = std::min(root[a] + (g[a] + 1) * G, root[3 + a]);
    }
    uint32_t i = 0;
    for (int depth = 0; depth < kMaxDepth; ++depth) {
      const DNode& nd = nodes[i];
      const uint32_t ax = nd.meta >> 30;
      if (ax == (uint32_t)kLeafAxis) break;
      const uint32_t c0 = nd.meta & kIndexMask;
      if (hi[ax] <= nd.split) i = c0;
      else if (lo[ax] >= nd.split) i = c0 + 1;
      else break;
    }
    out[(size_t)gi] = i;
  }
  return out;
}

// Bricks of element type T (float values, or float4 value + central differences) in the
// layout of the context's storage strategy; fills base (or gbase) of every patch record.
template <typename T>
amr_status upload_bricks(amr_ctx* c, const std::vector<std::vector<T>>& bricks,
                         std::vector<DPatch>& pt, bool gradient, cudaStream_t stream) {
  DeviceState& d = c->dev;
  const size_t P = c->patches.size();
  const int storage = c->storage;
  void*& pool = gradient ? d.gpool : d.pool;
  size_t& pool_bytes = gradient ? d.gpool_bytes : d.pool_bytes;
  auto set_base = [&](size_t p, long long v) { (gradient ? pt[p].gbase : pt[p].base) = v; };
  const cudaChannelFormatDesc ch = cudaCreateChannelDesc<T>();
  cudaTextureDesc td;
  std::memset(&td, 0, sizeof td);
  td.addressMode[0] = td.addressMode[1] = td.addressMode[2] = cudaAddressModeClamp;
  td.filterMode = cudaFilterModePoint;
  td.readMode = cudaReadModeElementType;
  td.normalizedCoords = 0;
  if (storage == AMR_STORE_PTR || storage == AMR_STORE_TEXOBJ) {
    // the kernels address a per-patch brick with 32-bit element offsets
    for (size_t p = 0; p < P; ++p)
      if (bricks[p].size() >= ((size_t)1 << 31))
        return fail(c, AMR_ERR_CAPACITY, "a brick holds 2^31 cells or more");
  }
  if (storage == AMR_STORE_PTR) {
    // one pool, each brick 128-byte aligned; the table holds the device addresses
    std::vector<size_t> off(P);
    size_t elems = 0;
    const size_t align = 128 / sizeof(T);
    for (size_t p = 0; p < P; ++p) {
      off[p] = elems;
      elems += (bricks[p].size() + align - 1) / align * align;
    }
    pool_bytes = elems * sizeof(T);
    CK(cudaMalloc(&pool, pool_bytes));
    for (size_t p = 0; p < P; ++p) {
      T* dst = (T*)pool + off[p];
      CK(cudaMemcpyAsync(dst, bricks[p].data(), bricks[p].size() * sizeof(T),
                         cudaMemcpyHostToDevice, stream));
      set_base(p, (long long)(uintptr_t)dst);
      pt[p].sy = pt[p].dim[0];
      pt[p].sz = pt[p].dim[0] * pt[p].dim[1];
    }
  } else if (storage == AMR_STORE_TEXOBJ) {
    std::vector<void*>& arrays = gradient ? d.garrays : d.arrays;
    std::vector<cudaTextureObject_t>& tex = gradient ? d.gtexobjs : d.texobjs;
    arrays.assign(P, nullptr);
    tex.assign(P, 0);
    pool_bytes = 0;
    for (size_t p = 0; p < P; ++p) {
      cudaExtent ext = make_cudaExtent(pt[p].dim[0], pt[p].dim[1], pt[p].dim[2]);
      cudaArray_t arr = nullptr;
      CK(cudaMalloc3DArray(&arr, &ch, ext));
      arrays[p] = arr;
      cudaMemcpy3DParms cp;
      std::memset(&cp, 0, sizeof cp);
      cp.srcPtr = make_cudaPitchedPtr((void*)bricks[p].data(), pt[p].dim[0] * sizeof(T),
                                      pt[p].dim[0], pt[p].dim[1]);
      cp.dstArray = arr;
      cp.extent = ext;
      cp.kind = cudaMemcpyHostToDevice;
      CK(cudaMemcpy3DAsync(&cp, stream));
      cudaResourceDesc rd;
      std::memset(&rd, 0, sizeof rd);
      rd.resType = cudaResourceTypeArray;
      rd.res.array.array = arr;
      cudaTextureObject_t t = 0;
      CK(cudaCreateTextureObject(&t, &rd, &td, nullptr));
      tex[p] = t;
      set_base(p, (long long)t);
      pool_bytes += bricks[p].size() * sizeof(T);
    }
    CK(cudaStreamSynchronize(stream));
  } else {
    // packed atlas (NFDH), linear memory or one 3D array
    const int64_t AX = c->packing.dims[0], AY = c->packing.dims[1], AZ = c->packing.dims[2];
    const size_t total = (size_t)(AX * AY * AZ);
    std::vector<T> img(total);
    std::memset((void*)img.data(), 0, total * sizeof(T));
    for (size_t p = 0; p < P; ++p) {
      const int64_t* o = &c->packing.org[3 * p];
      const int64_t d0 = pt[p].dim[0], d1 = pt[p].dim[1], d2 = pt[p].dim[2];
      for (int64_t k = 0; k < d2; ++k)
        for (int64_t j = 0; j < d1; ++j)
          std::memcpy((void*)&img[(size_t)(o[0] + AX * ((o[1] + j) + AY * (o[2] + k)))],
                      &bricks[p][(size_t)(d0 * (j + d1 * k))], sizeof(T) * (size_t)d0);
      for (int a = 0; a < 3; ++a) pt[p].org[a] = (int32_t)o[a];
      set_base(p, (long long)(o[0] + AX * (o[1] + AY * o[2])));
      pt[p].sy = (int32_t)AX;
      pt[p].sz = (int32_t)(AX * AY);
    }
    pool_bytes = total * sizeof(T);
    if (storage == AMR_STORE_ATLAS_LINEAR) {
      CK(cudaMalloc(&pool, pool_bytes));
      CK(cudaMemcpyAsync(pool, img.data(), pool_bytes, cudaMemcpyHostToDevice, stream));
      CK(cudaStreamSynchronize(stream));
    } else {
      cudaDeviceProp prop;
      CK(cudaGetDeviceProperties(&prop, d.device));
      if (AX > prop.maxTexture3D[0] || AY > prop.maxTexture3D[1] || AZ > prop.maxTexture3D[2])
        return fail(c, AMR_ERR_CAPACITY, "atlas exceeds the 3D texture extent limit");
      cudaExtent ext = make_cudaExtent(AX, AY, AZ);
      cudaArray_t arr = nullptr;
      CK(cudaMalloc3DArray(&arr, &ch, ext));
      (gradient ? d.gatlas_array : d.atlas_array) = arr;
      cudaMemcpy3DParms cp;
      std::memset(&cp, 0, sizeof cp);
      cp.srcPtr = make_cudaPitchedPtr(img.data(), AX * sizeof(T), AX, AY);
      cp.dstArray = arr;
      cp.extent = ext;
      cp.kind = cudaMemcpyHostToDevice;
      CK(cudaMemcpy3DAsync(&cp, stream));
      cudaResourceDesc rd;
      std::memset(&rd, 0, sizeof rd);
      rd.resType = cudaResourceTypeArray;
      rd.res.array.array = arr;
      CK(cudaCreateTextureObject(gradient ? &d.gatlas_tex : &d.atlas_tex, &rd, &td, nullptr));
      CK(cudaStreamSynchronize(stream));
    }
  }
  return AMR_OK;
}

// Stencil-maximum bricks of the pointer storage: a second pool with the value pool's
// offsets (the same brick sizes and alignment), so a brick's maximum brick lies at a fixed
// byte distance (mpool - pool) from it.
template <typename T>
amr_status upload_max_pool(amr_ctx* c, const std::vector<std::vector<T>>& mb, cudaStream_t stream) {
  DeviceState& d = c->dev;
  const size_t P = mb.size();
  const size_t align = 128 / sizeof(T);
  std::vector<size_t> off(P);
  size_t elems = 0;
  for (size_t p = 0; p < P; ++p) {
    off[p] = elems;
    elems += (mb[p].size() + align - 1) / align * align;
  }
  if (elems * sizeof(T) != d.pool_bytes)
    return fail(c, AMR_ERR_STATE, "stencil-maximum pool does not match the brick pool");
  CK(cudaMalloc(&d.mpool, elems * sizeof(T)));
  for (size_t p = 0; p < P; ++p)
    CK(cudaMemcpyAsync((T*)d.mpool + off[p], mb[p].data(), mb[p].size() * sizeof(T),
                       cudaMemcpyHostToDevice, stream));
  return AMR_OK;
}

}  // namespace

void release_device(amr_ctx* c) {
  DeviceState& d = c->dev;
  if (d.device >= 0) cudaSetDevice(d.device);
  if (d.atlas_tex) cudaDestroyTextureObject(d.atlas_tex);
  if (d.gatlas_tex) cudaDestroyTextureObject(d.gatlas_tex);
  for (auto t : d.texobjs)
    if (t) cudaDestroyTextureObject(t);
  for (auto t : d.gtexobjs)
    if (t) cudaDestroyTextureObject(t);
  for (void* a : d.arrays)
    if (a) cudaFreeArray((cudaArray_t)a);
  for (void* a : d.garrays)
    if (a) cudaFreeArray((cudaArray_t)a);
  if (d.atlas_array) cudaFreeArray((cudaArray_t)d.atlas_array);
  if (d.gatlas_array) cudaFreeArray((cudaArray_t)d.gatlas_array);
  cudaFree(d.gpool);
  cudaFree(d.mpool);
  cudaFree(d.nodes);
  cudaFree(d.lod);
  cudaFree(d.face_node);
  cudaFree(d.node_box);
  cudaFree(d.macro);
  cudaFree(d.leaves);
  cudaFree(d.patches);
  cudaFree(d.pool);
  cudaFree(d.counters);
  cudaFree(d.tf_scratch);
  cudaFree(d.proposal);
  cudaFree(d.img_scratch);
  cudaFree(d.log_counts);
  cudaFree(d.log_offsets);
  d = DeviceState();
  c->device_built = false;
}

amr_status upload(amr_ctx* c, void* stream_v) {
  cudaStream_t stream = (cudaStream_t)stream_v;
  if (c->device_built) release_device(c);
  DeviceState& d = c->dev;
  CK(cudaGetDevice(&d.device));
  const Tree& t = c->tree;
  const size_t P = c->patches.size();
  const size_t M = t.leaf_patch.size();
  if (t.axis.size() >= (size_t)kIndexMask || M >= (size_t)kIndexMask)
    return fail(c, AMR_ERR_CAPACITY, "tree too large for 30-bit node indices");
  std::vector<int32_t> lodv, slot_of;
  std::vector<int4> boxes;
  std::vector<int32_t> leaf_anc;
  std::vector<DNode> nodes = layout_nodes(t, c->root, lodv, slot_of, boxes, leaf_anc);
  if (fault_injected("corrupt_node") && nodes.size() > 1 &&
      (nodes[0].meta >> 30) != (uint32_t)kLeafAxis)
    nodes[0].meta &= ~kIndexMask;  // the root's children become slots 0 (itself) and 1
  std::vector<int32_t> face_slots(std::max<size_t>(1, t.face_node.size()), 0);
  for (size_t k = 0; k < t.face_node.size(); ++k) {
    const int32_t pre = t.face_node[k];
    face_slots[k] = t.axis[pre] < 0 ? (int32_t)(kFaceLeaf | (uint32_t)t.leaf[pre]) : slot_of[pre];
  }
  const size_t ML = t.lod_patch.size();
  if (M + ML >= ((size_t)1 << 26)) return fail(c, AMR_ERR_CAPACITY, "too many leaves");
  std::vector<DLeaf> leaves(M + ML);
  for (size_t m = 0; m < M + ML; ++m) {
    DLeaf& l = leaves[m];
    std::memset(&l, 0, sizeof l);
    const bool lod = m >= M;
    const int32_t* box = lod ? &t.lod_box[6 * (m - M)] : &t.leaf_box[6 * m];
    for (int k = 0; k < 6; ++k) (k < 3 ? l.lo[k] : l.hi[k - 3]) = box[k];
    l.patch = lod ? t.lod_patch[m - M] : t.leaf_patch[m];
    l.level = lod ? t.lod_level[m - M] : t.leaf_level[m];
    l.faces = (lod || t.leaf_faces.empty()) ? 0 : t.leaf_faces[m];
    l.lod_anc = lod ? -1 : leaf_anc[m];
    // the range of the cells as stored; rounding is monotone, so the rounded extremes
    // bound every rounded cell and empty-space skipping stays exact
    l.vmin = storage_round(c->dtype, c->leaf_vmin[m]);
    l.vmax = storage_round(c->dtype, c->leaf_vmax[m]);
  }
  std::vector<DPatch> pt(P);
  for (size_t p = 0; p < P; ++p) {
    std::memset(&pt[p], 0, sizeof(DPatch));
    for (int a = 0; a < 3; ++a) {
      // brick index = cell - lo + 1 in every kernel: a halo of H cells shifts lo by H - 1
      pt[p].lo[a] = (int32_t)(c->patches[p].box[a] - (c->halo - 1));
      pt[p].dim[a] = (int32_t)(c->patches[p].n[a] + 2 * c->halo);
    }
  }
  if (fault_injected("oom")) return fail(c, AMR_ERR_OOM, "injected device allocation failure");
  CK(cudaMalloc(&d.nodes, nodes.size() * sizeof(DNode)));
  CK(cudaMalloc(&d.lod, lodv.size() * sizeof(int32_t)));
  CK(cudaMalloc(&d.face_node, face_slots.size() * sizeof(int32_t)));
  CK(cudaMalloc(&d.node_box, boxes.size() * sizeof(int4)));
  CK(cudaMalloc(&d.leaves, std::max<size_t>(1, M + ML) * sizeof(DLeaf)));
  CK(cudaMalloc(&d.patches, P * sizeof(DPatch)));
  CK(cudaMalloc(&d.counters, kNumCounters * sizeof(unsigned long long)));
  const std::vector<uint32_t> macro = macro_grid(nodes, c->root, c->R, &d.macro_cell, d.macro_dims);
  CK(cudaMalloc(&d.macro, macro.size() * sizeof(uint32_t)));
  CK(cudaMemcpyAsync(d.macro, macro.data(), macro.size() * sizeof(uint32_t),
                     cudaMemcpyHostToDevice, stream));
  CK(cudaMemsetAsync(d.counters, 0, kNumCounters * sizeof(unsigned long long), stream));

  amr_status st;
  if (c->dtype == AMR_F32) {
    st = upload_bricks<float>(c, c->bricks, pt, false, stream);
    if (st != AMR_OK) return st;
    if (c->want_max && c->storage == AMR_STORE_PTR) {
      st = upload_max_pool<float>(c, c->mbricks, stream);
      if (st != AMR_OK) return st;
    }
    if (c->want_gradient) {
      st = upload_bricks<float4>(c, c->gbricks, pt, true, stream);
      if (st != AMR_OK) return st;
    }
  } else {
    // 16-bit cells (and 4 x 16-bit value + central differences)
    {
      std::vector<std::vector<uint16_t>> b16(P);
#pragma omp parallel for schedule(dynamic, 4)
      for (long long pi = 0; pi < (long long)P; ++pi) {
        const size_t p = (size_t)pi;
        const std::vector<float>& b = c->bricks[p];
        b16[p].resize(b.size());
        for (size_t i = 0; i < b.size(); ++i) b16[p][i] = storage_bits(c->dtype, b[i]);
      }
      st = upload_bricks<uint16_t>(c, b16, pt, false, stream);
      if (st != AMR_OK) return st;
      if (c->want_max && c->storage == AMR_STORE_PTR) {
        // the maximum of the rounded cells is the rounded maximum (rounding is monotone)
#pragma omp parallel for schedule(dynamic, 4)
        for (long long pi = 0; pi < (long long)P; ++pi) {
          const size_t p = (size_t)pi;
          const std::vector<float>& m = c->mbricks[p];
          for (size_t i = 0; i < m.size(); ++i) b16[p][i] = storage_bits(c->dtype, m[i]);
        }
        st = upload_max_pool<uint16_t>(c, b16, stream);
        if (st != AMR_OK) return st;
      }
    }
    if (c->want_gradient) {
      std::vector<std::vector<ushort4>> g16(P);
#pragma omp parallel for schedule(dynamic, 4)
      for (long long pi = 0; pi < (long long)P; ++pi) {
        const size_t p = (size_t)pi;
        const std::vector<float4>& g = c->gbricks[p];
        g16[p].resize(g.size());
        for (size_t i = 0; i < g.size(); ++i)
          g16[p][i] = make_ushort4(storage_bits(c->dtype, g[i].x), storage_bits(c->dtype, g[i].y),
                                   storage_bits(c->dtype, g[i].z), storage_bits(c->dtype, g[i].w));
      }
      st = upload_bricks<ushort4>(c, g16, pt, true, stream);
      if (st != AMR_OK) return st;
    }
  }
  CK(cudaMemcpyAsync(d.nodes, nodes.data(), nodes.size() * sizeof(DNode), cudaMemcpyHostToDevice,
                     stream));
  CK(cudaMemcpyAsync(d.lod, lodv.data(), lodv.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                     stream));
  CK(cudaMemcpyAsync(d.face_node, face_slots.data(), face_slots.size() * sizeof(int32_t),
                     cudaMemcpyHostToDevice, stream));
  CK(cudaMemcpyAsync(d.node_box, boxes.data(), boxes.size() * sizeof(int4), cudaMemcpyHostToDevice,
                     stream));
  for (DLeaf& l : leaves) {  // brick addressing, now that the bricks are placed
    const DPatch& q = pt[(size_t)l.patch];
    l.base = q.base;
    l.gbase = q.gbase;
    l.sy = q.sy;
    l.sz = q.sz;
    for (int a = 0; a < 3; ++a) {
      l.blo[a] = q.lo[a];
      l.dim[a] = q.dim[a];
    }
  }
  if (M + ML)
    CK(cudaMemcpyAsync(d.leaves, leaves.data(), (M + ML) * sizeof(DLeaf), cudaMemcpyHostToDevice,
                       stream));
  CK(cudaMemcpyAsync(d.patches, pt.data(), P * sizeof(DPatch), cudaMemcpyHostToDevice, stream));
  CK(cudaStreamSynchronize(stream));
  c->device_built = true;
  return AMR_OK;
}

}  // namespace amr
