"""GB300 single-pass raycaster for structured AMR data (Kaehler & Abel, arXiv 1212.3333).

A thin Python binding over the C ABI in include/amr.h.  It only marshals arguments:
the kD-tree build, brick packing and every step of the ray march run in the native
library (host C++ for the build, sm_103a CUDA kernels for rendering).  PyTorch provides
device memory and streams.  The functions keep the ABI's names.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence

import numpy as np

from . import _lib
from ._lib import (AMR_BF16, AMR_F16, AMR_F32, AMR_STORE_ATLAS_LINEAR,  # noqa: F401
                   AMR_STORE_ATLAS_TEX3D, AMR_STORE_GRADIENT, AMR_STORE_PTR, AMR_STORE_TEXOBJ,
                   DTYPES, STORAGES, amr_camera, amr_render_params, amr_stats)


class AmrError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_lib.STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def _check(status: int, ctx_handle) -> None:
    if status != _lib.AMR_OK:
        msg = _lib.load().amr_last_error(ctx_handle)
        raise AmrError(status, msg.decode() if msg else "")


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dptr(t) -> int:
    return int(t.data_ptr())


def make_camera(cam) -> amr_camera:
    """amr_camera from any object with eye/fwd/right/up/tan_half_fov_y/width/height."""
    c = amr_camera()
    for name in ("eye", "fwd", "right", "up"):
        getattr(c, name)[:] = [float(v) for v in np.asarray(getattr(cam, name), dtype=np.float64)]
    c.tan_half_fov_y = float(cam.tan_half_fov_y)
    c.width = int(cam.width)
    c.height = int(cam.height)
    return c


def amr_default_params(**overrides) -> amr_render_params:
    p = amr_render_params()
    _lib.load().amr_default_params(C.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise AttributeError(f"amr_render_params has no field {k}")
        setattr(p, k, v)
    return p


class AmrContext:
    """Owns one amr_ctx (created by amr_create, released by amr_destroy)."""

    def __init__(self, handle: int):
        self._h = C.c_void_p(handle)
        self._lib = _lib.load()

    # ----------------------------------------------------------------- lifecycle
    @staticmethod
    def _storage_code(storage, gradient: bool, halo: int = 1, maxbrick: bool = False) -> int:
        st = STORAGES[storage] if isinstance(storage, str) else int(storage)
        if halo not in (1, 2):
            raise ValueError("halo must be 1 or 2")
        return (st | (AMR_STORE_GRADIENT if gradient else 0) |
                (_lib.AMR_STORE_HALO2 if halo == 2 else 0) |
                (_lib.AMR_STORE_MAXBRICK if maxbrick else 0))

    def amr_build_kdtree(self, storage="ptr", stream=None, gradient: bool = False,
                         halo: int = 1, maxbrick: bool = False) -> None:
        st = self._storage_code(storage, gradient, halo, maxbrick)
        _check(self._lib.amr_build_kdtree(self._h, st, C.c_void_p(_stream_ptr(stream))), self._h)

    def amr_build_host(self, storage="ptr", gradient: bool = False, halo: int = 1,
                       maxbrick: bool = False) -> None:
        st = self._storage_code(storage, gradient, halo, maxbrick)
        _check(self._lib.amr_build_host(self._h, st), self._h)

    def amr_destroy(self) -> None:
        if self._h:
            self._lib.amr_destroy(self._h)
            self._h = C.c_void_p(None)

    def __del__(self):
        try:
            self.amr_destroy()
        except Exception:
            pass

    # ----------------------------------------------------------------- rendering
    def amr_render(self, camera, tf, params: amr_render_params, out, stream=None,
                   count_samples: bool = False) -> Optional[int]:
        """tf: CUDA float32 [n, 4]; out: CUDA float32 [rows, W, 4] (contiguous)."""
        cam = camera if isinstance(camera, amr_camera) else make_camera(camera)
        if not tf.is_contiguous() or not out.is_contiguous():
            raise ValueError("tf and out must be contiguous")
        smp = C.c_uint64(0)
        _check(self._lib.amr_render(self._h, C.byref(cam), C.c_void_p(_dptr(tf)), int(tf.shape[0]),
                                    C.byref(params), C.c_void_p(_dptr(out)),
                                    C.c_void_p(_stream_ptr(stream)),
                                    C.byref(smp) if count_samples else None), self._h)
        return int(smp.value) if count_samples else None

    def amr_render_host(self, camera, tf: np.ndarray, params: amr_render_params,
                        out: np.ndarray, stream=None, count_samples: bool = False):
        """Host buffers (numpy, or pinned torch CPU tensors via their data pointers)."""
        cam = camera if isinstance(camera, amr_camera) else make_camera(camera)
        tfp = tf.ctypes.data if isinstance(tf, np.ndarray) else tf.data_ptr()
        outp = out.ctypes.data if isinstance(out, np.ndarray) else out.data_ptr()
        n = tf.shape[0]
        smp = C.c_uint64(0)
        _check(self._lib.amr_render_host(self._h, C.byref(cam), C.c_void_p(tfp), int(n),
                                         C.byref(params), C.c_void_p(outp),
                                         C.c_void_p(_stream_ptr(stream)),
                                         C.byref(smp) if count_samples else None), self._h)
        return int(smp.value) if count_samples else None

    def amr_render_batch(self, views, tfs, params: amr_render_params, out, config=None,
                         stream=None, count_samples: bool = False) -> Optional[int]:
        """views: from make_views; tfs: CUDA float32 [n_tf, tf_n, 4]; out: CUDA float32 buffer
        of at least the views' total size; config: amr_batch_config or None (autotuned)."""
        smp = C.c_uint64(0)
        _check(self._lib.amr_render_batch(
            self._h, views, len(views), C.c_void_p(_dptr(tfs)), int(tfs.shape[0]),
            int(tfs.shape[1]), C.byref(params), C.c_void_p(_dptr(out)), int(out.numel()),
            C.byref(config) if config is not None else None, C.c_void_p(_stream_ptr(stream)),
            C.byref(smp) if count_samples else None), self._h)
        return int(smp.value) if count_samples else None

    def amr_batch_autotune(self, views, tfs, params: amr_render_params, out, reps: int = 3,
                           stream=None):
        """Returns (best amr_batch_config, mean ms of every candidate)."""
        best = _lib.amr_batch_config()
        ms = (C.c_float * _lib.AMR_BATCH_CANDIDATES)()
        _check(self._lib.amr_batch_autotune(
            self._h, views, len(views), C.c_void_p(_dptr(tfs)), int(tfs.shape[0]),
            int(tfs.shape[1]), C.byref(params), C.c_void_p(_dptr(out)), int(out.numel()),
            int(reps), C.c_void_p(_stream_ptr(stream)), C.byref(best), ms), self._h)
        return best, list(ms)

    def amr_trace(self, camera, leaf_seq, seq_len, max_len: int, t_seq=None, stream=None,
                  lod_pixels: float = 0.0) -> None:
        cam = camera if isinstance(camera, amr_camera) else make_camera(camera)
        _check(self._lib.amr_trace(self._h, C.byref(cam), float(lod_pixels),
                                   C.c_void_p(_dptr(leaf_seq)),
                                   C.c_void_p(_dptr(t_seq) if t_seq is not None else None),
                                   C.c_void_p(_dptr(seq_len)), int(max_len),
                                   C.c_void_p(_stream_ptr(stream))), self._h)

    # ----------------------------------------------------------------- inspection
    def amr_get_stats(self) -> amr_stats:
        s = amr_stats()
        _check(self._lib.amr_get_stats(self._h, C.byref(s)), self._h)
        return s

    def amr_get_leaves(self):
        n = C.c_int64(0)
        self._lib.amr_get_leaves(self._h, None, None, None, 0, C.byref(n))
        m = n.value
        box = np.zeros((m, 6), dtype=np.int32)
        patch = np.zeros(m, dtype=np.int32)
        level = np.zeros(m, dtype=np.int32)
        ip = C.POINTER(C.c_int32)
        _check(self._lib.amr_get_leaves(self._h, box.ctypes.data_as(ip), patch.ctypes.data_as(ip),
                                        level.ctypes.data_as(ip), m, C.byref(n)), self._h)
        return box, patch, level

    def amr_get_lod_leaves(self):
        """Type-(a) nodes in pruned-leaf id order: box int32[k,6], patch, level, pre-order id."""
        n = C.c_int64(0)
        self._lib.amr_get_lod_leaves(self._h, None, None, None, None, 0, C.byref(n))
        m = n.value
        box = np.zeros((m, 6), dtype=np.int32)
        arrs = [np.zeros(m, dtype=np.int32) for _ in range(3)]
        ip = lambda a: a.ctypes.data_as(C.POINTER(C.c_int32))  # noqa: E731
        _check(self._lib.amr_get_lod_leaves(self._h, ip(box), ip(arrs[0]), ip(arrs[1]),
                                            ip(arrs[2]), m, C.byref(n)), self._h)
        return box, arrs[0], arrs[1], arrs[2]

    def amr_get_leaf_faces(self):
        """Per leaf: face bits (DLeaf.faces) and the 12 neighbour-lookup start nodes."""
        n = C.c_int64(0)
        self._lib.amr_get_leaf_faces(self._h, None, None, 0, C.byref(n))
        m = n.value
        faces = np.zeros(m, dtype=np.int32)
        nodes = np.zeros((m, 12), dtype=np.int32)
        ip = lambda a: a.ctypes.data_as(C.POINTER(C.c_int32))  # noqa: E731
        _check(self._lib.amr_get_leaf_faces(self._h, ip(faces), ip(nodes), m, C.byref(n)),
               self._h)
        return faces, nodes

    def amr_get_nodes(self):
        n = C.c_int64(0)
        self._lib.amr_get_nodes(self._h, None, None, None, None, None, 0, C.byref(n))
        m = n.value
        arrs = [np.zeros(m, dtype=np.int32) for _ in range(5)]
        ip = C.POINTER(C.c_int32)
        _check(self._lib.amr_get_nodes(self._h, *[a.ctypes.data_as(ip) for a in arrs], m,
                                       C.byref(n)), self._h)
        return tuple(arrs)

    def amr_get_brick(self, patch: int) -> np.ndarray:
        n = C.c_int64(0)
        self._lib.amr_get_brick(self._h, int(patch), None, 0, C.byref(n))
        out = np.zeros(n.value, dtype=np.float32)
        _check(self._lib.amr_get_brick(self._h, int(patch),
                                       out.ctypes.data_as(C.POINTER(C.c_float)), n.value,
                                       C.byref(n)), self._h)
        return out


def amr_create(num_levels: int, refine_ratio: int, domain_lo: Sequence[float],
               h0: Sequence[float], patch_level, patch_box, cell_data, dtype=AMR_F32) -> AmrContext:
    """dtype: device cell type, an amr_dtype code or "f32" / "f16" / "bf16"."""
    lib = _lib.load()
    dtype = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    lvl = np.ascontiguousarray(patch_level, dtype=np.int32)
    box = np.ascontiguousarray(patch_box, dtype=np.int64).reshape(-1, 6)
    data = [np.ascontiguousarray(d, dtype=np.float32) for d in cell_data]
    P = lvl.shape[0]
    ptrs = (C.c_void_p * P)(*[d.ctypes.data for d in data])
    dlo = (C.c_double * 3)(*[float(v) for v in domain_lo])
    hh = (C.c_double * 3)(*[float(v) for v in h0])
    h = C.c_void_p(None)
    st = lib.amr_create(int(num_levels), int(refine_ratio), dlo, hh, P,
                        lvl.ctypes.data_as(C.POINTER(C.c_int32)),
                        box.ctypes.data_as(C.POINTER(C.c_int64)), ptrs, int(dtype), C.byref(h))
    _check(st, None)
    return AmrContext(h.value)


def make_views(cameras, tf_index):
    """Batch view table with the images packed back to back in camera order:
    returns (amr_view array, per-view float offsets, total floats)."""
    n = len(cameras)
    views = (_lib.amr_view * n)()
    offsets = []
    off = 0
    for v, (cam, t) in enumerate(zip(cameras, tf_index)):
        views[v].cam = cam if isinstance(cam, amr_camera) else make_camera(cam)
        views[v].tf_index = int(t)
        views[v].out_offset = off
        offsets.append(off)
        off += 4 * views[v].cam.width * views[v].cam.height
    return views, offsets, off


def batch_config(tile_w: int = 16, tile_h: int = 8, rays_per_thread: int = 1,
                 blocks_per_sm: int = 0, samples_per_iter: int = 0):
    return _lib.amr_batch_config(tile_w, tile_h, rays_per_thread, blocks_per_sm,
                                 samples_per_iter)


def from_hierarchy(hier, dtype=AMR_F32) -> AmrContext:
    """amr_create from an object with num_levels, ratio, domain_lo, h0, patch_level,
    patch_box and data (list of float32 [nz, ny, nx] arrays)."""
    return amr_create(hier.num_levels, hier.ratio, hier.domain_lo, hier.h0, hier.patch_level,
                      hier.patch_box, hier.data, dtype)
