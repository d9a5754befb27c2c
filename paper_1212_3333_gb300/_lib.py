"""ctypes declarations for libamr_gb300.so (the C ABI in include/amr.h).

There is no fallback: if the library is missing or fails to load, importing the binding
raises, so no code path can silently run without the CUDA kernels.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libamr_gb300.so")

AMR_OK, AMR_ERR_ARG, AMR_ERR_OVERLAP, AMR_ERR_NOT_TILED, AMR_ERR_STATE = 0, 1, 2, 3, 4
AMR_ERR_OOM, AMR_ERR_CUDA, AMR_ERR_CAPACITY, AMR_ERR_DEVICE = 5, 6, 7, 8
STATUS_NAMES = {0: "AMR_OK", 1: "AMR_ERR_ARG", 2: "AMR_ERR_OVERLAP", 3: "AMR_ERR_NOT_TILED",
                4: "AMR_ERR_STATE", 5: "AMR_ERR_OOM", 6: "AMR_ERR_CUDA", 7: "AMR_ERR_CAPACITY",
                8: "AMR_ERR_DEVICE"}

AMR_F32, AMR_F16, AMR_BF16 = 0, 1, 2
DTYPES = {"f32": AMR_F32, "f16": AMR_F16, "bf16": AMR_BF16}
AMR_STORE_PTR, AMR_STORE_TEXOBJ, AMR_STORE_ATLAS_LINEAR, AMR_STORE_ATLAS_TEX3D = 0, 1, 2, 3
AMR_STORE_GRADIENT = 0x100
AMR_STORE_HALO2 = 0x200
AMR_STORE_MAXBRICK = 0x400
AMR_MLP_FEATURES, AMR_MLP_PARAMS, AMR_MLP_PACKED_BYTES = 12, 9217, 23440
AMR_MLP_GRAD_BLOCKS = 152
AMR_MLP_GRAD_SCRATCH = AMR_MLP_GRAD_BLOCKS * (AMR_MLP_PARAMS + 1)
STORAGES = {"ptr": AMR_STORE_PTR, "texobj": AMR_STORE_TEXOBJ,
            "atlas_linear": AMR_STORE_ATLAS_LINEAR, "atlas_tex3d": AMR_STORE_ATLAS_TEX3D}


class amr_camera(C.Structure):
    _fields_ = [("eye", C.c_double * 3), ("fwd", C.c_double * 3), ("right", C.c_double * 3),
                ("up", C.c_double * 3), ("tan_half_fov_y", C.c_double), ("width", C.c_int32),
                ("height", C.c_int32)]


class amr_render_params(C.Structure):
    _fields_ = [("step_factor", C.c_double), ("kappa", C.c_double), ("ert_eps", C.c_double),
                ("vmin", C.c_double), ("vmax", C.c_double), ("ka", C.c_double),
                ("kd", C.c_double), ("ks", C.c_double), ("shininess", C.c_double),
                ("gamma", C.c_double), ("interp", C.c_int32), ("shade", C.c_int32),
                ("row0", C.c_int32), ("rows", C.c_int32), ("skip", C.c_int32),
                ("max_segments", C.c_int32), ("schedule", C.c_int32),
                ("learned", C.c_int32), ("tau", C.c_double), ("samples_per_iter", C.c_int32),
                ("coarse_factor", C.c_int32), ("lod_pixels", C.c_double),
                ("shadow", C.c_int32), ("light", C.c_double * 3), ("light_step", C.c_double),
                ("light_ambient", C.c_double), ("learned_min_samples", C.c_int32),
                ("reserved", C.c_int32)]


class amr_stats(C.Structure):
    _fields_ = [("num_nodes", C.c_int64), ("num_leaves", C.c_int64),
                ("num_patches", C.c_int64), ("num_cells", C.c_int64),
                ("brick_bytes", C.c_int64), ("tree_bytes", C.c_int64),
                ("atlas_dims", C.c_int32 * 3), ("atlas_efficiency", C.c_double),
                ("atlas_efficiency_halo", C.c_double), ("build_seconds", C.c_double),
                ("max_depth", C.c_int32), ("storage", C.c_int32),
                ("exact_paths", C.c_int64 * 3)]


AMR_MAX_BATCH_VIEWS = 128
AMR_SCHEDULE_AUTO = -1
AMR_BATCH_CANDIDATES = 13


class amr_view(C.Structure):
    _fields_ = [("cam", amr_camera), ("tf_index", C.c_int32), ("reserved", C.c_int32),
                ("out_offset", C.c_int64)]


class amr_batch_config(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("rays_per_thread", C.c_int32),
                ("blocks_per_sm", C.c_int32), ("samples_per_iter", C.c_int32)]


# every symbol include/amr.h declares, with its ctypes signature
_P = C.c_void_p
_SIGS = {
    "amr_default_params": (None, [C.POINTER(amr_render_params)]),
    "amr_create": (C.c_int, [C.c_int32, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_double),
                             C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int64),
                             C.POINTER(C.c_void_p), C.c_int, C.POINTER(_P)]),
    "amr_build_kdtree": (C.c_int, [_P, C.c_int, _P]),
    "amr_build_host": (C.c_int, [_P, C.c_int]),
    "amr_render": (C.c_int, [_P, C.POINTER(amr_camera), _P, C.c_int32,
                             C.POINTER(amr_render_params), _P, _P, C.POINTER(C.c_uint64)]),
    "amr_render_host": (C.c_int, [_P, C.POINTER(amr_camera), _P, C.c_int32,
                                  C.POINTER(amr_render_params), _P, _P, C.POINTER(C.c_uint64)]),
    "amr_render_host_noalloc": (C.c_int, [_P, C.POINTER(amr_camera), _P, C.c_int32,
                                          C.POINTER(amr_render_params), _P, _P,
                                          C.POINTER(C.c_uint64)]),
    "amr_render_batch": (C.c_int, [_P, C.POINTER(amr_view), C.c_int32, _P, C.c_int32, C.c_int32,
                                   C.POINTER(amr_render_params), _P, C.c_int64,
                                   C.POINTER(amr_batch_config), _P, C.POINTER(C.c_uint64)]),
    "amr_batch_autotune": (C.c_int, [_P, C.POINTER(amr_view), C.c_int32, _P, C.c_int32,
                                     C.c_int32, C.POINTER(amr_render_params), _P, C.c_int64,
                                     C.c_int32, _P, C.POINTER(amr_batch_config),
                                     C.POINTER(C.c_float)]),
    "amr_log_segments": (C.c_int, [_P, C.POINTER(amr_camera), _P, C.c_int32,
                                   C.POINTER(amr_render_params), _P, _P, C.c_int64, _P, C.c_float,
                                   C.c_uint32, _P]),
    "amr_mlp_pack": (C.c_int, [_P, _P, _P]),
    "amr_mlp_forward": (C.c_int, [_P, _P, C.c_int64, _P, _P]),
    "amr_mlp_loss_grad": (C.c_int, [_P, _P, _P, C.c_int64, C.c_int64, C.c_int64, C.c_int64,
                                    C.c_int64, _P, _P, _P, _P]),
    "amr_mlp_adam": (C.c_int, [_P, _P, _P, _P, C.c_float, C.c_float, C.c_float, C.c_float,
                               C.c_int32, _P]),
    "amr_set_proposal": (C.c_int, [_P, _P, _P]),
    "amr_destroy": (C.c_int, [_P]),
    "amr_last_error": (C.c_char_p, [_P]),
    "amr_get_stats": (C.c_int, [_P, C.POINTER(amr_stats)]),
    "amr_get_leaves": (C.c_int, [_P, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                 C.POINTER(C.c_int32), C.c_int64, C.POINTER(C.c_int64)]),
    "amr_get_nodes": (C.c_int, [_P, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                C.c_int64, C.POINTER(C.c_int64)]),
    "amr_get_lod_leaves": (C.c_int, [_P, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                     C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.c_int64,
                                     C.POINTER(C.c_int64)]),
    "amr_get_leaf_faces": (C.c_int, [_P, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.c_int64,
                                     C.POINTER(C.c_int64)]),
    "amr_get_brick": (C.c_int, [_P, C.c_int32, C.POINTER(C.c_float), C.c_int64,
                                C.POINTER(C.c_int64)]),
    "amr_trace": (C.c_int, [_P, C.POINTER(amr_camera), C.c_double, _P, _P, _P, C.c_int32, _P]),
}

_lock = threading.Lock()
_lib = None


def load() -> C.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(
                    f"{LIB_PATH} is missing: build it with "
                    "`python -c 'import __graft_entry__ as g; g.build()'` "
                    "(or paper_1212_3333_gb300.build.build()); there is no CPU fallback")
            lib = C.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def declared_symbols():
    return list(_SIGS)
