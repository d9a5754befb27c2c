"""FP64 CPU oracle for the AMR raycaster (test infrastructure only).

Only the tests, the smoke check and the CPU-baseline leg of the bench load this package.
It wraps `oracle.c` (plain C, double precision, compiled with -ffp-contract=off) through
ctypes and shares nothing with the product library.

Paper: Kaehler & Abel, "Single-Pass GPU-Raycasting for Structured Adaptive Mesh Refinement
Data".  Each function's docstring names the section it restates.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ORC_OK, ORC_ERR_ARG, ORC_ERR_OVERLAP, ORC_ERR_NOT_TILED, ORC_ERR_STATE = 0, -1, -2, -3, -4
ORC_ERR_OOM, ORC_ERR_CAPACITY = -5, -6


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (gcc, OpenMP, no FMA contraction)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Camera(C.Structure):
    _fields_ = [("eye", C.c_double * 3), ("fwd", C.c_double * 3), ("right", C.c_double * 3),
                ("up", C.c_double * 3), ("tan_half_fov_y", C.c_double), ("width", C.c_int),
                ("height", C.c_int)]


class _Params(C.Structure):
    _fields_ = [("step_factor", C.c_double), ("kappa", C.c_double), ("ert_eps", C.c_double),
                ("vmin", C.c_double), ("vmax", C.c_double), ("ka", C.c_double),
                ("kd", C.c_double), ("ks", C.c_double), ("shininess", C.c_double),
                ("gamma", C.c_double), ("world_step", C.c_double), ("interp", C.c_int),
                ("shade", C.c_int), ("lookup", C.c_int), ("max_segments", C.c_int),
                ("lod_pixels", C.c_double), ("shadow", C.c_int), ("light", C.c_double * 3),
                ("light_step", C.c_double), ("light_ambient", C.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB)
            P = C.c_void_p
            dp = C.POINTER(C.c_double)
            ip = C.POINTER(C.c_int)
            lp = C.POINTER(C.c_longlong)
            lib.orc_create.restype = P
            lib.orc_create.argtypes = [C.c_int, C.c_int, dp, dp, C.c_int, ip, lp,
                                       C.POINTER(C.c_void_p)]
            lib.orc_destroy.argtypes = [P]
            lib.orc_build.argtypes = [P]
            lib.orc_num_nodes.argtypes = [P]
            lib.orc_num_leaves.argtypes = [P]
            lib.orc_get_leaves.argtypes = [P, lp, ip, ip]
            lib.orc_get_nodes.argtypes = [P, ip, lp, ip, ip, ip]
            lib.orc_V.restype = C.c_double
            lib.orc_V.argtypes = [P, C.c_int, C.c_longlong, C.c_longlong, C.c_longlong]
            lib.orc_S.restype = C.c_double
            lib.orc_S.argtypes = [P, C.c_int, dp]
            lib.orc_F.restype = C.c_double
            lib.orc_F.argtypes = [P, dp, C.c_int, C.c_int]
            lib.orc_lookup_scan.argtypes = [P, dp, ip]
            lib.orc_lookup_leaf.argtypes = [P, dp]
            lib.orc_trace.argtypes = [P, C.POINTER(_Camera), C.c_int, C.c_int, ip, dp, dp, C.c_int]
            lib.orc_trace_lod.argtypes = [P, C.POINTER(_Camera), C.c_int, C.c_int, C.c_double,
                                          ip, dp, dp, C.c_int]
            lib.orc_get_node_labels.argtypes = [P, ip, ip, ip]
            lib.orc_shadow_T.restype = C.c_double
            lib.orc_shadow_T.argtypes = [P, C.POINTER(C.c_float), C.c_int, C.POINTER(_Params), dp]
            lib.orc_render_pixels.argtypes = [P, C.POINTER(_Camera), C.POINTER(C.c_float), C.c_int,
                                              C.POINTER(_Params), C.c_int, ip, ip, dp,
                                              C.POINTER(C.c_ulonglong), C.c_int]
            lib.orc_max_threads.restype = C.c_int
            lib.orc_mlp_forward.argtypes = [dp] * 8 + [C.c_int, dp, dp]
            lib.orc_mlp_loss_grad.restype = C.c_double
            lib.orc_mlp_loss_grad.argtypes = [dp] * 8 + [C.c_int, dp, dp] + [dp] * 8
            _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _lp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_longlong))


def camera_struct(cam) -> _Camera:
    c = _Camera()
    for name in ("eye", "fwd", "right", "up"):
        arr = np.asarray(getattr(cam, name), dtype=np.float64)
        getattr(c, name)[:] = [float(v) for v in arr]
    c.tan_half_fov_y = float(cam.tan_half_fov_y)
    c.width = int(cam.width)
    c.height = int(cam.height)
    return c


@dataclass
class OracleParams:
    """Render parameters (defaults: Phong constants ka 0.3, kd 0.6, ks 0.3, shininess 32,
    gradient floor gamma 1e-3, step factor 0.5, ERT epsilon 1e-4)."""
    vmin: float = 0.0
    vmax: float = 1.0
    step_factor: float = 0.5
    kappa: float = 8.0
    ert_eps: float = 1e-4
    interp: int = 1
    shade: int = 0
    ka: float = 0.3
    kd: float = 0.6
    ks: float = 0.3
    shininess: float = 32.0
    gamma: float = 1e-3
    world_step: float = 0.0
    lookup: int = 0
    max_segments: int = 0
    lod_pixels: float = 0.0  # > 0: level-of-detail pruning (Sec. 3.1 type-(a) nodes)
    shadow: int = 0          # 1: secondary rays to a point light
    light: tuple = (0.0, 0.0, 0.0)
    light_step: float = 0.0
    light_ambient: float = 0.2

    def struct(self) -> _Params:
        p = _Params()
        for f in ("step_factor", "kappa", "ert_eps", "vmin", "vmax", "ka", "kd", "ks",
                  "shininess", "gamma", "world_step", "lod_pixels", "light_step",
                  "light_ambient"):
            setattr(p, f, float(getattr(self, f)))
        for f in ("interp", "shade", "lookup", "max_segments", "shadow"):
            setattr(p, f, int(getattr(self, f)))
        p.light[:] = [float(v) for v in self.light]
        return p


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: oracle status {code}")
        self.code = code


class Oracle:
    """One AMR hierarchy with its oracle kD-tree (built on construction)."""

    def __init__(self, hier, build_tree: bool = True):
        lib = _load()
        self._lib = lib
        P = hier.num_patches
        self._levels = np.ascontiguousarray(hier.patch_level, dtype=np.int32)
        self._boxes = np.ascontiguousarray(hier.patch_box, dtype=np.int64).reshape(P, 6)
        self._data = [np.ascontiguousarray(d, dtype=np.float32) for d in hier.data]
        ptrs = (C.c_void_p * P)(*[d.ctypes.data for d in self._data])
        dlo = np.ascontiguousarray(hier.domain_lo, dtype=np.float64)
        h0 = np.ascontiguousarray(hier.h0, dtype=np.float64)
        self._h = lib.orc_create(int(hier.num_levels), int(hier.ratio), _dp(dlo), _dp(h0), P,
                                 _ip(self._levels), _lp(self._boxes), ptrs)
        if not self._h:
            raise OracleError(ORC_ERR_ARG, "orc_create")
        self._data = None  # the oracle keeps its own copy
        self.hier = hier
        if build_tree:
            rc = lib.orc_build(self._h)
            if rc != 0:
                lib.orc_destroy(self._h)
                self._h = None
                raise OracleError(rc, "orc_build")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_destroy(h)
            self._h = None

    # ------------------------------------------------------------------ tree (Sec. 3.1)
    @property
    def num_nodes(self) -> int:
        return int(self._lib.orc_num_nodes(self._h))

    @property
    def num_leaves(self) -> int:
        return int(self._lib.orc_num_leaves(self._h))

    def leaves(self):
        """Canonical leaves (pre-order): box int64[M,6] (finest cells), patch, level."""
        M = self.num_leaves
        box = np.zeros((M, 6), dtype=np.int64)
        patch = np.zeros(M, dtype=np.int32)
        level = np.zeros(M, dtype=np.int32)
        rc = self._lib.orc_get_leaves(self._h, _lp(box), _ip(patch), _ip(level))
        if rc < 0:
            raise OracleError(rc, "orc_get_leaves")
        return box, patch, level

    def nodes(self):
        """Pre-order nodes: axis (-1 leaf), split (finest), left, right, leaf id."""
        N = self.num_nodes
        axis = np.zeros(N, dtype=np.int32)
        split = np.zeros(N, dtype=np.int64)
        left = np.zeros(N, dtype=np.int32)
        right = np.zeros(N, dtype=np.int32)
        leaf = np.zeros(N, dtype=np.int32)
        rc = self._lib.orc_get_nodes(self._h, _ip(axis), _lp(split), _ip(left), _ip(right),
                                     _ip(leaf))
        if rc < 0:
            raise OracleError(rc, "orc_get_nodes")
        return axis, split, left, right, leaf

    def node_labels(self):
        """Pre-order node labels: patch, level (for an inner node: the patch of that level
        holding its whole box, -1 if none) and the node's pruned-leaf id (-1 if none)."""
        N = self.num_nodes
        patch = np.zeros(N, dtype=np.int32)
        level = np.zeros(N, dtype=np.int32)
        lod = np.zeros(N, dtype=np.int32)
        rc = self._lib.orc_get_node_labels(self._h, _ip(patch), _ip(level), _ip(lod))
        if rc < 0:
            raise OracleError(rc, "orc_get_node_labels")
        return patch, level, lod

    # ------------------------------------------------------------------ field (Sec. 2, 4)
    def V(self, l: int, i: int, j: int, k: int) -> float:
        return float(self._lib.orc_V(self._h, l, i, j, k))

    def S(self, l: int, x: Sequence[float]) -> float:
        xa = np.ascontiguousarray(x, dtype=np.float64)
        return float(self._lib.orc_S(self._h, l, _dp(xa)))

    def F(self, x: Sequence[float], interp: int = 1, lookup: int = 0) -> float:
        xa = np.ascontiguousarray(x, dtype=np.float64)
        return float(self._lib.orc_F(self._h, _dp(xa), interp, lookup))

    def lookup_scan(self, x):
        xa = np.ascontiguousarray(x, dtype=np.float64)
        p = np.zeros(1, dtype=np.int32)
        l = self._lib.orc_lookup_scan(self._h, _dp(xa), _ip(p))
        return int(l), int(p[0])

    def lookup_leaf(self, x) -> int:
        xa = np.ascontiguousarray(x, dtype=np.float64)
        return int(self._lib.orc_lookup_leaf(self._h, _dp(xa)))

    # ------------------------------------------------------------------ rays (Sec. 3.3)
    def trace(self, cam, i: int, j: int, cap: int = 1 << 16, lod_pixels: float = 0.0):
        """Leaf-id sequence and segment parameters of pixel (i, j); with lod_pixels > 0
        the pruned descent (pruned nodes have ids after the leaves)."""
        leaf = np.zeros(cap, dtype=np.int32)
        t0 = np.zeros(cap, dtype=np.float64)
        t1 = np.zeros(cap, dtype=np.float64)
        cs = camera_struct(cam)
        n = self._lib.orc_trace_lod(self._h, C.byref(cs), int(i), int(j), float(lod_pixels),
                                    _ip(leaf), _dp(t0), _dp(t1), cap)
        if n < 0:
            raise OracleError(n, "orc_trace")
        return leaf[:n].copy(), t0[:n].copy(), t1[:n].copy()

    def shadow_T(self, x, tf: np.ndarray, params: OracleParams) -> float:
        """Transmittance from world point x to params.light (secondary ray)."""
        tfa = np.ascontiguousarray(tf, dtype=np.float32).reshape(-1, 4)
        xa = np.ascontiguousarray(x, dtype=np.float64)
        ps = params.struct()
        return float(self._lib.orc_shadow_T(self._h, tfa.ctypes.data_as(C.POINTER(C.c_float)),
                                            tfa.shape[0], C.byref(ps), _dp(xa)))

    def render(self, cam, tf: np.ndarray, params: OracleParams,
               pixels: Optional[np.ndarray] = None, nthreads: int = 0):
        """Render all pixels (-> float64[H, W, 4]) or the listed (i, j) pixels
        (-> float64[n, 4]); also returns the per-pixel sample counts."""
        tfa = np.ascontiguousarray(tf, dtype=np.float32).reshape(-1, 4)
        W, H = int(cam.width), int(cam.height)
        if pixels is None:
            jj, ii = np.meshgrid(np.arange(H, dtype=np.int32), np.arange(W, dtype=np.int32),
                                 indexing="ij")
            px = np.ascontiguousarray(ii.ravel())
            py = np.ascontiguousarray(jj.ravel())
        else:
            pix = np.asarray(pixels, dtype=np.int32).reshape(-1, 2)
            px = np.ascontiguousarray(pix[:, 0])
            py = np.ascontiguousarray(pix[:, 1])
        n = px.shape[0]
        out = np.zeros((n, 4), dtype=np.float64)
        smp = np.zeros(n, dtype=np.uint64)
        cs = camera_struct(cam)
        ps = params.struct()
        rc = self._lib.orc_render_pixels(self._h, C.byref(cs),
                                         tfa.ctypes.data_as(C.POINTER(C.c_float)), tfa.shape[0],
                                         C.byref(ps), n, _ip(px), _ip(py), _dp(out),
                                         smp.ctypes.data_as(C.POINTER(C.c_ulonglong)),
                                         int(nthreads))
        if rc < 0:
            raise OracleError(rc, "orc_render_pixels")
        if pixels is None:
            return out.reshape(H, W, 4), smp.reshape(H, W)
        return out, smp


def max_threads() -> int:
    return int(_load().orc_max_threads())


# ---------------------------------------------------------------------- MLP (learned part)
MLP_SHAPES = [(64, 12), (64,), (64, 64), (64,), (64, 64), (64,), (1, 64), (1,)]


def mlp_forward(params: Sequence[np.ndarray], x: np.ndarray) -> np.ndarray:
    """sigmoid(W4 relu(W3 relu(W2 relu(W1 x + b1) + b2) + b3) + b4) in FP64, per row."""
    lib = _load()
    ps = [np.ascontiguousarray(p, dtype=np.float64) for p in params]
    xa = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 12)
    y = np.zeros(xa.shape[0], dtype=np.float64)
    lib.orc_mlp_forward(*[_dp(p) for p in ps], xa.shape[0], _dp(xa), _dp(y))
    return y


def mlp_loss_grad(params: Sequence[np.ndarray], x: np.ndarray, t: np.ndarray):
    """Mean BCE loss and its gradient for every parameter (FP64)."""
    lib = _load()
    ps = [np.ascontiguousarray(p, dtype=np.float64) for p in params]
    xa = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 12)
    ta = np.ascontiguousarray(t, dtype=np.float64).reshape(-1)
    gs = [np.zeros(s, dtype=np.float64) for s in MLP_SHAPES]
    loss = lib.orc_mlp_loss_grad(*[_dp(p) for p in ps], xa.shape[0], _dp(xa), _dp(ta),
                                 *[_dp(g) for g in gs])
    return float(loss), gs
