"""Learned segment proposal: logging, training and installation (orchestration only).

Every computation runs in the library's kernels (amr_log_segments, amr_mlp_loss_grad,
amr_mlp_adam, amr_mlp_pack, amr_mlp_forward); this module allocates the device tensors,
loops over views and minibatches and passes pointers.  The network (12-64-64-64-1, ReLU,
sigmoid) predicts a segment's opacity contribution A_out - A_in; segments predicted below
a threshold are skipped or sampled coarsely by the learned march.
"""
from __future__ import annotations

import ctypes as C
import math
from typing import Iterable, Optional, Tuple

import numpy as np

from . import AmrError, _check, _dptr, _stream_ptr, make_camera
from . import _lib

MLP_SHAPES = [(64, 12), (64,), (64, 64), (64,), (64, 64), (64,), (1, 64), (1,)]


def init_params(seed: int = 0) -> np.ndarray:
    """He-normal weights, zero biases, flattened in the library's parameter order."""
    rng = np.random.default_rng(seed)
    out = []
    for s in MLP_SHAPES:
        if len(s) == 2:
            out.append(rng.normal(0.0, math.sqrt(2.0 / s[1]), size=s).ravel())
        else:
            out.append(np.zeros(s))
    p = np.concatenate(out).astype(np.float32)
    assert p.size == _lib.AMR_MLP_PARAMS
    return p


def split_params(p: np.ndarray):
    """Flat parameter vector -> [W1, b1, W2, b2, W3, b3, W4, b4] arrays."""
    out, k = [], 0
    for s in MLP_SHAPES:
        n = int(np.prod(s))
        out.append(np.asarray(p[k:k + n]).reshape(s))
        k += n
    return out


def log_segments(ctx, cameras: Iterable, tf, params, capacity: int, keep_prob: float,
                 seed: int = 0, stream=None):
    """Run the plain march over `cameras` and collect (features [n,12], targets [n]) on the
    device; returns the tensors and the number of segments seen (before capacity)."""
    import torch

    lib = _lib.load()
    feats = torch.empty((capacity, _lib.AMR_MLP_FEATURES), dtype=torch.float32, device="cuda")
    tgts = torch.empty((capacity,), dtype=torch.float32, device="cuda")
    count = torch.zeros((1,), dtype=torch.int64, device="cuda")
    sp = C.c_void_p(_stream_ptr(stream))
    for v, cam in enumerate(cameras):
        cs = make_camera(cam)
        _check(lib.amr_log_segments(ctx._h, C.byref(cs), C.c_void_p(_dptr(tf)), int(tf.shape[0]),
                                    C.byref(params), C.c_void_p(_dptr(feats)),
                                    C.c_void_p(_dptr(tgts)), int(capacity),
                                    C.c_void_p(_dptr(count)), float(keep_prob),
                                    int((seed * 1000003 + v) & 0xffffffff), sp), ctx._h)
    torch.cuda.synchronize()
    seen = int(count.item())
    n = min(seen, capacity)
    return feats[:n], tgts[:n], seen


class Proposal:
    """FP32 master parameters with Adam state on the device, and their packed image."""

    def __init__(self, params: Optional[np.ndarray] = None, seed: int = 0):
        import torch

        p = init_params(seed) if params is None else np.asarray(params, dtype=np.float32)
        self.params = torch.as_tensor(p.copy(), device="cuda")
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.loss = torch.zeros((1,), dtype=torch.float32, device="cuda")
        # per-block partial sums of the gradient pass (reduced in a fixed order)
        self.scratch = torch.empty((_lib.AMR_MLP_GRAD_SCRATCH,), dtype=torch.float32,
                                   device="cuda")
        # 16-byte aligned buffer for the packed inference image
        self.packed = torch.zeros((_lib.AMR_MLP_PACKED_BYTES // 4,), dtype=torch.float32,
                                  device="cuda")
        self.step = 0
        self._lib = _lib.load()

    def loss_grad(self, x, t, first: int = 0, n: Optional[int] = None, perm_a: int = 1,
                  perm_b: int = 0, stream=None):
        N = int(x.shape[0])
        n = N if n is None else int(n)
        st = self._lib.amr_mlp_loss_grad(
            C.c_void_p(_dptr(self.params)), C.c_void_p(_dptr(x)), C.c_void_p(_dptr(t)), N,
            int(first), n, int(perm_a), int(perm_b), C.c_void_p(_dptr(self.grad)),
            C.c_void_p(_dptr(self.loss)), C.c_void_p(_dptr(self.scratch)),
            C.c_void_p(_stream_ptr(stream)))
        _check(st, None)

    def adam(self, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
             stream=None):
        self.step += 1
        st = self._lib.amr_mlp_adam(C.c_void_p(_dptr(self.params)), C.c_void_p(_dptr(self.grad)),
                                    C.c_void_p(_dptr(self.m)), C.c_void_p(_dptr(self.v)),
                                    float(lr), float(beta1), float(beta2), float(eps),
                                    self.step, C.c_void_p(_stream_ptr(stream)))
        _check(st, None)

    def train(self, x, t, epochs: int = 3, batch: int = 16384, lr: float = 2e-3, seed: int = 0,
              log_every: int = 0):
        """Adam over pseudo-randomly permuted minibatches (permutation computed in-kernel);
        returns the loss of the last minibatch of every epoch."""
        import torch

        N = int(x.shape[0])
        rng = np.random.default_rng(seed)
        losses = []
        for ep in range(epochs):
            a = int(rng.integers(1, N)) | 1
            while math.gcd(a, N) != 1:
                a += 2
            b = int(rng.integers(0, N))
            steps = (N + batch - 1) // batch
            for s in range(steps):
                first = s * batch
                n = min(batch, N - first)
                # cosine decay over the whole run
                frac = (ep * steps + s) / max(1, epochs * steps)
                self.loss_grad(x, t, first, n, a, b)
                self.adam(lr * 0.5 * (1.0 + math.cos(math.pi * frac)))
            torch.cuda.synchronize()
            losses.append(float(self.loss.item()))
        return losses

    def save(self, path: str) -> None:
        """Checkpoint: FP32 parameters, Adam moments and step count (.npz)."""
        np.savez(path, params=self.params.cpu().numpy(), m=self.m.cpu().numpy(),
                 v=self.v.cpu().numpy(), step=np.int64(self.step))

    @classmethod
    def load(cls, path: str) -> "Proposal":
        """Resume from a checkpoint written by save()."""
        import torch

        z = np.load(path)
        prop = cls(z["params"])
        prop.m.copy_(torch.as_tensor(z["m"]))
        prop.v.copy_(torch.as_tensor(z["v"]))
        prop.step = int(z["step"])
        return prop

    def pack(self, stream=None):
        _check(self._lib.amr_mlp_pack(C.c_void_p(_dptr(self.params)), C.c_void_p(_dptr(self.packed)),
                                      C.c_void_p(_stream_ptr(stream))), None)
        return self.packed

    def predict(self, x, stream=None):
        import torch

        self.pack(stream)
        y = torch.empty((int(x.shape[0]),), dtype=torch.float32, device="cuda")
        _check(self._lib.amr_mlp_forward(C.c_void_p(_dptr(self.packed)), C.c_void_p(_dptr(x)),
                                         int(x.shape[0]), C.c_void_p(_dptr(y)),
                                         C.c_void_p(_stream_ptr(stream))), None)
        return y

    def install(self, ctx, stream=None):
        """Pack the current parameters and install them in a rendering context."""
        self.pack(stream)
        _check(self._lib.amr_set_proposal(ctx._h, C.c_void_p(_dptr(self.packed)),
                                          C.c_void_p(_stream_ptr(stream))), ctx._h)


def psnr(img, ref) -> float:
    """10 log10(1 / MSE) over all channels of two images in [0, 1] (torch tensors)."""
    mse = float(((img.double() - ref.double()) ** 2).mean().item())
    return float("inf") if mse == 0.0 else 10.0 * math.log10(1.0 / mse)


__all__ = ["Proposal", "init_params", "split_params", "log_segments", "psnr", "AmrError"]
