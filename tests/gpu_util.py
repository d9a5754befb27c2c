"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and the FP64
oracle on the same seeded inputs with the same parameters."""
import numpy as np

import oracle

TOL_MAX = 5e-4   # per RGBA channel on [0, 1]
TOL_MEAN = 1e-5


def params_pair(amr, vmin, vmax, **kw):
    """Matching product and oracle parameter blocks."""
    p = amr.amr_default_params(vmin=float(vmin), vmax=float(vmax))
    for k, v in kw.items():
        setattr(p, k, v)
    o = oracle.OracleParams(vmin=float(vmin), vmax=float(vmax), step_factor=p.step_factor,
                            kappa=p.kappa, ert_eps=p.ert_eps, interp=p.interp, shade=p.shade,
                            ka=p.ka, kd=p.kd, ks=p.ks, shininess=p.shininess, gamma=p.gamma,
                            lod_pixels=p.lod_pixels, shadow=p.shadow, light=tuple(p.light),
                            light_step=p.light_step, light_ambient=p.light_ambient)
    return p, o


def gpu_render(ctx, cam, tf, p, count_samples=True):
    import torch

    tf_d = torch.as_tensor(np.ascontiguousarray(tf, dtype=np.float32), device="cuda")
    rows = cam.height - p.row0 if p.rows <= 0 else min(p.rows, cam.height - p.row0)
    out = torch.full((rows, cam.width, 4), float("nan"), dtype=torch.float32, device="cuda")
    n = ctx.amr_render(cam, tf_d, p, out, count_samples=count_samples)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64), n


def gpu_trace(ctx, cam, max_len=4096, lod_pixels=0.0):
    import torch

    npx = cam.width * cam.height
    seq = torch.full((npx * max_len,), -7, dtype=torch.int32, device="cuda")
    tseq = torch.zeros((npx * max_len * 2,), dtype=torch.float64, device="cuda")
    ln = torch.full((npx,), -7, dtype=torch.int32, device="cuda")
    ctx.amr_trace(cam, seq, ln, max_len, t_seq=tseq, lod_pixels=lod_pixels)
    torch.cuda.synchronize()
    return (seq.cpu().numpy().reshape(npx, max_len), tseq.cpu().numpy().reshape(npx, max_len, 2),
            ln.cpu().numpy())


def assert_image_close(got, want, tol_max=TOL_MAX, tol_mean=TOL_MEAN, what=""):
    assert got.shape == want.shape
    assert np.all(np.isfinite(got)), f"{what}: non-finite output"
    d = np.abs(got - want)
    mx = d.reshape(-1, 4).max(axis=0)
    mean = d.reshape(-1, 4).mean(axis=0)
    assert np.all(mx <= tol_max), f"{what}: max-abs per channel {mx}"
    assert np.all(mean <= tol_mean), f"{what}: mean-abs per channel {mean}"
    return mx, mean
