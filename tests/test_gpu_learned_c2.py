"""What the trained proposal gains over the method without it, on the learned-proposal
workload: the 5-level bench hierarchy, a network trained by the library's own kernels on
segments the plain march logs from 256 seeded poses, held-out 2048² Phong views.  The
learned coarse mode must keep PSNR >= 45 dB against the plain march and take strictly
fewer samples and less time than exact min/max empty-space skipping alone."""
import numpy as np
import pytest

import synth
from gpu_util import gpu_render, params_pair

pytestmark = pytest.mark.gpu


def _psnr(a, b):
    mse = float(np.mean((a - b) ** 2))
    return np.inf if mse == 0 else 10 * np.log10(1.0 / mse)


def test_learned_coarse_beats_minmax_skipping_on_c2():
    import torch

    import paper_1212_3333_gb300 as amr
    from paper_1212_3333_gb300 import proposal

    h = synth.make_c2(device="cuda")
    vmin, vmax = synth.amr.percentile_range(h)
    ctx = amr.from_hierarchy(h)
    ctx.amr_build_kdtree("ptr", gradient=True)
    tf = torch.as_tensor(synth.ramp_tf(), device="cuda")
    p_log = amr.amr_default_params(vmin=vmin, vmax=vmax, shade=0)
    poses = [synth.orbit_camera(1000 + s, 96, 96) for s in range(256)]
    feats, tgts, seen = proposal.log_segments(ctx, poses, tf, p_log, capacity=10_000_000,
                                              keep_prob=0.3, seed=1)
    prop = proposal.Proposal(seed=0)
    prop.train(feats, tgts, epochs=3, batch=16384, lr=2e-3)
    prop.install(ctx)

    size = 2048
    out = torch.empty((size, size, 4), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def timed(cam, prm, reps=3):
        ctx.amr_render(cam, tf, prm, out)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            ctx.amr_render(cam, tf, prm, out)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    base = dict(shade=1, schedule=0)
    cfg = {"plain": {}, "minmax": {"skip": 1},
           "learned": {"skip": 1, "learned": 2, "tau": 1e-2, "coarse_factor": 16}}
    res = {k: {"ms": 0.0, "samples": 0, "psnr": np.inf} for k in cfg}
    for s in range(2):
        cam = synth.orbit_camera(2000 + s, size, size)
        plain = None
        for name, kw in cfg.items():
            prm, _ = params_pair(amr, vmin, vmax, **base, **kw)
            img, n = gpu_render(ctx, cam, synth.ramp_tf(), prm)
            if name == "plain":
                plain = img
            res[name]["samples"] += n
            res[name]["psnr"] = min(res[name]["psnr"], _psnr(img, plain))
            res[name]["ms"] += timed(cam, prm)
    print("\nlearned on c2: " + ", ".join(f"{k} {v['ms']:.1f} ms {v['samples']} samples "
                                          f"{v['psnr']:.1f} dB" for k, v in res.items()))
    assert res["minmax"]["psnr"] == np.inf  # exact skipping changes nothing
    assert res["learned"]["psnr"] >= 45.0
    assert res["learned"]["samples"] < res["minmax"]["samples"]
    assert res["learned"]["ms"] < 0.9 * res["minmax"]["ms"], res
