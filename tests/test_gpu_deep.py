"""Deep 8-level hierarchy (finest spacing 1/16384, the depth of the deep configuration) at
about 1e8 cells, which generates in seconds: the levels where FP32 positions no longer
resolve a cell, so the kernel's FP64 fallbacks decide descents, sample counts and sample
positions.  Checked against the FP64 oracle: traversal bit for bit on sampled pixels,
exact sample totals with early termination off, and sampled pixels of a 2048² Phong view
with FP32, FP16 and BF16 cells (FP32 within the image tolerance; 16-bit cells by PSNR and
max-abs against the FP64 image of the original cells)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_image_close, gpu_render, gpu_trace, params_pair

pytestmark = pytest.mark.gpu

PSNR_MIN = {"f16": 70.0, "bf16": 50.0}


@pytest.fixture(scope="module")
def deep():
    import paper_1212_3333_gb300 as amr

    h = synth.amr.make_deep(device="cuda")
    # transfer-function range from the level-0 cells, which cover the domain once: the
    # deep levels refine the densest regions, so their values sit at the opaque top of the
    # ramp (a range over all cells, most of them deep, leaves the view nearly transparent)
    lvl0 = np.concatenate([d.ravel() for d, l in zip(h.data, h.patch_level) if l == 0])
    vmin, vmax = float(lvl0.min()), float(np.percentile(lvl0, 99.9))
    print(f"\ndeep: {h.num_patches} patches {h.patches_per_level()}, {h.n_cells():.3e} cells")
    ctx = amr.from_hierarchy(h)
    ctx.amr_build_kdtree("ptr", gradient=True)
    return amr, h, vmin, vmax, oracle.Oracle(h), ctx


def test_deep_hierarchy_shape(deep):
    amr, h, vmin, vmax, o, ctx = deep
    assert h.num_levels == 8
    assert all(n > 0 for n in h.patches_per_level())
    np.testing.assert_allclose(h.h0 / 2 ** 7, 1.0 / 16384, rtol=0, atol=0)
    b, p, lv = ctx.amr_get_leaves()
    ob, op, olv = o.leaves()
    np.testing.assert_array_equal(b, ob)
    np.testing.assert_array_equal(p, op)
    np.testing.assert_array_equal(lv, olv)
    assert lv.max() == 7


def test_deep_trace_sampled_bit_exact(deep):
    amr, h, vmin, vmax, o, ctx = deep
    W = 256
    cam = synth.orbit_camera(3, W, W)
    seq, tseq, ln = gpu_trace(ctx, cam, max_len=2048)
    rng = np.random.default_rng(30)
    pix = np.stack([rng.integers(0, W, 2000), rng.integers(0, W, 2000)], 1)
    olv = o.leaves()[2]
    deepest = 0
    for i, j in pix:
        leaf, t0, t1 = o.trace(cam, int(i), int(j))
        q = j * W + i
        assert ln[q] == len(leaf), (i, j)
        np.testing.assert_array_equal(seq[q, :len(leaf)], leaf)
        assert np.array_equal(tseq[q, :len(leaf), 0], t0), (i, j)
        assert np.array_equal(tseq[q, :len(leaf), 1], t1), (i, j)
        if len(leaf):
            deepest = max(deepest, int(olv[leaf].max()))
    assert deepest >= 6  # the sample reaches the deep levels


def test_deep_exact_sample_total_without_ert(deep):
    amr, h, vmin, vmax, o, ctx = deep
    cam = synth.orbit_camera(3, 192, 160)
    tf = synth.ramp_tf()
    p, op = params_pair(amr, vmin, vmax, shade=0, ert_eps=0.0)
    _, n = gpu_render(ctx, cam, tf, p)
    _, smp = o.render(cam, tf, op)
    assert n == int(smp.sum())


def test_deep_sampled_pixels_per_cell_type(deep):
    amr, h, vmin, vmax, o, ctx32 = deep
    cam = synth.orbit_camera(3, 2048, 2048)
    tf = synth.ramp_tf()
    p, op = params_pair(amr, vmin, vmax, shade=1)
    rng = np.random.default_rng(33)
    pix = np.concatenate([np.stack([rng.integers(0, 2048, 1200), rng.integers(0, 2048, 1200)], 1),
                          np.stack([np.arange(2048), np.full(2048, 1024)], 1)]).astype(np.int32)
    ref, _ = o.render(cam, tf, op, pixels=pix)
    res = {}
    for dtype in ("f32", "f16", "bf16"):
        ctx = ctx32 if dtype == "f32" else amr.from_hierarchy(h, dtype)
        if dtype != "f32":
            ctx.amr_build_kdtree("ptr", gradient=True)
        img, n = gpu_render(ctx, cam, tf, p)
        exact = list(ctx.amr_get_stats().exact_paths)
        got = img[pix[:, 1], pix[:, 0]]
        mse = float(np.mean((got - ref) ** 2))
        res[dtype] = (10 * np.log10(1 / mse) if mse > 0 else np.inf,
                      float(np.abs(got - ref).max()), n, exact)
        if dtype == "f32":
            assert_image_close(got, ref, what="deep f32")
        else:
            ctx.amr_destroy()
    print("deep 2048 sampled: " + "; ".join(
        f"{k} PSNR {v[0]:.1f} dB max-abs {v[1]:.2e} samples {v[2]} "
        f"fp64 fallbacks (descent, count, position) {v[3]}" for k, v in res.items()))
    assert ref[:, 3].max() > 0.3  # the view sees the volume
    for dtype, lim in PSNR_MIN.items():
        assert res[dtype][0] >= lim, (dtype, res[dtype])
    assert res["f16"][2] > 0 and res["bf16"][2] > 0
