"""GPU checks of batched multi-view rendering: every view of a persistent batched launch
equals its own single-view render bit for bit (same per-pixel arithmetic), for every tile
shape and rays-per-thread setting, with the per-ray loop or deferred shading; a CUDA-graph
replay of the call gives the same images; the autotuner's choice is kept; malformed
batches are rejected before any launch."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_image_close, gpu_render, params_pair

pytestmark = pytest.mark.gpu

SHAPES = [(8, 8), (16, 8), (16, 16)]


@pytest.fixture(scope="module")
def amr():
    import paper_1212_3333_gb300 as m

    return m


@pytest.fixture(scope="module")
def c1():
    return synth.c1_workload()


def _views(n, seed, lo=17, hi=130):
    rng = np.random.default_rng(seed)
    cams, tfi = [], []
    for v in range(n):
        w, h = int(rng.integers(lo, hi)), int(rng.integers(lo, hi))
        cams.append(synth.orbit_camera(100 + v, w, h))
        tfi.append(int(rng.integers(0, 4)))
    return cams, tfi


def _singles(amr, ctx, cams, tfi, tfs_h, p):
    imgs, total = [], 0
    for cam, t in zip(cams, tfi):
        img, n = gpu_render(ctx, cam, tfs_h[t], p)
        imgs.append(img)
        total += n
    return imgs, total


def _split(out, cams, offsets):
    o = out.cpu().numpy().astype(np.float64)
    return [o[off:off + 4 * c.width * c.height].reshape(c.height, c.width, 4)
            for c, off in zip(cams, offsets)]


@pytest.mark.parametrize("gradient", [False, True])
@pytest.mark.parametrize("shade,schedule", [(0, 0), (1, 0), (1, 3)])
def test_batch_equals_single_view_renders(amr, c1, gradient, shade, schedule):
    import torch

    w = c1
    ctx = amr.from_hierarchy(w["hier"])
    ctx.amr_build_kdtree("ptr", gradient=gradient)
    tfs_h = synth.tf_variants()
    tfs = torch.as_tensor(np.stack(tfs_h), device="cuda")
    cams, tfi = _views(11, 5 + shade)
    p, _ = params_pair(amr, w["vmin"], w["vmax"], shade=shade)
    # schedule 3 (deferred shading) gives the per-ray loop's images bit for bit
    pb, _ = params_pair(amr, w["vmin"], w["vmax"], shade=shade, schedule=schedule)
    want, n_want = _singles(amr, ctx, cams, tfi, tfs_h, p)
    views, offsets, total = amr.make_views(cams, tfi)
    for tw, th in SHAPES:
        for rpt in (1, 2, 4):
            out = torch.full((total + 8,), float("nan"), device="cuda")
            n = ctx.amr_render_batch(views, tfs, pb, out, config=amr.batch_config(tw, th, rpt),
                                     count_samples=True)
            assert n == n_want, (tw, th, rpt)
            for v, img in enumerate(_split(out, cams, offsets)):
                assert np.array_equal(img, want[v]), (tw, th, rpt, v)
            assert torch.isnan(out[total:]).all()  # nothing written past the images


def test_batch_view_against_oracle(amr, c1):
    import torch

    w = c1
    ctx = amr.from_hierarchy(w["hier"])
    ctx.amr_build_kdtree("ptr", gradient=True)
    tfs_h = synth.tf_variants()
    cams, tfi = _views(3, 9, lo=40, hi=80)
    p, op = params_pair(amr, w["vmin"], w["vmax"], shade=1)
    views, offsets, total = amr.make_views(cams, tfi)
    out = torch.empty((total,), device="cuda")
    ctx.amr_render_batch(views, torch.as_tensor(np.stack(tfs_h), device="cuda"), p, out)
    torch.cuda.synchronize()
    o = oracle.Oracle(w["hier"])
    for v, img in enumerate(_split(out, cams, offsets)):
        ref, _ = o.render(cams[v], tfs_h[tfi[v]], op)
        assert_image_close(img, ref, what=f"batch view {v}")


def test_batch_graph_replay_and_autotune(amr, c1):
    import torch

    w = c1
    ctx = amr.from_hierarchy(w["hier"])
    ctx.amr_build_kdtree("ptr", gradient=True)
    tfs_h = synth.tf_variants()
    tfs = torch.as_tensor(np.stack(tfs_h), device="cuda")
    cams, tfi = _views(20, 11, lo=30, hi=200)
    p, _ = params_pair(amr, w["vmin"], w["vmax"], shade=1)
    views, offsets, total = amr.make_views(cams, tfi)
    out = torch.zeros((total,), device="cuda")
    # the default schedule (AMR_SCHEDULE_AUTO) renders Phong batches with deferred shading,
    # so the autotuner also searches samples per iteration on the best tile
    best, ms = ctx.amr_batch_autotune(views, tfs, p, out, reps=2)
    assert len(ms) == 13 and all(m > 0 for m in ms)
    assert (best.tile_w, best.tile_h) in SHAPES and best.rays_per_thread in (1, 2, 4)
    k = int(np.argmin(ms))
    if k < 9:
        assert best.samples_per_iter == 0
        assert k == SHAPES.index((best.tile_w, best.tile_h)) * 3 + (1, 2, 4).index(best.rays_per_thread)
    else:
        assert best.samples_per_iter == (4, 8, 16, 32)[k - 9]
    # the per-ray schedule has no samples-per-iteration knob
    p0, _ = params_pair(amr, w["vmin"], w["vmax"], shade=1, schedule=0)
    _, ms0 = ctx.amr_batch_autotune(views, tfs, p0, out, reps=1)
    assert all(m > 0 for m in ms0[:9]) and all(m == -1.0 for m in ms0[9:])
    ctx.amr_batch_autotune(views, tfs, p, out, reps=2)  # keep the deferred choice
    n_ref = ctx.amr_render_batch(views, tfs, p, out, count_samples=True)  # autotuned config
    ref = out.clone()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        ctx.amr_render_batch(views, tfs, p, out, stream=s)  # warm-up before capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
        ctx.amr_render_batch(views, tfs, p, out, stream=s)
    out.zero_()
    torch.cuda.synchronize()
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    assert ctx.amr_get_stats() is not None and n_ref > 0


def test_batch_rejects_malformed_batches(amr, c1):
    import torch

    from paper_1212_3333_gb300 import _lib

    w = c1
    ctx = amr.from_hierarchy(w["hier"])
    ctx.amr_build_kdtree("ptr")
    tfs = torch.as_tensor(np.stack(synth.tf_variants()), device="cuda")
    cams, tfi = _views(4, 3)
    p, _ = params_pair(amr, w["vmin"], w["vmax"])
    views, offsets, total = amr.make_views(cams, tfi)
    out = torch.zeros((total,), device="cuda")

    def rejects(v=views, o=out, cfg=None, prm=p, c=ctx):
        with pytest.raises(amr.AmrError) as e:
            c.amr_render_batch(v, tfs, prm, o, config=cfg)
        assert e.value.status == _lib.AMR_ERR_ARG

    rejects(o=out[: total - 4])                       # last image past the buffer
    v2, _, _ = amr.make_views(cams, tfi)
    v2[1].out_offset = v2[0].out_offset + 4           # overlapping images
    rejects(v=v2)
    v3, _, _ = amr.make_views(cams, tfi)
    v3[2].out_offset += 2                             # not 16-byte aligned
    rejects(v=v3)
    v4, _, _ = amr.make_views(cams, [0, 1, 2, 9])     # no such transfer function
    rejects(v=v4)
    rejects(cfg=amr.batch_config(32, 8, 1))           # unsupported tile
    rejects(cfg=amr.batch_config(16, 8, 0))
    rejects(cfg=amr.batch_config(16, 8, 1, 0, 65))    # samples per iteration beyond 64
    big, _, tot = amr.make_views([cams[0]] * 129, [0] * 129)
    rejects(v=big, o=torch.zeros((tot,), device="cuda"))
    p2, _ = params_pair(amr, w["vmin"], w["vmax"], row0=3)
    rejects(prm=p2)
    tex = amr.from_hierarchy(w["hier"])
    tex.amr_build_kdtree("texobj")
    rejects(c=tex)
    # the context still renders after the rejections
    n = ctx.amr_render_batch(views, tfs, p, out, count_samples=True)
    assert n > 0
