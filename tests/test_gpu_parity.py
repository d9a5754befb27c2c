"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the same seeded
inputs.  Leaf boxes, leaf ids and per-pixel traversal sequences must match bit for bit;
images within max-abs 5e-4 and mean-abs 1e-5 per RGBA channel (FP32 kernel vs FP64)."""
import numpy as np
import pytest

import oracle
import synth
from synth.amr import look_camera, random_hierarchy
from gpu_util import assert_image_close, gpu_render, gpu_trace, params_pair

pytestmark = pytest.mark.gpu

STORAGES = ["ptr", "texobj", "atlas_linear", "atlas_tex3d"]


@pytest.fixture(scope="module")
def amr():
    import paper_1212_3333_gb300 as m

    return m


@pytest.fixture(scope="module")
def c1():
    w = synth.c1_workload()
    return w, oracle.Oracle(w["hier"])


@pytest.fixture(scope="module")
def c1_ctx(amr, c1):
    ctxs = {}
    for st in STORAGES:
        ctx = amr.from_hierarchy(c1[0]["hier"])
        ctx.amr_build_kdtree(st)
        ctxs[st] = ctx
    return ctxs


def test_trace_c1_bit_exact(c1, c1_ctx):
    w, o = c1
    cam = w["camera"]
    ctx = c1_ctx["ptr"]
    seq, tseq, ln = gpu_trace(ctx, cam, max_len=512)
    # leaves themselves are bit-identical too
    b, p, lv = ctx.amr_get_leaves()
    ob, op, olv = o.leaves()
    np.testing.assert_array_equal(b, ob)
    np.testing.assert_array_equal(p, op)
    np.testing.assert_array_equal(lv, olv)
    hits = 0
    for j in range(cam.height):
        for i in range(cam.width):
            q = j * cam.width + i
            leaf, t0, t1 = o.trace(cam, i, j)
            assert ln[q] == len(leaf), (i, j)
            if len(leaf):
                hits += 1
                np.testing.assert_array_equal(seq[q, :len(leaf)], leaf)
                assert np.array_equal(tseq[q, :len(leaf), 0], t0), (i, j)
                assert np.array_equal(tseq[q, :len(leaf), 1], t1), (i, j)
    assert hits > 20000


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("shade", [0, 1])
@pytest.mark.parametrize("interp", [1, 0])
@pytest.mark.parametrize("schedule", [0, 1])
def test_image_c1(amr, c1, c1_ctx, storage, shade, interp, schedule):
    w, o = c1
    p, op = params_pair(amr, w["vmin"], w["vmax"], shade=shade, interp=interp, schedule=schedule)
    img, n = gpu_render(c1_ctx[storage], w["camera"], w["tf"], p)
    ref, smp = o.render(w["camera"], w["tf"], op)
    assert_image_close(img, ref, what=f"{storage} shade={shade} interp={interp} sched={schedule}")
    assert abs(int(n) - int(smp.sum())) <= 0.001 * smp.sum()


@pytest.fixture(scope="module")
def c1_gctx(amr, c1):
    """C1 with gradient bricks (float4 value + central differences per cell)."""
    ctxs = {}
    for st in STORAGES:
        ctx = amr.from_hierarchy(c1[0]["hier"])
        ctx.amr_build_kdtree(st, gradient=True)
        ctxs[st] = ctx
    return ctxs


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("schedule", [0, 1])
def test_image_c1_gradient_bricks(amr, c1, c1_ctx, c1_gctx, storage, schedule):
    w, o = c1
    p, op = params_pair(amr, w["vmin"], w["vmax"], shade=1, schedule=schedule)
    img, n = gpu_render(c1_gctx[storage], w["camera"], w["tf"], p)
    ref, smp = o.render(w["camera"], w["tf"], op)
    assert_image_close(img, ref, what=f"gradient bricks {storage} sched={schedule}")
    plain, n2 = gpu_render(c1_ctx[storage], w["camera"], w["tf"], p)
    assert np.max(np.abs(img - plain)) < 1e-5 and abs(int(n) - int(n2)) <= 0.001 * n2


@pytest.mark.parametrize("storage", ["ptr", "atlas_tex3d"])
@pytest.mark.parametrize("schedule", [0, 1])
def test_sample_count_exact_without_ert(amr, c1, c1_ctx, storage, schedule):
    w, o = c1
    p, op = params_pair(amr, w["vmin"], w["vmax"], ert_eps=0.0, shade=1, schedule=schedule)
    img, n = gpu_render(c1_ctx[storage], w["camera"], w["tf"], p)
    ref, smp = o.render(w["camera"], w["tf"], op)
    assert int(n) == int(smp.sum())
    assert_image_close(img, ref)


@pytest.mark.parametrize("seed", [0, 1, 2, 3, 4, 5])
def test_random_hierarchies_ragged_images(amr, seed):
    rng = np.random.default_rng(seed)
    h = random_hierarchy(seed, n0=8, num_levels=3, patches_per_level=6, max_size=12, tiles=4)
    o = oracle.Oracle(h)
    W, H = int(rng.integers(9, 61)), int(rng.integers(9, 61))  # ragged against 8x16 tiles
    cam = synth.orbit_camera(200 + seed, W, H)
    tf = synth.ramp_tf()
    vmin, vmax = h.value_range()
    storage = STORAGES[seed % 4]
    ctx = amr.from_hierarchy(h)
    ctx.amr_build_kdtree(storage)
    for shade in (0, 1):
        p, op = params_pair(amr, vmin, vmax, shade=shade, kappa=20.0, schedule=seed % 2)
        img, _ = gpu_render(ctx, cam, tf, p)
        ref, _ = o.render(cam, tf, op)
        assert_image_close(img, ref, what=f"seed {seed} {storage} shade {shade}")
    seq, tseq, ln = gpu_trace(ctx, cam, max_len=256)
    for j in range(H):
        for i in range(W):
            leaf, t0, t1 = o.trace(cam, i, j)
            q = j * W + i
            assert ln[q] == len(leaf)
            np.testing.assert_array_equal(seq[q, :len(leaf)], leaf)
            assert np.array_equal(tseq[q, :len(leaf), 0], t0)


def test_edge_cameras(amr, c1, c1_ctx):
    w, o = c1
    ctx = c1_ctx["ptr"]
    tf = w["tf"]
    p, op = params_pair(amr, w["vmin"], w["vmax"], shade=1)
    cams = [
        look_camera((0.5, 0.45, 0.55), (1.0, 0.9, 0.2), (0, 0, 1), 70.0, 33, 17),   # inside
        look_camera((3.0, 3.0, 3.0), (6.0, 6.0, 6.0), (0, 0, 1), 10.0, 8, 8),       # looks away
        look_camera((0.3, 0.55, -1.0), (0.3, 0.55, 0.5), (0, 1, 0), 30.0, 9, 7),    # d_x = d_y = 0
        look_camera((-1.0, 0.5, 0.5), (0.5, 0.5, 0.5), (0, 0, 1), 45.0, 1, 1),      # one pixel
    ]
    for cam in cams:
        img, _ = gpu_render(ctx, cam, tf, p)
        ref, _ = o.render(cam, tf, op)
        assert_image_close(img, ref, what=f"camera {cam.eye}")
        seq, tseq, ln = gpu_trace(ctx, cam, max_len=512)
        for j in range(cam.height):
            for i in range(cam.width):
                leaf, t0, t1 = o.trace(cam, i, j)
                q = j * cam.width + i
                assert ln[q] == len(leaf)
                np.testing.assert_array_equal(seq[q, :len(leaf)], leaf)
    away, _ = gpu_render(ctx, cams[1], tf, p)
    assert np.all(away == 0)


@pytest.mark.parametrize("schedule", [0, 1])
def test_bands_skip_and_host_path(amr, c1, c1_ctx, schedule):
    import torch

    w, _ = c1
    ctx = c1_ctx["atlas_linear"]
    cam = w["camera"]
    p, _ = params_pair(amr, w["vmin"], w["vmax"], shade=1, schedule=schedule)
    full, n_full = gpu_render(ctx, cam, w["tf"], p)
    again, n_again = gpu_render(ctx, cam, w["tf"], p)
    assert np.array_equal(full, again) and n_full == n_again  # deterministic
    # image-space bands (the multi-GPU partition) on 4-row boundaries stitch bit for bit:
    # a warp covers 8x4 pixels, so each warp sees the same rays as in the full frame
    parts = []
    for r0, r1 in [(0, 80), (80, 200), (200, 256)]:
        pb, _ = params_pair(amr, w["vmin"], w["vmax"], shade=1, row0=r0, rows=r1 - r0,
                            schedule=schedule)
        parts.append(gpu_render(ctx, cam, w["tf"], pb)[0])
    assert np.array_equal(np.concatenate(parts, axis=0), full)
    # exact empty-space skipping removes only transparent samples (the wavefront schedule
    # may sum the remaining contributions in another order)
    ps, _ = params_pair(amr, w["vmin"], w["vmax"], shade=1, skip=1, schedule=schedule)
    skipped, n_skip = gpu_render(ctx, cam, w["tf"], ps)
    assert np.max(np.abs(skipped - full)) <= (0.0 if schedule == 0 else 2e-6)
    assert n_skip < n_full
    # host-buffer entry point
    out = np.zeros((cam.height, cam.width, 4), dtype=np.float32)
    n_host = ctx.amr_render_host(cam, np.ascontiguousarray(w["tf"]), p, out, count_samples=True)
    torch.cuda.synchronize()
    assert np.array_equal(out.astype(np.float64), full) and n_host == n_full


def test_capacity_bound_reports_status(amr, c1, c1_ctx):
    w, _ = c1
    p, _ = params_pair(amr, w["vmin"], w["vmax"], max_segments=1)
    with pytest.raises(amr.AmrError) as e:
        gpu_render(c1_ctx["ptr"], w["camera"], w["tf"], p)
    assert "CAPACITY" in str(e.value)
    # the context stays usable
    p2, _ = params_pair(amr, w["vmin"], w["vmax"])
    img, _ = gpu_render(c1_ctx["ptr"], w["camera"], w["tf"], p2)
    assert np.all(np.isfinite(img))


# ------------------------------------------------------------------ cosmology-like hierarchy

@pytest.fixture(scope="module")
def c2():
    h = synth.make_c2(device="cuda")
    vmin, vmax = synth.amr.percentile_range(h)
    return h, vmin, vmax, oracle.Oracle(h)


def _sample_pixels(W, H, n, seed):
    rng = np.random.default_rng(seed)
    pix = np.stack([rng.integers(0, W, n), rng.integers(0, H, n)], axis=1)
    row = np.stack([np.arange(W), np.full(W, H // 2)], axis=1)  # one full row too
    return np.concatenate([pix, row], axis=0).astype(np.int32)


@pytest.mark.parametrize("size,storage,schedule,gradient", [
    (1024, "ptr", 0, False), (1024, "texobj", 0, False), (1024, "atlas_linear", 0, False),
    (1024, "atlas_tex3d", 0, False), (1024, "ptr", 1, False), (1024, "atlas_linear", 0, True),
    (2048, "ptr", 0, True), (2048, "ptr", 0, False)])
def test_c2_sampled_pixels(amr, c2, size, storage, schedule, gradient):
    h, vmin, vmax, o = c2
    ctx = amr.from_hierarchy(h)
    ctx.amr_build_kdtree(storage, gradient=gradient)
    cam = synth.orbit_camera(2, size, size)
    tf = synth.ramp_tf()
    p, op = params_pair(amr, vmin, vmax, shade=1, schedule=schedule)
    img, n = gpu_render(ctx, cam, tf, p)
    pix = _sample_pixels(size, size, 1200 if size == 1024 else 800, size)
    ref, _ = o.render(cam, tf, op, pixels=pix)
    got = img[pix[:, 1], pix[:, 0]]
    assert_image_close(got, ref, what=f"c2 {size} {storage} sched {schedule}")
    assert n > 0


def test_c2_trace_sampled(amr, c2):
    import torch

    h, vmin, vmax, o = c2
    ctx = amr.from_hierarchy(h)
    ctx.amr_build_kdtree("ptr")
    b, p, lv = ctx.amr_get_leaves()
    ob, op, olv = o.leaves()
    np.testing.assert_array_equal(b, ob)
    np.testing.assert_array_equal(p, op)
    cam = synth.orbit_camera(2, 512, 512)
    seq, tseq, ln = gpu_trace(ctx, cam, max_len=1024)
    pix = _sample_pixels(512, 512, 3000, 7)
    for i, j in pix:
        leaf, t0, t1 = o.trace(cam, int(i), int(j))
        q = j * 512 + i
        assert ln[q] == len(leaf)
        np.testing.assert_array_equal(seq[q, :len(leaf)], leaf)
        assert np.array_equal(tseq[q, :len(leaf), 0], t0)
        assert np.array_equal(tseq[q, :len(leaf), 1], t1)
    del torch


def test_c2_exact_sample_total_1024_without_ert(amr, c2):
    # the bench hierarchy at 1024²: with early termination off the sample total is fixed by
    # the traversal and the per-segment counts alone, so GPU and FP64 oracle agree exactly
    h, vmin, vmax, o = c2
    ctx = amr.from_hierarchy(h)
    ctx.amr_build_kdtree("ptr")
    cam = synth.orbit_camera(2, 1024, 1024)
    tf = synth.ramp_tf()
    p, op = params_pair(amr, vmin, vmax, shade=0, ert_eps=0.0)
    _, n = gpu_render(ctx, cam, tf, p)
    _, smp = o.render(cam, tf, op)
    assert n == int(smp.sum()) and n > 10 ** 8
