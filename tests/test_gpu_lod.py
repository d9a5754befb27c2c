"""GPU parity of level-of-detail pruning (Sec. 3.1 type-(a) nodes, Sec. 3.3): the pruned
traversal (leaf and pruned-node ids, entry and exit parameters) bit-exact against the FP64
oracle, images within the usual tolerance for every storage and schedule, the extreme
threshold equal to the level-0 hierarchy, batched views equal to single renders."""
import dataclasses

import numpy as np
import pytest

import oracle
import synth
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


def _mid_lod(h, cam, level=0):
    """Threshold that puts X(t) = hmin^level near the middle of the volume's depth."""
    hmin = float(np.min(h.h0) / h.ratio ** level)
    t_mid = float(np.linalg.norm(np.asarray(cam.eye) - 0.5))
    return hmin / (2.0 * cam.tan_half_fov_y / cam.height * t_mid)


def test_pruned_trace_bit_exact_c1(amr, c1):
    w, o = c1
    ctx = amr.from_hierarchy(w["hier"])
    ctx.amr_build_kdtree("ptr")
    cam = synth.orbit_camera(4, 96, 80)
    lod = _mid_lod(w["hier"], cam)
    seq, tseq, ln = gpu_trace(ctx, cam, max_len=512, lod_pixels=lod)
    M = o.num_leaves
    pruned = 0
    for j in range(cam.height):
        for i in range(cam.width):
            leaf, t0, t1 = o.trace(cam, i, j, lod_pixels=lod)
            q = j * cam.width + i
            assert ln[q] == len(leaf), (i, j)
            if len(leaf):
                np.testing.assert_array_equal(seq[q, :len(leaf)], leaf)
                assert np.array_equal(tseq[q, :len(leaf), 0], t0)
                assert np.array_equal(tseq[q, :len(leaf), 1], t1)
                pruned += int((leaf >= M).sum())
    assert pruned > 100


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("gradient", [False, True])
def test_pruned_images_c1(amr, c1, storage, gradient):
    w, o = c1
    ctx = amr.from_hierarchy(w["hier"])
    ctx.amr_build_kdtree(storage, gradient=gradient)
    cam = synth.orbit_camera(4, 96, 80)
    lod = _mid_lod(w["hier"], cam)
    for shade in (0, 1):
        p, op = params_pair(amr, w["vmin"], w["vmax"], shade=shade, lod_pixels=lod)
        img, n = gpu_render(ctx, cam, w["tf"], p)
        ref, smp = o.render(cam, w["tf"], op)
        assert_image_close(img, ref, what=f"lod {storage} grad={gradient} shade={shade}")
        assert abs(int(n) - int(smp.sum())) <= 0.001 * smp.sum()
        p2, _ = params_pair(amr, w["vmin"], w["vmax"], shade=shade, lod_pixels=lod, schedule=2)
        img2, n2 = gpu_render(ctx, cam, w["tf"], p2)
        assert np.array_equal(img, img2) and n == n2
        pf, _ = params_pair(amr, w["vmin"], w["vmax"], shade=shade)
        _, nf = gpu_render(ctx, cam, w["tf"], pf)
        assert n < nf


def test_huge_threshold_equals_level_zero_hierarchy(amr, c1):
    w, _ = c1
    h = w["hier"]
    keep = h.patch_level == 0
    h0 = dataclasses.replace(h, patch_level=h.patch_level[keep], patch_box=h.patch_box[keep],
                             data=[d for d, k in zip(h.data, keep) if k])
    a_ctx = amr.from_hierarchy(h)
    a_ctx.amr_build_kdtree("ptr")
    b_ctx = amr.from_hierarchy(h0)
    b_ctx.amr_build_kdtree("ptr")
    for shade in (0, 1):
        p, _ = params_pair(amr, w["vmin"], w["vmax"], shade=shade, lod_pixels=1e9, ert_eps=0.0)
        pb, _ = params_pair(amr, w["vmin"], w["vmax"], shade=shade, ert_eps=0.0)
        a, na = gpu_render(a_ctx, w["camera"], w["tf"], p)
        b, nb = gpu_render(b_ctx, w["camera"], w["tf"], pb)
        assert na == nb
        assert_image_close(a, b, tol_max=1e-6, tol_mean=1e-8, what=f"level 0 shade={shade}")


def test_pruned_batch_equals_single(amr, c1):
    import torch

    w, _ = c1
    ctx = amr.from_hierarchy(w["hier"])
    ctx.amr_build_kdtree("ptr", gradient=True)
    tfs_h = synth.tf_variants()
    cams = [synth.orbit_camera(30 + v, 40 + 9 * v, 36 + 7 * v) for v in range(5)]
    tfi = [v % 4 for v in range(5)]
    p, _ = params_pair(amr, w["vmin"], w["vmax"], shade=1, lod_pixels=2.0)
    views, offsets, total = amr.make_views(cams, tfi)
    out = torch.zeros((total,), device="cuda")
    ctx.amr_render_batch(views, torch.as_tensor(np.stack(tfs_h), device="cuda"), p, out)
    torch.cuda.synchronize()
    o = out.cpu().numpy().astype(np.float64)
    for cam, t, off in zip(cams, tfi, offsets):
        single, _ = gpu_render(ctx, cam, tfs_h[t], p)
        got = o[off:off + 4 * cam.width * cam.height].reshape(cam.height, cam.width, 4)
        assert np.array_equal(got, single)


def test_pruning_rejections(amr, c1):
    from paper_1212_3333_gb300 import _lib, proposal

    w, _ = c1
    ctx = amr.from_hierarchy(w["hier"])
    ctx.amr_build_kdtree("ptr")
    proposal.Proposal(seed=1).install(ctx)
    for kw in (dict(lod_pixels=-1.0), dict(lod_pixels=float("nan")),
               dict(lod_pixels=2.0, schedule=1), dict(lod_pixels=2.0, learned=1)):
        p, _ = params_pair(amr, w["vmin"], w["vmax"], **kw)
        with pytest.raises(amr.AmrError) as e:
            gpu_render(ctx, w["camera"], w["tf"], p)
        assert e.value.status == _lib.AMR_ERR_ARG, kw


@pytest.fixture(scope="module")
def c2():
    h = synth.make_c2(device="cuda")
    vmin, vmax = synth.amr.percentile_range(h)
    return h, vmin, vmax, oracle.Oracle(h)


@pytest.mark.parametrize("lod", [1.0, 4.0])
def test_pruned_c2_sampled(amr, c2, lod):
    h, vmin, vmax, o = c2
    ctx = amr.from_hierarchy(h)
    ctx.amr_build_kdtree("ptr", gradient=True)
    cam = synth.orbit_camera(2, 1024, 1024)
    tf = synth.ramp_tf()
    p, op = params_pair(amr, vmin, vmax, shade=1, lod_pixels=lod)
    img, n = gpu_render(ctx, cam, tf, p)
    pf, _ = params_pair(amr, vmin, vmax, shade=1)
    full, nf = gpu_render(ctx, cam, tf, pf)
    rng = np.random.default_rng(5)
    pix = np.stack([rng.integers(0, 1024, 800), rng.integers(0, 1024, 800)], 1).astype(np.int32)
    ref, _ = o.render(cam, tf, op, pixels=pix)
    assert_image_close(img[pix[:, 1], pix[:, 0]], ref, what=f"c2 lod {lod}")
    mse = float(np.mean((img - full) ** 2))
    print(f"\nc2 1024 lod {lod}: samples {n / nf:.3f} of full, PSNR vs full "
          f"{10 * np.log10(1 / mse) if mse > 0 else np.inf:.1f} dB")
    assert n < nf
    # traversal on sampled pixels
    seq, tseq, ln = gpu_trace(ctx, synth.orbit_camera(2, 256, 256), max_len=2048, lod_pixels=lod)
    cam2 = synth.orbit_camera(2, 256, 256)
    for i, j in pix[:200] // 4:
        leaf, t0, t1 = o.trace(cam2, int(i), int(j), lod_pixels=lod)
        q = j * 256 + i
        assert ln[q] == len(leaf)
        if len(leaf):
            np.testing.assert_array_equal(seq[q, :len(leaf)], leaf)
            assert np.array_equal(tseq[q, :len(leaf), 0], t0)


def test_pruned_16bit_cells(amr, c1):
    """Pruning with FP16 cells: the pruned traversal is the FP32 one (it depends on the
    geometry only), and the image stays close to the FP32-cell pruned image."""
    w, o = c1
    cam = synth.orbit_camera(4, 96, 80)
    lod = _mid_lod(w["hier"], cam)
    c32 = amr.from_hierarchy(w["hier"])
    c32.amr_build_kdtree("ptr", gradient=True)
    c16 = amr.from_hierarchy(w["hier"], "f16")
    c16.amr_build_kdtree("ptr", gradient=True)
    p, _ = params_pair(amr, w["vmin"], w["vmax"], shade=1, lod_pixels=lod, ert_eps=0.0)
    a, na = gpu_render(c32, cam, w["tf"], p)
    b, nb = gpu_render(c16, cam, w["tf"], p)
    assert na == nb
    assert np.abs(a - b).max() < 2e-3
    s32 = gpu_trace(c32, cam, max_len=512, lod_pixels=lod)
    s16 = gpu_trace(c16, cam, max_len=512, lod_pixels=lod)
    for x, y in zip(s32, s16):
        assert np.array_equal(x, y)
