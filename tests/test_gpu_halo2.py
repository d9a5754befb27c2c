"""GPU parity of the two-cell-halo layout (AMR_STORE_HALO2): bricks with two halo layers
and leaf faces onto the same level marked, so gradient neighbours up to one cell beyond
such a face read the sample's own brick (Sec. 4: gradients across block boundaries).  The
images must match the FP64 oracle within the usual tolerance for every storage, with and
without gradient bricks, under pruning, on ragged random hierarchies and on the bench
hierarchy; the per-ray and deferred schedules stay bit-identical to each other."""
import numpy as np
import pytest

import oracle
import synth
from synth.amr import random_hierarchy
from gpu_util import assert_image_close, gpu_render, params_pair

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


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("gradient", [False, True])
def test_halo2_c1_images(amr, c1, storage, gradient):
    w, o = c1
    ctx = amr.from_hierarchy(w["hier"])
    ctx.amr_build_kdtree(storage, gradient=gradient, halo=2)
    for shade, interp in ((0, 1), (1, 1), (1, 0)):
        if gradient and interp == 0:
            continue
        p, op = params_pair(amr, w["vmin"], w["vmax"], shade=shade, interp=interp, schedule=0)
        img, n = gpu_render(ctx, w["camera"], w["tf"], p)
        ref, smp = o.render(w["camera"], w["tf"], op)
        assert_image_close(img, ref, what=f"halo2 {storage} grad={gradient} shade={shade} "
                                          f"interp={interp}")
        assert abs(int(n) - int(smp.sum())) <= 0.001 * smp.sum()
    # the one-cell layout renders the same image up to rounding
    ctx1 = amr.from_hierarchy(w["hier"])
    ctx1.amr_build_kdtree(storage, gradient=gradient)
    p, _ = params_pair(amr, w["vmin"], w["vmax"], shade=1, schedule=0)
    a, _ = gpu_render(ctx, w["camera"], w["tf"], p)
    b, _ = gpu_render(ctx1, w["camera"], w["tf"], p)
    assert np.max(np.abs(a - b)) < 2e-5


@pytest.mark.parametrize("seed", [0, 1, 2, 3, 4, 5])
def test_halo2_random_hierarchies(amr, seed):
    rng = np.random.default_rng(seed)
    h = random_hierarchy(seed, n0=8, num_levels=3, patches_per_level=6, max_size=12, tiles=4)
    o = oracle.Oracle(h)
    W, H = int(rng.integers(9, 61)), int(rng.integers(9, 61))
    cam = synth.orbit_camera(200 + seed, W, H)
    tf = synth.ramp_tf()
    vmin, vmax = h.value_range()
    storage = STORAGES[seed % 4]
    ctx = amr.from_hierarchy(h)
    ctx.amr_build_kdtree(storage, gradient=storage in ("ptr", "atlas_linear"), halo=2)
    imgs = {}
    for schedule in (0, 3):
        p, op = params_pair(amr, vmin, vmax, shade=1, kappa=20.0, schedule=schedule)
        imgs[schedule], _ = gpu_render(ctx, cam, tf, p)
        ref, _ = o.render(cam, tf, op)
        assert_image_close(imgs[schedule], ref, what=f"halo2 seed {seed} sched {schedule}")
    assert np.array_equal(imgs[0], imgs[3])


@pytest.mark.parametrize("lod", [1.0, 3.0])
def test_halo2_pruned_c1(amr, c1, lod):
    w, o = c1
    ctx = amr.from_hierarchy(w["hier"])
    ctx.amr_build_kdtree("ptr", gradient=True, halo=2)
    p, op = params_pair(amr, w["vmin"], w["vmax"], shade=1, lod_pixels=lod)
    img, _ = gpu_render(ctx, w["camera"], w["tf"], p)
    ref, _ = o.render(w["camera"], w["tf"], op)
    assert_image_close(img, ref, what=f"halo2 lod {lod}")


@pytest.fixture(scope="module")
def c2():
    h = synth.make_c2(device="cuda")
    vmin, vmax = synth.amr.percentile_range(h)
    return h, vmin, vmax, oracle.Oracle(h)


@pytest.mark.parametrize("size,schedule", [(2048, 0), (1024, 3)])
def test_halo2_c2_sampled(amr, c2, size, schedule):
    h, vmin, vmax, o = c2
    ctx = amr.from_hierarchy(h)
    ctx.amr_build_kdtree("ptr", gradient=True, halo=2)
    cam = synth.orbit_camera(2, size, size)
    tf = synth.ramp_tf()
    p, op = params_pair(amr, vmin, vmax, shade=1, schedule=schedule)
    img, n = gpu_render(ctx, cam, tf, p)
    rng = np.random.default_rng(size + 7)
    pix = np.concatenate([np.stack([rng.integers(0, size, 900), rng.integers(0, size, 900)], 1),
                          np.stack([np.arange(size), np.full(size, size // 2)], 1)]).astype(np.int32)
    ref, _ = o.render(cam, tf, op, pixels=pix)
    assert_image_close(img[pix[:, 1], pix[:, 0]], ref, what=f"halo2 c2 {size}")
    assert n > 0
