"""GPU checks of the stencil-maximum bricks (AMR_STORE_MAXBRICK): a sample whose eight
stencil cells' maximum maps to zero opacity is decided by one load instead of eight.  The
test is exact, so images and sample counts must equal those rendered without the bricks
bit for bit - per-ray and deferred schedules, unshaded and Phong, with gradient bricks,
FP32 and 16-bit cells, both halos, ragged random hierarchies, ERT on and off, pruning - and
match the FP64 oracle."""
import numpy as np
import pytest

import oracle
import synth
from synth.amr import random_hierarchy
from gpu_util import assert_image_close, gpu_render, params_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amr():
    import paper_1212_3333_gb300 as m

    return m


@pytest.fixture(scope="module")
def c1():
    w = synth.c1_workload()
    return w, oracle.Oracle(w["hier"])


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("gradient,halo", [(False, 1), (True, 1), (True, 2)])
def test_maxbrick_images_bit_identical_c1(amr, c1, dtype, gradient, halo):
    w, o = c1
    a = amr.from_hierarchy(w["hier"], dtype)
    a.amr_build_kdtree("ptr", gradient=gradient, halo=halo)
    b = amr.from_hierarchy(w["hier"], dtype)
    b.amr_build_kdtree("ptr", gradient=gradient, halo=halo, maxbrick=True)
    for shade, schedule, ert, lod in ((0, 0, 1e-4, 0.0), (1, 0, 1e-4, 0.0), (1, 3, 1e-4, 0.0),
                                      (1, 0, 0.0, 0.0), (1, 3, 1e-4, 3.0), (0, 0, 0.0, 2.0)):
        p, op = params_pair(amr, w["vmin"], w["vmax"], shade=shade, schedule=schedule,
                            ert_eps=ert, lod_pixels=lod)
        ia, na = gpu_render(a, w["camera"], w["tf"], p)
        ib, nb = gpu_render(b, w["camera"], w["tf"], p)
        assert na == nb, (shade, schedule, ert, lod)
        assert np.array_equal(ia, ib), (shade, schedule, ert, lod)
        if dtype == "f32" and lod == 0.0:
            ref, _ = o.render(w["camera"], w["tf"], op)
            assert_image_close(ib, ref, what=f"maxbrick shade {shade} schedule {schedule}")


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_maxbrick_random_hierarchies(amr, seed):
    rng = np.random.default_rng(seed)
    h = random_hierarchy(seed, n0=8, num_levels=3, patches_per_level=6, max_size=12, tiles=4)
    W, H = int(rng.integers(9, 61)), int(rng.integers(9, 61))
    cam = synth.orbit_camera(300 + seed, W, H)
    vmin, vmax = h.value_range()
    # transfer functions with long transparent stretches, in the middle and at the top too
    tfs = [synth.ramp_tf(alpha_start=0.5), synth.tf_variants()[2], synth.tf_variants()[3]]
    a, b = amr.from_hierarchy(h), amr.from_hierarchy(h)
    a.amr_build_kdtree("ptr", gradient=True)
    b.amr_build_kdtree("ptr", gradient=True, maxbrick=True)
    for tf in tfs:
        for schedule in (0, 3):
            p, _ = params_pair(amr, vmin, vmax, shade=1, kappa=20.0, schedule=schedule)
            ia, na = gpu_render(a, cam, tf, p)
            ib, nb = gpu_render(b, cam, tf, p)
            assert na == nb and np.array_equal(ia, ib)


def test_maxbrick_c2_bench_configuration(amr):
    # the bench's storage (pointer table, gradient bricks, two-cell halo) at 2048^2
    h = synth.make_c2(device="cuda")
    vmin, vmax = synth.amr.percentile_range(h)
    a, b = amr.from_hierarchy(h), amr.from_hierarchy(h)
    a.amr_build_kdtree("ptr", gradient=True, halo=2)
    b.amr_build_kdtree("ptr", gradient=True, halo=2, maxbrick=True)
    cam = synth.orbit_camera(2, 2048, 2048)
    for schedule in (0, 3):
        p, _ = params_pair(amr, vmin, vmax, shade=1, schedule=schedule)
        ia, na = gpu_render(a, cam, synth.ramp_tf(), p)
        ib, nb = gpu_render(b, cam, synth.ramp_tf(), p)
        assert na == nb and np.array_equal(ia, ib)


def test_maxbrick_needs_the_pointer_storage(amr, c1):
    from paper_1212_3333_gb300 import _lib

    w, _ = c1
    for storage in ("texobj", "atlas_linear", "atlas_tex3d"):
        ctx = amr.from_hierarchy(w["hier"])
        with pytest.raises(amr.AmrError) as e:
            ctx.amr_build_kdtree(storage, maxbrick=True)
        assert e.value.status == _lib.AMR_ERR_ARG


@pytest.mark.parametrize("schedule", [0, 3])
def test_maxbrick_batches_bit_identical(amr, c1, schedule):
    # batched views read each view's transfer function and its prefix table from their own
    # places in shared memory: with the bricks they still equal the renders without
    import torch

    w, _ = c1
    a, b = amr.from_hierarchy(w["hier"]), amr.from_hierarchy(w["hier"])
    a.amr_build_kdtree("ptr", gradient=True)
    b.amr_build_kdtree("ptr", gradient=True, maxbrick=True)
    tfs = torch.as_tensor(np.stack(synth.tf_variants()), device="cuda")
    rng = np.random.default_rng(9)
    cams = [synth.orbit_camera(900 + v, int(rng.integers(20, 90)), int(rng.integers(20, 90)))
            for v in range(9)]
    tfi = [v % 4 for v in range(9)]
    views, offsets, total = amr.make_views(cams, tfi)
    p, _ = params_pair(amr, w["vmin"], w["vmax"], shade=1, schedule=schedule)
    outs = []
    for ctx in (a, b):
        out = torch.zeros((total,), device="cuda")
        n = ctx.amr_render_batch(views, tfs, p, out, config=amr.batch_config(8, 8, 1),
                                 count_samples=True)
        outs.append((out.cpu().numpy(), n))
    assert outs[0][1] == outs[1][1] and np.array_equal(outs[0][0], outs[1][0])
    # and each view equals its single render with the bricks
    for v, cam in enumerate(cams):
        img, _ = gpu_render(b, cam, synth.tf_variants()[tfi[v]], p)
        got = outs[1][0][offsets[v]:offsets[v] + 4 * cam.width * cam.height].reshape(img.shape)
        assert np.array_equal(got, img.astype(np.float32)), v


@pytest.mark.parametrize("schedule", [0, 3])
def test_maxbrick_secondary_rays_bit_identical(amr, c1, schedule):
    # light samples whose stencil maximum maps to zero opacity multiply T by exactly 1
    w, _ = c1
    a, b = amr.from_hierarchy(w["hier"]), amr.from_hierarchy(w["hier"])
    a.amr_build_kdtree("ptr", gradient=True)
    b.amr_build_kdtree("ptr", gradient=True, maxbrick=True)
    cam = synth.orbit_camera(1, 96, 80)
    p, _ = params_pair(amr, w["vmin"], w["vmax"], shade=1, schedule=schedule, shadow=1,
                       light=(0.5, 0.5, 0.5), light_step=1.0 / 128, light_ambient=0.15)
    ia, na = gpu_render(a, cam, w["tf"], p)
    ib, nb = gpu_render(b, cam, w["tf"], p)
    assert na == nb and np.array_equal(ia, ib)


def test_maxbrick_learned_march_bit_identical(amr, c1):
    from paper_1212_3333_gb300 import proposal

    w, _ = c1
    a, b = amr.from_hierarchy(w["hier"]), amr.from_hierarchy(w["hier"])
    a.amr_build_kdtree("ptr")
    b.amr_build_kdtree("ptr", maxbrick=True)
    prop = proposal.Proposal(seed=7)
    prop.install(a)
    prop.install(b)
    for mode, tau in ((1, 0.3), (2, 0.3), (1, 0.0)):
        p, _ = params_pair(amr, w["vmin"], w["vmax"], shade=1, learned=mode, tau=tau)
        ia, na = gpu_render(a, w["camera"], w["tf"], p)
        ib, nb = gpu_render(b, w["camera"], w["tf"], p)
        assert na == nb and np.array_equal(ia, ib), (mode, tau)


@pytest.mark.parametrize("gradient", [False, True])
def test_maxbrick_every_sample_opaque_bit_identical(amr, c1, gradient):
    # every sample opaque (a transfer function with non-zero opacity everywhere, no early
    # termination): the stencil-maximum test never proves a sample transparent, and the
    # image and the sample count equal those of the per-ray loop without the bricks bit
    # for bit
    w, o = c1
    tf = np.array(synth.ramp_tf(), dtype=np.float64)
    tf[:, 3] = 0.02 + 0.05 * np.linspace(0.0, 1.0, tf.shape[0])
    tf = tf.astype(np.float32)
    a, b = amr.from_hierarchy(w["hier"]), amr.from_hierarchy(w["hier"])
    a.amr_build_kdtree("ptr", gradient=gradient, halo=2)
    b.amr_build_kdtree("ptr", gradient=gradient, halo=2, maxbrick=True)
    cam = synth.orbit_camera(5, 128, 96)
    p, op = params_pair(amr, w["vmin"], w["vmax"], shade=1, schedule=0, ert_eps=0.0)
    ia, na = gpu_render(a, cam, tf, p)
    ib, nb = gpu_render(b, cam, tf, p)
    assert na == nb and np.array_equal(ia, ib)
    ref, _ = o.render(cam, tf, op)
    assert_image_close(ib, ref, what="every sample opaque")
