"""GPU parity of secondary rays to a point light (the global-illumination example of
Sec. 5): images against the FP64 oracle (whose transmittance is pinned by closed forms),
for a light inside and outside the domain, unshaded and Phong, with and without gradient
bricks, in both linear storages; unsupported combinations are rejected."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_image_close, gpu_render, params_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amr():
    import paper_1212_3333_gb300 as m

    return m


@pytest.fixture(scope="module")
def c1():
    w = synth.c1_workload(width=96, height=80)
    return w, oracle.Oracle(w["hier"])


@pytest.mark.parametrize("storage", ["ptr", "atlas_linear"])
@pytest.mark.parametrize("gradient", [False, True])
@pytest.mark.parametrize("light", [(0.5, 0.5, 0.5), (1.6, -0.4, 0.9)])
def test_shadow_image_c1(amr, c1, storage, gradient, light):
    w, o = c1
    ctx = amr.from_hierarchy(w["hier"])
    ctx.amr_build_kdtree(storage, gradient=gradient)
    # unshaded (per-ray loop), Phong with the per-ray loop (each lane marches its light
    # rays) and Phong with deferred shading (the warp marches each light ray)
    for shade, schedule in ((0, 0), (1, 0), (1, 3)):
        p, op = params_pair(amr, w["vmin"], w["vmax"], shade=shade, shadow=1, light=light,
                            light_step=1.0 / 128, light_ambient=0.15, schedule=schedule)
        img, n = gpu_render(ctx, w["camera"], w["tf"], p)
        ref, smp = o.render(w["camera"], w["tf"], op)
        assert_image_close(img, ref, what=f"shadow {storage} grad={gradient} shade={shade} "
                                          f"schedule={schedule}")
        assert int(n) == int(smp.sum()) or abs(int(n) - int(smp.sum())) <= 0.001 * smp.sum()
        plain, _ = gpu_render(ctx, w["camera"], w["tf"], params_pair(
            amr, w["vmin"], w["vmax"], shade=shade)[0])
        assert np.all(img[..., :3] <= plain[..., :3] + 1e-6)
        assert np.array_equal(img[..., 3], plain[..., 3])
        assert np.mean(img[..., :3]) < 0.95 * np.mean(plain[..., :3])


def test_shadow_rejections(amr, c1):
    import torch

    from paper_1212_3333_gb300 import _lib

    w, _ = c1
    p, _ = params_pair(amr, w["vmin"], w["vmax"], shadow=1, light=(0.5, 0.5, 0.5),
                       light_step=0.01)
    for storage, dtype in (("texobj", "f32"), ("ptr", "f16")):
        ctx = amr.from_hierarchy(w["hier"], dtype)
        ctx.amr_build_kdtree(storage)
        with pytest.raises(amr.AmrError) as e:
            gpu_render(ctx, w["camera"], w["tf"], p)
        assert e.value.status == _lib.AMR_ERR_ARG
    ctx = amr.from_hierarchy(w["hier"])
    ctx.amr_build_kdtree("ptr")
    for kw in (dict(schedule=1), dict(schedule=2), dict(interp=0), dict(light_step=0.0),
               dict(light_ambient=1.5), dict(light=(np.nan, 0.0, 0.0)),
               dict(schedule=3, shade=0)):
        base = dict(shadow=1, light=(0.5, 0.5, 0.5), light_step=0.01)
        base.update(kw)
        p, _ = params_pair(amr, w["vmin"], w["vmax"], **base)
        with pytest.raises(amr.AmrError) as e:
            gpu_render(ctx, w["camera"], w["tf"], p)
        assert e.value.status == _lib.AMR_ERR_ARG, kw
    views, offsets, total = amr.make_views([w["camera"]], [0])
    out = torch.zeros((total,), device="cuda")
    tfs = torch.as_tensor(np.stack(synth.tf_variants()), device="cuda")
    p, _ = params_pair(amr, w["vmin"], w["vmax"], shadow=1, light=(0.5, 0.5, 0.5),
                       light_step=0.01)
    with pytest.raises(amr.AmrError) as e:
        ctx.amr_render_batch(views, tfs, p, out)
    assert e.value.status == _lib.AMR_ERR_ARG


def test_shadow_schedules_agree_to_rounding(amr, c1):
    # the per-ray loop multiplies a light ray's factors sample by sample, the deferred
    # schedule 32 at a time: the same transmittance up to FP32 rounding
    w, _ = c1
    ctx = amr.from_hierarchy(w["hier"])
    ctx.amr_build_kdtree("ptr", gradient=True)
    imgs = []
    for schedule in (0, 3):
        p, _ = params_pair(amr, w["vmin"], w["vmax"], shade=1, shadow=1, light=(0.5, 0.5, 0.5),
                           light_step=1.0 / 256, light_ambient=0.1, schedule=schedule)
        imgs.append(gpu_render(ctx, w["camera"], w["tf"], p))
    (a, na), (b, nb) = imgs
    assert na == nb
    assert np.array_equal(a[..., 3], b[..., 3])
    assert np.max(np.abs(a - b)) <= 2e-6


@pytest.fixture(scope="module")
def c2():
    h = synth.make_c2(device="cuda")
    vmin, vmax = synth.amr.percentile_range(h)
    return h, vmin, vmax, oracle.Oracle(h)


@pytest.mark.parametrize("schedule", [3, 0])
def test_shadow_c2_sampled_pixels(amr, c2, schedule):
    # the bench hierarchy (5 levels, 2,219 patches) with the light at the domain centre:
    # sampled pixels of a 512^2 Phong view against the FP64 oracle
    h, vmin, vmax, o = c2
    ctx = amr.from_hierarchy(h)
    ctx.amr_build_kdtree("ptr", gradient=True)
    cam = synth.orbit_camera(2, 512, 512)
    tf = synth.ramp_tf()
    p, op = params_pair(amr, vmin, vmax, shade=1, shadow=1, light=(0.5, 0.5, 0.5),
                        light_step=0.5 / 128, light_ambient=0.2, schedule=schedule)
    img, n = gpu_render(ctx, cam, tf, p)
    rng = np.random.default_rng(52)
    pix = np.concatenate([np.stack([rng.integers(0, 512, 700), rng.integers(0, 512, 700)], 1),
                          np.stack([np.arange(512), np.full(512, 256)], 1)]).astype(np.int32)
    ref, _ = o.render(cam, tf, op, pixels=pix)
    got = img[pix[:, 1], pix[:, 0]]
    assert_image_close(got, ref, what=f"c2 shadow schedule {schedule}")
    plain, _ = gpu_render(ctx, cam, tf, params_pair(amr, vmin, vmax, shade=1)[0])
    assert np.array_equal(img[..., 3], plain[..., 3])
    assert np.all(img[..., :3] <= plain[..., :3] + 1e-6)
    assert np.max(plain[..., :3] - img[..., :3]) > 1e-3  # the light rays do shade
