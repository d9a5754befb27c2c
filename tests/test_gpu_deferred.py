"""GPU checks of the warp-synchronous march with deferred shading (schedule 3): every pixel
sees the same samples, opacities and colour terms as under the per-ray loop, added to its
colour in the same order (only the moment of each addition moves), so images and sample
counts must equal the per-ray schedule's bit for bit - for every storage, gradient bricks
or not, early termination, skipping, pruning, 16-bit cells, bands and samples-per-step
setting - and stay within the FP64 oracle's tolerance on ragged random hierarchies and on
the C2 hierarchy."""
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
    return synth.c1_workload()


def _same(amr, ctx, cam, tf, vmin, vmax, spis=(1, 4, 16), **kw):
    p0, _ = params_pair(amr, vmin, vmax, schedule=0, shade=1, **kw)
    a, na = gpu_render(ctx, cam, tf, p0)
    for spi in spis:
        p3, _ = params_pair(amr, vmin, vmax, schedule=3, shade=1, samples_per_iter=spi, **kw)
        b, nb = gpu_render(ctx, cam, tf, p3)
        assert na == nb, (kw, spi)
        assert np.array_equal(a, b), (kw, spi, np.abs(a - b).max())
    return a


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("gradient", [False, True])
def test_deferred_equals_per_ray_c1(amr, c1, storage, gradient):
    w = c1
    ctx = amr.from_hierarchy(w["hier"])
    ctx.amr_build_kdtree(storage, gradient=gradient)
    for ert in (0.0, 1e-4, 0.3):
        for skip in (0, 1):
            _same(amr, ctx, w["camera"], w["tf"], w["vmin"], w["vmax"], ert_eps=ert, skip=skip)


@pytest.mark.parametrize("dtype", ["f16", "bf16"])
def test_deferred_equals_per_ray_16bit(amr, c1, dtype):
    w = c1
    for storage in ("ptr", "atlas_linear"):
        ctx = amr.from_hierarchy(w["hier"], dtype)
        ctx.amr_build_kdtree(storage, gradient=True)
        _same(amr, ctx, w["camera"], w["tf"], w["vmin"], w["vmax"])


def test_deferred_equals_per_ray_with_pruning(amr, c1):
    w = c1
    ctx = amr.from_hierarchy(w["hier"])
    ctx.amr_build_kdtree("ptr", gradient=True)
    for lod in (0.5, 2.0, 8.0):
        _same(amr, ctx, w["camera"], w["tf"], w["vmin"], w["vmax"], spis=(4,), lod_pixels=lod)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_deferred_ragged_images_and_bands(amr, seed):
    h = random_hierarchy(seed, n0=8 + seed, num_levels=3)
    ctx = amr.from_hierarchy(h)
    ctx.amr_build_kdtree("ptr", gradient=bool(seed & 1))
    vmin, vmax = h.value_range()
    tf = synth.ramp_tf()
    cam = synth.orbit_camera(seed, 37 + 5 * seed, 29 + 3 * seed)  # partial tiles
    full = _same(amr, ctx, cam, tf, vmin, vmax, kappa=20.0)
    o = oracle.Oracle(h)
    _, op = params_pair(amr, vmin, vmax, shade=1, kappa=20.0)
    ref, _ = o.render(cam, tf, op)
    assert_image_close(full, ref)
    cuts = [0, 5, 11, 30, cam.height]
    parts = []
    for r0, r1 in zip(cuts[:-1], cuts[1:]):
        if r0 >= cam.height:
            continue
        p, _ = params_pair(amr, vmin, vmax, shade=1, kappa=20.0, schedule=3,
                           row0=r0, rows=min(r1, cam.height) - r0)
        parts.append(gpu_render(ctx, cam, tf, p)[0])
    assert np.array_equal(np.concatenate(parts, axis=0), full)


def test_deferred_rejects_bad_settings(amr, c1):
    from paper_1212_3333_gb300 import _lib

    w = c1
    ctx = amr.from_hierarchy(w["hier"])
    ctx.amr_build_kdtree("ptr")
    for kw in (dict(shade=0), dict(interp=0), dict(samples_per_iter=0),
               dict(samples_per_iter=65), dict(shadow=1), dict(learned=1)):
        base = dict(shade=1)
        base.update(kw)
        p, _ = params_pair(amr, w["vmin"], w["vmax"], schedule=3, **base)
        with pytest.raises(amr.AmrError) as e:
            gpu_render(ctx, w["camera"], w["tf"], p)
        assert e.value.status in (_lib.AMR_ERR_ARG, _lib.AMR_ERR_STATE)


@pytest.fixture(scope="module")
def c2():
    h = synth.make_c2(device="cuda")
    vmin, vmax = synth.amr.percentile_range(h)
    return h, vmin, vmax, oracle.Oracle(h)


@pytest.mark.parametrize("size", [512, 2048])
def test_deferred_c2(amr, c2, size):
    h, vmin, vmax, o = c2
    ctx = amr.from_hierarchy(h)
    ctx.amr_build_kdtree("ptr", gradient=True)
    cam = synth.orbit_camera(2, size, size)
    tf = synth.ramp_tf()
    img = _same(amr, ctx, cam, tf, vmin, vmax, spis=(16,))
    rng = np.random.default_rng(size)
    pix = np.stack([rng.integers(0, size, 600), rng.integers(0, size, 600)], 1).astype(np.int32)
    _, op = params_pair(amr, vmin, vmax, shade=1)
    ref, _ = o.render(cam, tf, op, pixels=pix)
    assert_image_close(img[pix[:, 1], pix[:, 0]], ref, what=f"c2 deferred {size}")
