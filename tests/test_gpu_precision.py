"""GPU checks of 16-bit brick cells (FP16 / BF16 storage, FP32 interpolation, gradients and
compositing, FP64-exact ray/leaf entry and exit).

Rounding happens once, at upload.  On single-level hierarchies every brick cell is a copy
of a patch cell, so a 16-bit render must equal, bit for bit, the FP32-storage render of
the cells rounded here by numpy / torch; on nested hierarchies the halo cells that hold an
interpolated coarser value are rounded after the interpolation, so there the 16-bit image
is compared with the FP64 oracle on the original cells, with the error reported as PSNR
and max-abs per dtype next to FP32 storage."""
import dataclasses

import numpy as np
import pytest

import oracle
import synth
from synth.amr import random_hierarchy
from gpu_util import assert_image_close, gpu_render, params_pair

pytestmark = pytest.mark.gpu

# lower bounds on PSNR (dB, all channels) against the FP64 oracle on the original cells
PSNR_MIN = {"f32": 90.0, "f16": 70.0, "bf16": 50.0}


@pytest.fixture(scope="module")
def amr():
    import paper_1212_3333_gb300 as m

    return m


def _round(data, dtype):
    import torch

    if dtype == "f16":
        return [np.ascontiguousarray(d.astype(np.float16).astype(np.float32)) for d in data]
    return [torch.as_tensor(d).to(torch.bfloat16).to(torch.float32).numpy() for d in data]


def _psnr(a, b):
    mse = float(np.mean((a - b) ** 2))
    return float("inf") if mse == 0.0 else 10.0 * np.log10(1.0 / mse)


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("dtype", ["f16", "bf16"])
@pytest.mark.parametrize("storage", ["ptr", "atlas_linear"])
def test_single_level_16bit_equals_fp32_of_rounded_cells(amr, seed, dtype, storage):
    h = random_hierarchy(40 + seed, n0=24, num_levels=1, tiles=7)
    hr = dataclasses.replace(h, data=_round(h.data, dtype))
    c16 = amr.from_hierarchy(h, dtype)
    c16.amr_build_kdtree(storage)
    c32 = amr.from_hierarchy(hr)
    c32.amr_build_kdtree(storage)
    vmin, vmax = h.value_range()
    tf = synth.ramp_tf()
    cam = synth.orbit_camera(seed, 96, 80)
    for shade in (0, 1):
        for skip in (0, 1):
            p, _ = params_pair(amr, vmin, vmax, shade=shade, skip=skip, ert_eps=0.0)
            a, na = gpu_render(c16, cam, tf, p)
            b, nb = gpu_render(c32, cam, tf, p)
            assert np.array_equal(a, b), (shade, skip, np.abs(a - b).max())
            assert na == nb
    # and the oracle on the rounded cells within the FP32 kernel's tolerance
    p, op = params_pair(amr, vmin, vmax, shade=1)
    img, _ = gpu_render(c16, cam, tf, p)
    ref, _ = oracle.Oracle(hr).render(cam, tf, op)
    assert_image_close(img, ref, what=f"{dtype} {storage} seed {seed}")


@pytest.fixture(scope="module")
def c1():
    w = synth.c1_workload()
    return w, oracle.Oracle(w["hier"])


@pytest.mark.parametrize("gradient", [False, True])
@pytest.mark.parametrize("storage", ["ptr", "atlas_linear"])
def test_c1_error_against_fp64_oracle(amr, c1, storage, gradient):
    w, o = c1
    p, op = params_pair(amr, w["vmin"], w["vmax"], shade=1)
    ref, _ = o.render(w["camera"], w["tf"], op)
    res = {}
    counts = {}
    for dtype in ("f32", "f16", "bf16"):
        ctx = amr.from_hierarchy(w["hier"], dtype)
        ctx.amr_build_kdtree(storage, gradient=gradient)
        img, counts[dtype] = gpu_render(ctx, w["camera"], w["tf"], p)
        assert np.all(np.isfinite(img))
        res[dtype] = (_psnr(img, ref), float(np.abs(img - ref).max()))
    print(f"\nc1 {storage} gradient={gradient}: " +
          ", ".join(f"{k} PSNR {v[0]:.1f} dB max-abs {v[1]:.2e}" for k, v in res.items()))
    for dtype, (ps, _) in res.items():
        assert ps >= PSNR_MIN[dtype], (dtype, ps)
    assert res["f32"][1] <= 5e-4
    assert res["f16"][1] <= res["bf16"][1] + 1e-6


def test_c1_sample_counts_and_exact_skipping(amr, c1):
    w, _ = c1
    p, _ = params_pair(amr, w["vmin"], w["vmax"], shade=1, ert_eps=0.0)
    ps, _ = params_pair(amr, w["vmin"], w["vmax"], shade=1, ert_eps=0.0, skip=1)
    c32 = amr.from_hierarchy(w["hier"])
    c32.amr_build_kdtree("ptr")
    _, n32 = gpu_render(c32, w["camera"], w["tf"], p)
    for dtype in ("f16", "bf16"):
        for storage in ("ptr", "atlas_linear"):
            ctx = amr.from_hierarchy(w["hier"], dtype)
            ctx.amr_build_kdtree(storage)
            full, n = gpu_render(ctx, w["camera"], w["tf"], p)
            assert n == n32  # sample positions depend on the geometry only
            skipped, n_skip = gpu_render(ctx, w["camera"], w["tf"], ps)
            assert np.array_equal(skipped, full) and n_skip < n


def test_16bit_rejects_unsupported_modes(amr, c1):
    import torch

    from paper_1212_3333_gb300 import _lib, proposal

    w, _ = c1
    ctx = amr.from_hierarchy(w["hier"], "bf16")
    ctx.amr_build_kdtree("ptr")
    for kw in (dict(interp=0), dict(schedule=1), dict(learned=1)):
        p, _ = params_pair(amr, w["vmin"], w["vmax"], **kw)
        with pytest.raises(amr.AmrError) as e:
            gpu_render(ctx, w["camera"], w["tf"], p)
        assert e.value.status == _lib.AMR_ERR_ARG, kw
    p, _ = params_pair(amr, w["vmin"], w["vmax"])
    tf = torch.as_tensor(w["tf"], device="cuda")
    with pytest.raises(amr.AmrError) as e:
        proposal.log_segments(ctx, [w["camera"]], tf, p, capacity=16, keep_prob=1.0)
    assert e.value.status == _lib.AMR_ERR_ARG
    # the context stays usable
    img, n = gpu_render(ctx, w["camera"], w["tf"], p)
    assert n > 0 and np.all(np.isfinite(img))


@pytest.fixture(scope="module")
def c2():
    h = synth.make_c2(device="cuda")
    vmin, vmax = synth.amr.percentile_range(h)
    return h, vmin, vmax, oracle.Oracle(h)


@pytest.mark.parametrize("dtype", ["f16", "bf16"])
def test_c2_sampled_error_against_fp64_oracle(amr, c2, dtype):
    h, vmin, vmax, o = c2
    cam = synth.orbit_camera(2, 1024, 1024)
    tf = synth.ramp_tf()
    p, op = params_pair(amr, vmin, vmax, shade=1)
    rng = np.random.default_rng(3)
    pix = np.stack([rng.integers(0, 1024, 1500), rng.integers(0, 1024, 1500)], axis=1)
    pix = pix.astype(np.int32)
    ref, _ = o.render(cam, tf, op, pixels=pix)
    out = {}
    for dt in ("f32", dtype):
        ctx = amr.from_hierarchy(h, dt)
        ctx.amr_build_kdtree("ptr", gradient=True)
        img, _ = gpu_render(ctx, cam, tf, p)
        got = img[pix[:, 1], pix[:, 0]]
        out[dt] = (_psnr(got, ref), float(np.abs(got - ref).max()))
    print(f"\nc2 1024 sampled: " +
          ", ".join(f"{k} PSNR {v[0]:.1f} dB max-abs {v[1]:.2e}" for k, v in out.items()))
    assert out[dtype][0] >= PSNR_MIN[dtype]
    assert out["f32"][1] <= 5e-4
