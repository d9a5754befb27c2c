"""16-bit brick cells, host side: the library's rounding of FP32 cells to IEEE binary16 and
to bfloat16 (round to nearest, ties to even) against numpy's binary16 and torch's bfloat16
conversions, the range check, and which storages accept 16-bit cells."""
import numpy as np
import pytest

amr = pytest.importorskip("paper_1212_3333_gb300")
from paper_1212_3333_gb300 import _lib  # noqa: E402


def _edge_values() -> np.ndarray:
    """Cells spanning the binary16 normal and subnormal ranges, exact ties of both formats,
    values either side of the binary16 overflow threshold, zeros and negatives."""
    rng = np.random.default_rng(5)
    mags = np.exp2(rng.uniform(-30.0, 15.9, size=300))
    v = list(mags * rng.choice([-1.0, 1.0], size=300))
    one = 1.0
    v += [0.0, -0.0, 65504.0, 65519.0, -65519.0, 6.1035156e-05, 5.9604645e-08, 2.0 ** -25,
          1.5 * 2.0 ** -25, 2.0 ** -26]
    # binary16 ties (half an ulp above 1 and 3 halves) and bfloat16 ties
    v += [one + 2.0 ** -11, one + 3 * 2.0 ** -11, one + 2.0 ** -8, one + 3 * 2.0 ** -8,
          -(one + 2.0 ** -11), 2048.0 + 1.0, 2048.0 + 3.0, 256.0 + 1.0, 256.0 + 3.0]
    v += list(rng.normal(size=512 - len(v)))
    return np.asarray(v, dtype=np.float32)


def _ctx(values: np.ndarray, dtype):
    d = values.reshape(8, 8, 8)
    return amr.amr_create(1, 2, (0, 0, 0), (0.125, 0.125, 0.125), [0], [[0, 0, 0, 8, 8, 8]],
                          [d], dtype=dtype)


def _f16(x):
    return x.astype(np.float16).astype(np.float32)


def _bf16(x):
    torch = pytest.importorskip("torch")
    return torch.as_tensor(x).to(torch.bfloat16).to(torch.float32).numpy()


@pytest.mark.parametrize("dtype,ref", [("f16", _f16), ("bf16", _bf16)])
@pytest.mark.parametrize("storage", ["ptr", "atlas_linear"])
def test_brick_cells_are_rounded_to_nearest_even(dtype, ref, storage):
    v = _edge_values()
    c32 = _ctx(v, "f32")
    c32.amr_build_host(storage)
    b32 = c32.amr_get_brick(0)
    c16 = _ctx(v, dtype)
    c16.amr_build_host(storage)
    b16 = c16.amr_get_brick(0)
    want = ref(b32)
    np.testing.assert_array_equal(b16.view(np.uint32), want.view(np.uint32))
    # spot checks of the ties, independent of the reference conversion
    if dtype == "f16":
        assert np.float32(1 + 2.0 ** -11) in b32 and 1.0 in b16
    else:
        assert np.float32(1 + 3 * 2.0 ** -8) in b32 and np.float32(1 + 2.0 ** -6) in b16


def test_f16_range_is_checked_and_bf16_is_not_limited():
    v = _edge_values()
    v[7] = 65520.0  # rounds to infinity in binary16
    c = _ctx(v, "f16")
    with pytest.raises(amr.AmrError) as e:
        c.amr_build_host("ptr")
    assert e.value.status == _lib.AMR_ERR_ARG and "FP16" in str(e.value)
    c = _ctx(v, "bf16")
    c.amr_build_host("ptr")
    assert np.isfinite(c.amr_get_brick(0)).all()
    # central differences of in-range cells may overflow: checked with gradient bricks
    w = np.full((8, 8, 8), 40000.0, dtype=np.float32)
    w[:, :, 4:] = -40000.0  # x-difference -80000 across i = 3..4
    c = _ctx(w, "f16")
    c.amr_build_host("ptr")
    c = _ctx(w, "f16")
    with pytest.raises(amr.AmrError) as e:
        c.amr_build_host("ptr", gradient=True)
    assert e.value.status == _lib.AMR_ERR_ARG


@pytest.mark.parametrize("storage", ["texobj", "atlas_tex3d"])
def test_16bit_cells_need_a_linear_storage(storage):
    c = _ctx(_edge_values(), "bf16")
    with pytest.raises(amr.AmrError) as e:
        c.amr_build_host(storage)
    assert e.value.status == _lib.AMR_ERR_ARG
    c.amr_build_host("atlas_linear", gradient=True)


@pytest.mark.parametrize("dtype,ref", [("f16", _f16), ("bf16", _bf16)])
def test_rounding_over_random_bit_patterns(dtype, ref):
    """200k random float32 bit patterns across every binade the cell type can hold."""
    rng = np.random.default_rng(11 if dtype == "f16" else 12)
    bits = rng.integers(0, 1 << 32, size=64 * 64 * 48, dtype=np.uint64).astype(np.uint32)
    v = bits.view(np.float32).copy()
    lim = 65504.0 if dtype == "f16" else 1e30
    bad = ~np.isfinite(v) | (np.abs(v) > lim)
    v[bad] = rng.uniform(-1, 1, size=int(bad.sum())).astype(np.float32)
    d = v.reshape(48, 64, 64)
    c32 = amr.amr_create(1, 2, (0, 0, 0), (1, 1, 1), [0], [[0, 0, 0, 64, 64, 48]], [d])
    c32.amr_build_host("ptr")
    c16 = amr.amr_create(1, 2, (0, 0, 0), (1, 1, 1), [0], [[0, 0, 0, 64, 64, 48]], [d],
                         dtype=dtype)
    c16.amr_build_host("ptr")
    b32 = c32.amr_get_brick(0)
    np.testing.assert_array_equal(c16.amr_get_brick(0).view(np.uint32), ref(b32).view(np.uint32))
