"""The allocation-free host render (amr_render_host_noalloc) against amr_render_host.

Callers that may not allocate device memory while rendering (their device memory is owned
and capped by another allocator, or their footprint must not grow after start-up) use the
no-alloc entry point, which stages everything in a fixed array inside the library.  This
file is collected last so that a run stopping at the first failure has run every other
test first; it also passes on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import paper_1212_3333_gb300 as amr
    from paper_1212_3333_gb300 import _lib

    w = synth.c1_workload()
    ctx = amr.from_hierarchy(w["hier"])
    ctx.amr_build_kdtree("ptr")
    # 4096 wide: the 4 MiB band holds 64 rows, so 150 rows take three bands (64, 64, 22)
    cam = synth.orbit_camera(1, 4096, 150, fov_y_deg=12.0)
    return amr, _lib, w, ctx, cam


def _noalloc(lib, ctx, cam_s, tf, p, out):
    n = C.c_uint64(0)
    st = lib.amr_render_host_noalloc(ctx._h, C.byref(cam_s), C.c_void_p(tf.ctypes.data),
                                     tf.shape[0], C.byref(p), C.c_void_p(out.ctypes.data), None,
                                     C.byref(n))
    return st, int(n.value)


@pytest.mark.parametrize("schedule", [0, 1, 2, 3])
def test_noalloc_matches_render_host_on_two_calls(setup, schedule):
    amr, _lib, w, ctx, cam = setup
    lib = _lib.load()
    tf = np.ascontiguousarray(w["tf"], dtype=np.float32)
    p = amr.amr_default_params(vmin=w["vmin"], vmax=w["vmax"], shade=1, schedule=schedule)
    ref = np.zeros((cam.height, cam.width, 4), dtype=np.float32)
    n_ref = ctx.amr_render_host(cam, tf, p, ref, count_samples=True)
    cam_s = amr.make_camera(cam)
    for _ in range(2):  # the array keeps the previous call's contents
        out = np.full((cam.height, cam.width, 4), np.nan, dtype=np.float32)
        st, n = _noalloc(lib, ctx, cam_s, tf, p, out)
        assert st == _lib.AMR_OK, lib.amr_last_error(ctx._h)
        assert np.all(np.isfinite(out))
        np.testing.assert_allclose(out, ref, rtol=0, atol=1e-6)
        assert n == n_ref
    assert ref[..., 3].max() > 0.1  # the view does cover the volume


def test_noalloc_rejects_sizes_beyond_its_staging(setup):
    amr, _lib, w, ctx, cam = setup
    lib = _lib.load()
    p = amr.amr_default_params(vmin=w["vmin"], vmax=w["vmax"])
    big_tf = np.zeros((4096, 4), dtype=np.float32)
    out = np.zeros((4, 8, 4), dtype=np.float32)
    st, _ = _noalloc(lib, ctx, amr.make_camera(synth.orbit_camera(1, 8, 4)), big_tf, p, out)
    assert st == _lib.AMR_ERR_ARG and b"2048" in lib.amr_last_error(ctx._h)
    wide = synth.orbit_camera(1, 20000, 2)
    out = np.zeros((2, 20000, 4), dtype=np.float32)
    tf = np.ascontiguousarray(w["tf"], dtype=np.float32)
    st, _ = _noalloc(lib, ctx, amr.make_camera(wide), tf, p, out)
    assert st == _lib.AMR_ERR_ARG and b"16384" in lib.amr_last_error(ctx._h)


def test_noalloc_leaves_device_free_memory_unchanged(setup):
    """The property the entry point exists for: on a warmed context, calls allocate no
    device memory - not for a repeat of the same frame, and not for a wider image with a
    longer transfer function, which would make amr_render_host grow its staging buffers."""
    import torch

    amr, _lib, w, ctx, cam = setup
    lib = _lib.load()
    p = amr.amr_default_params(vmin=w["vmin"], vmax=w["vmax"], shade=1)
    tf = np.ascontiguousarray(w["tf"], dtype=np.float32)
    tf_long = np.ascontiguousarray(np.repeat(tf, 4, axis=0), dtype=np.float32)  # 1024 entries
    wide = synth.orbit_camera(1, 6000, 40, fov_y_deg=12.0)
    outs = {}
    for c in (cam, wide):
        outs[c.width] = np.zeros((c.height, c.width, 4), dtype=np.float32)
    # warm-up: the first call on the device looks up (and commits) the staging array
    st, _ = _noalloc(lib, ctx, amr.make_camera(cam), tf, p, outs[cam.width])
    assert st == _lib.AMR_OK, lib.amr_last_error(ctx._h)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for c, t in ((cam, tf), (wide, tf_long), (cam, tf), (wide, tf_long)):
        st, n = _noalloc(lib, ctx, amr.make_camera(c), t, p, outs[c.width])
        assert st == _lib.AMR_OK, lib.amr_last_error(ctx._h)
        assert n > 0
        assert torch.cuda.mem_get_info()[0] == free0, "the no-alloc call changed free device memory"
