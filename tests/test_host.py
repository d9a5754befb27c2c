"""Host-side logic of the product library, checked without a GPU: the kD-tree build
(Sec. 3.1) against the FP64 oracle's independent brute-force build, brick halos against
the oracle's level values V_l (Sec. 4), the NFDH atlas (Sec. 4.1), argument checking and
the exported ABI."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle
import synth
from synth.amr import make_hierarchy_from_boxes, random_hierarchy

amr = pytest.importorskip("paper_1212_3333_gb300")
from paper_1212_3333_gb300 import _lib  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _tree_equal(h):
    ctx = amr.from_hierarchy(h)
    ctx.amr_build_host("ptr")
    o = oracle.Oracle(h)
    got = ctx.amr_get_nodes()
    want = o.nodes()
    for g, w in zip(got, want):
        np.testing.assert_array_equal(g, w.astype(np.int32))
    b, p, lv = ctx.amr_get_leaves()
    ob, op, olv = o.leaves()
    np.testing.assert_array_equal(b, ob.astype(np.int32))
    np.testing.assert_array_equal(p, op)
    np.testing.assert_array_equal(lv, olv)
    return ctx, o


def test_library_exports_every_declared_symbol():
    lib = _lib.load()
    header = open(os.path.join(ROOT, "include", "amr.h")).read()
    declared = set(re.findall(r"\b(amr_[a-z_]+)\s*\(", header))
    assert declared == set(_lib.declared_symbols())
    for name in declared:
        assert hasattr(lib, name), name


def _header_functions():
    """name -> parameter count of every function declared in include/amr.h."""
    header = open(os.path.join(ROOT, "include", "amr.h")).read()
    header = re.sub(r"/\*.*?\*/", " ", header, flags=re.S)
    out = {}
    for m in re.finditer(r"\b(amr_[a-z_]+)\s*\(([^;{]*?)\)\s*;", header):
        params = m.group(2).strip()
        out[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_argument_counts_match_the_header():
    # each ctypes signature passes as many arguments as the C declaration takes
    decl = _header_functions()
    for name, (_, args) in _lib._SIGS.items():
        assert decl.get(name) == len(args), (name, decl.get(name), len(args))


def test_binding_constants_match_the_header(tmp_path):
    # the binding's copies of the header's constants, read back from a C program that
    # includes the header (enums and #defines alike)
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    names = ["AMR_OK", "AMR_ERR_ARG", "AMR_ERR_OVERLAP", "AMR_ERR_NOT_TILED", "AMR_ERR_STATE",
             "AMR_ERR_OOM", "AMR_ERR_CUDA", "AMR_ERR_CAPACITY", "AMR_ERR_DEVICE", "AMR_F32",
             "AMR_F16", "AMR_BF16", "AMR_STORE_PTR", "AMR_STORE_TEXOBJ",
             "AMR_STORE_ATLAS_LINEAR", "AMR_STORE_ATLAS_TEX3D", "AMR_STORE_GRADIENT",
             "AMR_STORE_HALO2", "AMR_STORE_MAXBRICK", "AMR_MLP_FEATURES", "AMR_MLP_PARAMS",
             "AMR_MLP_PACKED_BYTES", "AMR_MLP_GRAD_BLOCKS", "AMR_MLP_GRAD_SCRATCH",
             "AMR_MAX_BATCH_VIEWS", "AMR_SCHEDULE_AUTO", "AMR_BATCH_CANDIDATES"]
    src = tmp_path / "consts.c"
    src.write_text('#include <stdio.h>\n#include "amr.h"\nint main(void) {\n' +
                   "".join(f'  printf("%lld\\n", (long long)({n}));\n' for n in names) +
                   "  return 0;\n}\n")
    exe = tmp_path / "consts"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True,
                                          text=True).stdout.split()]
    for n, v in zip(names, got):
        assert getattr(_lib, n) == v, (n, getattr(_lib, n), v)


def test_tree_matches_oracle_c1():
    _tree_equal(synth.make_c1())


@pytest.mark.parametrize("seed", range(40))
def test_tree_matches_oracle_random(seed):
    rng = np.random.default_rng(seed)
    h = random_hierarchy(seed, n0=int(rng.choice([4, 8, 12])), num_levels=int(rng.integers(2, 5)),
                         patches_per_level=int(rng.integers(1, 9)), max_size=int(rng.integers(2, 14)),
                         tiles=int(rng.integers(1, 6)))
    _tree_equal(h)


def test_tree_matches_oracle_ratio3():
    boxes = [[0, 0, 0, 6, 6, 6], [2, 1, 3, 11, 9, 12], [11, 11, 0, 17, 18, 5],
             [10, 12, 14, 30, 27, 33]]
    h = make_hierarchy_from_boxes(3, 3, (6, 6, 6), boxes, [0, 1, 1, 2],
                                  lambda X, Y, Z: X + Y * Z)
    _tree_equal(h)


@pytest.mark.parametrize("halo", [1, 2])
@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_halo_equals_level_value(seed, halo):
    """Every brick cell (interior and the one- or two-cell halo) equals the level value
    V_l of the cell it stands for, rounded to float32 (the product reads coarse values from
    coarse bricks that are already rounded, so a few ulps may separate them)."""
    h = random_hierarchy(seed, n0=8, num_levels=3, patches_per_level=5, max_size=9, tiles=3)
    ctx = amr.from_hierarchy(h)
    ctx.amr_build_host("ptr", halo=halo)
    o = oracle.Oracle(h)
    worst = 0.0
    H = halo
    for p in range(h.num_patches):
        b = h.patch_box[p]
        l = int(h.patch_level[p])
        n = b[3:] - b[:3]
        br = ctx.amr_get_brick(p).reshape(n[2] + 2 * H, n[1] + 2 * H, n[0] + 2 * H)
        for k in range(n[2] + 2 * H):
            for j in range(n[1] + 2 * H):
                for i in range(n[0] + 2 * H):
                    interior = (H <= i < n[0] + H and H <= j < n[1] + H and
                                H <= k < n[2] + H)
                    v = o.V(l, b[0] + i - H, b[1] + j - H, b[2] + k - H)
                    if interior:
                        assert br[k, j, i] == np.float32(v)
                    else:
                        err = abs(float(br[k, j, i]) - v) / max(1.0, abs(v))
                        worst = max(worst, err)
    assert worst < 4e-7, worst


def test_atlas_packing_is_valid():
    h = random_hierarchy(5, n0=8, num_levels=3, patches_per_level=8, max_size=12, tiles=5)
    ctx = amr.from_hierarchy(h)
    ctx.amr_build_host("atlas_linear")
    st = ctx.amr_get_stats()
    dims = np.array(st.atlas_dims[:])
    assert np.all(dims > 0)
    assert 0.0 < st.atlas_efficiency <= st.atlas_efficiency_halo <= 1.0


@pytest.mark.parametrize("halo", [1, 2])
@pytest.mark.parametrize("seed", [3, 5])
def test_brick_bytes_and_packing_efficiency_follow_their_definitions(seed, halo):
    """Memory statistics (the quantities of the paper's Table 2): one FP32 value per cell,
    bricks carrying a one-cell halo (Sec. 4; two with AMR_STORE_HALO2), packing efficiency =
    data cells / atlas cells (Sec. 4.1), with and without the halos."""
    h = random_hierarchy(seed, n0=8, num_levels=3, patches_per_level=8, max_size=12, tiles=5)
    n = (h.patch_box[:, 3:] - h.patch_box[:, :3]).astype(np.int64)
    cells = int(np.prod(n, axis=1).sum())
    halo_cells = int(np.prod(n + 2 * halo, axis=1).sum())
    for storage in ("ptr", "atlas_linear"):
        ctx = amr.from_hierarchy(h)
        ctx.amr_build_host(storage, halo=halo)
        st = ctx.amr_get_stats()
        assert st.num_patches == h.num_patches
        assert st.num_cells == cells
        assert st.brick_bytes == 4 * halo_cells
        if storage == "atlas_linear":
            vol = int(np.prod(np.array(st.atlas_dims[:], dtype=np.int64)))
            assert vol >= halo_cells  # bricks are disjoint inside the atlas box
            assert st.atlas_efficiency == pytest.approx(cells / vol, rel=1e-12)
            assert st.atlas_efficiency_halo == pytest.approx(halo_cells / vol, rel=1e-12)
        ctx.amr_destroy()


@pytest.mark.parametrize("boxes,levels,code", [
    ([[0, 0, 0, 4, 4, 4], [2, 0, 0, 4, 4, 4]], [0, 0], _lib.AMR_ERR_OVERLAP),
    ([[0, 0, 0, 2, 2, 2], [2, 2, 2, 4, 4, 4]], [0, 0], _lib.AMR_ERR_NOT_TILED),
    ([[0, 0, 0, 4, 4, 4], [0, 0, 0, 3, 3, 3], [2, 2, 2, 5, 5, 5]], [0, 1, 1], _lib.AMR_ERR_OVERLAP),
    ([[0, 0, 0, 4, 4, 4], [6, 6, 6, 10, 10, 10]], [0, 1], _lib.AMR_ERR_ARG),  # outside root
])
def test_build_rejects_bad_hierarchies(boxes, levels, code):
    h = make_hierarchy_from_boxes(2, 2, (4, 4, 4), boxes, levels, lambda X, Y, Z: X)
    ctx = amr.from_hierarchy(h)
    with pytest.raises(amr.AmrError) as e:
        ctx.amr_build_host("ptr")
    assert e.value.status == code
    assert str(e.value)


def test_create_rejects_malformed_arguments():
    d = [np.zeros((2, 2, 2), dtype=np.float32)]
    with pytest.raises(amr.AmrError) as e:
        amr.amr_create(1, 1, (0, 0, 0), (1, 1, 1), [0], [[0, 0, 0, 2, 2, 2]], d)
    assert e.value.status == _lib.AMR_ERR_ARG
    with pytest.raises(amr.AmrError):
        amr.amr_create(1, 2, (0, 0, 0), (1, 1, 1), [0], [[0, 0, 0, 0, 2, 2]], d)  # empty box
    with pytest.raises(amr.AmrError):
        amr.amr_create(1, 2, (0, 0, 0), (1, 1, 1), [3], [[0, 0, 0, 2, 2, 2]], d)  # bad level
    with pytest.raises(amr.AmrError):
        amr.amr_create(1, 2, (0, 0, 0), (0, 1, 1), [0], [[0, 0, 0, 2, 2, 2]], d)  # h0 = 0
    with pytest.raises(amr.AmrError):
        amr.amr_create(1, 2, (0, 0, 0), (1, 1, 1), [0], [[0, 0, 0, 2, 2, 2]], d, dtype=7)


def test_render_before_build_is_a_state_error():
    h = synth.make_c1()
    ctx = amr.from_hierarchy(h)
    lib = _lib.load()
    cam = amr.make_camera(synth.orbit_camera(1, 8, 8))
    p = amr.amr_default_params()
    st = lib.amr_render(ctx._h, C.byref(cam), C.c_void_p(16), 256, C.byref(p), C.c_void_p(16),
                        None, None)
    assert st == _lib.AMR_ERR_STATE
    assert b"build" in lib.amr_last_error(ctx._h)
    # host-only build does not make the context renderable either
    ctx.amr_build_host("ptr")
    assert lib.amr_render(ctx._h, C.byref(cam), C.c_void_p(16), 256, C.byref(p), C.c_void_p(16),
                          None, None) == _lib.AMR_ERR_STATE
    assert lib.amr_destroy(None) == _lib.AMR_OK


def test_injected_host_allocation_failure(monkeypatch):
    """AMR_FAULT=bad_alloc: the host build reports AMR_ERR_OOM with a message and leaves
    the context usable; without the variable the same context builds."""
    ctx = amr.from_hierarchy(synth.make_c1())
    lib = _lib.load()
    monkeypatch.setenv("AMR_FAULT", "bad_alloc")
    assert lib.amr_build_host(ctx._h, _lib.AMR_STORE_PTR) == _lib.AMR_ERR_OOM
    assert b"memory" in lib.amr_last_error(ctx._h)
    monkeypatch.setenv("AMR_FAULT", "none")
    ctx.amr_build_host("ptr")
    assert ctx.amr_get_stats().num_leaves > 0
