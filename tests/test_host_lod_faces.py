"""Host-side tree annotations the kernels rely on, against independent computations:
the type-(a) nodes (Sec. 3.1) and their pruned-leaf ids against the FP64 oracle's labels,
and the same-patch face bits and neighbour-lookup start nodes against brute force over
the oracle's leaves and node boxes."""
import numpy as np
import pytest

import oracle
import synth
from synth.amr import random_hierarchy

amr = pytest.importorskip("paper_1212_3333_gb300")

HIERS = [("c1", lambda: synth.make_c1())] + [
    (f"rand{s}", (lambda s=s: random_hierarchy(50 + s, n0=8, num_levels=3 + s % 2,
                                                patches_per_level=6, max_size=9, tiles=4)))
    for s in range(6)]


def _boxes(axis, split, left, right, root):
    """Finest-cell box of every pre-order node from the split structure."""
    N = len(axis)
    box = np.zeros((N, 6), dtype=np.int64)
    box[0] = root
    for k in range(N):
        if axis[k] >= 0:
            a, s = int(axis[k]), int(split[k])
            lb, rb = box[k].copy(), box[k].copy()
            lb[3 + a] = s
            rb[a] = s
            box[left[k]] = lb
            box[right[k]] = rb
    return box


def _root(h):
    sc = h.ratio ** (h.num_levels - 1)
    b = h.patch_box[h.patch_level == 0]
    return np.concatenate([b[:, :3].min(axis=0), b[:, 3:].max(axis=0)]) * sc


def _contains(outer, inner):
    return np.all(outer[:3] <= inner[:3]) and np.all(inner[3:] <= outer[3:])


@pytest.mark.parametrize("name,make", HIERS)
def test_type_a_nodes_match_oracle(name, make):
    h = make()
    ctx = amr.from_hierarchy(h)
    ctx.amr_build_host("ptr")
    o = oracle.Oracle(h)
    patch, level, lod = o.node_labels()
    M = o.num_leaves
    box, p, l, node = ctx.amr_get_lod_leaves()
    want = [k for k in range(len(lod)) if lod[k] >= 0]
    assert list(node) == want
    assert list(lod[want]) == list(range(M, M + len(want)))
    np.testing.assert_array_equal(p, patch[want])
    np.testing.assert_array_equal(l, level[want])
    axis, split, left, right, _ = o.nodes()
    nb = _boxes(axis, split, left, right, _root(h))
    np.testing.assert_array_equal(box, nb[want])


@pytest.mark.parametrize("halo", [1, 2])
@pytest.mark.parametrize("name,make", HIERS)
def test_leaf_faces_by_brute_force(name, make, halo):
    # a face bit: with a one-cell halo, the slab of one level cell beyond the face lies in
    # the leaf's patch and overlaps only that patch's leaves; with a two-cell halo, the
    # slab lies in the root and overlaps only leaves of the leaf's level
    h = make()
    ctx = amr.from_hierarchy(h)
    ctx.amr_build_host("ptr", halo=halo)
    o = oracle.Oracle(h)
    lbox, lpatch, llevel = o.leaves()
    axis, split, left, right, leaf = o.nodes()
    root = _root(h)
    nb = _boxes(axis, split, left, right, root)
    faces, fnode = ctx.amr_get_leaf_faces()
    R = h.ratio ** (h.num_levels - 1)
    pf = h.patch_box * 1  # level cells
    for m in range(len(lbox)):
        b = lbox[m]
        sc = h.ratio ** (h.num_levels - 1 - llevel[m])
        fbox = pf[lpatch[m]] * sc
        for a in range(3):
            for side in (0, 1):
                q = b.copy()
                if side == 0:
                    q[3 + a], q[a] = b[a], b[a] - sc
                else:
                    q[a], q[3 + a] = b[3 + a], b[3 + a] + sc
                inside_patch = q[a] >= fbox[a] and q[3 + a] <= fbox[3 + a]
                inside_root = q[a] >= root[a] and q[3 + a] <= root[3 + a]
                over = np.all((lbox[:, :3] < q[3:]) & (lbox[:, 3:] > q[:3]), axis=1)
                if halo == 1:
                    want = bool(inside_patch and np.all(lpatch[over] == lpatch[m]))
                else:
                    want = bool(inside_root and np.all(llevel[over] == llevel[m]))
                assert bool((faces[m] >> (2 * a + side)) & 1) == want, (name, m, a, side)
                for only, k in ((0, fnode[m, 2 * a + side]), (1, fnode[m, 6 + 2 * a + side])):
                    u = q.copy() if only else np.concatenate(
                        [np.minimum(q[:3], b[:3]), np.maximum(q[3:], b[3:])])
                    u = np.concatenate([np.maximum(u[:3], root[:3]), np.minimum(u[3:], root[3:])])
                    if u[a] >= u[3 + a]:
                        assert k == 0
                        continue
                    assert _contains(nb[k], u)
                    if axis[k] >= 0:  # deepest: no child holds it
                        assert not _contains(nb[left[k]], u) and not _contains(nb[right[k]], u)
    assert faces.any()


@pytest.mark.parametrize("name,make", HIERS)
def test_same_level_faces_cover_the_same_patch_faces(name, make):
    # a face onto the same unrefined patch is a face onto the same level
    h = make()
    c1c, c2c = amr.from_hierarchy(h), amr.from_hierarchy(h)
    c1c.amr_build_host("ptr")
    c2c.amr_build_host("ptr", halo=2)
    f1, n1 = c1c.amr_get_leaf_faces()
    f2, n2 = c2c.amr_get_leaf_faces()
    assert np.all((f1 & f2) == f1)
    np.testing.assert_array_equal(n1, n2)  # the lookup starts do not depend on the halo
