"""Pins for the oracle's kD-tree build (Sec. 3.1, kD-tree construction)."""
import numpy as np
import pytest

import oracle
import synth
from synth.amr import make_hierarchy_from_boxes, random_hierarchy
from golden_util import brute_finest_level, finest_boxes, read_kd_golden


def _const(X, Y, Z):
    return np.ones_like(X)


def _check_tree(o, nodes, leaves):
    axis, split, left, right, leaf = o.nodes()
    got = np.stack([np.arange(len(axis)), axis, split, left, right, leaf], axis=1)
    np.testing.assert_array_equal(got, nodes)
    box, patch, level = o.leaves()
    got_l = np.concatenate([np.arange(len(patch))[:, None], box, patch[:, None], level[:, None]],
                           axis=1)
    np.testing.assert_array_equal(got_l, leaves)


def test_golden_inner_patch():
    h = make_hierarchy_from_boxes(2, 2, (8, 8, 8), [[0, 0, 0, 8, 8, 8], [4, 4, 4, 12, 12, 12]],
                                  [0, 1], _const)
    nodes, leaves = read_kd_golden("kd_inner_patch.txt")
    _check_tree(oracle.Oracle(h), nodes, leaves)


def test_golden_tiling_2x2x2():
    boxes = []
    for p in range(8):
        i, j, k = p & 1, (p >> 1) & 1, p >> 2
        boxes.append([16 * i, 16 * j, 16 * k, 16 * i + 16, 16 * j + 16, 16 * k + 16])
    h = make_hierarchy_from_boxes(1, 2, (32, 32, 32), boxes, [0] * 8, _const)
    nodes, leaves = read_kd_golden("kd_tiling_2x2x2.txt")
    _check_tree(oracle.Oracle(h), nodes, leaves)


def test_single_patch_is_one_leaf():
    h = make_hierarchy_from_boxes(1, 2, (5, 7, 3), [[0, 0, 0, 5, 7, 3]], [0], _const)
    o = oracle.Oracle(h)
    assert o.num_nodes == 1 and o.num_leaves == 1
    box, patch, level = o.leaves()
    assert box.tolist() == [[0, 0, 0, 5, 7, 3]] and patch[0] == 0 and level[0] == 0


def test_fully_covering_fine_patch_relabels_leaf():
    # a level-1 patch covering the whole root turns the single leaf into a level-1 leaf
    h = make_hierarchy_from_boxes(2, 2, (4, 4, 4), [[0, 0, 0, 4, 4, 4], [0, 0, 0, 8, 8, 8]],
                                  [0, 1], _const)
    o = oracle.Oracle(h)
    box, patch, level = o.leaves()
    assert o.num_leaves == 1 and patch[0] == 1 and level[0] == 1


def test_validation_errors():
    # overlapping level-0 patches
    h = make_hierarchy_from_boxes(1, 2, (4, 4, 4), [[0, 0, 0, 4, 4, 4], [2, 0, 0, 4, 4, 4]],
                                  [0, 0], _const)
    with pytest.raises(oracle.OracleError) as e:
        oracle.Oracle(h)
    assert e.value.code == oracle.ORC_ERR_OVERLAP
    # level 0 does not tile its bounding box
    h = make_hierarchy_from_boxes(1, 2, (4, 4, 4), [[0, 0, 0, 2, 2, 2], [2, 2, 2, 4, 4, 4]],
                                  [0, 0], _const)
    with pytest.raises(oracle.OracleError) as e:
        oracle.Oracle(h)
    assert e.value.code == oracle.ORC_ERR_NOT_TILED
    # overlapping fine patches
    h = make_hierarchy_from_boxes(2, 2, (4, 4, 4), [[0, 0, 0, 4, 4, 4], [0, 0, 0, 3, 3, 3],
                                                    [2, 2, 2, 5, 5, 5]], [0, 1, 1], _const)
    with pytest.raises(oracle.OracleError) as e:
        oracle.Oracle(h)
    assert e.value.code == oracle.ORC_ERR_OVERLAP


def _invariants(h):
    o = oracle.Oracle(h)
    box, patch, level = o.leaves()
    fb = finest_boxes(h)
    root = np.concatenate([fb[h.patch_level == 0][:, :3].min(0), fb[h.patch_level == 0][:, 3:].max(0)])
    vol = np.prod(box[:, 3:] - box[:, :3], axis=1)
    # 1. leaves tile the root: volumes add up and no two overlap
    assert vol.sum() == np.prod(root[3:] - root[:3])
    assert np.all(vol > 0)
    M = len(box)
    lo = np.maximum(box[:, None, :3], box[None, :, :3])
    hi = np.minimum(box[:, None, 3:], box[None, :, 3:])
    inter = np.all(hi > lo, axis=2)
    np.fill_diagonal(inter, False)
    assert not inter.any()
    for m in range(M):
        # 2. each leaf lies inside its patch
        pb = fb[patch[m]]
        assert np.all(box[m, :3] >= pb[:3]) and np.all(box[m, 3:] <= pb[3:])
        assert h.patch_level[patch[m]] == level[m]
        # 3. its level is the finest level of any patch it overlaps
        ov = np.all(np.minimum(fb[:, 3:], box[m, 3:]) > np.maximum(fb[:, :3], box[m, :3]), axis=1)
        assert h.patch_level[ov].max() == level[m]
    return o


def test_invariants_c1():
    _invariants(synth.make_c1())


@pytest.mark.parametrize("seed", range(12))
def test_invariants_random(seed):
    h = random_hierarchy(seed, n0=8, num_levels=3, patches_per_level=5, max_size=9, tiles=4)
    _invariants(h)


@pytest.mark.parametrize("seed", [0, 3, 7])
def test_kd_lookup_equals_patch_scan(seed):
    # pin 4: the level found by descending the tree equals the finest level among all
    # patches containing the point, on random points away from cell faces
    h = random_hierarchy(seed, n0=8, num_levels=3, patches_per_level=6, max_size=10, tiles=3)
    o = oracle.Oracle(h)
    box, patch, level = o.leaves()
    rng = np.random.default_rng(seed)
    hf = h.h0 / h.ratio ** (h.num_levels - 1)
    n_checked = 0
    for x in rng.uniform(0.0, 1.0, size=(20000, 3)):
        q = x / hf
        if np.any(np.abs(q - np.round(q)) < 1e-6):
            continue
        lf = o.lookup_leaf(x)
        want = brute_finest_level(h, x)
        assert want is not None
        assert level[lf] == want[0] and patch[lf] == want[1]
        assert o.lookup_scan(x) == want
        n_checked += 1
    assert n_checked > 19000
