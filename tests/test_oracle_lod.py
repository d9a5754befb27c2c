"""Pins for the oracle's level-of-detail pruning (Sec. 3.1: type-(a) nodes cover a region
held by at least two levels; Sec. 3.3: the descent may stop at such a node when the
coarser level's cells project small enough, and the node is sampled at that level).

On a properly nested hierarchy, stopping at every type-(a) node of level >= k+1 must give
exactly the render of the hierarchy truncated to levels <= k+1: same segments, samples,
values and gradients.  These pins fix that at both ends and in between, plus the stopping
rule itself on a non-nested hierarchy."""
import dataclasses
import math

import numpy as np

import oracle
import synth
from synth.amr import gaussians_fn, look_camera, make_hierarchy_from_boxes, random_hierarchy


def _nested3():
    """Levels 0..2 (ratio 2), every level-(l+1) patch inside the level-l patches."""
    b0 = [[i * 8, j * 8, k * 8, i * 8 + 8, j * 8 + 8, k * 8 + 8]
          for k in range(2) for j in range(2) for i in range(2)]
    b1 = [[4, 4, 4, 20, 16, 14], [20, 18, 6, 28, 30, 26]]
    b2 = [[10, 10, 10, 30, 28, 24], [42, 38, 14, 54, 58, 50]]
    boxes = b0 + b1 + b2
    levels = [0] * 8 + [1] * 2 + [2] * 2
    rng = np.random.default_rng(21)
    return make_hierarchy_from_boxes(3, 2, (16, 16, 16), boxes, levels, gaussians_fn(rng, 6))


def _truncate(h, top):
    keep = h.patch_level <= top
    return dataclasses.replace(h, patch_level=h.patch_level[keep], patch_box=h.patch_box[keep],
                               data=[d for d, k in zip(h.data, keep) if k])


def _hmin(h, l):
    return float(np.min(h.h0) / h.ratio ** l)


def _params(h, **kw):
    lo, hi = h.value_range()
    return oracle.OracleParams(vmin=lo, vmax=hi, shade=1, kappa=12.0, **kw)


def test_tiny_threshold_is_the_unpruned_march():
    h = _nested3()
    o = oracle.Oracle(h)
    cam = synth.orbit_camera(3, 40, 32)
    tf = synth.ramp_tf()
    a, na = o.render(cam, tf, _params(h))
    b, nb = o.render(cam, tf, _params(h, lod_pixels=1e-9))
    assert np.array_equal(a, b) and np.array_equal(na, nb)


def test_huge_threshold_renders_level_zero_only():
    h = _nested3()
    o = oracle.Oracle(h)
    o0 = oracle.Oracle(_truncate(h, 0))
    cam = synth.orbit_camera(5, 40, 32)
    tf = synth.ramp_tf()
    a, na = o.render(cam, tf, _params(h, lod_pixels=1e9))
    b, nb = o0.render(cam, tf, _params(h))
    assert np.array_equal(a, b) and np.array_equal(na, nb)
    full, nf = o.render(cam, tf, _params(h))
    assert nf.sum() > na.sum() and not np.array_equal(full, a)
    # the pruned segments are the level-0 pieces: same parameters, pruned ids after leaves
    M = o.num_leaves
    for j in range(0, 32, 3):
        for i in range(0, 40, 3):
            l1, s0, s1 = o.trace(cam, i, j, lod_pixels=1e9)
            l2, u0, u1 = o0.trace(cam, i, j)
            assert np.array_equal(s0, u0) and np.array_equal(s1, u1)
            assert len(l1) == len(l2)


def test_far_view_between_levels_renders_the_truncation():
    h = _nested3()
    o = oracle.Oracle(h)
    o1 = oracle.Oracle(_truncate(h, 1))
    D = 20.0
    cam = look_camera((0.5 + D * 0.6, 0.5 + D * 0.48, 0.5 + D * 0.64), (0.5, 0.5, 0.5),
                      (0.0, 0.0, 1.0), 4.0, 36, 30)
    # X(t) = lod (2 tan / H) t stays inside (hmin^1, hmin^0) for t in [D - 1, D + 1]
    lod = math.sqrt(_hmin(h, 0) * _hmin(h, 1)) / (2.0 * cam.tan_half_fov_y / cam.height * D)
    for t in (D - 1.0, D + 1.0):
        X = lod * (2.0 * cam.tan_half_fov_y / cam.height) * t
        assert _hmin(h, 1) < X < _hmin(h, 0)
    tf = synth.ramp_tf()
    a, na = o.render(cam, tf, _params(h, lod_pixels=lod))
    b, nb = o1.render(cam, tf, _params(h))
    assert np.array_equal(a, b) and np.array_equal(na, nb)
    assert np.any(a[..., 3] > 0.05)


def test_stop_rule_on_a_non_nested_hierarchy():
    h = random_hierarchy(7, n0=8, num_levels=4, patches_per_level=6, max_size=10, tiles=5)
    o = oracle.Oracle(h)
    axis, split, left, right, leaf = o.nodes()
    patch, level, lod = o.node_labels()
    N = len(axis)
    parent = np.full(N, -1)
    for k in range(N):
        if axis[k] >= 0:
            parent[left[k]] = k
            parent[right[k]] = k
    M = o.num_leaves
    node_of = {int(lod[k]): k for k in range(N) if lod[k] >= 0}
    assert all(axis[k] >= 0 and patch[k] >= 0 for k in node_of.values())
    cam = synth.orbit_camera(9, 30, 26)
    scale = 2.0 * cam.tan_half_fov_y / cam.height
    lod_px = 6.0
    pruned = 0
    for j in range(0, 26, 2):
        for i in range(0, 30, 2):
            ids, t0, t1 = o.trace(cam, i, j, lod_pixels=lod_px)
            full, f0, f1 = o.trace(cam, i, j)
            if len(ids) == 0:
                assert len(full) == 0
                continue
            assert t0[0] == f0[0] and t1[-1] == f1[-1]
            assert np.array_equal(t0[1:], t1[:-1])  # segments abut
            assert len(ids) <= len(full)
            for q, s in enumerate(ids):
                X = lod_px * scale * t0[q]
                k = node_of[int(s)] if s >= M else int(np.nonzero(leaf == s)[0][0])
                if s >= M:
                    pruned += 1
                    assert _hmin(h, level[k]) <= X
                a = parent[k]
                while a >= 0:  # no labelled ancestor qualified earlier
                    if patch[a] >= 0:
                        assert _hmin(h, level[a]) > X
                    a = parent[a]
    assert pruned > 0
