"""Pins for the oracle's rays, kd-restart traversal, sampling and compositing
(Sec. 3 outline: front-to-back emission-absorption; Sec. 3.3 ray traversal; Sec. 5 on
the emission-absorption model)."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
import synth
from synth.amr import look_camera, make_hierarchy_from_boxes, make_uniform, random_hierarchy
from golden_util import ray_of_pixel, slab


def _const_tf(rgba):
    return np.tile(np.asarray(rgba, dtype=np.float32), (256, 1))


# ------------------------------------------------------------------------------ traversal

def _leaf_world_boxes(h, box):
    hf = h.h0 / h.ratio ** (h.num_levels - 1)
    return h.domain_lo + box[:, :3] * hf, h.domain_lo + box[:, 3:] * hf


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_trace_properties_and_bruteforce(seed):
    h = random_hierarchy(seed, n0=8, num_levels=3, patches_per_level=5, max_size=9, tiles=4)
    o = oracle.Oracle(h)
    box, patch, level = o.leaves()
    lo, hi = _leaf_world_boxes(h, box)
    cam = synth.orbit_camera(100 + seed, 24, 20)
    compared = 0
    for j in range(cam.height):
        for i in range(cam.width):
            leaf, t0, t1 = o.trace(cam, i, j)
            orig, d = ray_of_pixel(cam, i, j)
            if len(leaf) == 0:
                assert slab(orig, d, np.zeros(3), np.ones(3)) is None or \
                    slab(orig, d, np.zeros(3), np.ones(3))[1] <= slab(orig, d, np.zeros(3), np.ones(3))[0]
                continue
            # ordered, abutting, positive length, covering [t_in, t_out]
            assert np.all(t1 > t0)
            assert np.all(t0[1:] == t1[:-1])
            t_in, t_out = slab(orig, d, np.zeros(3), np.ones(3))
            assert abs(t0[0] - t_in) < 1e-12 and abs(t1[-1] - t_out) < 1e-12
            # each segment's midpoint lies in its leaf
            for k in range(len(leaf)):
                m = orig + 0.5 * (t0[k] + t1[k]) * d
                assert np.all(m >= lo[leaf[k]] - 1e-9) and np.all(m <= hi[leaf[k]] + 1e-9)
            # brute force: every leaf slab interval of positive length, sorted by entry
            iv = []
            for m in range(len(box)):
                s = slab(orig, d, lo[m], hi[m])
                if s is not None and s[1] - s[0] > 1e-9:
                    iv.append((s[0], m))
            iv.sort()
            ent = np.array([v[0] for v in iv])
            if len(ent) > 1 and np.min(np.diff(ent)) < 1e-9:
                continue  # the ray grazes an edge: entry order is not unique
            assert [v[1] for v in iv] == leaf.tolist()
            compared += 1
    assert compared > 200


def test_axis_aligned_ray_zero_direction_components():
    # odd image sizes put the centre pixel exactly on the optical axis: d has two zero
    # components and the traversal takes the d_a == 0 branches
    h = random_hierarchy(5, n0=8, num_levels=3, patches_per_level=5, max_size=9, tiles=4)
    o = oracle.Oracle(h)
    box, _, _ = o.leaves()
    lo, hi = _leaf_world_boxes(h, box)
    cam = look_camera((0.3, 0.55, -1.0), (0.3, 0.55, 0.5), (0, 1, 0), 30.0, 5, 5)
    orig, d = ray_of_pixel(cam, 2, 2)
    assert d[0] == 0.0 and d[1] == 0.0
    leaf, t0, t1 = o.trace(cam, 2, 2)
    zs = orig[2] + np.concatenate([t0, t1[-1:]]) * d[2]
    assert abs(zs[0] - 0.0) < 1e-12 and abs(zs[-1] - 1.0) < 1e-12
    for k, m in enumerate(leaf):
        assert lo[m][0] <= 0.3 < hi[m][0] and lo[m][1] <= 0.55 < hi[m][1]
        assert abs(orig[2] + t0[k] * d[2] - lo[m][2]) < 1e-12


def test_miss_gives_zero():
    h = make_uniform(4, lambda X, Y, Z: X)
    o = oracle.Oracle(h)
    cam = look_camera((3.0, 3.0, 3.0), (6.0, 6.0, 6.0), (0, 0, 1), 10.0, 8, 8)  # looks away
    img, smp = o.render(cam, synth.ramp_tf(), oracle.OracleParams())
    assert np.all(img == 0) and np.all(smp == 0)


# ------------------------------------------------------------------------------ closed forms

@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("step", [0.5, 0.37])
def test_constant_field_alpha_closed_form(seed, step):
    """Constant field and colour: A = 1 - exp(-sigma L), C = rgb A, for any hierarchy and
    any step, since the per-sample transmittances multiply to exp(-sigma L)."""
    h = random_hierarchy(seed, n0=8, num_levels=3, patches_per_level=5, max_size=9, tiles=4,
                         fn=lambda X, Y, Z: np.full_like(X, 0.5))
    o = oracle.Oracle(h)
    rgba = (0.2, 0.5, 0.9, 0.7)
    kappa = 3.0
    cam = synth.orbit_camera(7 + seed, 16, 12)
    pr = oracle.OracleParams(vmin=0.0, vmax=1.0, kappa=kappa, ert_eps=0.0, step_factor=step)
    img, smp = o.render(cam, _const_tf(rgba), pr)
    rgba32 = np.asarray(rgba, dtype=np.float32).astype(np.float64)
    for j in range(cam.height):
        for i in range(cam.width):
            orig, d = ray_of_pixel(cam, i, j)
            s = slab(orig, d, np.zeros(3), np.ones(3))
            if s is None or s[1] <= s[0]:
                assert np.all(img[j, i] == 0)
                continue
            L = np.linalg.norm(d) * (s[1] - s[0])
            A = 1.0 - math.exp(-kappa * rgba32[3] * L)
            assert abs(img[j, i, 3] - A) < 1e-12
            np.testing.assert_allclose(img[j, i, :3], rgba32[:3] * A, atol=1e-12)


def test_ert_stops_at_threshold():
    h = make_uniform(8, lambda X, Y, Z: np.full_like(X, 0.5))
    o = oracle.Oracle(h)
    cam = look_camera((0.5, 0.5, -1.0), (0.5, 0.5, 0.5), (0, 1, 0), 5.0, 3, 3)
    tf = _const_tf((1.0, 1.0, 1.0, 1.0))
    pr = oracle.OracleParams(kappa=200.0, ert_eps=1e-2)
    img, smp = o.render(cam, tf, pr)
    pr0 = oracle.OracleParams(kappa=200.0, ert_eps=0.0)
    img0, smp0 = o.render(cam, tf, pr0)
    assert np.all(img[..., 3] >= 1 - 1e-2)
    assert np.all(smp < smp0)
    assert np.max(np.abs(img - img0)) <= 1e-2


def _linear_z_setup(n=16):
    h = make_uniform(n, lambda X, Y, Z: Z)
    tf = np.zeros((256, 4), dtype=np.float32)
    u = np.arange(256) / 255.0
    tf[:, 0] = u
    tf[:, 1] = 1 - u
    tf[:, 2] = 0.5
    tf[:, 3] = 1.0
    return h, tf


def _exact_emission(h, cam, i, j, kappa, n):
    """Emission-absorption integral of the exact field along the ray: the trilinear
    interpolant of v = z on an n^3 grid is z itself between the first and last cell
    centres and constant beyond (edge replication)."""
    orig, d = ray_of_pixel(cam, i, j)
    t_in, t_out = slab(orig, d, np.zeros(3), np.ones(3))
    dn = np.linalg.norm(d)
    L = dn * (t_out - t_in)
    lo, hi = 0.5 / n, 1.0 - 0.5 / n
    vmin, vmax = lo, hi

    def z_of(s):
        return orig[2] + (t_in + s / dn) * d[2]

    def red(s):
        v = min(max(z_of(s), lo), hi)
        return (v - vmin) / (vmax - vmin)

    brk = []
    for zb in (lo, hi):
        if d[2] != 0:
            s = ((zb - orig[2]) / d[2] - t_in) * dn
            if 0 < s < L:
                brk.append(s)
    val, _ = integrate.quad(lambda s: red(s) * kappa * math.exp(-kappa * s), 0.0, L,
                            points=brk or None, epsabs=1e-13, epsrel=1e-13, limit=200)
    return val, 1.0 - math.exp(-kappa * L), vmin, vmax


def test_midpoint_quadrature_converges_second_order():
    """A field linear along the ray with constant extinction: the composited colour
    converges to the emission-absorption integral with error ~ step^2 (midpoint rule)."""
    n = 16
    h, tf = _linear_z_setup(n)
    o = oracle.Oracle(h)
    cam = look_camera((0.41, 0.37, -0.9), (0.52, 0.6, 0.5), (0, 1, 0), 20.0, 7, 5)
    kappa = 2.5
    errs = []
    for f in (0.5, 0.25, 0.125):
        e = []
        pr = None
        for (i, j) in [(3, 2), (6, 4), (2, 3)]:
            want_r, want_a, vmin, vmax = _exact_emission(h, cam, i, j, kappa, n)
            pr = oracle.OracleParams(vmin=vmin, vmax=vmax, kappa=kappa, ert_eps=0.0,
                                     step_factor=f)
            got, _ = o.render(cam, tf, pr, pixels=[(i, j)])
            assert abs(got[0, 3] - want_a) < 1e-12
            e.append(abs(got[0, 0] - want_r))
        errs.append(max(e))
    assert errs[-1] < 2e-5, errs
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.6 and 3.5 < r2 < 4.6, errs


def test_prolonged_trilinear_hierarchy_renders_like_uniform():
    """Fine patches holding samples of a global trilinear field: F is the same function
    as on the uniform grid, so images differ only by quadrature placement, which shrinks
    as the (level-independent) world step shrinks."""
    c = np.array([0.25, 0.5, -0.25, 0.75, 0.125, 0.0, -0.5, 0.25])

    def fn(X, Y, Z):
        return (c[0] + c[1] * X + c[2] * Y + c[3] * Z + c[4] * X * Y + c[5] * Y * Z
                + c[6] * Z * X + c[7] * X * Y * Z)

    # fine patches keep two coarse cells away from the domain boundary, where edge
    # replication (not the polynomial) defines the field; the level-2 patch straddles the
    # two level-1 patches
    boxes = [[0, 0, 0, 4, 8, 8], [4, 0, 0, 8, 8, 8],
             [4, 4, 4, 9, 11, 8], [9, 5, 6, 12, 12, 12],
             [9, 9, 9, 20, 15, 14], [16, 16, 16, 24, 24, 24]]
    amr = make_hierarchy_from_boxes(3, 2, (8, 8, 8), boxes, [0, 0, 1, 1, 2, 2], fn)
    uni = make_hierarchy_from_boxes(1, 2, (8, 8, 8), [[0, 0, 0, 8, 8, 8]], [0], fn)
    oa, ou = oracle.Oracle(amr), oracle.Oracle(uni)
    # keep the TF support inside the region where F is exact: only mid-range values opaque
    tf = synth.ramp_tf()
    cam = look_camera((0.5, 0.5, -1.5), (0.5, 0.5, 0.5), (0, 1, 0), 8.0, 12, 12)
    diffs = []
    for ws in (1 / 64, 1 / 256):
        pr = oracle.OracleParams(vmin=-0.5, vmax=1.5, kappa=4.0, ert_eps=0.0, world_step=ws)
        ia, _ = oa.render(cam, tf, pr)
        iu, _ = ou.render(cam, tf, pr)
        diffs.append(np.max(np.abs(ia - iu)))
    assert diffs[1] < diffs[0] / 3 and diffs[1] < 1e-4, diffs
