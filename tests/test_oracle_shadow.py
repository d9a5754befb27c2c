"""Pins for the oracle's secondary rays to a point light (the global-illumination example
of Sec. 5; no formula in the paper): closed forms on constant fields, where the midpoint
product of (1 - alpha) is exactly exp(-kappa a len) for any step, and the lighting of
rendered samples."""
import math

import numpy as np
import pytest

import oracle
import synth
from synth.amr import make_hierarchy_from_boxes, make_uniform


def _const_tf(a):
    tf = np.zeros((256, 4), dtype=np.float32)
    tf[:, :3] = 1.0
    tf[:, 3] = a
    return tf


def _params(**kw):
    base = dict(vmin=0.0, vmax=1.0, kappa=3.0, shadow=1, light_step=0.013, light_ambient=0.2)
    base.update(kw)
    return oracle.OracleParams(**base)


@pytest.mark.parametrize("step", [0.013, 0.05, 0.3])
def test_light_inside_the_domain(step):
    o = oracle.Oracle(make_uniform(12, lambda X, Y, Z: 0.5 + 0 * X))
    tf = _const_tf(0.4)
    light = (0.7, 0.35, 0.6)
    for x in [(0.1, 0.2, 0.3), (0.5, 0.5, 0.5), (0.95, 0.02, 0.5)]:
        T = o.shadow_T(x, tf, _params(light=light, light_step=step))
        d = math.dist(x, light)
        a = float(np.float32(0.4))  # the table holds float32 opacities
        assert T == pytest.approx(math.exp(-3.0 * a * d), rel=1e-12)


def test_light_outside_counts_only_the_path_inside():
    # two level-0 patches tiling [0,1]^3 (the second half along x), constant field
    h = make_hierarchy_from_boxes(1, 2, (8, 8, 8), [[0, 0, 0, 4, 8, 8], [4, 0, 0, 8, 8, 8]],
                                  [0, 0], lambda X, Y, Z: 0.5 + 0 * X)
    o = oracle.Oracle(h)
    tf = _const_tf(0.25)
    light = (3.0, 0.5, 0.5)
    x = (0.2, 0.5, 0.5)
    T = o.shadow_T(x, tf, _params(light=light))
    assert T == pytest.approx(math.exp(-3.0 * 0.25 * 0.8), rel=1e-12)
    # diagonal: exits through y = 1 first
    light = (0.5, 4.0, 2.0)
    x = np.array((0.5, 0.5, 0.5))
    s = (1.0 - 0.5) / (4.0 - 0.5)
    T = o.shadow_T(x, tf, _params(light=light))
    assert T == pytest.approx(math.exp(-3.0 * 0.25 * s * math.dist(x, light)), rel=1e-12)


def test_opaque_path_cuts_to_zero_and_transparent_path_is_one():
    o = oracle.Oracle(make_uniform(10, lambda X, Y, Z: 0.5 + 0 * X))
    assert o.shadow_T((0.5, 0.5, 0.5), _const_tf(0.0), _params(light=(2, 2, 2))) == 1.0
    assert o.shadow_T((0.5, 0.5, 0.5), _const_tf(1.0), _params(light=(0.5, 0.5, 3.0),
                                                                kappa=60.0)) == 0.0


def test_lighting_scales_the_rendered_colour():
    """A transparent light path (TF alpha 0 above 0.6, the field below it along the light
    direction) gives I = 1: shadowed and plain renders agree; an ambient-only light (TF
    opaque towards the light) scales every channel but alpha by the ambient factor."""
    o = oracle.Oracle(make_uniform(10, lambda X, Y, Z: 0.5 + 0 * X))
    cam = synth.orbit_camera(3, 16, 12)
    tf = _const_tf(0.3)
    plain, n0 = o.render(cam, tf, oracle.OracleParams(vmin=0.0, vmax=1.0, kappa=3.0))
    dark, n1 = o.render(cam, tf, _params(light=(0.5, 0.5, 0.5), kappa=3.0, light_step=0.01,
                                         light_ambient=0.2))
    assert np.array_equal(n0, n1)
    assert np.array_equal(dark[..., 3], plain[..., 3])
    # every sample is lit by I in [0.2, 1]: colour between 0.2x and 1x the plain colour
    assert np.all(dark[..., :3] <= plain[..., :3] + 1e-15)
    assert np.all(dark[..., :3] >= 0.2 * plain[..., :3] - 1e-15)
    assert np.any(dark[..., :3] < 0.99 * plain[..., :3])
