"""Pins for the oracle's field evaluation: V_l, S_l and the AMR field F (Sec. 2; Sec. 4 on
interpolation across resolution changes)."""
import numpy as np
import pytest

import oracle
from synth.amr import make_hierarchy_from_boxes, random_hierarchy


def _poly(c):
    """A global trilinear polynomial: span{1, x, y, z, xy, yz, zx, xyz}."""
    def fn(X, Y, Z):
        return (c[0] + c[1] * X + c[2] * Y + c[3] * Z + c[4] * X * Y + c[5] * Y * Z
                + c[6] * Z * X + c[7] * X * Y * Z)
    return fn


def _poly_eval(c, x):
    X, Y, Z = x
    return (c[0] + c[1] * X + c[2] * Y + c[3] * Z + c[4] * X * Y + c[5] * Y * Z + c[6] * Z * X
            + c[7] * X * Y * Z)


@pytest.mark.parametrize("seed", [1, 2, 5, 11])
def test_trilinear_polynomial_reproduced(seed):
    """Trilinear interpolation reproduces trilinear polynomials, and the coarse fallback
    (a cell no level-l patch holds takes S of the finest coarser level holding its centre)
    keeps that exactness across level interfaces: F equals the polynomial at every point
    far enough from the domain boundary (edge replication changes the outer shell)."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(-1, 1, size=8)
    # float32 storage must hold the samples exactly: use dyadic coefficients on a grid
    # whose cell centres are dyadic too
    c = np.round(c * 8) / 8
    h = random_hierarchy(seed, n0=8, num_levels=3, patches_per_level=6, max_size=10, tiles=3,
                         fn=_poly(c))
    o = oracle.Oracle(h)
    pts = rng.uniform(0.25 + 1e-3, 0.75 - 1e-3, size=(3000, 3))  # 2 h^0 from the boundary
    for x in pts:
        want = _poly_eval(c, x)
        assert abs(o.F(x) - want) <= 1e-12 * max(1.0, abs(want))
        # every level's interpolant reproduces it as well, wherever it is defined
        for l in range(h.num_levels):
            assert abs(o.S(l, x) - want) <= 1e-12 * max(1.0, abs(want))


def test_V_direct_and_fallback():
    # level 0: 4^3 cells with value = 100*i + 10*j + k (cell indices); level 1 patch
    # [2,6)^3 holds value 1000 + 100*i + 10*j + k (level-1 indices)
    def lvl0(X, Y, Z):
        i, j, k = np.floor(X * 4), np.floor(Y * 4), np.floor(Z * 4)
        return 100 * i + 10 * j + k

    h = make_hierarchy_from_boxes(2, 2, (4, 4, 4), [[0, 0, 0, 4, 4, 4], [2, 2, 2, 6, 6, 6]],
                                  [0, 1], lvl0)
    h.data[1][:] = 1000 + (100 * np.arange(2, 6)[None, None, :] + 10 * np.arange(2, 6)[None, :, None]
                           + np.arange(2, 6)[:, None, None])
    o = oracle.Oracle(h)
    # stored values
    assert o.V(0, 1, 2, 3) == 123
    assert o.V(1, 3, 4, 5) == 1000 + 345
    # clamping replicates the edge
    assert o.V(0, -5, 2, 9) == 0 * 100 + 20 + 3
    # a level-1 cell outside the fine patch: S_0 at its centre.  Level-1 cell (0,0,0) has
    # centre (1/16,1/16,1/16); level-0 xi = 1/16*4 - 0.5 = -0.25 -> corners clamp to
    # cell 0 in every axis -> value of level-0 cell (0,0,0) = 0
    assert o.V(1, 0, 0, 0) == 0.0
    # level-1 cell (1,1,1): centre 3/16 -> xi = 0.25: w = 0.25 on corners 0 and 1
    want = 0.75 * 0 + 0.25 * 100  # x
    want = want + 0.25 * 10  # y adds 0.25*10 everywhere (linear)
    want = want + 0.25 * 1
    assert abs(o.V(1, 1, 1, 1) - want) < 1e-12


def test_injected_nearest_equals_uniform():
    """Fine patches holding injected coarse values render, with nearest sampling, the
    same field as the coarse grid alone: F agrees everywhere, boundary shell included."""
    rng = np.random.default_rng(4)
    vals = rng.uniform(0, 1, size=(8, 8, 8)).astype(np.float32)

    def coarse(X, Y, Z):
        i = np.clip(np.floor(X * 8).astype(int), 0, 7)
        j = np.clip(np.floor(Y * 8).astype(int), 0, 7)
        k = np.clip(np.floor(Z * 8).astype(int), 0, 7)
        return vals[k, j, i]

    amr = random_hierarchy(9, n0=8, num_levels=3, patches_per_level=6, max_size=10, tiles=3,
                           fn=coarse)
    uni = make_hierarchy_from_boxes(1, 2, (8, 8, 8), [[0, 0, 0, 8, 8, 8]], [0], coarse)
    oa, ou = oracle.Oracle(amr), oracle.Oracle(uni)
    for x in rng.uniform(-0.1, 1.1, size=(4000, 3)):
        assert oa.F(x, interp=0) == ou.F(x, interp=0)
