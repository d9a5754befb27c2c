"""Pins for the oracle's gradient and Phong shading (Sec. 4, Fig. 6: central differences
through the AMR field across block boundaries; headlight Phong).

A field linear in z has the exact central difference g = (0, 0, slope) at every sample
whose neighbours stay where the field is linear - on every level and across leaf and
level boundaries, since every level's cells (data or coarse-filled) sample the same linear
function and trilinear interpolation reproduces it.  With a transfer function of constant
colour, every opaque sample of a ray then has the same shaded colour, so a pixel's colour
divided by its opacity is the Phong formula itself at |n.L| = |d_z| / |d| (headlight
L = -d / |d|).  A second pin activates the gradient floor (n = g / max(|g|, gamma (vmax -
vmin) / h)), which fixes the central difference's 1/2h scale and the floor's 1/h."""
import numpy as np
import pytest

import oracle
from synth.amr import look_camera, make_hierarchy_from_boxes, make_uniform
from golden_util import ray_of_pixel

RGB = (0.3, 0.5, 0.2)


def _box_tf(lo_u, hi_u, a=0.8):
    """Constant colour; opacity a for u in [lo_u, hi_u], zero elsewhere."""
    tf = np.zeros((256, 4), dtype=np.float32)
    tf[:, :3] = RGB
    u = np.arange(256) / 255.0
    tf[(u >= lo_u) & (u <= hi_u), 3] = a
    return tf


def _phong(ndl, ka=0.3, kd=0.6, ks=0.3, shininess=32.0):
    rgb = np.asarray(RGB, dtype=np.float32).astype(np.float64)
    return np.clip(rgb * (ka + kd * ndl) + ks * ndl ** shininess, 0.0, 1.0)


def _check(img, cam, ndl_of, min_alpha=1e-3, tol=1e-9):
    hit = 0
    for j in range(cam.height):
        for i in range(cam.width):
            A = img[j, i, 3]
            if A < min_alpha:
                continue
            hit += 1
            _, d = ray_of_pixel(cam, i, j)
            want = _phong(ndl_of(d))
            np.testing.assert_allclose(img[j, i, :3] / A, want, rtol=0, atol=tol,
                                       err_msg=f"pixel {(i, j)}")
    return hit


def test_linear_field_shading_across_levels_is_phong_of_the_true_normal():
    # a three-level non-nested hierarchy (the level-2 patch straddles two level-1 patches)
    boxes = [[0, 0, 0, 4, 8, 8], [4, 0, 0, 8, 8, 8],
             [4, 4, 4, 9, 11, 8], [9, 5, 6, 12, 12, 12],
             [9, 9, 9, 20, 15, 14], [16, 16, 16, 24, 24, 24]]
    h = make_hierarchy_from_boxes(3, 2, (8, 8, 8), boxes, [0, 0, 1, 1, 2, 2],
                                  lambda X, Y, Z: Z)
    o = oracle.Oracle(h)
    # opaque only for z in [0.3, 0.7]: every opaque sample and its neighbours (one level
    # cell, at most 1/8, away) lie where the field is z exactly
    tf = _box_tf(0.3, 0.7)
    cam = look_camera((0.45, 0.1, -1.2), (0.55, 0.5, 0.5), (0, 1, 0), 30.0, 13, 11)
    pr = oracle.OracleParams(vmin=0.0, vmax=1.0, kappa=6.0, ert_eps=0.0, shade=1)
    img, _ = o.render(cam, tf, pr)
    hit = _check(img, cam, lambda d: abs(d[2]) / np.linalg.norm(d))
    assert hit > 100
    # unshaded, the same opacities: only the colour changes
    img0, _ = o.render(cam, tf, oracle.OracleParams(vmin=0.0, vmax=1.0, kappa=6.0,
                                                    ert_eps=0.0, shade=0))
    np.testing.assert_allclose(img[..., 3], img0[..., 3], rtol=0, atol=1e-15)
    np.testing.assert_allclose(img0[..., :3], np.asarray(RGB, np.float32) * img0[..., 3:4],
                               rtol=0, atol=1e-12)


@pytest.mark.parametrize("interp", [1, 0])
@pytest.mark.parametrize("gamma", [0.5, 2.0])
def test_gradient_floor_scales_the_normal(gamma, interp):
    # one level, h = 1/16: g = (0, 0, 1) also under nearest sampling (the neighbours' cells
    # are the sample's cell +- one, whose centres differ by 2h); floor gamma * 1 / h = 16 gamma
    n = 16
    h = make_uniform(n, lambda X, Y, Z: Z)
    o = oracle.Oracle(h)
    tf = _box_tf(0.3, 0.7)
    cam = look_camera((0.4, 0.2, -1.0), (0.5, 0.55, 0.5), (0, 1, 0), 30.0, 9, 8)
    pr = oracle.OracleParams(vmin=0.0, vmax=1.0, kappa=6.0, ert_eps=0.0, shade=1,
                             gamma=gamma, interp=interp)
    img, _ = o.render(cam, tf, pr)
    floor = gamma * 1.0 * n
    hit = _check(img, cam, lambda d: abs(d[2]) / (floor * np.linalg.norm(d)))
    assert hit > 30


def test_gradient_floor_takes_the_segment_level_across_levels():
    # two levels: level 0 is 16^3 (h = 1/16), a level-1 slab x in [0.375, 0.625) covers all
    # of y and z (h = 1/32).  With gamma 0.5 the floor is 8 in coarse leaves and 16 in fine
    # ones, both above |g| = 1, so |n.L| = |d_z| / (floor_l |d|) with l the level of the
    # sample's own leaf.  Rays run nearly along +z; a pixel is checked when all of its
    # opaque samples (z in [0.3, 0.7]) lie in one region: coarse, the slab's interior, or
    # the slab's outer fine cells, whose x-neighbours at +-1/32 lie in a coarse leaf (where
    # a floor taken from a neighbour's level instead of the segment's would be 8, not 16)
    h = make_hierarchy_from_boxes(2, 2, (16, 16, 16),
                                  [[0, 0, 0, 16, 16, 16], [12, 0, 0, 20, 32, 32]], [0, 1],
                                  lambda X, Y, Z: Z)
    o = oracle.Oracle(h)
    tf = _box_tf(0.3, 0.7)
    W, H = 61, 5
    dist = 40.0
    # horizontal half-width 0.36 at the volume's centre: pixels span x in [0.14, 0.86]
    fov_y = 2.0 * np.degrees(np.arctan(0.36 / (dist + 0.5) * H / W))
    cam = look_camera((0.5, 0.5, -dist), (0.5, 0.5, 0.5), (0, 1, 0), fov_y, W, H)
    gamma = 0.5
    pr = oracle.OracleParams(vmin=0.0, vmax=1.0, kappa=6.0, ert_eps=0.0, shade=1, gamma=gamma)
    img, _ = o.render(cam, tf, pr)
    lo_f, hi_f, hf = 0.375, 0.625, 1.0 / 32
    seen = {"coarse": 0, "fine": 0, "fine_edge": 0}
    for j in range(H):
        for i in range(W):
            o_, d = ray_of_pixel(cam, i, j)
            xs = [o_[0] + (z - o_[2]) / d[2] * d[0] for z in (0.29, 0.71)]
            x0, x1 = min(xs), max(xs)
            if x1 < lo_f - 1e-3 or x0 >= hi_f + 1e-3:
                region, floor = "coarse", gamma * 16
            elif x0 >= lo_f + hf + 1e-3 and x1 < hi_f - hf - 1e-3:
                region, floor = "fine", gamma * 32
            elif (x0 >= lo_f + 1e-3 and x1 < lo_f + hf - 1e-3) or \
                    (x0 >= hi_f - hf + 1e-3 and x1 < hi_f - 1e-3):
                region, floor = "fine_edge", gamma * 32
            else:
                continue
            A = img[j, i, 3]
            assert A > 1e-3, (i, j)
            want = _phong(abs(d[2]) / (floor * np.linalg.norm(d)))
            np.testing.assert_allclose(img[j, i, :3] / A, want, rtol=0, atol=1e-9,
                                       err_msg=f"pixel {(i, j)} ({region})")
            seen[region] += 1
    assert seen["coarse"] >= 20 and seen["fine"] >= 10 and seen["fine_edge"] >= 5, seen
