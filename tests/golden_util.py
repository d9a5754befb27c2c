"""Readers for the hand-derived fixtures under tests/golden/ and small pure-Python
brute-force checkers used to pin the oracle (they restate nothing from the oracle's code:
they test geometric facts directly)."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_kd_golden(name):
    nodes, leaves = [], []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            if parts[0] == "L":
                leaves.append([int(v) for v in parts[1:]])
            else:
                nodes.append([int(v) for v in parts])
    return np.array(nodes, dtype=np.int64), np.array(leaves, dtype=np.int64)


def finest_boxes(hier):
    """Patch boxes scaled to the finest level's index space."""
    L, r = hier.num_levels, hier.ratio
    sc = np.array([r ** (L - 1 - int(l)) for l in hier.patch_level], dtype=np.int64)
    return hier.patch_box * sc[:, None]


def brute_finest_level(hier, x):
    """Finest level among patches whose half-open world box contains x (None if none)."""
    best = None
    for p in range(hier.num_patches):
        l = int(hier.patch_level[p])
        h = hier.h0 / hier.ratio ** l
        b = hier.patch_box[p]
        lo = hier.domain_lo + b[:3] * h
        hi = hier.domain_lo + b[3:] * h
        if np.all(lo <= x) and np.all(x < hi):
            if best is None or l > best[0]:
                best = (l, p)
    return best


def slab(o, d, lo, hi):
    """Parameter interval [t_enter, t_exit] of the ray o + t d inside box [lo, hi]."""
    t0, t1 = -np.inf, np.inf
    for a in range(3):
        if d[a] == 0.0:
            if not (lo[a] <= o[a] < hi[a]):
                return None
            continue
        ta = (lo[a] - o[a]) / d[a]
        tb = (hi[a] - o[a]) / d[a]
        t0 = max(t0, min(ta, tb))
        t1 = min(t1, max(ta, tb))
    return (max(t0, 0.0), t1)


def ray_of_pixel(cam, i, j):
    W, H = cam.width, cam.height
    u = (2.0 * (i + 0.5) / W - 1.0) * cam.tan_half_fov_y * (W / H)
    v = (1.0 - 2.0 * (j + 0.5) / H) * cam.tan_half_fov_y
    d = cam.fwd + u * cam.right + v * cam.up
    return np.asarray(cam.eye, dtype=np.float64), d
