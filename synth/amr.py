"""Seeded synthetic AMR hierarchies, cameras and transfer functions.

The paper measures on three cosmology SAMR datasets that are not available here; these
generators stand in for their shapes (block-structured refinement with ratio 2, patches
of 8-64 cells per axis clustered on density peaks, fine patches that straddle coarse
parents).  Everything is deterministic for a given seed.

Conventions shared by every consumer:
  * level l has spacing h^l = h^0 / r^l per axis (Sec. 2 of the paper);
  * a patch box is half-open [lo, hi) in level-l cell indices, int64[6] = lo xyz, hi xyz;
  * cell data is float32, shape [nz, ny, nx], C-contiguous, so x is fastest:
    value(i, j, k) = data[k, j, i] = flat[i + nx * (j + ny * k)];
  * the domain is [domain_lo, domain_lo + n0 * h^0) per axis.
"""
from __future__ import annotations

import hashlib
import math
import os
from dataclasses import dataclass, field
from typing import Callable, List, Optional, Sequence

import numpy as np

# ----------------------------------------------------------------------------------------
# containers
# ----------------------------------------------------------------------------------------


@dataclass
class Hierarchy:
    num_levels: int
    ratio: int
    domain_lo: np.ndarray  # float64[3]
    h0: np.ndarray  # float64[3]
    patch_level: np.ndarray  # int32[P]
    patch_box: np.ndarray  # int64[P, 6]
    data: List[np.ndarray]  # float32[nz, ny, nx] per patch
    name: str = "hierarchy"
    meta: dict = field(default_factory=dict)

    @property
    def num_patches(self) -> int:
        return int(self.patch_level.shape[0])

    def n_cells(self) -> int:
        return int(sum(int(d.size) for d in self.data))

    def nbytes(self) -> int:
        return int(sum(int(d.nbytes) for d in self.data))

    def root_cells(self) -> np.ndarray:
        """Level-0 extent (cells per axis) of the bounding box of the level-0 patches."""
        b = self.patch_box[self.patch_level == 0]
        return b[:, 3:].max(axis=0) - b[:, :3].min(axis=0)

    def value_range(self):
        lo = min(float(d.min()) for d in self.data)
        hi = max(float(d.max()) for d in self.data)
        return lo, hi

    def patches_per_level(self):
        return [int((self.patch_level == l).sum()) for l in range(self.num_levels)]


@dataclass
class Camera:
    eye: np.ndarray  # float64[3]
    fwd: np.ndarray  # float64[3]
    right: np.ndarray  # float64[3]
    up: np.ndarray  # float64[3]
    tan_half_fov_y: float
    width: int
    height: int


# ----------------------------------------------------------------------------------------
# cameras and transfer functions
# ----------------------------------------------------------------------------------------


def look_camera(eye, target, world_up, fov_y_deg: float, width: int, height: int) -> Camera:
    eye = np.asarray(eye, dtype=np.float64)
    target = np.asarray(target, dtype=np.float64)
    world_up = np.asarray(world_up, dtype=np.float64)
    fwd = target - eye
    fwd = fwd / np.linalg.norm(fwd)
    right = np.cross(fwd, world_up)
    if np.linalg.norm(right) < 1e-12:  # looking along world_up: pick any perpendicular
        right = np.cross(fwd, np.array([1.0, 0.0, 0.0]))
        if np.linalg.norm(right) < 1e-12:
            right = np.cross(fwd, np.array([0.0, 1.0, 0.0]))
    right = right / np.linalg.norm(right)
    up = np.cross(right, fwd)
    return Camera(eye, fwd, right, up, float(math.tan(math.radians(fov_y_deg) / 2.0)),
                  int(width), int(height))


def orbit_camera(seed: int, width: int, height: int, radius: float = 2.0,
                 fov_y_deg: float = 40.0, center=(0.5, 0.5, 0.5)) -> Camera:
    """Orbit pose around `center`: azimuth U[0, 2pi), elevation U[-60, 60] degrees, up = +z."""
    rng = np.random.default_rng(seed)
    az = rng.uniform(0.0, 2.0 * math.pi)
    el = math.radians(rng.uniform(-60.0, 60.0))
    c = np.asarray(center, dtype=np.float64)
    eye = c + radius * np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az),
                                 math.sin(el)])
    return look_camera(eye, c, (0.0, 0.0, 1.0), fov_y_deg, width, height)


def ramp_tf(n: int = 256, alpha_start: float = 0.1,
            rgb_lo=(0.0, 0.2, 1.0), rgb_hi=(1.0, 0.3, 0.0)) -> np.ndarray:
    """Piecewise-linear RGBA ramp: rgb linear from rgb_lo to rgb_hi, alpha 0 below
    `alpha_start`, then linear to 1 at the top entry.  float32[n, 4]."""
    t = np.arange(n, dtype=np.float64) / (n - 1)
    tf = np.zeros((n, 4), dtype=np.float64)
    for c in range(3):
        tf[:, c] = (1.0 - t) * rgb_lo[c] + t * rgb_hi[c]
    tf[:, 3] = np.clip((t - alpha_start) / (1.0 - alpha_start), 0.0, 1.0)
    return tf.astype(np.float32)


def tf_variants(n: int = 256) -> List[np.ndarray]:
    """Four distinct 256-entry RGBA transfer functions (used for multi-view batches)."""
    out = [ramp_tf(n)]
    out.append(ramp_tf(n, alpha_start=0.3, rgb_lo=(0.1, 0.1, 0.1), rgb_hi=(1.0, 1.0, 0.9)))
    t = np.arange(n, dtype=np.float64) / (n - 1)
    bump = np.zeros((n, 4))
    bump[:, 0] = 0.5 + 0.5 * np.sin(6.0 * t)
    bump[:, 1] = t
    bump[:, 2] = 1.0 - t
    bump[:, 3] = np.exp(-((t - 0.6) / 0.08) ** 2)
    out.append(bump.astype(np.float32))
    step = np.zeros((n, 4))
    step[:, :3] = np.stack([t, t * t, np.sqrt(t)], axis=1)
    step[:, 3] = (t > 0.5) * 0.7
    out.append(step.astype(np.float32))
    return out


# ----------------------------------------------------------------------------------------
# generic construction helpers
# ----------------------------------------------------------------------------------------


def _cell_centres(lo: int, hi: int, h: float, dlo: float) -> np.ndarray:
    return dlo + (np.arange(lo, hi, dtype=np.float64) + 0.5) * h


def make_hierarchy_from_boxes(num_levels: int, ratio: int, n0: Sequence[int],
                              boxes: Sequence[Sequence[int]], levels: Sequence[int],
                              fn: Callable[[np.ndarray, np.ndarray, np.ndarray], np.ndarray],
                              name: str = "custom", domain_lo=(0.0, 0.0, 0.0),
                              extent=(1.0, 1.0, 1.0)) -> Hierarchy:
    """Sample `fn(X, Y, Z)` (broadcast float64 arrays of cell-centre coordinates) on every
    patch at its own level."""
    n0 = np.asarray(n0, dtype=np.int64)
    dlo = np.asarray(domain_lo, dtype=np.float64)
    h0 = np.asarray(extent, dtype=np.float64) / n0
    data = []
    for b, l in zip(boxes, levels):
        h = h0 / (ratio ** l)
        xs = _cell_centres(b[0], b[3], h[0], dlo[0])
        ys = _cell_centres(b[1], b[4], h[1], dlo[1])
        zs = _cell_centres(b[2], b[5], h[2], dlo[2])
        Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
        data.append(np.ascontiguousarray(fn(X, Y, Z), dtype=np.float32))
    return Hierarchy(num_levels, ratio, dlo, h0, np.asarray(levels, dtype=np.int32),
                     np.asarray(boxes, dtype=np.int64).reshape(-1, 6), data, name)


def make_uniform(n: int, fn, name: str = "uniform") -> Hierarchy:
    """One level-0 patch of n^3 cells on [0,1]^3."""
    return make_hierarchy_from_boxes(1, 2, (n, n, n), [[0, 0, 0, n, n, n]], [0], fn, name)


def gaussians_fn(rng: np.random.Generator, count: int = 8):
    c = rng.uniform(0.0, 1.0, size=(count, 3))
    s = rng.uniform(0.05, 0.15, size=count)
    a = rng.uniform(0.2, 1.0, size=count)

    def fn(X, Y, Z):
        v = np.zeros(np.broadcast(X, Y, Z).shape, dtype=np.float64)
        for m in range(count):
            r2 = (X - c[m, 0]) ** 2 + (Y - c[m, 1]) ** 2 + (Z - c[m, 2]) ** 2
            v += a[m] * np.exp(-r2 / (2.0 * s[m] ** 2))
        return v

    return fn


def _disjoint(a, b) -> bool:
    return any(a[3 + k] <= b[k] or b[3 + k] <= a[k] for k in range(3))


def random_hierarchy(seed: int, n0: int = 8, num_levels: int = 3, ratio: int = 2,
                     patches_per_level: int = 4, max_size: int = 8,
                     tiles: int = 3, fn=None) -> Hierarchy:
    """Small random hierarchy for property tests: level 0 is a random guillotine tiling
    of an n0^3 root into `tiles`+ boxes; level l >= 1 holds up to `patches_per_level`
    disjoint random boxes anywhere in the level-l index space (nesting not enforced,
    so fine patches may straddle coarse parents or poke outside them)."""
    rng = np.random.default_rng(seed)
    boxes = [[0, 0, 0, n0, n0, n0]]
    for _ in range(tiles - 1):
        idx = int(rng.integers(len(boxes)))
        b = boxes[idx]
        axes = [a for a in range(3) if b[3 + a] - b[a] >= 2]
        if not axes:
            continue
        a = int(rng.choice(axes))
        s = int(rng.integers(b[a] + 1, b[3 + a]))
        left = list(b)
        right = list(b)
        left[3 + a] = s
        right[a] = s
        boxes[idx] = left
        boxes.append(right)
    levels = [0] * len(boxes)
    for l in range(1, num_levels):
        n_l = n0 * ratio ** l
        placed = []
        for _ in range(patches_per_level):
            for _try in range(50):
                size = np.minimum(rng.integers(1, max_size + 1, size=3), n_l)
                lo = np.array([rng.integers(0, n_l - size[k] + 1) for k in range(3)])
                cand = [int(lo[0]), int(lo[1]), int(lo[2]), int(lo[0] + size[0]),
                        int(lo[1] + size[1]), int(lo[2] + size[2])]
                if all(_disjoint(cand, p) for p in placed):
                    placed.append(cand)
                    break
        boxes.extend(placed)
        levels.extend([l] * len(placed))
    if fn is None:
        fn = gaussians_fn(rng, 4)
    return make_hierarchy_from_boxes(num_levels, ratio, (n0, n0, n0), boxes, levels, fn,
                                     name=f"random{seed}")


# ----------------------------------------------------------------------------------------
# configuration 1: tiny 2-level hierarchy
# ----------------------------------------------------------------------------------------


def make_c1(seed: int = 1) -> Hierarchy:
    """Level 0: 2x2x2 patches of 16^3 tiling [0,1]^3 (h^0 = 1/32).  Level 1 (ratio 2,
    a 64^3 index space): 4 disjoint patches with per-axis sizes U{16..24} at seeded
    cell-aligned positions; patch 0 straddles x = 32, the face between two level-0
    parents.  Field: sum of 8 seeded isotropic Gaussians at cell centres."""
    rng = np.random.default_rng(seed)
    boxes, levels = [], []
    for k in range(2):
        for j in range(2):
            for i in range(2):
                boxes.append([16 * i, 16 * j, 16 * k, 16 * i + 16, 16 * j + 16, 16 * k + 16])
                levels.append(0)
    placed = []
    while len(placed) < 4:
        size = rng.integers(16, 25, size=3)
        lo = [int(rng.integers(0, 64 - size[a] + 1)) for a in range(3)]
        if not placed:  # force a straddle of the x = 32 face
            lo[0] = int(rng.integers(32 - size[0] + 1, 32))
        cand = [lo[0], lo[1], lo[2], lo[0] + int(size[0]), lo[1] + int(size[1]),
                lo[2] + int(size[2])]
        if all(_disjoint(cand, p) for p in placed):
            placed.append(cand)
    boxes.extend(placed)
    levels.extend([1] * 4)
    fn = gaussians_fn(rng, 8)
    return make_hierarchy_from_boxes(2, 2, (32, 32, 32), boxes, levels, fn, name="c1")


def c1_workload(seed: int = 1, width: int = 256, height: int = 256, camera_seed: int = 1):
    hier = make_c1(seed)
    vmin, vmax = hier.value_range()
    return dict(hier=hier, camera=orbit_camera(camera_seed, width, height), tf=ramp_tf(),
                vmin=vmin, vmax=vmax, kappa=8.0, step_factor=0.5, ert_eps=1e-4,
                shade=False, name=f"c1_{width}x{height}")


# ----------------------------------------------------------------------------------------
# configuration 2 (and deeper variants): lognormal field with clustered refinement
# ----------------------------------------------------------------------------------------


class GaussianRandomField:
    """delta(x) = sum_m sqrt(2/M) cos(k_m . x + phi_m): unit variance, isotropic, with
    |k| uniform in [2 pi k_lo, 2 pi k_hi] so that the power per |k| shell is flat, i.e.
    P(k) proportional to k^-2 in 3D.  rho = exp(delta) is the lognormal density."""

    def __init__(self, seed: int, M: int = 2048, k_lo: float = 1.0, k_hi: float = 64.0):
        rng = np.random.default_rng(seed)
        kmag = rng.uniform(2 * math.pi * k_lo, 2 * math.pi * k_hi, size=M)
        cost = rng.uniform(-1.0, 1.0, size=M)
        phi = rng.uniform(0.0, 2 * math.pi, size=M)
        sint = np.sqrt(1.0 - cost ** 2)
        self.k = np.stack([kmag * sint * np.cos(phi), kmag * sint * np.sin(phi), kmag * cost],
                          axis=1)
        self.phase = rng.uniform(0.0, 2 * math.pi, size=M)
        self.amp = math.sqrt(2.0 / M)
        self.M = M

    def sample_box(self, xs: np.ndarray, ys: np.ndarray, zs: np.ndarray, device=None):
        """delta on the tensor grid xs x ys x zs -> float64[nz, ny, nx]."""
        import torch

        dev = torch.device(device) if device is not None else torch.device("cpu")
        k = torch.as_tensor(self.k, dtype=torch.float64, device=dev)
        ph = torch.as_tensor(self.phase, dtype=torch.float64, device=dev)
        x = torch.as_tensor(xs, dtype=torch.float64, device=dev)
        y = torch.as_tensor(ys, dtype=torch.float64, device=dev)
        z = torch.as_tensor(zs, dtype=torch.float64, device=dev)
        nx, ny, nz = x.numel(), y.numel(), z.numel()
        out = torch.zeros(nz, ny * nx, dtype=torch.float64, device=dev)
        chunk = max(1, min(self.M, (1 << 24) // max(1, ny * nx)))
        for m0 in range(0, self.M, chunk):
            m1 = min(self.M, m0 + chunk)
            kk = k[m0:m1]
            X = torch.polar(torch.ones(m1 - m0, nx, dtype=torch.float64, device=dev),
                            kk[:, 0:1] * x[None, :])
            Y = torch.polar(torch.ones(m1 - m0, ny, dtype=torch.float64, device=dev),
                            kk[:, 1:2] * y[None, :])
            Z = torch.polar(torch.full((m1 - m0, nz), self.amp, dtype=torch.float64, device=dev),
                            kk[:, 2:3] * z[None, :] + ph[m0:m1, None])
            YX = (Y[:, :, None] * X[:, None, :]).reshape(m1 - m0, ny * nx)
            out += (Z.transpose(0, 1) @ YX).real
        return out.reshape(nz, ny, nx).cpu().numpy()


def _tile_patches(flag_idx: np.ndarray, n_l: np.ndarray, tile: int, offset: int,
                  min_cells: int) -> List[List[int]]:
    """Cluster flagged level-l cells (int64[F, 3]) into one box per tile of a global tile
    grid (size `tile`, shifted by `offset`): the bounding box of the tile's flagged cells,
    grown by one cell, clipped to the tile and the domain, then widened inside the tile to
    at least `min_cells` per axis.  Boxes of different tiles are disjoint."""
    if flag_idx.shape[0] == 0:
        return []
    t = (flag_idx + offset) // tile
    order = np.lexsort((t[:, 0], t[:, 1], t[:, 2]))
    t = t[order]
    f = flag_idx[order]
    brk = np.nonzero(np.any(t[1:] != t[:-1], axis=1))[0] + 1
    starts = np.concatenate([[0], brk])
    ends = np.concatenate([brk, [t.shape[0]]])
    boxes = []
    for s, e in zip(starts, ends):
        tt = t[s]
        tlo = np.maximum(tt * tile - offset, 0)
        thi = np.minimum(tt * tile - offset + tile, n_l)
        lo = f[s:e].min(axis=0) - 1
        hi = f[s:e].max(axis=0) + 2
        lo = np.maximum(lo, tlo)
        hi = np.minimum(hi, thi)
        for a in range(3):
            while hi[a] - lo[a] < min_cells:
                if hi[a] < thi[a]:
                    hi[a] += 1
                if hi[a] - lo[a] < min_cells and lo[a] > tlo[a]:
                    lo[a] -= 1
        boxes.append([int(lo[0]), int(lo[1]), int(lo[2]), int(hi[0]), int(hi[1]), int(hi[2])])
    return boxes


def _cache_path(key: str) -> Optional[str]:
    root = os.environ.get("AMR_SYNTH_CACHE", "/tmp/amr_synth_cache")
    try:
        os.makedirs(root, exist_ok=True)
    except OSError:
        return None
    return os.path.join(root, hashlib.sha1(key.encode()).hexdigest()[:16] + ".npz")


def _box_cells(bs) -> int:
    return int(sum((b[3] - b[0]) * (b[4] - b[1]) * (b[5] - b[2]) for b in bs))


def _fit_budget(fl, vals, coarse, n_l, tile, ratio, budget):
    """Raise the refinement threshold until the refined patches hold at most `budget`
    finer cells: keep the densest flagged cells (fl, densities vals), their number scaled
    by the budget over the current cell count, and re-cluster (a few passes)."""
    cells = _box_cells(coarse) * ratio ** 3
    if cells <= budget:
        return coarse
    order = np.argsort(-vals, kind="stable")
    keep = fl.shape[0]
    for _ in range(8):
        keep = max(1, int(keep * budget / cells * 0.97))
        sel = fl[np.sort(order[:keep])]
        coarse = _tile_patches(sel.astype(np.int64), n_l, tile, tile // 2, 4)
        cells = _box_cells(coarse) * ratio ** 3
        if cells <= budget:
            break
    return coarse


def make_lognormal(seed: int = 2, num_levels: int = 5, n0: int = 128, patch0: int = 32,
                   threshold: float = 4.0, level_growth: float = 2.25, tile: int = 32,
                   M: int = 2048, device=None, name: str = "c2",
                   use_cache: bool = True, cell_budget: Optional[int] = None) -> Hierarchy:
    """Cosmology-like SAMR hierarchy.

    Level 0: (n0/patch0)^3 patches of patch0^3 cells on [0,1]^3.  The density is
    rho = exp(delta), delta a unit-variance Gaussian random field with P(k) ~ k^-2
    (`GaussianRandomField`).  Level l+1 refines the level-l cells with
    rho > threshold * mean(rho) * level_growth^l (mean over the domain, e^{1/2}); flagged
    cells are clustered per tile of `tile` level-l cells on a global grid shifted by
    tile/2, so fine patches straddle coarse parents (non-nested refinement) and are
    8..2*tile fine cells per axis.  Each patch samples rho at its own cell centres.

    cell_budget (optional) caps the cells of every refined level: when the patches of the
    flagged cells would hold more, the threshold is raised to a quantile of the level's
    flagged densities (refining the densest cells first) until they fit.
    """
    key = f"lognormal:{seed}:{num_levels}:{n0}:{patch0}:{threshold}:{level_growth}:{tile}:{M}"
    if cell_budget is not None:
        key += f":budget{int(cell_budget)}"
    path = _cache_path(key) if use_cache else None
    if path and os.path.exists(path):
        z = np.load(path, allow_pickle=False)
        P = z["patch_level"].shape[0]
        return Hierarchy(int(z["num_levels"]), int(z["ratio"]), z["domain_lo"], z["h0"],
                         z["patch_level"], z["patch_box"], [z[f"d{p}"] for p in range(P)],
                         name, dict(key=key, cached=True))
    grf = GaussianRandomField(seed, M=M)
    if device is None:
        try:
            import torch

            device = "cuda" if torch.cuda.is_available() else "cpu"
        except Exception:  # pragma: no cover
            device = "cpu"
    ratio = 2
    h0 = np.full(3, 1.0 / n0)
    mean_rho = math.exp(0.5)
    boxes: List[List[int]] = []
    levels: List[int] = []
    data: List[np.ndarray] = []
    m = n0 // patch0
    cur = []
    for k in range(m):
        for j in range(m):
            for i in range(m):
                cur.append([i * patch0, j * patch0, k * patch0, (i + 1) * patch0,
                            (j + 1) * patch0, (k + 1) * patch0])
    for l in range(num_levels):
        h = 1.0 / (n0 * ratio ** l)
        flags = []
        fvals = []
        thr = threshold * mean_rho * level_growth ** l
        for b in cur:
            xs = (np.arange(b[0], b[3]) + 0.5) * h
            ys = (np.arange(b[1], b[4]) + 0.5) * h
            zs = (np.arange(b[2], b[5]) + 0.5) * h
            rho = np.exp(grf.sample_box(xs, ys, zs, device=device))
            boxes.append(b)
            levels.append(l)
            data.append(np.ascontiguousarray(rho, dtype=np.float32))
            if l + 1 < num_levels:
                kk, jj, ii = np.nonzero(rho > thr)
                if kk.size:
                    flags.append(np.stack([ii + b[0], jj + b[1], kk + b[2]], axis=1))
                    if cell_budget is not None:
                        fvals.append(rho[kk, jj, ii])
        if l + 1 == num_levels:
            break
        fl = np.concatenate(flags, axis=0) if flags else np.zeros((0, 3), dtype=np.int64)
        n_l = np.full(3, n0 * ratio ** l, dtype=np.int64)
        coarse = _tile_patches(fl.astype(np.int64), n_l, tile, tile // 2, 4)
        if cell_budget is not None and coarse:
            coarse = _fit_budget(fl, np.concatenate(fvals), coarse, n_l, tile, ratio,
                                 int(cell_budget))
        cur = [[c * ratio for c in b] for b in coarse]
        if not cur:
            num_levels = l + 1
            break
    hier = Hierarchy(num_levels, ratio, np.zeros(3), h0, np.asarray(levels, dtype=np.int32),
                     np.asarray(boxes, dtype=np.int64).reshape(-1, 6), data, name,
                     dict(key=key, cached=False))
    if path:
        arrs = {f"d{p}": d for p, d in enumerate(hier.data)}
        tmp = path + f".{os.getpid()}.tmp.npz"
        np.savez(tmp, num_levels=hier.num_levels, ratio=hier.ratio, domain_lo=hier.domain_lo,
                 h0=hier.h0, patch_level=hier.patch_level, patch_box=hier.patch_box, **arrs)
        os.replace(tmp, path)
    return hier


def make_c2(seed: int = 2, device=None, use_cache: bool = True) -> Hierarchy:
    return make_lognormal(seed=seed, num_levels=5, device=device, name="c2", use_cache=use_cache)


def make_c3(seed: int = 3, device=None, use_cache: bool = False,
            cell_budget: int = 140_000_000) -> Hierarchy:
    """Deep hierarchy: the C2 generator with 8 levels (finest spacing 1/16384), the density
    threshold fixed at 4x the mean on every level, and each refined level capped at
    `cell_budget` cells (about 1e9 cells and 2e4 patches in all)."""
    return make_lognormal(seed=seed, num_levels=8, level_growth=1.0, device=device, name="c3",
                          use_cache=use_cache, cell_budget=cell_budget)


def make_deep(seed: int = 3, device=None, use_cache: bool = True,
              cell_budget: int = 12_000_000) -> Hierarchy:
    """The deep configuration's shape at a size that generates in seconds: the C3 generator
    (8 levels, finest spacing 1/16384, threshold 4x the mean on every level) with each
    refined level capped at `cell_budget` cells (about 1e8 cells in all instead of 1e9)."""
    return make_lognormal(seed=seed, num_levels=8, level_growth=1.0, device=device,
                          name="deep", use_cache=use_cache, cell_budget=cell_budget)


def percentile_range(hier: Hierarchy, q: float = 99.9):
    allv = np.concatenate([d.ravel() for d in hier.data])
    return float(allv.min()), float(np.percentile(allv, q))


def c2_workload(width: int = 1024, height: Optional[int] = None, seed: int = 2,
                camera_seed: int = 2, device=None, shade: bool = True):
    hier = make_c2(seed, device=device)
    vmin, vmax = percentile_range(hier)
    h = width if height is None else height
    return dict(hier=hier, camera=orbit_camera(camera_seed, width, h), tf=ramp_tf(),
                vmin=vmin, vmax=vmax, kappa=8.0, step_factor=0.5, ert_eps=1e-4,
                shade=shade, name=f"c2_{width}x{h}")
