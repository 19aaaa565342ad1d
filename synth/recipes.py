"""Seeded synthetic workloads standing in for the paper's datasets (Table 1).

Each recipe returns a Scene: the bricked hierarchy (dense levels or a
procedural cell field), the leaf value ranges the data source supplies, the
initially resident bricks, and frame descriptions.  Nothing here renders.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import (Cells, Frame, bricks_from_dense, blobs_u8, hue_rgb, leaf_ranges, look_at, lod_thresholds,
               mean_levels, orbit, seeded_subset, tf_ramp, TF)


@dataclass
class Scene:
    name: str
    dims: tuple               # level-0 voxels (x, y, z)
    spacing: tuple
    m: int
    k: int
    B: int
    leaf: tuple
    value_bits: int
    levels: list = None       # levels[c][l] dense arrays, or None (procedural)
    cells: Cells = None
    leaf_min: np.ndarray = None   # (m, lz, ly, lx) int64, -1 = no metadata
    leaf_max: np.ndarray = None
    resident: list = field(default_factory=list)  # (c, l, bx, by, bz)
    frames: list = field(default_factory=list)
    keep_axes: list = None        # per level: bit a set = axis a not halved going to the next level

    def level_dims(self, l):
        d = list(self.dims)
        for q in range(l):
            keep = 0 if self.keep_axes is None else self.keep_axes[q]
            d = [v if (keep >> a) & 1 else (v + 1) // 2 for a, v in enumerate(d)]
        return tuple(d)

    def n_bricks_axis(self, l):
        return tuple(-(-v // self.B) for v in self.level_dims(l))

    def all_bricks(self, channels=None, levels=None):
        out = []
        for c in (range(self.m) if channels is None else channels):
            for l in (range(self.k) if levels is None else levels):
                nx, ny, nz = self.n_bricks_axis(l)
                for z in range(nz):
                    for y in range(ny):
                        for x in range(nx):
                            out.append((c, l, x, y, z))
        return out

    def bricks(self, keys) -> np.ndarray:
        """Voxels of the given (c, l, bx, by, bz) bricks with their border."""
        keys = np.asarray(keys, np.int32).reshape(-1, 5)
        if self.cells is not None:
            return self.cells.bricks_mixed(self.B, keys)
        E = self.B + 2
        dt = np.uint8 if self.value_bits == 8 else np.uint16
        out = np.empty((keys.shape[0], E, E, E), dt)
        for i, (c, l, x, y, z) in enumerate(keys):
            out[i] = bricks_from_dense(self.levels[c][l], self.B, [(x, y, z)])[0]
        return out


def _exact_meta(levels_per_channel, leaf):
    mins, maxs = [], []
    for ch in levels_per_channel:
        mn, mx = leaf_ranges(ch[0], leaf)
        mins.append(mn.astype(np.int64))
        maxs.append(mx.astype(np.int64))
    return np.stack(mins), np.stack(maxs)


def blobs128(seed=1, dims=(128, 128, 128), W=256, H=256) -> Scene:
    """One-channel 128^3 u8 volume of 40 Gaussian blobs plus noise <= 4,
    32^3 bricks, 3 mean levels, every brick resident, 256^2 orthographic view
    along +z at 0.5 voxel per pixel, step 0.5, TF ramp 8 -> 255."""
    v0 = blobs_u8(dims, seed)
    levels = [mean_levels(v0, 3)]
    mn, mx = _exact_meta(levels, (16, 16, 16))
    s = Scene("blobs128", tuple(dims), (1.0, 1.0, 1.0), 1, 3, 32, (16, 16, 16), 8, levels=levels,
              leaf_min=mn, leaf_max=mx)
    s.resident = s.all_bricks()
    cx, cy, cz = (d / 2.0 for d in dims)
    pix = dims[0] / W
    cam = look_at((cx, cy, -8.0), (cx, cy, cz), (0.0, -1.0, 0.0), W, H, ortho_pixel=pix)
    tf = tf_ramp(8, 255)
    lod = [0.0] + [float("inf")] * 15
    s.frames.append(Frame(W, H, cam, [tf], 0.5, lod, [0], [0]))
    d = np.array([1.0, 2.0, 3.0]) / math.sqrt(14.0)
    eye = np.array([cx, cy, cz]) - 200.0 * d
    cam2 = look_at(tuple(eye), (cx, cy, cz), (0.0, 0.0, 1.0), W, H, ortho_pixel=pix * 1.4)
    s.frames.append(Frame(W, H, cam2, [tf], 0.5, lod, [0], [0]))
    return s


def _cell_tfs(m, lo=400.0, hi=12000.0, alpha_max=0.5):
    return [tf_ramp(lo, hi, rgb=hue_rgb(c / m), alpha_max=alpha_max) for c in range(m)]


def cells_slab(seed=2, m=4, dims=(1024, 1024, 64), ncells=20000, k=5, resident_l0=0.3, W=1024, H=1024,
               n_views=16, dense=True, fovy=40.0, radius=None, elevation=35.0) -> Scene:
    """m-channel u16 slab (spacing 1:1:4) of Poisson ellipsoid cells, 32^3
    bricks, k levels, leaves 16x16x4; every level >= 1 resident plus a seeded
    fraction of level 0; perspective views orbiting the slab normal."""
    spacing = (1.0, 1.0, 4.0)
    cells = Cells(seed, ncells, m, dims, spacing)
    leaf = (16, 16, 4)
    if dense:
        levels = [mean_levels(cells.dense(c), k) for c in range(m)]
        mn, mx = _exact_meta(levels, leaf)
        s = Scene("cells_slab", tuple(dims), spacing, m, k, 32, leaf, 16, levels=levels, leaf_min=mn, leaf_max=mx)
    else:
        mins, maxs = zip(*[cells.leaf_bounds(c, leaf) for c in range(m)])
        s = Scene("cells_slab", tuple(dims), spacing, m, k, 32, leaf, 16, cells=cells,
                  leaf_min=np.stack(mins).astype(np.int64), leaf_max=np.stack(maxs).astype(np.int64))
    coarse = s.all_bricks(levels=range(1, k))
    fine = s.all_bricks(levels=[0])
    pick = seeded_subset(seed, len(fine), int(round(resident_l0 * len(fine))))
    s.resident = coarse + [fine[i] for i in pick]
    center = tuple(d * sp / 2.0 for d, sp in zip(dims, spacing))
    ext = math.hypot(dims[0] * spacing[0], dims[1] * spacing[1])
    r = radius if radius is not None else 0.55 * ext / math.tan(math.radians(fovy) / 2.0)
    tfs = _cell_tfs(m)
    lod = lod_thresholds(min(spacing), H, fovy, k)
    for v in range(n_views):
        cam = orbit(center, r, elevation, 360.0 * v / n_views + 7.0, W, H, fovy)
        s.frames.append(Frame(W, H, cam, tfs, 0.5 * min(spacing), lod, [0] * m, [k - 1] * m))
    return s


def cells_large(seed=3, m=16, dims=(4096, 4096, 96), ncells=480000, k=7, W=1920, H=1080, n_views=16, fovy=40.0,
                radius=1500.0, elevation=35.0, close_up=True, arc_deg=360.0, lod_bias=1.0) -> Scene:
    """16-channel 4096x4096x96 u16 procedural slab (spacing 1:1:4) of the
    same cell model, bricks generated on request; 1920x1080 perspective orbit
    about the slab normal around the centre (close-up: one pixel ~ one
    level-0 voxel at the focus), n_views views spread over arc_deg degrees;
    lod_bias scales the level thresholds."""
    spacing = (1.0, 1.0, 4.0)
    cells = Cells(seed, ncells, m, dims, spacing)
    leaf = (16, 16, 4)
    mins, maxs = zip(*[cells.leaf_bounds(c, leaf) for c in range(m)])
    s = Scene("cells_large", tuple(dims), spacing, m, k, 32, leaf, 16, cells=cells,
              leaf_min=np.stack(mins).astype(np.int64), leaf_max=np.stack(maxs).astype(np.int64))
    center = tuple(d * sp / 2.0 for d, sp in zip(dims, spacing))
    r = radius if close_up else 0.55 * math.hypot(dims[0], dims[1]) / math.tan(math.radians(fovy) / 2.0)
    tfs = _cell_tfs(m)
    lod = lod_thresholds(min(spacing), H, fovy, k, bias=lod_bias)
    for v in range(n_views):
        cam = orbit(center, r, elevation, arc_deg * v / n_views + 7.0, W, H, fovy)
        s.frames.append(Frame(W, H, cam, tfs, 0.5 * min(spacing), lod, [0] * m, [k - 1] * m))
    return s


VIEW_SIZES = ((256, 256), (512, 512), (1024, 768), (1920, 1080))


def cells_views(seed=5, m=16, dims=(1024, 1024, 64), ncells=20000, k=5, n_views=64, sizes=VIEW_SIZES, fovy=40.0,
                elevation=(25.0, 60.0), distance=(0.6, 1.2), leaf=(16, 16, 4)) -> Scene:
    """m-channel u16 slab (spacing 1:1:4) of the cell model, bricks generated
    on request; n_views seeded perspective cameras around the slab, each with
    an image size drawn uniformly from `sizes`, a seeded azimuth, elevation and
    distance (a multiple of the distance that frames the whole slab); leaf:
    the octree's leaf extent in level-0 voxels."""
    spacing = (1.0, 1.0, 4.0)
    cells = Cells(seed, ncells, m, dims, spacing)
    leaf = tuple(int(v) for v in leaf)
    mins, maxs = zip(*[cells.leaf_bounds(c, leaf) for c in range(m)])
    s = Scene("cells_views", tuple(dims), spacing, m, k, 32, leaf, 16, cells=cells,
              leaf_min=np.stack(mins).astype(np.int64), leaf_max=np.stack(maxs).astype(np.int64))
    center = tuple(d * sp / 2.0 for d, sp in zip(dims, spacing))
    ext = math.hypot(dims[0] * spacing[0], dims[1] * spacing[1])
    r0 = 0.55 * ext / math.tan(math.radians(fovy) / 2.0)
    rng = np.random.default_rng(seed)
    tfs = _cell_tfs(m)
    for v in range(n_views):
        W, H = sizes[int(rng.integers(len(sizes)))]
        az = float(rng.uniform(0.0, 360.0))
        el = float(rng.uniform(*elevation))
        r = r0 * float(rng.uniform(*distance))
        cam = orbit(center, r, el, az, W, H, fovy)
        lod = lod_thresholds(min(spacing), H, fovy, k)
        s.frames.append(Frame(W, H, cam, tfs, 0.5 * min(spacing), lod, [0] * m, [k - 1] * m))
    return s
