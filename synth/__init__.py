"""Seeded synthetic inputs for the residency-octree ray caster.

This package is the data source of the paper's system (Sec. 4: a server
provides a bricked multi-resolution multi-volume hierarchy and, optionally,
per-region min/max metadata).  It makes the voxel data, the coarser levels,
bricks with a one-voxel border, per-leaf value ranges, transfer functions and
cameras.  It contains none of the rendering method's arithmetic (no octree, no
page table, no traversal, no compositing), so that both the CUDA library's
callers and the independent CPU oracle can take their inputs from it.

Volumes are numpy arrays in C order [z][y][x] (x fastest).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "libsynth.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile libsynth.so with the host C compiler (x86-64 or aarch64)."""
    src = os.path.join(_HERE, "synth.c")
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-D_GNU_SOURCE",
                               "-fvisibility=hidden", src, "-o", tmp, "-lpthread", "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        c_void_p, c_int, c_double, c_uint32, c_uint64 = (ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                                                         ctypes.c_uint32, ctypes.c_uint64)
        L.sy_noise.restype = c_uint32
        L.sy_noise.argtypes = [c_uint64] + [c_uint32] * 6
        L.sy_blobs_u8.argtypes = [c_uint64, c_int, c_int, c_int, c_int, c_double, c_double, c_double, c_double,
                                  c_uint32, c_void_p]
        L.sy_downsample.argtypes = [c_int, c_int, c_int, c_int, c_void_p, c_void_p]
        L.sy_downsample_axes.argtypes = [c_int, c_int, c_int, c_int, c_int, c_void_p, c_void_p]
        L.sy_bricks_from_dense.argtypes = [c_int, c_int, c_int, c_int, c_void_p, c_int, c_int, c_void_p, c_void_p]
        L.sy_leaf_ranges.argtypes = [c_int, c_int, c_int, c_int, c_void_p, c_int, c_int, c_int, c_void_p, c_void_p]
        L.sy_cells_create.restype = c_void_p
        L.sy_cells_create.argtypes = [c_uint64, c_int, c_int, c_int, c_int, c_int, c_double, c_double, c_double,
                                      c_double, c_double, c_double, c_double, c_double, c_uint32, c_double]
        L.sy_cells_free.argtypes = [c_void_p]
        L.sy_cells_dense.argtypes = [c_void_p, c_int, c_void_p]
        L.sy_cells_bricks.argtypes = [c_void_p, c_int, c_int, c_int, c_int, c_void_p, c_void_p]
        L.sy_cells_bricks_mixed.argtypes = [c_void_p, c_int, c_int, c_void_p, c_void_p]
        L.sy_cells_leaf_bounds.argtypes = [c_void_p, c_int, c_int, c_int, c_int, c_void_p, c_void_p]
        L.sy_cells_count.restype = ctypes.c_int64
        L.sy_cells_count.argtypes = [c_void_p, c_int]
        L.sy_set_threads.argtypes = [c_int]
        L.sy_vcache_create.restype = c_void_p
        L.sy_vcache_create.argtypes = [c_void_p, c_int, ctypes.c_int64]
        L.sy_vcache_free.argtypes = [c_void_p]
        L.sy_vcache_bricks.restype = ctypes.c_int64
        L.sy_vcache_bricks.argtypes = [c_void_p]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def set_threads(n: int) -> None:
    lib().sy_set_threads(int(n))


def noise(seed, c, l, x, y, z, nmax) -> int:
    return int(lib().sy_noise(seed, c, l, x, y, z, nmax))


# ----------------------------------------------------------------- volumes

def blobs_u8(dims_xyz, seed, n_blobs=40, sigma=(3.0, 10.0), amp=(60.0, 180.0), noise_max=4) -> np.ndarray:
    nx, ny, nz = dims_xyz
    out = np.empty((nz, ny, nx), np.uint8)
    rc = lib().sy_blobs_u8(seed, nx, ny, nz, n_blobs, sigma[0], sigma[1], amp[0], amp[1], noise_max, _ptr(out))
    if rc != 0:
        raise ValueError(f"sy_blobs_u8 failed ({rc})")
    return out


def downsample(vol: np.ndarray, keep: int = 0) -> np.ndarray:
    """Rounded mean over blocks of 2 voxels along each halved axis (bit a of
    keep set: axis a (x, y, z) keeps its resolution)."""
    nz, ny, nx = vol.shape
    bpv = vol.dtype.itemsize
    f = [1 if (keep >> a) & 1 else 2 for a in range(3)]
    out = np.empty((-(-nz // f[2]), -(-ny // f[1]), -(-nx // f[0])), vol.dtype)
    vol = np.ascontiguousarray(vol)
    if lib().sy_downsample_axes(bpv, nx, ny, nz, int(keep), _ptr(vol), _ptr(out)) != 0:
        raise ValueError("sy_downsample failed")
    return out


def mean_levels(vol0: np.ndarray, k: int, keep_axes=None) -> list:
    """Level 0 .. k-1 of the hierarchy, each the rounded mean of the previous;
    keep_axes[l] (default 0) names the axes level l + 1 keeps unhalved."""
    levels = [np.ascontiguousarray(vol0)]
    for l in range(1, k):
        levels.append(downsample(levels[-1], 0 if keep_axes is None else keep_axes[l - 1]))
    return levels


def bricks_from_dense(level: np.ndarray, B: int, coords) -> np.ndarray:
    """(n, B+2, B+2, B+2) bricks with a clamped one-voxel border."""
    coords = np.ascontiguousarray(np.asarray(coords, np.int32).reshape(-1, 3))
    n = coords.shape[0]
    nz, ny, nx = level.shape
    out = np.empty((n, B + 2, B + 2, B + 2), level.dtype)
    level = np.ascontiguousarray(level)
    if lib().sy_bricks_from_dense(level.dtype.itemsize, nx, ny, nz, _ptr(level), B, n, _ptr(coords), _ptr(out)):
        raise ValueError("sy_bricks_from_dense failed")
    return out


def leaf_ranges(vol0: np.ndarray, leaf_extent_xyz):
    """Exact per-leaf (min, max) of the level-0 voxels whose trilinear
    support reaches the leaf; arrays of shape (lz, ly, lx)."""
    nz, ny, nx = vol0.shape
    ex, ey, ez = leaf_extent_xyz
    lx, ly, lz = -(-nx // ex), -(-ny // ey), -(-nz // ez)
    mn = np.empty((lz, ly, lx), np.uint32)
    mx = np.empty((lz, ly, lx), np.uint32)
    vol0 = np.ascontiguousarray(vol0)
    if lib().sy_leaf_ranges(vol0.dtype.itemsize, nx, ny, nz, _ptr(vol0), ex, ey, ez, _ptr(mn), _ptr(mx)):
        raise ValueError("sy_leaf_ranges failed")
    return mn, mx


class Cells:
    """Poisson field of rotated ellipsoidal cells, one intensity per channel."""

    def __init__(self, seed, ncells, m, dims_xyz, spacing_xyz, r=(4.0, 12.0), p_express=0.3,
                 median=8000.0, sigma_ln=0.6, noise_max=200, bin_edge=24.0):
        self.dims = tuple(int(v) for v in dims_xyz)
        self.spacing = tuple(float(v) for v in spacing_xyz)
        self.m = m
        self.noise_max = noise_max
        self._h = lib().sy_cells_create(seed, ncells, m, *self.dims, *self.spacing, r[0], r[1], p_express,
                                        median, sigma_ln, noise_max, bin_edge)
        if not self._h:
            raise ValueError("sy_cells_create failed")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.sy_cells_free(h)
            self._h = None

    def count(self, ch=-1) -> int:
        return int(lib().sy_cells_count(self._h, ch))

    def dense(self, ch) -> np.ndarray:
        nx, ny, nz = self.dims
        out = np.empty((nz, ny, nx), np.uint16)
        if lib().sy_cells_dense(self._h, ch, _ptr(out)):
            raise ValueError("sy_cells_dense failed")
        return out

    def bricks(self, ch, l, B, coords) -> np.ndarray:
        coords = np.ascontiguousarray(np.asarray(coords, np.int32).reshape(-1, 3))
        out = np.empty((coords.shape[0], B + 2, B + 2, B + 2), np.uint16)
        if lib().sy_cells_bricks(self._h, ch, l, B, coords.shape[0], _ptr(coords), _ptr(out)):
            raise ValueError("sy_cells_bricks failed")
        return out

    def bricks_mixed(self, B, keys, out=None) -> np.ndarray:
        """keys: (n, 5) int32 rows (channel, level, bx, by, bz)."""
        keys = np.ascontiguousarray(np.asarray(keys, np.int32).reshape(-1, 5))
        if out is None:
            out = np.empty((keys.shape[0], B + 2, B + 2, B + 2), np.uint16)
        if lib().sy_cells_bricks_mixed(self._h, B, keys.shape[0], _ptr(keys), _ptr(out)):
            raise ValueError("sy_cells_bricks_mixed failed")
        return out

    def voxel_source(self, B, capacity=1 << 20):
        """A lazily filled voxel source over this field (see VoxelSource)."""
        return VoxelSource(self, B, capacity)

    def leaf_bounds(self, ch, leaf_extent_xyz):
        nx, ny, nz = self.dims
        ex, ey, ez = leaf_extent_xyz
        lx, ly, lz = -(-nx // ex), -(-ny // ey), -(-nz // ez)
        mn = np.empty((lz, ly, lx), np.uint32)
        mx = np.empty((lz, ly, lx), np.uint32)
        if lib().sy_cells_leaf_bounds(self._h, ch, ex, ey, ez, _ptr(mn), _ptr(mx)):
            raise ValueError("sy_cells_leaf_bounds failed")
        return mn, mx


class VoxelSource:
    """Voxel-at-a-time access to a cell field for readers that cannot hold
    the volume densely: bricks of B^3 level-l voxels are generated on first
    touch and kept.  `fn` / `ctx` are the C function pointer and its context
    for a C consumer."""

    def __init__(self, cells: "Cells", B: int, capacity: int):
        self.cells = cells          # keeps the field alive
        L = lib()
        self._h = L.sy_vcache_create(cells._h, int(B), int(capacity))
        if not self._h:
            raise ValueError("sy_vcache_create failed")
        self.fn = ctypes.cast(L.sy_vcache_voxel, ctypes.c_void_p).value
        self.ctx = self._h

    def bricks_generated(self) -> int:
        return int(lib().sy_vcache_bricks(self._h))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.sy_vcache_free(h)
            self._h = None


# ------------------------------------------------- transfer functions

@dataclass
class TF:
    """Per-channel transfer function: a raw value v maps to the LUT
    coordinate clamp((v - lo) * scale, 0, 255); lut is 256 RGBA knots."""
    lo: float
    scale: float
    lut: np.ndarray  # (256, 4) float32


def tf_ramp(lo, hi, rgb=(1.0, 1.0, 1.0), alpha_max=1.0) -> TF:
    """Opacity rising linearly from 0 at raw value lo to alpha_max at hi,
    constant colour rgb."""
    lut = np.zeros((256, 4), np.float32)
    j = np.arange(256, dtype=np.float64)
    lut[:, 0], lut[:, 1], lut[:, 2] = rgb
    lut[:, 3] = (alpha_max * j / 255.0).astype(np.float32)
    scale = np.float32(255.0 / (float(hi) - float(lo)))
    return TF(float(np.float32(lo)), float(scale), lut)


def hue_rgb(h: float):
    """Fully saturated colour of hue h in [0, 1)."""
    h6 = (h % 1.0) * 6.0
    i = int(h6)
    f = h6 - i
    return [(1, f, 0), (1 - f, 1, 0), (0, 1, f), (0, 1 - f, 1), (f, 0, 1), (1, 0, 1 - f)][i % 6]


# ------------------------------------------------------------ cameras

@dataclass
class Camera:
    """Pinhole or orthographic camera in physical coordinates.

    ortho: pixel (i, j) starts at eye + a*right + b*up with
      a = (i + 0.5 - W/2) * pixel, b = (H/2 - j - 0.5) * pixel, along forward.
    perspective: rays start at eye along normalize(forward + a*right + b*up),
      a = (2 (i + 0.5)/W - 1) * tan_x, b = (1 - 2 (j + 0.5)/H) * tan_y.
    """
    eye: tuple
    forward: tuple
    right: tuple
    up: tuple
    perspective: bool
    tan_x: float = 0.0
    tan_y: float = 0.0
    pixel: float = 1.0
    fovy_deg: float = 0.0


def _norm(v):
    v = np.asarray(v, np.float64)
    return v / np.linalg.norm(v)


def look_at(eye, target, up_hint, W, H, fovy_deg=None, ortho_pixel=None) -> Camera:
    f = _norm(np.asarray(target, np.float64) - np.asarray(eye, np.float64))
    r = _norm(np.cross(f, up_hint))
    u = np.cross(r, f)
    f32 = lambda v: tuple(float(x) for x in np.asarray(v, np.float32))
    if fovy_deg is not None:
        ty = math.tan(math.radians(fovy_deg) / 2.0)
        return Camera(f32(eye), f32(f), f32(r), f32(u), True, float(np.float32(ty * W / H)),
                      float(np.float32(ty)), 1.0, float(fovy_deg))
    return Camera(f32(eye), f32(f), f32(r), f32(u), False, 0.0, 0.0, float(np.float32(ortho_pixel)))


def orbit(center, radius, elevation_deg, azimuth_deg, W, H, fovy_deg, up=(0.0, 0.0, 1.0)) -> Camera:
    """Perspective camera on a circle about the up axis through center."""
    el, az = math.radians(elevation_deg), math.radians(azimuth_deg)
    d = np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])
    eye = np.asarray(center, np.float64) + radius * d
    return look_at(eye, center, np.asarray(up, np.float64), W, H, fovy_deg=fovy_deg)


def lod_thresholds(min_spacing, H, fovy_deg, k, bias=1.0):
    """Distances tau_l (l = 1..k-1) at which the footprint of one pixel
    reaches 2^l level-0 voxels: tau_l = bias * 2^l * s_min * H / (2 tan(fovy/2)),
    computed in double and rounded to float32; index 0 is unused."""
    t = [0.0] * 16
    ty = math.tan(math.radians(fovy_deg) / 2.0)
    for l in range(1, 16):
        t[l] = float(np.float32(bias * (2.0 ** l) * min_spacing * H / (2.0 * ty))) if l < k else float("inf")
    return t


def seeded_subset(seed, n_total, n_pick) -> np.ndarray:
    """n_pick distinct indices of range(n_total), chosen by a seeded shuffle."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.sort(rng.permutation(n_total)[:n_pick])


@dataclass
class Frame:
    """Everything one rendered frame takes besides the volume: image size,
    camera, one transfer function per channel, lattice spacing dt (physical),
    lod thresholds lod_t[1..k-1] (index 0 unused), per-channel level range,
    octree start depth, empty-space skipping switch and early-termination
    threshold on transmittance (0 = off)."""
    W: int
    H: int
    camera: Camera
    tfs: list
    dt: float
    lod_t: list
    lmin: list
    lmax: list
    start_depth: int = 0
    skip: bool = True
    ert: float = 2.0 ** -10
