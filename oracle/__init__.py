"""CPU oracle of the residency-octree ray caster (test infrastructure).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may use
this package.  It loads liboracle.so, built from oracle.c with the host C
compiler and -ffp-contract=off, and shares no code with the CUDA library.
See oracle.c for what each entry point computes and which passage of the
paper it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

MAXC, MAXL = 16, 16


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "oracle.c")
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-D_GNU_SOURCE",
                               "-ffp-contract=off", "-fno-fast-math", "-fexcess-precision=standard",
                               "-fvisibility=hidden", src, "-o", tmp, "-lpthread", "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _Volume(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int32 * 3), ("spacing", ctypes.c_float * 3),
                ("m", ctypes.c_int32), ("k", ctypes.c_int32), ("B", ctypes.c_int32), ("bpv", ctypes.c_int32),
                ("leaf", ctypes.c_int32 * 3), ("levels", ctypes.POINTER(ctypes.c_void_p)),
                ("resident", ctypes.c_void_p), ("leaf_min", ctypes.c_void_p), ("leaf_max", ctypes.c_void_p),
                ("voxel_fn", ctypes.c_void_p), ("voxel_ctx", ctypes.c_void_p), ("sample_format", ctypes.c_int32),
                ("node_min", ctypes.c_void_p), ("node_max", ctypes.c_void_p),
                ("keep_axes", ctypes.c_int32 * MAXL)]


class _Params(ctypes.Structure):
    _fields_ = [("W", ctypes.c_int32), ("H", ctypes.c_int32), ("perspective", ctypes.c_int32),
                ("eye", ctypes.c_float * 3), ("fwd", ctypes.c_float * 3), ("right", ctypes.c_float * 3),
                ("up", ctypes.c_float * 3), ("tan_x", ctypes.c_float), ("tan_y", ctypes.c_float),
                ("pixel", ctypes.c_float), ("dt", ctypes.c_float), ("lod_t", ctypes.c_float * MAXL),
                ("lmin", ctypes.c_int32 * MAXC), ("lmax", ctypes.c_int32 * MAXC),
                ("start_depth", ctypes.c_int32), ("skip", ctypes.c_int32), ("ert", ctypes.c_float),
                ("tf_lo", ctypes.c_float * MAXC), ("tf_scale", ctypes.c_float * MAXC),
                ("lut", ctypes.c_void_p)]


class _Outputs(ctypes.Structure):
    _fields_ = [("rgba32", ctypes.c_void_p), ("rgba64", ctypes.c_void_p), ("hash", ctypes.c_void_p),
                ("n_eval", ctypes.c_void_p), ("i_end", ctypes.c_void_p), ("n_bs", ctypes.c_void_p),
                ("req", ctypes.c_void_p), ("used", ctypes.c_void_p), ("node_req", ctypes.c_void_p)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        V, P, O = ctypes.POINTER(_Volume), ctypes.POINTER(_Params), ctypes.POINTER(_Outputs)
        vp, i64 = ctypes.c_void_p, ctypes.c_int64
        L.or_brick_index.restype = i64
        L.or_brick_index.argtypes = [V] + [ctypes.c_int] * 5
        L.or_brick_count.restype = i64
        L.or_brick_count.argtypes = [V]
        L.or_depth.argtypes = [V]
        L.or_node_count.restype = i64
        L.or_node_count.argtypes = [V]
        L.or_node_words.argtypes = [V, vp]
        L.or_render.argtypes = [V, vp, P, vp, i64, O]
        L.or_flags_to_ids.restype = i64
        L.or_flags_to_ids.argtypes = [V, vp, vp, i64, ctypes.POINTER(i64)]
        L.or_traversal_depth.argtypes = [V, ctypes.c_float, ctypes.c_int]
        L.or_bucket_occupancy.argtypes = [V, P, vp]
        L.or_brick_id.restype = ctypes.c_uint32
        L.or_brick_id.argtypes = [V] + [ctypes.c_int] * 5
        L.or_set_threads.argtypes = [ctypes.c_int]
        L.or_threads_used.restype = ctypes.c_int
        L.or_round_fmt.restype = ctypes.c_double
        L.or_round_fmt.argtypes = [ctypes.c_double, ctypes.c_int]
        L.or_lerp_fmt.restype = ctypes.c_double
        L.or_lerp_fmt.argtypes = [ctypes.c_double] * 3 + [ctypes.c_int]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def round_fmt(x: float, fmt: int) -> float:
    """Round-to-nearest-even of x to binary16 (fmt 1) or bfloat16 (fmt 2)."""
    return float(lib().or_round_fmt(float(x), int(fmt)))


def lerp_fmt(f: float, a: float, b: float, fmt: int) -> float:
    """One low-precision lerp: q(f * q(b - a) + a), each q a single rounding."""
    return float(lib().or_lerp_fmt(float(f), float(a), float(b), int(fmt)))


def set_threads(n: int) -> None:
    lib().or_set_threads(int(n))


def threads_used() -> int:
    return int(lib().or_threads_used())


class Volume:
    """Dense multi-channel, multi-level volume plus residency and leaf
    metadata, as the oracle sees it.

    levels[c][l]: numpy array [z][y][x] (uint8 or uint16) of level l.
    resident: iterable of (c, l, bx, by, bz) bricks resident in the cache.
    leaf_min / leaf_max: arrays (m, lz, ly, lx) int64, -1 = no metadata.
    node_min / node_max: ranges given for inner nodes, arrays (m, n_nodes)
    int64 by node index (depth-major), -1 = none (entries of leaves unused).
    keep_axes: per level l, bit a set = axis a keeps its resolution from
    level l to level l + 1 (default: every level halves every axis).
    sample_format: 0 = raw values with binary32 lerps, 1 = binary16,
    2 = bfloat16 samples (the brick cache's format).
    provider: instead of levels, (m, k, dims_xyz, bytes_per_voxel, fn, ctx)
    where fn is a C function pointer uint32_t(void*, int c, int l, int64 x,
    int64 y, int64 z) and ctx its first argument (a voxel source for
    volumes too large to hold densely).
    """

    def __init__(self, levels, spacing, B, leaf_extent, resident=(), leaf_min=None, leaf_max=None, provider=None,
                 sample_format=0, node_min=None, node_max=None, keep_axes=None):
        self.s = _Volume()
        self.s.sample_format = int(sample_format)
        ka = list(keep_axes or []) + [0] * MAXL
        self.s.keep_axes[:] = [int(v) for v in ka[:MAXL]]
        if provider is None:
            self.m = len(levels)
            self.k = len(levels[0])
            self.levels = [[np.ascontiguousarray(a) for a in ch] for ch in levels]
            nz, ny, nx = self.levels[0][0].shape
            self.dims = (nx, ny, nz)
            self.bpv = self.levels[0][0].dtype.itemsize
            self._ptrs = (ctypes.c_void_p * (self.m * self.k))()
            for c in range(self.m):
                for l in range(self.k):
                    assert self.levels[c][l].dtype == self.levels[0][0].dtype
                    self._ptrs[c * self.k + l] = self.levels[c][l].ctypes.data
            self.s.levels = ctypes.cast(self._ptrs, ctypes.POINTER(ctypes.c_void_p))
        else:
            self.m, self.k, self.dims, self.bpv, fn, fctx = provider
            nx, ny, nz = self.dims
            self.levels = None
            self.s.levels = None
            self.s.voxel_fn = fn
            self.s.voxel_ctx = fctx
        self.s.dims[:] = list(self.dims)
        self.s.spacing[:] = [float(np.float32(v)) for v in spacing]
        self.s.m, self.s.k, self.s.B, self.s.bpv = self.m, self.k, int(B), self.bpv
        self.s.leaf[:] = list(leaf_extent)
        self.n_bricks = int(lib().or_brick_count(ctypes.byref(self.s)))
        self.resident = np.zeros(self.n_bricks, np.uint8)
        self.s.resident = self.resident.ctypes.data
        self.set_resident(resident)
        ex, ey, ez = leaf_extent
        self.leaf_shape = (-(-nz // ez), -(-ny // ey), -(-nx // ex))
        n_leaves = int(np.prod(self.leaf_shape))
        self.leaf_min = np.full((self.m, n_leaves), -1, np.int64)
        self.leaf_max = np.full((self.m, n_leaves), -1, np.int64)
        if leaf_min is not None:
            self.leaf_min[:] = np.asarray(leaf_min, np.int64).reshape(self.m, n_leaves)
            self.leaf_max[:] = np.asarray(leaf_max, np.int64).reshape(self.m, n_leaves)
        self.s.leaf_min = self.leaf_min.ctypes.data
        self.s.leaf_max = self.leaf_max.ctypes.data
        self.set_node_ranges(node_min, node_max)

    def set_node_ranges(self, node_min, node_max):
        """Ranges the data source gave for inner nodes ((m, n_nodes) int64,
        -1 = none), or None for none."""
        if node_min is None:
            self.node_min = self.node_max = None
            self.s.node_min = self.s.node_max = None
            return
        n = self.n_nodes
        self.node_min = np.ascontiguousarray(np.asarray(node_min, np.int64).reshape(self.m, n))
        self.node_max = np.ascontiguousarray(np.asarray(node_max, np.int64).reshape(self.m, n))
        self.s.node_min = self.node_min.ctypes.data
        self.s.node_max = self.node_max.ctypes.data

    @property
    def depth(self) -> int:
        return int(lib().or_depth(ctypes.byref(self.s)))

    @property
    def n_nodes(self) -> int:
        return int(lib().or_node_count(ctypes.byref(self.s)))

    def brick_index(self, c, l, bx, by, bz) -> int:
        return int(lib().or_brick_index(ctypes.byref(self.s), c, l, bx, by, bz))

    def set_resident(self, bricks) -> None:
        self.resident[:] = 0
        for (c, l, bx, by, bz) in bricks:
            i = self.brick_index(c, l, bx, by, bz)
            if i < 0:
                raise ValueError(f"brick out of range: {(c, l, bx, by, bz)}")
            self.resident[i] = 1

    def node_words(self) -> np.ndarray:
        w = np.zeros((self.n_nodes, self.m), np.uint32)
        if lib().or_node_words(ctypes.byref(self.s), _p(w)) != 0:
            raise ValueError("or_node_words failed")
        return w

    def brick_id(self, c, l, bx, by, bz) -> int:
        return int(lib().or_brick_id(ctypes.byref(self.s), c, l, bx, by, bz))

    def flags_to_ids(self, flags: np.ndarray) -> np.ndarray:
        total = ctypes.c_int64()
        ids = np.zeros(max(1, int(flags.sum())), np.uint32)
        n = lib().or_flags_to_ids(ctypes.byref(self.s), _p(flags), _p(ids), ids.size, ctypes.byref(total))
        return ids[:n]

    def traversal_depth(self, dt, l) -> int:
        return int(lib().or_traversal_depth(ctypes.byref(self.s), float(dt), int(l)))


def _params(vol: Volume, frame) -> _Params:
    cam = frame.camera
    p = _Params()
    p.W, p.H, p.perspective = frame.W, frame.H, int(cam.perspective)
    p.eye[:], p.fwd[:], p.right[:], p.up[:] = cam.eye, cam.forward, cam.right, cam.up
    p.tan_x, p.tan_y, p.pixel = cam.tan_x, cam.tan_y, cam.pixel
    p.dt = frame.dt
    p.lod_t[:] = list(frame.lod_t) + [float("inf")] * (MAXL - len(frame.lod_t))
    lmin = list(frame.lmin) + [0] * (MAXC - len(frame.lmin))
    lmax = list(frame.lmax) + [0] * (MAXC - len(frame.lmax))
    p.lmin[:], p.lmax[:] = lmin, lmax
    p.start_depth, p.skip, p.ert = frame.start_depth, int(frame.skip), frame.ert
    p.tf_lo[:] = [t.lo for t in frame.tfs] + [0.0] * (MAXC - len(frame.tfs))
    p.tf_scale[:] = [t.scale for t in frame.tfs] + [0.0] * (MAXC - len(frame.tfs))
    return p


def bucket_occupancy(vol: Volume, frame) -> np.ndarray:
    lut = np.ascontiguousarray(np.stack([t.lut for t in frame.tfs]).astype(np.float32))
    p = _params(vol, frame)
    p.lut = lut.ctypes.data
    out = np.zeros((vol.m, 256), np.uint8)
    lib().or_bucket_occupancy(ctypes.byref(vol.s), ctypes.byref(p), _p(out))
    return out


def render(vol: Volume, words: np.ndarray, frame, pixels=None) -> dict:
    """March the given pixels ((n, 2) int32 of (px, py); default: all)."""
    if pixels is None:
        jj, ii = np.meshgrid(np.arange(frame.H), np.arange(frame.W), indexing="ij")
        pixels = np.stack([ii.ravel(), jj.ravel()], 1)
    pixels = np.ascontiguousarray(np.asarray(pixels, np.int32).reshape(-1, 2))
    n = pixels.shape[0]
    lut = np.ascontiguousarray(np.stack([t.lut for t in frame.tfs]).astype(np.float32))
    p = _params(vol, frame)
    p.lut = lut.ctypes.data
    o = dict(rgba32=np.zeros((n, 4), np.float32), rgba64=np.zeros((n, 4), np.float64),
             hash=np.zeros(n, np.uint32), n_eval=np.zeros(n, np.uint32), i_end=np.zeros(n, np.uint32),
             n_bs=np.zeros(n, np.uint32), req=np.zeros(vol.n_bricks, np.uint8),
             used=np.zeros(vol.n_bricks, np.uint8), node_req=np.zeros(vol.n_nodes * vol.m, np.uint8))
    outs = _Outputs(*[o[k].ctypes.data for k in ("rgba32", "rgba64", "hash", "n_eval", "i_end", "n_bs",
                                                  "req", "used", "node_req")])
    words = np.ascontiguousarray(words, np.uint32)
    rc = lib().or_render(ctypes.byref(vol.s), _p(words), ctypes.byref(p), _p(pixels), n, ctypes.byref(outs))
    if rc != 0:
        raise ValueError(f"or_render failed ({rc})")
    o["req_ids"] = vol.flags_to_ids(o["req"])
    o["used_ids"] = vol.flags_to_ids(o["used"])
    o["node_req_ids"] = np.nonzero(o["node_req"])[0].astype(np.uint32)
    o["pixels"] = pixels
    return o
