"""Thin ctypes binding of the C ABI in include/ro.h.

Argument marshalling only: every step of the path runs in libro.so's CUDA
kernels.  Device memory comes from torch (one uint8 arena per context, sized
by ro_query_sizes); the CUDA stream is torch's current stream unless another
is given.  If the library cannot be loaded this module raises: there is no
fallback path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

RO_MAX_CHANNELS = 16
RO_MAX_LEVELS = 16
RO_MAX_VIEWS = 256
RO_NONE = 0xFFFFFFFF
STATUS = {0: "RO_OK", 1: "RO_ERR_INVALID_ARG", 2: "RO_ERR_CUDA", 3: "RO_ERR_CAPACITY", 4: "RO_ERR_TIMEOUT",
          5: "RO_ERR_INTERNAL"}
EXPORTS = ["ro_query_sizes", "ro_create", "ro_destroy", "ro_upload_bricks", "ro_update_residency_octree", "ro_render",
           "ro_read_requests", "ro_get_stats", "ro_debug_read", "ro_brick_index", "ro_set_timeout", "ro_last_error",
           "ro_compact_flags_noalloc", "ro_render_batch", "ro_autotune_batch", "ro_replace_channel",
           "ro_update_node_metadata", "ro_upload_bricks_async", "ro_upload_wait"]
RO_UNKNOWN_DEPTH = 254


class RoError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Desc(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_uint32 * 3), ("spacing", ctypes.c_float * 3), ("channels", ctypes.c_uint32),
                ("value_bits", ctypes.c_uint32), ("brick", ctypes.c_uint32), ("levels", ctypes.c_uint32),
                ("leaf_extent", ctypes.c_uint32 * 3), ("cache_slots", ctypes.c_uint32),
                ("max_requests", ctypes.c_uint32), ("max_upload", ctypes.c_uint32), ("max_meta", ctypes.c_uint32),
                ("max_batch_tiles", ctypes.c_uint32), ("sample_format", ctypes.c_uint32),
                ("keep_axes", ctypes.c_uint32 * RO_MAX_LEVELS)]


class Sizes(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("cache", "page_table", "octree", "req_flags", "node_req_flags",
                                                "used_flags", "last_used", "staging", "frame", "lists", "scratch",
                                                "total", "slot_pitch", "n_bricks", "n_nodes")] + \
               [("depth", ctypes.c_uint32), ("channel_stride", ctypes.c_uint32), ("batch", ctypes.c_uint64)]


class Camera(ctypes.Structure):
    _fields_ = [("eye", ctypes.c_float * 3), ("forward", ctypes.c_float * 3), ("right", ctypes.c_float * 3),
                ("up", ctypes.c_float * 3), ("perspective", ctypes.c_uint32), ("tan_x", ctypes.c_float),
                ("tan_y", ctypes.c_float), ("pixel", ctypes.c_float)]


class TF(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_float), ("scale", ctypes.c_float), ("lut", ctypes.c_void_p)]


class RenderParams(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_float), ("lod_t", ctypes.c_float * RO_MAX_LEVELS),
                ("lmin", ctypes.c_uint32 * RO_MAX_CHANNELS), ("lmax", ctypes.c_uint32 * RO_MAX_CHANNELS),
                ("start_depth", ctypes.c_uint32), ("skip", ctypes.c_uint32), ("ert", ctypes.c_float),
                ("debug_hash", ctypes.c_void_p), ("debug_n_eval", ctypes.c_void_p),
                ("debug_i_end", ctypes.c_void_p), ("debug_n_bs", ctypes.c_void_p), ("order", ctypes.c_uint32)]


class View(ctypes.Structure):
    _fields_ = [("camera", Camera), ("params", RenderParams), ("image", ctypes.c_void_p), ("W", ctypes.c_uint32),
                ("H", ctypes.c_uint32)]


class Schedule(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_uint32), ("order", ctypes.c_uint32)]


class LeafMeta(ctypes.Structure):
    _fields_ = [("leaf", ctypes.c_uint32), ("channel", ctypes.c_uint32), ("vmin", ctypes.c_uint32),
                ("vmax", ctypes.c_uint32)]


_lib = None


def library_path() -> str:
    return _build.SO


def load(build_if_missing: bool = True):
    """Load libro.so (building it first if asked and absent)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.SO):
        if not build_if_missing:
            raise RoError(2, f"libro.so not built at {_build.SO}")
        _build.build()
    L = ctypes.CDLL(_build.SO)
    vp, u32, u64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
    L.ro_query_sizes.argtypes = [ctypes.POINTER(Desc), ctypes.POINTER(Sizes)]
    L.ro_create.argtypes = [ctypes.POINTER(Desc), vp, u64, vp, ctypes.POINTER(vp)]
    L.ro_destroy.argtypes = [vp]
    L.ro_upload_bricks.argtypes = [vp, u32, vp, vp, vp, vp]
    L.ro_upload_bricks_async.argtypes = [vp, u32, vp, vp, vp, vp, vp]
    L.ro_upload_wait.argtypes = [vp]
    L.ro_update_residency_octree.argtypes = [vp, u32, vp]
    L.ro_update_node_metadata.argtypes = [vp, u32, vp]
    L.ro_render.argtypes = [vp, ctypes.POINTER(Camera), vp, ctypes.POINTER(RenderParams), vp, u32, u32]
    L.ro_read_requests.argtypes = [vp, vp, u32, vp, vp, vp, u32, vp]
    L.ro_get_stats.argtypes = [vp, vp]
    L.ro_debug_read.argtypes = [vp, u32, vp, u64]
    L.ro_brick_index.restype = u32
    L.ro_brick_index.argtypes = [vp, u32]
    L.ro_set_timeout.argtypes = [vp, u32]
    L.ro_last_error.restype = ctypes.c_char_p
    L.ro_last_error.argtypes = [vp]
    L.ro_compact_flags_noalloc.argtypes = [vp, u64, vp, u32, vp, vp]
    L.ro_render_batch.argtypes = [vp, u32, vp, vp, ctypes.POINTER(Schedule)]
    L.ro_replace_channel.argtypes = [vp, u32]
    L.ro_autotune_batch.argtypes = [vp, u32, vp, vp, ctypes.POINTER(Schedule), ctypes.POINTER(ctypes.c_float)]
    for f in EXPORTS:
        getattr(L, f).restype = getattr(L, f).restype if f in ("ro_brick_index", "ro_last_error") else ctypes.c_int
    _lib = L
    return L


def make_desc(dims, spacing, channels, value_bits, brick, levels, leaf_extent, cache_slots, max_requests=65536,
              max_upload=1024, max_meta=65536, max_batch_tiles=0, sample_format=0, keep_axes=None) -> Desc:
    """sample_format: 0 raw values with binary32 lerps, 1 binary16, 2 bfloat16.
    keep_axes: per level l, bit a set = axis a keeps its resolution from
    level l to l + 1 (default: every level halves every axis)."""
    d = Desc()
    d.dims[:] = [int(v) for v in dims]
    d.spacing[:] = [float(v) for v in spacing]
    d.channels, d.value_bits, d.brick, d.levels = int(channels), int(value_bits), int(brick), int(levels)
    d.leaf_extent[:] = [int(v) for v in leaf_extent]
    d.cache_slots, d.max_requests, d.max_upload, d.max_meta = int(cache_slots), int(max_requests), int(max_upload), \
        int(max_meta)
    d.max_batch_tiles = int(max_batch_tiles)
    d.sample_format = int(sample_format)
    ka = list(keep_axes or []) + [0] * RO_MAX_LEVELS
    d.keep_axes[:] = [int(v) for v in ka[:RO_MAX_LEVELS]]
    return d


def query_sizes(desc: Desc) -> Sizes:
    L = load()
    s = Sizes()
    rc = L.ro_query_sizes(ctypes.byref(desc), ctypes.byref(s))
    if rc != 0:
        raise RoError(rc, L.ro_last_error(None).decode())
    return s


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


class Context:
    """One residency-octree renderer over a torch-allocated device arena."""

    def __init__(self, desc: Desc, stream=None, device=None):
        import torch
        self.torch = torch
        self.L = load()
        self.desc = desc
        self.sizes = query_sizes(desc)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.arena = torch.empty(int(self.sizes.total), dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        rc = self.L.ro_create(ctypes.byref(desc), ctypes.c_void_p(self.arena.data_ptr()), int(self.sizes.total),
                              ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if rc != 0:
            raise RoError(rc, self.L.ro_last_error(None).decode())
        self.h = h
        self.m = int(desc.channels)
        self.k = int(desc.levels)

    def _check(self, rc):
        if rc != 0:
            raise RoError(rc, self.L.ro_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            rc = self.L.ro_destroy(self.h)
            self.h = None
            self._check_destroy(rc)

    def _check_destroy(self, rc):
        if rc != 0:
            raise RoError(rc, "ro_destroy failed")

    def __del__(self):
        try:
            if getattr(self, "h", None):
                self.L.ro_destroy(self.h)
                self.h = None
        except Exception:
            pass

    def set_timeout(self, ms: int):
        self._check(self.L.ro_set_timeout(self.h, int(ms)))

    # ------------------------------------------------------------ calls
    def upload_bricks(self, ids, voxels):
        ids = np.ascontiguousarray(np.asarray(ids, np.uint32))
        voxels = np.ascontiguousarray(voxels)
        n = ids.size
        slots = np.zeros(n, np.uint32)
        evicted = np.zeros(n, np.uint32)
        self._check(self.L.ro_upload_bricks(self.h, n, _ptr(ids), _ptr(voxels), _ptr(slots), _ptr(evicted)))
        return slots, evicted

    def upload_bricks_async(self, ids, voxels, copy_stream):
        """ro_upload_bricks_async: voxels a page-locked CPU tensor (or a view
        of one: a numpy array over pinned memory), kept unchanged until
        upload_wait(); copy_stream a torch.cuda.Stream."""
        ids = np.ascontiguousarray(np.asarray(ids, np.uint32))
        n = ids.size
        slots = np.zeros(n, np.uint32)
        evicted = np.zeros(n, np.uint32)
        ptr = voxels.data_ptr() if hasattr(voxels, "data_ptr") else voxels.ctypes.data
        self._check(self.L.ro_upload_bricks_async(self.h, n, _ptr(ids), ctypes.c_void_p(ptr), _ptr(slots),
                                                  _ptr(evicted), ctypes.c_void_p(copy_stream.cuda_stream)))
        return slots, evicted

    def upload_wait(self):
        self._check(self.L.ro_upload_wait(self.h))

    def update_residency_octree(self, meta=None):
        """meta: (n, 4) uint32 rows (leaf, channel, vmin, vmax) or None."""
        if meta is None or len(meta) == 0:
            self._check(self.L.ro_update_residency_octree(self.h, 0, None))
            return
        meta = np.ascontiguousarray(np.asarray(meta, np.uint32).reshape(-1, 4))
        self._check(self.L.ro_update_residency_octree(self.h, meta.shape[0], _ptr(meta)))

    def update_node_metadata(self, meta):
        """meta: (n, 4) uint32 rows (node, channel, vmin, vmax), nodes numbered
        as node requests number them (depth-major, leaves last)."""
        meta = np.ascontiguousarray(np.asarray(meta, np.uint32).reshape(-1, 4))
        self._check(self.L.ro_update_node_metadata(self.h, meta.shape[0], _ptr(meta) if meta.size else None))

    def render(self, camera: Camera, tfs, params: RenderParams, image, W: int, H: int):
        """tfs: list of (lo, scale, lut (256, 4) float32); image: cuda float32 tensor with W*H*4 elements."""
        assert image.is_cuda and image.dtype == self.torch.float32 and image.numel() >= W * H * 4
        luts = [np.ascontiguousarray(np.asarray(t[2], np.float32).reshape(256, 4)) for t in tfs]
        arr = (TF * len(tfs))()
        for i, (lo, sc, _) in enumerate(tfs):
            arr[i].lo, arr[i].scale, arr[i].lut = float(lo), float(sc), luts[i].ctypes.data
        self._check(self.L.ro_render(self.h, ctypes.byref(camera), arr, ctypes.byref(params),
                                     ctypes.c_void_p(image.data_ptr()), int(W), int(H)))

    def _tf_array(self, tfs):
        luts = [np.ascontiguousarray(np.asarray(t[2], np.float32).reshape(256, 4)) for t in tfs]
        arr = (TF * len(tfs))()
        for i, (lo, sc, _) in enumerate(tfs):
            arr[i].lo, arr[i].scale, arr[i].lut = float(lo), float(sc), luts[i].ctypes.data
        return arr, luts

    def render_batch(self, views, tfs, tile_w=8, order=0):
        """views: list of (Camera, RenderParams, image cuda tensor, W, H); tfs as for render."""
        arr, luts = self._tf_array(tfs)
        vs = (View * len(views))()
        for i, (cam, par, img, W, H) in enumerate(views):
            assert img.is_cuda and img.dtype == self.torch.float32 and img.numel() >= W * H * 4
            vs[i].camera, vs[i].params, vs[i].image, vs[i].W, vs[i].H = cam, par, img.data_ptr(), int(W), int(H)
        sched = Schedule(int(tile_w), int(order))
        self._check(self.L.ro_render_batch(self.h, len(views), vs, arr, ctypes.byref(sched)))

    def autotune_batch(self, views, tfs):
        """Returns ((tile_w, order), ms) of the fastest schedule for this batch."""
        arr, luts = self._tf_array(tfs)
        vs = (View * len(views))()
        for i, (cam, par, img, W, H) in enumerate(views):
            vs[i].camera, vs[i].params, vs[i].image, vs[i].W, vs[i].H = cam, par, img.data_ptr(), int(W), int(H)
        best, ms = Schedule(), ctypes.c_float()
        self._check(self.L.ro_autotune_batch(self.h, len(views), vs, arr, ctypes.byref(best), ctypes.byref(ms)))
        return (int(best.tile_w), int(best.order)), float(ms.value)

    def replace_channel(self, ch: int):
        """Free channel slot ch for another data-set channel (ro_replace_channel)."""
        self._check(self.L.ro_replace_channel(self.h, int(ch)))

    def read_requests(self, cap=None, node_cap=None):
        cap = int(self.desc.max_requests if cap is None else cap)
        node_cap = int(self.desc.max_requests if node_cap is None else node_cap)
        ids = np.zeros(max(cap, 1), np.uint32)
        nodes = np.zeros(max(node_cap, 1), np.uint32)
        n, ov, nn = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
        self._check(self.L.ro_read_requests(self.h, _ptr(ids), cap, ctypes.byref(n), ctypes.byref(ov), _ptr(nodes),
                                            node_cap, ctypes.byref(nn)))
        return ids[:n.value].copy(), int(ov.value), nodes[:nn.value].copy()

    def stats(self) -> np.ndarray:
        out = np.zeros(8, np.uint64)
        self._check(self.L.ro_get_stats(self.h, _ptr(out)))
        return out

    def debug_read(self, what: int) -> np.ndarray:
        s = self.sizes
        shape = {0: (int(s.n_nodes) * int(s.channel_stride), np.uint32), 1: (int(s.n_bricks), np.uint32),
                 2: (int(self.desc.cache_slots), np.uint32), 3: (int(s.n_bricks), np.uint8),
                 4: (int(self.desc.cache_slots), np.uint8),
                 5: (int(self.desc.cache_slots) * int(s.slot_pitch), np.uint8)}[what]
        out = np.zeros(shape[0], shape[1])
        self._check(self.L.ro_debug_read(self.h, int(what), _ptr(out), out.nbytes))
        return out

    def octree_words(self) -> np.ndarray:
        """(n_nodes, channels) node words, channel padding stripped."""
        w = self.debug_read(0).reshape(int(self.sizes.n_nodes), int(self.sizes.channel_stride))
        return np.ascontiguousarray(w[:, :self.m])

    def brick_index(self, brick_id: int) -> int:
        return int(self.L.ro_brick_index(self.h, int(brick_id)))


def compact_flags_noalloc(flags, ids, total, stream=None):
    """ro_compact_flags_noalloc on torch cuda tensors: flags (uint8, length a
    multiple of 16), ids (int32 capacity), total (int32, one element), all on
    one device; the call runs with that device current.  No device memory is
    allocated by the call."""
    import torch
    L = load()
    with torch.cuda.device(flags.device):
        st = stream if stream is not None else torch.cuda.current_stream(flags.device)
        rc = L.ro_compact_flags_noalloc(ctypes.c_void_p(flags.data_ptr()), flags.numel(),
                                        ctypes.c_void_p(ids.data_ptr()), ids.numel(),
                                        ctypes.c_void_p(total.data_ptr()), ctypes.c_void_p(st.cuda_stream))
    if rc != 0:
        raise RoError(rc, "ro_compact_flags_noalloc failed")


def brick_id(c, l, bx, by, bz, k) -> int:
    """32-bit brick ID: page table c*k + l in bits 31:24, then z, y, x."""
    return ((c * k + l) << 24) | (bz << 16) | (by << 8) | bx


def camera_struct(cam) -> Camera:
    c = Camera()
    c.eye[:], c.forward[:], c.right[:], c.up[:] = cam.eye, cam.forward, cam.right, cam.up
    c.perspective = int(cam.perspective)
    c.tan_x, c.tan_y, c.pixel = cam.tan_x, cam.tan_y, cam.pixel
    return c


def params_struct(frame, debug=None, order=0) -> RenderParams:
    p = RenderParams()
    p.dt = frame.dt
    p.lod_t[:] = list(frame.lod_t) + [float("inf")] * (RO_MAX_LEVELS - len(frame.lod_t))
    p.lmin[:] = list(frame.lmin) + [0] * (RO_MAX_CHANNELS - len(frame.lmin))
    p.lmax[:] = list(frame.lmax) + [0] * (RO_MAX_CHANNELS - len(frame.lmax))
    p.start_depth, p.skip, p.ert = int(frame.start_depth), int(frame.skip), float(frame.ert)
    p.order = int(order)
    if debug is not None:
        p.debug_hash, p.debug_n_eval, p.debug_i_end, p.debug_n_bs = [int(t.data_ptr()) for t in debug]
    return p


def render_batch(ctx: Context, frames, images=None, tile_w=8, order=0, debug=False):
    """Render several synth.Frame-like views (same TFs: those of frames[0])
    in one batch launch.  Returns the list of (H, W, 4) images and, with
    debug=True, the per-view debug tensors."""
    torch = ctx.torch
    if images is None:
        images = [torch.empty((int(f.H), int(f.W), 4), dtype=torch.float32, device=ctx.device) for f in frames]
    dbgs = []
    views = []
    for f, img in zip(frames, images):
        dbg = None
        if debug:
            dbg = [torch.zeros((int(f.H), int(f.W)), dtype=torch.int32, device=ctx.device) for _ in range(4)]
        dbgs.append(dbg)
        views.append((camera_struct(f.camera), params_struct(f, dbg), img, int(f.W), int(f.H)))
    ctx.render_batch(views, [(t.lo, t.scale, t.lut) for t in frames[0].tfs], tile_w=tile_w, order=order)
    return images, dbgs


def render_frame(ctx: Context, frame, image=None, debug=False, order=0):
    """Render one frame described by a synth.Frame-like object (W, H, camera,
    tfs, dt, lod_t, lmin, lmax, start_depth, skip, ert).  Returns the (H, W, 4)
    float32 cuda image and, with debug=True, per-pixel (hash, n_eval, i_end,
    n_bs) uint32 cuda tensors."""
    torch = ctx.torch
    W, H = int(frame.W), int(frame.H)
    if image is None:
        image = torch.empty((H, W, 4), dtype=torch.float32, device=ctx.device)
    dbg = None
    if debug:
        dbg = [torch.zeros((H, W), dtype=torch.int32, device=ctx.device) for _ in range(4)]
    ctx.render(camera_struct(frame.camera), [(t.lo, t.scale, t.lut) for t in frame.tfs],
               params_struct(frame, dbg, order), image, W, H)
    return image, dbg
