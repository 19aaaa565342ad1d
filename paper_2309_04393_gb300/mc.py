"""Thin ctypes binding of include/ro_mc.h (the learned miss compensator).

Argument marshalling only: upsample, the network, its gradients and Adam run
in libro.so's CUDA kernels.  Device memory comes from torch (one uint8 arena
sized by ro_mc_query_bytes); grids are torch cuda tensors.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import ro

EDGE = 34
VOXELS = EDGE ** 3
PARAMS = 57121
LAYERS = ((1, 32), (32, 32), (32, 32), (32, 1))


# every entry point include/ro_mc.h declares
EXPORTS = ["ro_mc_query_bytes", "ro_mc_create", "ro_mc_destroy", "ro_mc_set_params", "ro_mc_get_params",
           "ro_mc_upsample", "ro_mc_forward", "ro_mc_gradients", "ro_mc_train_step", "ro_mc_apply_gradients",
           "ro_mc_get_moments", "ro_compensate_bricks"]


class McDesc(ctypes.Structure):
    _fields_ = [("max_batch", ctypes.c_uint32)]


def _lib():
    L = ro.load()
    if not getattr(L, "_mc_typed", False):
        vp, u32 = ctypes.c_void_p, ctypes.c_uint32
        L.ro_mc_query_bytes.argtypes = [ctypes.POINTER(McDesc), ctypes.POINTER(ctypes.c_uint64)]
        L.ro_mc_create.argtypes = [ctypes.POINTER(McDesc), vp, ctypes.c_uint64, vp, ctypes.POINTER(vp)]
        L.ro_mc_destroy.argtypes = [vp]
        L.ro_mc_set_params.argtypes = [vp, vp]
        L.ro_mc_get_params.argtypes = [vp, vp]
        L.ro_mc_upsample.argtypes = [vp, u32, vp, vp, vp]
        L.ro_mc_forward.argtypes = [vp, u32, vp, vp]
        L.ro_mc_gradients.argtypes = [vp, u32, vp, vp, vp, vp]
        L.ro_mc_train_step.argtypes = [vp, u32, vp, vp, ctypes.c_float, vp]
        L.ro_mc_apply_gradients.argtypes = [vp, vp, ctypes.c_float]
        L.ro_mc_get_moments.argtypes = [vp, vp, vp, ctypes.POINTER(u32)]
        L.ro_compensate_bricks.argtypes = [vp, vp, u32, vp, vp]
        for f in EXPORTS:
            getattr(L, f).restype = ctypes.c_int
        L._mc_typed = True
    return L


def flatten(params) -> np.ndarray:
    """[(W[27, ci, co], b[co]) x 4] -> the RO_MC_PARAMS float32 vector."""
    return np.concatenate([np.concatenate([np.asarray(W).ravel(), np.asarray(b).ravel()]) for W, b in params]) \
        .astype(np.float32)


def unflatten(v: np.ndarray):
    out, o = [], 0
    for ci, co in LAYERS:
        W = v[o:o + 27 * ci * co].reshape(27, ci, co)
        o += 27 * ci * co
        b = v[o:o + co]
        o += co
        out.append((W, b))
    return out


def init_params(seed: int = 0) -> np.ndarray:
    """Seeded He-normal weights (the last layer 100x smaller, so the network
    starts near y = x0) and zero biases, as the RO_MC_PARAMS vector."""
    rng = np.random.default_rng(seed)
    parts = []
    for i, (ci, co) in enumerate(LAYERS):
        std = np.sqrt(2.0 / (27 * ci)) * (0.01 if i == len(LAYERS) - 1 else 1.0)
        parts.append(rng.normal(0.0, std, 27 * ci * co))
        parts.append(np.zeros(co))
    return np.concatenate(parts).astype(np.float32)


class Compensator:
    def __init__(self, max_batch: int, stream=None, device=None):
        import torch
        self.torch = torch
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.L = _lib()
        self.desc = McDesc(int(max_batch))
        nbytes = ctypes.c_uint64()
        self._check(self.L.ro_mc_query_bytes(ctypes.byref(self.desc), ctypes.byref(nbytes)))
        self.arena = torch.empty(int(nbytes.value), dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        self._check(self.L.ro_mc_create(ctypes.byref(self.desc), ctypes.c_void_p(self.arena.data_ptr()), nbytes.value,
                                        ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self.h = h

    @staticmethod
    def _check(rc):
        if rc != 0:
            raise ro.RoError(rc, "compensator call failed")

    def close(self):
        if self.h:
            self._check(self.L.ro_mc_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params):
        v = np.ascontiguousarray(flatten(params) if isinstance(params, (list, tuple)) else params, np.float32)
        assert v.size == PARAMS
        self._check(self.L.ro_mc_set_params(self.h, v.ctypes.data_as(ctypes.c_void_p)))

    def get_params(self) -> np.ndarray:
        v = np.zeros(PARAMS, np.float32)
        self._check(self.L.ro_mc_get_params(self.h, v.ctypes.data_as(ctypes.c_void_p)))
        return v

    def _grid(self, n):
        return self.torch.empty((n, EDGE, EDGE, EDGE), dtype=self.torch.float32, device=self.device)

    def upsample(self, slots, octants):
        """slots: cuda int16/uint16 tensor (n, 34, 34, 34) of raw level-1 values;
        octants: cuda int32 tensor (n,) with bits x, y, z."""
        n = slots.shape[0]
        x0 = self._grid(n)
        self._check(self.L.ro_mc_upsample(self.h, n, ctypes.c_void_p(slots.data_ptr()),
                                          ctypes.c_void_p(octants.data_ptr()), ctypes.c_void_p(x0.data_ptr())))
        return x0

    def forward(self, x0):
        y = self._grid(x0.shape[0])
        self._check(self.L.ro_mc_forward(self.h, x0.shape[0], ctypes.c_void_p(x0.data_ptr()),
                                         ctypes.c_void_p(y.data_ptr())))
        return y

    def gradients(self, x0, target):
        g = self.torch.empty(PARAMS, dtype=self.torch.float32, device=self.device)
        loss = self.torch.zeros(1, dtype=self.torch.float32, device=self.device)
        self._check(self.L.ro_mc_gradients(self.h, x0.shape[0], ctypes.c_void_p(x0.data_ptr()),
                                           ctypes.c_void_p(target.data_ptr()), ctypes.c_void_p(g.data_ptr()),
                                           ctypes.c_void_p(loss.data_ptr())))
        return g, loss

    def train_step(self, x0, target, lr, loss=None):
        """One Adam step; loss (cuda float32, one element) receives the batch loss."""
        ptr = ctypes.c_void_p(loss.data_ptr()) if loss is not None else None
        self._check(self.L.ro_mc_train_step(self.h, x0.shape[0], ctypes.c_void_p(x0.data_ptr()),
                                            ctypes.c_void_p(target.data_ptr()), ctypes.c_float(lr), ptr))

    def apply_gradients(self, grads, lr):
        """One Adam step on given gradients (cuda float32 tensor of PARAMS)."""
        assert grads.numel() == PARAMS and grads.dtype == self.torch.float32 and grads.is_contiguous()
        self._check(self.L.ro_mc_apply_gradients(self.h, ctypes.c_void_p(grads.data_ptr()), ctypes.c_float(lr)))

    def get_moments(self):
        """(m, v, step): the Adam moment estimates and the step count."""
        m, v, step = np.zeros(PARAMS, np.float32), np.zeros(PARAMS, np.float32), ctypes.c_uint32()
        self._check(self.L.ro_mc_get_moments(self.h, m.ctypes.data_as(ctypes.c_void_p),
                                             v.ctypes.data_as(ctypes.c_void_p), ctypes.byref(step)))
        return m, v, int(step.value)


def compensate_bricks(ctx, comp: Compensator, ids) -> np.ndarray:
    """ro_compensate_bricks: predicted level-0 bricks for the given IDs
    (their level-1 parents resident); returns the slots."""
    ids = np.ascontiguousarray(np.asarray(ids, np.uint32))
    slots = np.zeros(max(1, ids.size), np.uint32)
    ctx._check(_lib().ro_compensate_bricks(ctx.h, comp.h, ids.size, ids.ctypes.data_as(ctypes.c_void_p),
                                           slots.ctypes.data_as(ctypes.c_void_p)))
    return slots[:ids.size]
