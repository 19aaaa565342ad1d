"""Oracle of the learned miss compensator (test infrastructure; only tests/,
__graft_entry__.smoke() and bench.py's CPU leg may use it).

A missing level-0 brick is predicted from its resident level-1 parent (the
paper substitutes the coarser brick, Sec. 6.1; the compensator refines that
substitute).  Plain binary64 numpy, written from the definitions:

upsample  the level-0 apron grid (B+2)^3 of brick b0, each voxel X sampled
          trilinearly from the level-1 apron slot of the parent b1 = b0 // 2
          at the level-1 coordinate u = (X + 0.5) / 2 - 0.5 (the voxel-centre
          convention of the renderer's trilinear step), values scaled by
          2^-S (S = 16 for u16 data).
network   y = x0 + f(x0): f is four 3x3x3 convolutions with zero padding
          ("same" size), 1 -> C -> C -> C -> 1 channels, bias, ReLU after
          the first three.  Weight layout W[tap, ci, co], tap = (dz * 3 +
          dy) * 3 + dx; activations channels-last [z, y, x, c].
loss      mean squared error against the true level-0 apron slot (scaled).
precision the GPU runs every product on the tensor cores with bfloat16
          operands (binary32 sums); forward(..., bf16_inputs=(0, 1, 2, 3))
          mirrors that rounding of the layer inputs, and
          loss_and_grads(..., bf16_grads=(0, 1, 2, 3)) the rounding of the
          output gradients that enter the layers' weight- and input-
          gradient products (their bias gradients sum the unrounded values).
adam      one step of Adam (Kingma and Ba, 2015, Algorithm 1): exponential
          moving averages of the gradient and its square, both divided by
          their bias corrections 1 - beta^t, then a step of lr * m_hat /
          (sqrt(v_hat) + eps).

Parity unpinned where the GPU's binary32 accumulation order differs: the
GPU kernels are compared within a tolerance derived from that order.
"""
from __future__ import annotations

import numpy as np

C = 32           # hidden channels
LAYERS = ((1, C), (C, C), (C, C), (C, 1))


def upsample(l1_slot: np.ndarray, octant, B: int = 32) -> np.ndarray:
    """l1_slot: (B+2)^3 level-1 apron slot [z, y, x] (raw values, origin at
    level-1 voxel 32*b1 - 1); octant (ox, oy, oz) in {0, 1}^3: which child.
    Returns the (B+2)^3 level-0 grid of child b0 = 2*b1 + octant, origin at
    level-0 voxel 32*b0 - 1, as float64 (raw units)."""
    E = B + 2
    v = np.asarray(l1_slot, np.float64)
    idx, frac = [], []
    for a, o in enumerate(octant):
        X = np.arange(E) - 1 + B * o               # level-0 voxel relative to 32 * (2 * b1)
        u = (X + 0.5) / 2.0 - 0.5                  # level-1 coordinate relative to 32 * b1
        i0 = np.floor(u).astype(np.int64)
        idx.append(i0 + 1)                         # slot index (the slot starts at voxel -1)
        frac.append(u - i0)
    ix, iy, iz = idx
    fx, fy, fz = frac
    out = np.zeros((E, E, E))
    for dz in (0, 1):
        wz = fz if dz else 1.0 - fz
        for dy in (0, 1):
            wy = fy if dy else 1.0 - fy
            for dx in (0, 1):
                wx = fx if dx else 1.0 - fx
                out += (wz[:, None, None] * wy[None, :, None] * wx[None, None, :]) * \
                    v[np.ix_(iz + dz, iy + dy, ix + dx)]
    return out


def conv3(x: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """'same' 3x3x3 convolution (cross-correlation) with zero padding.
    x [Z, Y, X, ci], W [27, ci, co], b [co] -> [Z, Y, X, co]."""
    Z, Y, X, _ = x.shape
    xp = np.pad(x, ((1, 1), (1, 1), (1, 1), (0, 0)))
    out = np.broadcast_to(b, (Z, Y, X, W.shape[2])).astype(np.float64).copy()
    for t in range(27):
        dz, dy, dx = t // 9, (t // 3) % 3, t % 3
        out += np.einsum("zyxi,io->zyxo", xp[dz:dz + Z, dy:dy + Y, dx:dx + X], W[t])
    return out


def conv3_backward(x: np.ndarray, W: np.ndarray, g: np.ndarray):
    """Gradients of conv3 given dL/dout g: (dL/dx, dL/dW, dL/db)."""
    Z, Y, X, _ = x.shape
    xp = np.pad(x, ((1, 1), (1, 1), (1, 1), (0, 0)))
    dW = np.zeros_like(W, dtype=np.float64)
    dxp = np.zeros(xp.shape)
    for t in range(27):
        dz, dy, dx = t // 9, (t // 3) % 3, t % 3
        dW[t] = np.einsum("zyxi,zyxo->io", xp[dz:dz + Z, dy:dy + Y, dx:dx + X], g)
        dxp[dz:dz + Z, dy:dy + Y, dx:dx + X] += np.einsum("zyxo,io->zyxi", g, W[t])
    return dxp[1:-1, 1:-1, 1:-1], dW, g.sum(axis=(0, 1, 2))


def init_params(seed: int = 0):
    """He-scaled normal weights (the last layer 100x smaller, so the net
    starts near the identity y = x0), zero biases."""
    rng = np.random.default_rng(seed)
    params = []
    for i, (ci, co) in enumerate(LAYERS):
        std = np.sqrt(2.0 / (27 * ci)) * (0.01 if i == len(LAYERS) - 1 else 1.0)
        params.append((rng.normal(0.0, std, (27, ci, co)), np.zeros(co)))
    return params


def forward(params, x0: np.ndarray, bf16_inputs=()):
    """x0 [Z, Y, X] (scaled) -> (y [Z, Y, X], the input of every layer).
    bf16_inputs: layers whose input enters rounded to bfloat16 (the layers
    the GPU runs on the tensor cores)."""
    a = x0[..., None]
    acts = []
    for i, (W, b) in enumerate(params):
        if i in bf16_inputs:
            a = bf16(a)
        acts.append(a)
        a = conv3(a, W, b)
        if i < len(params) - 1:
            a = np.maximum(a, 0.0)
    return x0 + a[..., 0], acts


def loss_and_grads(params, x0: np.ndarray, target: np.ndarray, bf16_inputs=(), bf16_grads=()):
    """Mean squared error of forward(x0) against target and its gradients
    with respect to every weight and bias.  bf16_grads: layers whose output
    gradient enters the weight- and input-gradient products rounded to
    bfloat16 (the bias gradient is summed from the unrounded values)."""
    y, acts = forward(params, x0, bf16_inputs)
    n = y.size
    d = y - target
    loss = float((d * d).sum() / n)
    g = (2.0 / n) * d[..., None]
    grads = [None] * len(params)
    for i in range(len(params) - 1, -1, -1):
        W, _ = params[i]
        gx, gW, _ = conv3_backward(acts[i], W, bf16(g) if i in bf16_grads else g)
        gb = g.sum(axis=(0, 1, 2))
        grads[i] = (gW, gb)
        if i > 0:
            g = gx * (acts[i] > 0.0)
    return loss, grads


def bf16(x: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), via the float32 bits."""
    f = np.asarray(x, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def adam_step(p: np.ndarray, g: np.ndarray, m: np.ndarray, v: np.ndarray, t: int, lr: float,
              beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """Adam step t >= 1 (Kingma and Ba, 2015, Algorithm 1), binary64, on flat
    arrays: returns the new parameters and the new first and second moment
    estimates."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** t)
    v_hat = v / (1.0 - beta2 ** t)
    return p - lr * m_hat / (np.sqrt(v_hat) + eps), m, v
