"""Pins of the CPU oracle to things other than itself (CPU only).

Each test fixes part of the oracle against the paper's definitions worked
out by a different route (voxel-level enumeration instead of interval
arithmetic, exactly representable ray positions, closed forms, a textbook
front-to-back loop built on scipy's trilinear interpolation), so that a
dropped term, wrong index or transposed operand in oracle.c fails one of them.
"""
import math
import os

import numpy as np
import pytest
from scipy import ndimage

import oracle
import synth

INF = float("inf")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def lod_none():
    return [0.0] + [INF] * 15


def frame(cam, W, H, tfs, dt=0.5, lmin=None, lmax=None, **kw):
    m = len(tfs)
    return synth.Frame(W, H, cam, tfs, dt, kw.pop("lod_t", lod_none()), lmin or [0] * m, lmax or [0] * m, **kw)


def all_bricks(levels_c, B, channels):
    out = []
    for c in channels:
        for l, a in enumerate(levels_c[c]):
            nz, ny, nx = a.shape
            for z in range(-(-nz // B)):
                for y in range(-(-ny // B)):
                    for x in range(-(-nx // B)):
                        out.append((c, l, x, y, z))
    return out


def exact_meta(levels, leaf):
    mins, maxs = [], []
    for ch in levels:
        mn, mx = synth.leaf_ranges(ch[0], leaf)
        mins.append(mn.astype(np.int64))
        maxs.append(mx.astype(np.int64))
    return np.stack(mins), np.stack(maxs)


# ------------------------------------------------------------ bit layouts

def test_golden_bit_layouts():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "brick_id_layout.txt")) if l.strip() and l[0] != "#"]
    ids = [r for r in rows if len(r) == 7]
    words = [r for r in rows if len(r) == 4]
    assert len(ids) == 5 and len(words) == 3
    for k, c, l, bx, by, bz, h in ids:
        k = int(k)
        lv = [[np.zeros((1, 1, 1), np.uint8)] * k]
        v = oracle.Volume(lv, (1, 1, 1), 1, (1, 1, 1))
        assert v.brick_id(int(c), int(l), int(bx), int(by), int(bz)) == int(h, 16)
    # node word: one node (the root), resident bricks at levels 0 and 2, range [3, 200]
    lv = [np.zeros((8, 8, 8), np.uint8), np.zeros((4, 4, 4), np.uint8), np.zeros((2, 2, 2), np.uint8)]
    v = oracle.Volume([lv], (1, 1, 1), 4, (8, 8, 8), [(0, 0, 1, 1, 0), (0, 2, 0, 0, 0)],
                      np.array([[3]]), np.array([[200]]))
    w = v.node_words()
    mask, mn, mx, want = words[0]
    assert (int(mask, 16), int(mn), int(mx)) == (5, 3, 200)
    assert w.shape == (1, 1) and int(w[0, 0]) == int(want, 16)


# ------------------------------------------------------ residency (O-a)

def brute_words(dims, B, leaf, k, m, resident, lmin, lmax, bpv):
    """Node words by enumerating level-0 voxels: bit l is set iff some voxel of
    the node lies in a resident brick of level l; the range is taken over the
    leaves that own the node's voxels."""
    nx, ny, nz = dims
    ex, ey, ez = leaf
    nl = [-(-nx // ex), -(-ny // ey), -(-nz // ez)]
    D = max(max(0, math.ceil(math.log2(n))) if n > 1 else 0 for n in nl)
    res = set(resident)
    out = []
    for d in range(D + 1):
        E = [ex << (D - d), ey << (D - d), ez << (D - d)]
        nn = [-(-nx // E[0]), -(-ny // E[1]), -(-nz // E[2])]
        for jz in range(nn[2]):
            for jy in range(nn[1]):
                for jx in range(nn[0]):
                    vox = [(x, y, z) for z in range(jz * E[2], min((jz + 1) * E[2], nz))
                           for y in range(jy * E[1], min((jy + 1) * E[1], ny))
                           for x in range(jx * E[0], min((jx + 1) * E[0], nx))]
                    leaves = {(x // ex, y // ey, z // ez) for (x, y, z) in vox}
                    row = []
                    for c in range(m):
                        mask = 0
                        for l in range(k):
                            BL = B << l
                            if any((c, l, x // BL, y // BL, z // BL) in res for (x, y, z) in vox):
                                mask |= 1 << l
                        vals = [(lmin[c][lz][ly][lx], lmax[c][lz][ly][lx]) for (lx, ly, lz) in leaves]
                        if any(a < 0 for a, _ in vals):
                            q0, q1 = 255, 254      # INVALID, no valid ancestor: UNKNOWN
                        else:
                            a, b = min(v[0] for v in vals), max(v[1] for v in vals)
                            q0, q1 = (a, b) if bpv == 1 else (a >> 8, b >> 8)
                        row.append(mask | (q0 << 16) | (q1 << 24))
                    out.append(row)
    return np.array(out, np.uint32)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_residency_matches_voxel_enumeration(seed):
    rng = np.random.default_rng(seed)
    dims, B, leaf, k, m = (12, 10, 7), 4, (2, 2, 1), 3, 2
    bpv = 2 if seed == 2 else 1
    dt = np.uint16 if bpv == 2 else np.uint8
    lv = [[np.zeros((1, 1, 1), dt)] for _ in range(m)]
    # the oracle only reads level shapes for residency; build real shapes
    for c in range(m):
        a = np.zeros((dims[2], dims[1], dims[0]), dt)
        lv[c] = synth.mean_levels(a, k)
    cand = all_bricks(lv, B, range(m))
    resident = [b for b in cand if rng.random() < 0.3]
    nl = (-(-dims[2] // leaf[2]), -(-dims[1] // leaf[1]), -(-dims[0] // leaf[0]))
    hi = 65535 if bpv == 2 else 255
    lmin = rng.integers(0, hi // 2, size=(m,) + nl).astype(np.int64)
    lmax = lmin + rng.integers(0, hi // 2, size=(m,) + nl)
    missing = rng.random((m,) + nl) < 0.08
    lmin[missing] = -1
    lmax[missing] = -1
    v = oracle.Volume(lv, (1, 1, 1), B, leaf, resident, lmin, lmax)
    got = v.node_words()
    want = brute_words(dims, B, leaf, k, m, resident, lmin, lmax, bpv)
    assert got.shape == want.shape
    assert np.array_equal(got, want)


def test_residency_structural_invariants():
    """Parent mask = OR of the child masks (Sec. 5.3); a parent's range is the
    hull of its children's; INVALID propagates to every ancestor."""
    rng = np.random.default_rng(5)
    dims, B, leaf, k = (64, 48, 40), 8, (4, 4, 2), 4
    a = np.zeros((dims[2], dims[1], dims[0]), np.uint8)
    lv = [synth.mean_levels(a, k)]
    resident = [b for b in all_bricks(lv, B, [0]) if rng.random() < 0.2]
    nl = (20, 12, 16)
    lmin = rng.integers(0, 120, size=(1,) + nl).astype(np.int64)
    lmax = lmin + rng.integers(0, 120, size=(1,) + nl)
    lmin[0, 3, 4, 5] = lmax[0, 3, 4, 5] = -1
    v = oracle.Volume(lv, (1, 1, 1), B, leaf, resident, lmin, lmax)
    w = v.node_words()[:, 0]
    D = v.depth
    ext = lambda d: [leaf[0] << (D - d), leaf[1] << (D - d), leaf[2] << (D - d)]
    cnt = lambda d: [-(-dims[i] // ext(d)[i]) for i in range(3)]
    off = [0]
    for d in range(D + 1):
        off.append(off[-1] + int(np.prod(cnt(d))))
    n_invalid = 0
    for d in range(D):
        nc, nn = cnt(d + 1), cnt(d)
        for jz in range(nn[2]):
            for jy in range(nn[1]):
                for jx in range(nn[0]):
                    p = w[off[d] + (jz * nn[1] + jy) * nn[0] + jx]
                    kids = [w[off[d + 1] + (cz * nc[1] + cy) * nc[0] + cx]
                            for cz in (2 * jz, 2 * jz + 1) for cy in (2 * jy, 2 * jy + 1)
                            for cx in (2 * jx, 2 * jx + 1) if cx < nc[0] and cy < nc[1] and cz < nc[2]]
                    assert kids
                    orr = 0
                    for kw in kids:
                        orr |= int(kw) & 0xFFFF
                    assert int(p) & 0xFFFF == orr
                    kmin = [(int(kw) >> 16) & 255 for kw in kids]
                    kmax = [int(kw) >> 24 for kw in kids]
                    if any(a > b for a, b in zip(kmin, kmax)):
                        assert ((int(p) >> 16) & 255) > (int(p) >> 24)
                        n_invalid += 1
                    else:
                        assert (int(p) >> 16) & 255 == min(kmin) and int(p) >> 24 == max(kmax)
    assert n_invalid == D          # exactly the ancestors of the one leaf without metadata


def test_traversal_depth_closed_form():
    lv = [[np.zeros((128, 128, 128), np.uint8)]]
    v = oracle.Volume(lv, (1, 1, 1), 32, (16, 16, 16))
    assert v.depth == 3
    # node extent 16*2^(3-d) voxels; deepest d with extent >= 0.5*2^l
    for l in range(6):
        assert v.traversal_depth(0.5, l) == 3
    assert v.traversal_depth(0.5, 6) == 2 and v.traversal_depth(0.5, 7) == 1
    assert v.traversal_depth(0.5, 8) == 0 and v.traversal_depth(0.5, 12) == 0
    # anisotropic leaf 16x16x4 at spacing 1:1:4 is 16 physical units per axis
    lv = [[np.zeros((64, 256, 256), np.uint16)]]
    v = oracle.Volume(lv, (1, 1, 4), 32, (16, 16, 4))
    assert v.depth == 4 and v.traversal_depth(0.5, 5) == 4 and v.traversal_depth(0.5, 6) == 3


def test_bucket_occupancy_closed_forms():
    lv = [[np.zeros((4, 4, 4), np.uint8)]]
    v = oracle.Volume(lv, (1, 1, 1), 4, (4, 4, 4))
    lut = np.zeros((256, 4), np.float32)
    lut[[5, 100, 101, 255], 3] = 0.5
    fr = frame(synth.look_at((2, 2, -1), (2, 2, 2), (0, -1, 0), 4, 4, ortho_pixel=1), 4, 4,
               [synth.TF(0.0, 1.0, lut)])
    occ = oracle.bucket_occupancy(v, fr)[0]
    assert set(np.nonzero(occ)[0]) == {5, 100, 101, 255}
    # 16-bit buckets of 256 raw values, window [1000, 2000]: only buckets whose
    # top value exceeds 1000 reach a knot with alpha > 0
    lv = [[np.zeros((4, 4, 4), np.uint16)]]
    v = oracle.Volume(lv, (1, 1, 1), 4, (4, 4, 4))
    fr.tfs = [synth.tf_ramp(1000, 2000)]
    occ = oracle.bucket_occupancy(v, fr)[0]
    assert set(np.nonzero(occ)[0]) == set(range(3, 256))


# ------------------------------------------------- closed forms (O-b, O-c)

def slab_scene(value, dtype, k=1, B=32):
    a = np.full((32, 32, 32), value, dtype)
    lv = [synth.mean_levels(a, k)]
    mn, mx = exact_meta(lv, (16, 16, 16))
    return oracle.Volume(lv, (1, 1, 1), B, (16, 16, 16), all_bricks(lv, B, [0]), mn, mx), lv


def const_tf(alpha, rgb=(0.2, 0.6, 1.0)):
    lut = np.zeros((256, 4), np.float32)
    lut[:, :3] = rgb
    lut[:, 3] = alpha
    return synth.TF(0.0, 1.0, lut)


def axis_camera(W=8, H=8, center=16.0):
    # rays along +z through exactly representable positions
    return synth.look_at((center, center, -10.0), (center, center, 0.0), (0, -1, 0), W, H, ortho_pixel=1.0)


@pytest.mark.parametrize("dtype,value", [(np.uint8, 77), (np.uint16, 77 * 257)])
@pytest.mark.parametrize("s", [0, 1, 2])
def test_constant_slab_opacity_closed_form(dtype, value, s):
    """n lattice samples of constant opacity alpha at step 2^s: opacity
    1 - (1 - alpha)^(n), colour rgb * (1 - (1 - alpha)^n) with n counted in
    base lattice steps (opacity correction of the adaptive step, Sec. 6.1)."""
    alpha = float(np.float32(0.03))         # the LUT holds binary32 knots
    vol, _ = slab_scene(value, dtype, k=3)
    fr = frame(axis_camera(), 8, 8, [const_tf(alpha)], lmin=[s], lmax=[s], ert=0.0)
    o = oracle.render(vol, vol.node_words(), fr)
    n = 64                                  # t in [10, 42): i = 0..63 base steps
    assert np.all(o["n_eval"] == n // (1 << s))
    want_a = 1.0 - (1.0 - alpha) ** n
    assert np.allclose(o["rgba64"][:, 3], want_a, rtol=0, atol=1e-12)
    rgb = np.array([0.2, 0.6, 1.0], np.float32).astype(np.float64)
    assert np.allclose(o["rgba64"][:, :3], rgb * want_a, rtol=0, atol=1e-12)
    assert np.allclose(o["rgba32"], o["rgba64"], atol=1e-5)
    if dtype == np.uint8:                  # homogeneous nodes: no brick is read (Sec. 5.2)
        assert np.all(o["n_bs"] == 0) and o["used_ids"].size == 0
    else:                                  # 16-bit data never takes the homogeneous path
        assert np.all(o["n_bs"] == n // (1 << s))


def test_two_identical_channels_closed_form():
    alpha = float(np.float32(0.02))
    a = np.full((32, 32, 32), 77, np.uint16)
    lv = [[a], [a.copy()]]
    mn, mx = exact_meta(lv, (16, 16, 16))
    vol = oracle.Volume(lv, (1, 1, 1), 32, (16, 16, 16), all_bricks(lv, 32, [0, 1]), mn, mx)
    fr = frame(axis_camera(), 8, 8, [const_tf(alpha), const_tf(alpha)], ert=0.0)
    o = oracle.render(vol, vol.node_words(), fr)
    q = (1 - alpha) ** 2
    n = 64
    assert np.allclose(o["rgba64"][:, 3], 1 - q ** n, atol=1e-12)
    # colour per sample 2*alpha*rgb, weighted by T before the sample
    want = 2 * alpha * np.array([0.2, 0.6, 1.0], np.float32).astype(np.float64) * (1 - q ** n) / (1 - q)
    assert np.allclose(o["rgba64"][:, :3], np.minimum(want, 1.0), atol=1e-9)


def test_early_ray_termination_closed_form():
    """alpha = 1/2: T = 2^-n exactly; T < 2^-10 first after the 11th sample."""
    vol, _ = slab_scene(50, np.uint16)
    fr = frame(axis_camera(), 8, 8, [const_tf(0.5)], ert=2.0 ** -10)
    o = oracle.render(vol, vol.node_words(), fr)
    assert np.all(o["n_eval"] == 11) and np.all(o["i_end"] == 10)
    assert np.all(o["rgba32"][:, 3] == np.float32(1 - 2.0 ** -11))


# ---------------------------------------- textbook DVR (FP64, scipy trilinear)

def textbook_dvr(vol0, spacing, cam, W, H, dt, tf, n_samples):
    """Front-to-back emission-absorption DVR of a trilinear field, written
    independently: rays in binary64, scipy map_coordinates(order=1) for the
    trilinear field (voxel centres at integer + 0.5), np.interp for the TF."""
    nz, ny, nx = vol0.shape
    dims = np.array([nx, ny, nz], np.float64)
    s = np.array(spacing, np.float64)
    out = np.zeros((H * W, 4))
    field = vol0.astype(np.float64)
    knots = np.arange(256, dtype=np.float64)
    for py in range(H):
        for px in range(W):
            idx = py * W + px
            n = int(n_samples[idx])
            if n == 0:
                continue
            if cam.perspective:
                a = (2 * (px + 0.5) / W - 1) * cam.tan_x
                b = (1 - 2 * (py + 0.5) / H) * cam.tan_y
                d = np.array(cam.forward) + a * np.array(cam.right) + b * np.array(cam.up)
                d /= np.linalg.norm(d)
                o = np.array(cam.eye, np.float64)
            else:
                a = (px + 0.5 - W / 2) * cam.pixel
                b = (H / 2 - py - 0.5) * cam.pixel
                o = np.array(cam.eye) + a * np.array(cam.right) + b * np.array(cam.up)
                d = np.array(cam.forward, np.float64)
            ov, dv = o / s, d / s
            with np.errstate(divide="ignore"):
                ta, tb = (0 - ov) / dv, (dims - ov) / dv
            t0 = max(np.max(np.minimum(ta, tb)[dv != 0]), 0.0)
            t = t0 + dt * np.arange(n)
            x = np.clip(ov[None, :] + t[:, None] * dv[None, :], 0, dims - 1e-9)
            u = np.clip(x - 0.5, 0, dims - 1)
            val = ndimage.map_coordinates(field, [u[:, 2], u[:, 1], u[:, 0]], order=1, mode="nearest")
            xq = np.clip((val - tf.lo) * tf.scale, 0, 255)
            rgba = np.stack([np.interp(xq, knots, tf.lut[:, ch].astype(np.float64)) for ch in range(4)], 1)
            T, C = 1.0, np.zeros(3)
            for i in range(n):
                al = min(max(rgba[i, 3], 0.0), 1.0)
                C += T * al * rgba[i, :3]
                T *= 1 - al
            out[idx, :3] = np.minimum(C, 1.0)
            out[idx, 3] = 1 - T
    return out


@pytest.mark.parametrize("persp", [False, True])
def test_textbook_dvr_single_level(persp):
    vol0 = synth.blobs_u8((40, 36, 32), 11, n_blobs=6, amp=(80, 200))
    lv = [[vol0]]
    mn, mx = exact_meta(lv, (8, 8, 8))
    vol = oracle.Volume(lv, (1, 1, 1), 16, (8, 8, 8), all_bricks(lv, 16, [0]), mn, mx)
    W = H = 24
    if persp:
        cam = synth.look_at((-30.0, 70.0, 60.0), (20.0, 18.0, 16.0), (0, 0, 1), W, H, fovy_deg=35.0)
    else:
        cam = synth.look_at((-20.0, -25.0, -30.0), (20.0, 18.0, 16.0), (0, 0, 1), W, H, ortho_pixel=2.2)
    tf = synth.tf_ramp(8, 255, rgb=(0.9, 0.5, 0.2), alpha_max=0.3)
    fr = frame(cam, W, H, [tf], dt=0.5, skip=False, ert=0.0)
    o = oracle.render(vol, vol.node_words(), fr)
    assert o["n_eval"].sum() > 5000
    want = textbook_dvr(vol0, (1, 1, 1), cam, W, H, 0.5, tf, o["n_eval"])
    assert np.abs(o["rgba64"] - want).max() < 1e-4
    assert np.abs(o["rgba32"] - want).max() < 2e-3


def test_empty_space_skipping_invariant_all_resident():
    """All bricks resident, level 0: skipping (Algorithm 1, skipNode) leaves
    the float image bit-identical to the march without skipping."""
    vol0 = synth.blobs_u8((64, 64, 64), 4, n_blobs=12)
    lv = [synth.mean_levels(vol0, 2)]
    mn, mx = exact_meta(lv, (8, 8, 8))
    vol = oracle.Volume(lv, (1, 1, 1), 16, (8, 8, 8), all_bricks(lv, 16, [0]), mn, mx)
    cam = synth.look_at((-40.0, -30.0, 90.0), (32.0, 32.0, 32.0), (0, 0, 1), 48, 48, fovy_deg=40.0)
    tf = synth.tf_ramp(8, 255)
    w = vol.node_words()
    on = oracle.render(vol, w, frame(cam, 48, 48, [tf], skip=True))
    off = oracle.render(vol, w, frame(cam, 48, 48, [tf], skip=False))
    assert np.array_equal(on["rgba32"], off["rgba32"])
    assert np.array_equal(on["rgba64"], off["rgba64"])
    assert on["n_eval"].sum() < 0.8 * off["n_eval"].sum()
    assert np.array_equal(np.sort(on["used_ids"]), np.sort(off["used_ids"]))


# --------------------------------------- requests and brick selection

def exact_scene(B=16, k=3, seed=9):
    vol0 = synth.blobs_u8((64, 64, 64), seed, n_blobs=10, amp=(60, 200))
    lv = [synth.mean_levels(vol0, k)]
    mn, mx = exact_meta(lv, (8, 8, 8))
    return vol0, lv, mn, mx


def walk_positions(W, H, n):
    """Exact positions of the axis camera at center 32 over a 64^3 volume."""
    return [(px + 0.5, py + 0.5, 0.5 * i) for py in range(H) for px in range(W) for i in range(n)]


def test_requests_with_nothing_resident():
    """Nothing resident: no node is partially mapped, so every non-empty
    sample requests its desired brick (Algorithm 1); with skipping on, the ray
    skips the node after its first request."""
    vol0, lv, mn, mx = exact_scene()
    vol = oracle.Volume(lv, (1, 1, 1), 16, (8, 8, 8), [], mn, mx)
    cam = axis_camera(64, 64, 32.0)
    tf = synth.tf_ramp(8, 255)
    w = vol.node_words()
    off = oracle.render(vol, w, frame(cam, 64, 64, [tf], skip=False))
    # root is non-empty, so every lattice sample of every ray requests its brick
    want = {vol.brick_id(0, 0, int(x) // 16, int(y) // 16, int(z) // 16) for (x, y, z) in walk_positions(64, 64, 128)}
    assert set(off["req_ids"].tolist()) == want
    assert off["used_ids"].size == 0 and np.all(off["rgba32"] == 0)
    on = oracle.render(vol, w, frame(cam, 64, 64, [tf], skip=True))
    want_on = {vol.brick_id(0, 0, px // 16, py // 16, 0) for py in range(64) for px in range(64)}
    assert set(on["req_ids"].tolist()) == want_on
    assert np.all(on["n_eval"] == 0)


@pytest.mark.parametrize("skip", [False, True])
def test_substitution_by_coarser_level_exact(skip):
    """Desired level 0; level 2 fully resident, level 1 absent, half of level
    0 resident: a non-empty sample reads its level-0 brick if resident, else
    requests it and reads level 2 (the next coarser resident level), and the
    step grows to 2^2 (Sec. 6.1)."""
    vol0, lv, mn, mx = exact_scene()
    rng = np.random.default_rng(4)
    l0 = [b for b in all_bricks(lv, 16, [0]) if b[1] == 0 and rng.random() < 0.5]
    l2 = [b for b in all_bricks(lv, 16, [0]) if b[1] == 2]
    vol = oracle.Volume(lv, (1, 1, 1), 16, (8, 8, 8), l0 + l2, mn, mx)
    res0 = {(b[2], b[3], b[4]) for b in l0}
    lut = np.zeros((256, 4), np.float32)
    lut[:, :3] = 1.0
    lut[40:, 3] = np.linspace(0.001, 0.05, 216, dtype=np.float32)
    tf = synth.TF(0.0, 1.0, lut)
    cam = axis_camera(32, 32, 32.0)  # rays x, y in [16, 48)
    o = oracle.render(vol, vol.node_words(), frame(cam, 32, 32, [tf], skip=skip, ert=0.0))
    req, used, n_bs = set(), set(), []
    for py in range(32):
        for px in range(32):
            x, y = px + 16.5, py + 16.5
            i, cnt = 0, 0
            while i < 128:
                z = 0.5 * i
                leaf_max = mx[0, int(z) // 8, int(y) // 8, int(x) // 8]
                if leaf_max < 40:               # empty leaf for this TF
                    i += 1
                    continue
                b0 = (int(x) // 16, int(y) // 16, int(z) // 16)
                cnt += 1
                if b0 in res0:
                    used.add(vol.brick_id(0, 0, *b0))
                    i += 1
                else:
                    req.add(vol.brick_id(0, 0, *b0))
                    used.add(vol.brick_id(0, 2, int(x) // 64, int(y) // 64, int(z) // 64))
                    i += 4
            n_bs.append(cnt)
    assert set(o["req_ids"].tolist()) == req
    assert set(o["used_ids"].tolist()) == used
    assert np.array_equal(o["n_bs"], np.array(n_bs, np.uint32))


def test_level_range_restricts_selection():
    vol0, lv, mn, mx = exact_scene()
    vol = oracle.Volume(lv, (1, 1, 1), 16, (8, 8, 8), all_bricks(lv, 16, [0]), mn, mx)
    cam = synth.look_at((-40.0, -30.0, 90.0), (32.0, 32.0, 32.0), (0, 0, 1), 32, 32, fovy_deg=40.0)
    o = oracle.render(vol, vol.node_words(), frame(cam, 32, 32, [synth.tf_ramp(8, 255)], lmin=[1], lmax=[1]))
    levels = (o["used_ids"] >> 24) & 0xFF
    assert o["used_ids"].size > 0 and np.all(levels == 1)
    assert o["req_ids"].size == 0


def test_channel_order_changes_image_only_by_rounding():
    vol0, lv, mn, mx = exact_scene()
    vol1 = synth.blobs_u8((64, 64, 64), 77, n_blobs=10, amp=(60, 200))
    lv2 = synth.mean_levels(vol1, 3)
    mn2, mx2 = exact_meta([lv2], (8, 8, 8))
    cam = synth.look_at((-40.0, -30.0, 90.0), (32.0, 32.0, 32.0), (0, 0, 1), 32, 32, fovy_deg=40.0)
    tfa = synth.tf_ramp(8, 255, rgb=(1, 0, 0), alpha_max=0.2)
    tfb = synth.tf_ramp(20, 200, rgb=(0, 1, 0.5), alpha_max=0.3)
    outs = []
    for order in ([lv[0], lv2], [lv2, lv[0]]):
        m0 = np.concatenate([mn, mn2]) if order[0] is lv[0] else np.concatenate([mn2, mn])
        m1 = np.concatenate([mx, mx2]) if order[0] is lv[0] else np.concatenate([mx2, mx])
        v = oracle.Volume(order, (1, 1, 1), 16, (8, 8, 8), all_bricks(order, 16, [0, 1]), m0, m1)
        tfs = [tfa, tfb] if order[0] is lv[0] else [tfb, tfa]
        outs.append(oracle.render(v, v.node_words(), frame(cam, 32, 32, tfs, ert=0.0)))
    assert np.abs(outs[0]["rgba64"] - outs[1]["rgba64"]).max() < 1e-12
    assert np.abs(outs[0]["rgba32"] - outs[1]["rgba32"]).max() < 1e-5
