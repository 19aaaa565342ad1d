"""Pins of the oracle's coarser-level sampling and of its level choice
(CPU only), each against a closed form worked out independently of the
oracle's code.

Sample value at level l (Sec. 6.2, mixing resolutions; the trilinear reading
with voxel centres at integer + 0.5): a linear field stays linear under the
2x2x2 mean of Sec. 3's hierarchy, and trilinear interpolation reproduces a
linear field exactly, so the value a ray reads at level l has a closed form
in the sample position, whatever l is.  A missing -0.5 in the level-l
coordinate shifts it by half a level-l voxel, a missing lower clamp
extrapolates below the first voxel centre: both fail here.

Level choice (Sec. 6.2): the desired level is the number of thresholds
tau_l (l >= 1) that the sample distance t has reached, then clamped to the
channel's level range; the step grows to 2^s with s the finest level read
(Sec. 6.1).  On an axis-aligned ray with exactly representable t the level
of every sample follows by hand, including the sample that lands exactly on
a threshold.
"""
import numpy as np
import pytest

import oracle
import synth

INF = float("inf")

# level-0 field v(x, y, z) = A + bx x + by y + bz z on voxel indices; the
# slopes sum to an even number, so every 2x2x2 mean stays an integer
DIMS = (96, 80, 64)
A0, SLOPE = 1000, (212, 156, 98)
ALPHA = 0.5


def linear_levels(k):
    z, y, x = np.meshgrid(*[np.arange(n) for n in DIMS[::-1]], indexing="ij")
    v0 = (A0 + SLOPE[0] * x + SLOPE[1] * y + SLOPE[2] * z).astype(np.uint16)
    return synth.mean_levels(v0, k)


def closed_level(l, shape_zyx):
    """Level-l voxel j of the field: the level-0 field at the level-l voxel
    centre (j + 0.5) 2^l - 0.5 in level-0 index units."""
    z, y, x = np.meshgrid(*[np.arange(n) for n in shape_zyx], indexing="ij")
    f = float(2 ** l)
    return A0 + sum(s * (f * j + (f - 1) / 2) for s, j in zip(SLOPE, (x, y, z)))


def closed_value(x64, l):
    """Value read at level l for a level-0 position x (binary64): per axis
    u = clamp(x / 2^l - 0.5, 0, dims_l - 1), then the linear field at u."""
    f = float(2 ** l)
    out = np.full(x64.shape[0], float(A0))
    for a in range(3):
        dl = DIMS[a]
        for _ in range(l):
            dl = (dl + 1) // 2
        u = np.clip(x64[:, a] / f - 0.5, 0.0, dl - 1.0)
        out += SLOPE[a] * (f * u + (f - 1.0) / 2.0)
    return out


def value_tf():
    """Constant opacity 1/2; red = LUT coordinate / 256 (exact knots), so the
    red channel of one sample is a' * xq / 256 with xq = v * scale."""
    lut = np.zeros((256, 4), np.float32)
    lut[:, 0] = np.arange(256) / 256.0
    lut[:, 3] = ALPHA
    return synth.TF(0.0, float(np.float32(255.0 / 65535.0)), lut)


def oblique_camera(W=160, H=160, pixel=0.83):
    """Orthographic pixel origins on a plane through the volume centre, tilted
    so that it crosses all six faces: origins near every border."""
    c = np.array(DIMS, np.float64) / 2.0
    d = np.array([1.0, 2.0, 3.0]) / np.sqrt(14.0)
    return synth.look_at(tuple(c), tuple(c + d), (0.0, 0.0, 1.0), W, H, ortho_pixel=pixel)


def first_sample_positions(cam, W, H):
    """Binary64 pixel origins (the oracle's binary64 ray), and which of them
    lie inside the volume with a margin (their first sample is the origin)."""
    e, r, u = (np.array(v, np.float64) for v in (cam.eye, cam.right, cam.up))
    jj, ii = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    a = ((ii.ravel() + 0.5) - 0.5 * W) * cam.pixel
    b = (0.5 * H - (jj.ravel() + 0.5)) * cam.pixel
    o = e[None, :] + a[:, None] * r[None, :] + b[:, None] * u[None, :]
    inside = np.all((o > 1e-3) & (o < np.array(DIMS, np.float64) - 1e-3), axis=1)
    return o, inside


@pytest.mark.parametrize("desired,resident_levels", [(0, (0, 1, 2)), (1, (0, 1, 2)), (2, (0, 1, 2)),
                                                     (0, (1, 2)), (0, (2,)), (1, (2,))])
def test_level_sample_value_closed_form(desired, resident_levels):
    """One sample per ray (early termination right after it): the red channel
    gives back the value read, which must equal the linear field at the
    clamped level-l coordinate.  With the desired level's bricks absent the
    ray reads the next coarser resident level (Sec. 6.1 getAlternativeBrick),
    and the same closed form holds at that level."""
    k = 3
    lv = linear_levels(k)
    for l in range(k):
        assert np.array_equal(lv[l].astype(np.float64), closed_level(l, lv[l].shape)), f"level {l} not linear"
    mn, mx = synth.leaf_ranges(lv[0], (16, 16, 16))
    bricks = []
    for l in resident_levels:
        nz, ny, nx = lv[l].shape
        bricks += [(0, l, x, y, z) for z in range(-(-nz // 32)) for y in range(-(-ny // 32)) for x in range(-(-nx // 32))]
    vol = oracle.Volume([lv], (1, 1, 1), 32, (16, 16, 16), bricks, mn[None].astype(np.int64), mx[None].astype(np.int64))
    read = min(l for l in resident_levels if l >= desired)
    W = H = 160
    cam = oblique_camera(W, H)
    tf = value_tf()
    fr = synth.Frame(W, H, cam, [tf], 0.5, [0.0] + [INF] * 15, [desired], [desired], ert=2.0)
    o = oracle.render(vol, vol.node_words(), fr)
    x64, inside = first_sample_positions(cam, W, H)
    assert inside.sum() > 2000
    sel = np.nonzero(inside)[0]
    assert np.all(o["n_eval"][sel] == 1) and np.all(o["i_end"][sel] == 0)
    # every brick read is of the expected level; absent desired bricks are requested
    assert o["used_ids"].size > 0 and np.all(((o["used_ids"] >> 24) & 0xFF) == read)
    assert (o["req_ids"].size > 0) == (read != desired)
    ap = 1.0 - 0.5 ** (2 ** read)
    got = o["rgba64"][sel, 0] * 256.0 / (ap * tf.scale)
    want = closed_value(x64[sel], read)
    assert np.abs(got - want).max() < 1e-6
    # the border clamp is exercised: some origins lie below the first and
    # above the last level-l voxel centre
    f = 2.0 ** read
    assert np.any(x64[sel] < 0.5 * f) and np.any(x64[sel] > np.array(DIMS) - 0.5 * f)
    # binary32 image within binary32 rounding of the binary64 one
    assert np.abs(o["rgba32"][sel].astype(np.float64) - o["rgba64"][sel]).max() < 1e-5
    assert np.allclose(o["rgba64"][sel, 3], ap, atol=1e-15)


def test_closed_form_separates_coordinate_mistakes():
    """The closed form is sensitive to the two mistakes it is meant to catch:
    without the -0.5 a level-l value moves by sum(slopes) * 2^(l-1) (at least
    233 raw units here), without the lower clamp a position below the first
    voxel centre extrapolates; the tolerance above is 1e-6."""
    x = np.array([[40.3, 33.7, 20.2]])
    vals = [closed_value(x, l)[0] for l in range(3)]
    assert abs(vals[0] - vals[1]) < 1e-9 and abs(vals[0] - vals[2]) < 1e-9
    for l in (1, 2):
        f = 2.0 ** l
        no_half = A0 + sum(s * (f * (x[0, a] / f) + (f - 1.0) / 2.0) for a, s in enumerate(SLOPE))
        assert abs(no_half - vals[l]) >= 233.0 * 2 ** (l - 1) - 1e-9
    edge = np.array([[0.7, 33.7, 20.2]])
    clamped = closed_value(edge, 2)[0]
    extrapolated = A0 + sum(s * (edge[0, a] - 0.5) for a, s in enumerate(SLOPE))
    assert abs(clamped - extrapolated) > 100.0


# ------------------------------------------------------------ lod(t)

def fnv_words(h, words):
    for w in words:
        for b in range(4):
            h ^= (int(w) >> (8 * b)) & 0xFF
            h = (h * 16777619) & 0xFFFFFFFF
    return h


def lod_scene(m):
    rng = np.random.default_rng(5)
    v0 = rng.integers(1000, 60000, (8, 8, 64)).astype(np.uint16)
    lv = [synth.mean_levels(v0, 3) for _ in range(m)]
    mn, mx = synth.leaf_ranges(lv[0][0], (8, 8, 8))
    bricks = [(c, l, x, 0, 0) for c in range(m) for l in range(3) for x in range(2 if l == 0 else 1)]
    vol = oracle.Volume(lv, (1, 1, 1), 32, (8, 8, 8), bricks, np.stack([mn] * m).astype(np.int64),
                        np.stack([mx] * m).astype(np.int64))
    return vol


@pytest.mark.parametrize("ranges", [[(0, 2)], [(0, 2), (1, 1)]])
def test_lod_thresholds_exact(ranges):
    """A ray along +x from x = 0 at dt = 1/2: t_i = i / 2 exactly.  With
    thresholds tau_1 = 8, tau_2 = 16 the desired level is 0 below t = 8, 1
    from t = 8 on (the sample at t = 8 itself is at level 1), 2 from t = 16;
    each channel clamps it to its range, the step is 2^(finest level read).
    The per-sample selection hash, the evaluated count, the end index and the
    used bricks all follow from this sequence."""
    m = len(ranges)
    vol = lod_scene(m)
    cam = synth.look_at((0.0, 4.25, 3.75), (1.0, 4.25, 3.75), (0.0, 0.0, 1.0), 1, 1, ortho_pixel=1.0)
    lut = np.zeros((256, 4), np.float32)
    lut[:, :3] = 1.0
    lut[:, 3] = np.float32(0.001)
    tf = synth.TF(0.0, float(np.float32(255.0 / 65535.0)), lut)
    lod_t = [0.0, 8.0, 16.0] + [INF] * 13
    fr = synth.Frame(1, 1, cam, [tf] * m, 0.5, lod_t, [r[0] for r in ranges], [r[1] for r in ranges], ert=0.0)
    o = oracle.render(vol, vol.node_words(), fr)

    h, i, n, used = 2166136261, 0, 0, set()
    while 0.5 * i < 64.0:
        t = 0.5 * i
        lod = (t >= 8.0) + (t >= 16.0)
        levels = [min(max(lod, lo), hi) for lo, hi in ranges]
        for c, l in enumerate(levels):
            bx = int(t) // (32 << l)
            bid = ((c * 3 + l) << 24) | bx
            h = fnv_words(h, [i, c, l, bid])
            used.add(bid)
        n += 1
        i += 1 << min(levels)
    assert int(o["hash"][0]) == h
    assert int(o["n_eval"][0]) == n and int(o["i_end"][0]) == i
    assert set(o["used_ids"].tolist()) == used
    # the sample exactly at t = 8 (i = 16) was read at level 1, not 0
    assert 16 in range(0, i) and (((0 * 3 + 1) << 24) | 0) in used
    if m == 1:
        assert n == 16 + 8 + 24 and i == 128
    else:
        assert n == 16 + 8 + 48 and i == 128


# ------------------------------------------- anisotropic downsampling

def level_shifts(keep_axes, l):
    """log2 of the level-l voxel extent per axis: halvings so far."""
    return [sum(0 if (keep_axes[i] >> a) & 1 else 1 for i in range(l)) for a in range(3)]


def closed_value_aniso(x64, l, keep_axes):
    e = level_shifts(keep_axes, l)
    out = np.full(x64.shape[0], float(A0))
    for a in range(3):
        f = float(2 ** e[a])
        dl = DIMS[a]
        for i in range(l):
            if not (keep_axes[i] >> a) & 1:
                dl = (dl + 1) // 2
        u = np.clip(x64[:, a] / f - 0.5, 0.0, dl - 1.0)
        out += SLOPE[a] * (f * u + (f - 1.0) / 2.0)
    return out


@pytest.mark.parametrize("keep_axes", [[4, 0], [4, 4], [1, 6], [3, 0]])
@pytest.mark.parametrize("read", [1, 2])
def test_anisotropic_level_value_closed_form(keep_axes, read):
    """Levels that halve only some axes (Sec. 8: downsampling in two
    dimensions; Sec. 9: anisotropic subdivision): the 2x2x1 (or 2x1x1) means
    of a linear field stay linear, the level-l value is the field at the
    per-axis clamped coordinate x / 2^e_a - 0.5, and the opacity correction
    uses the level's step exponent, min over axes of e_a at unit spacing."""
    k = 3
    lv = synth.mean_levels(linear_levels(1)[0], k, keep_axes)
    for l in range(k):
        e = level_shifts(keep_axes, l)
        z, y, x = np.meshgrid(*[np.arange(n) for n in lv[l].shape], indexing="ij")
        want = A0 + sum(s * (2.0 ** ea * j + (2.0 ** ea - 1) / 2) for s, j, ea in zip(SLOPE, (x, y, z), e))
        assert np.array_equal(lv[l].astype(np.float64), want), f"level {l} not linear"
    mn, mx = synth.leaf_ranges(lv[0], (16, 16, 16))
    bricks = []
    for l in range(k):
        nz, ny, nx = lv[l].shape
        bricks += [(0, l, x, y, z) for z in range(-(-nz // 32)) for y in range(-(-ny // 32)) for x in range(-(-nx // 32))]
    vol = oracle.Volume([lv], (1, 1, 1), 32, (16, 16, 16), bricks, mn[None].astype(np.int64), mx[None].astype(np.int64),
                        keep_axes=keep_axes)
    W = H = 160
    cam = oblique_camera(W, H)
    tf = value_tf()
    fr = synth.Frame(W, H, cam, [tf], 0.5, [0.0] + [INF] * 15, [read], [read], ert=2.0)
    o = oracle.render(vol, vol.node_words(), fr)
    x64, inside = first_sample_positions(cam, W, H)
    sel = np.nonzero(inside)[0]
    assert np.all(o["n_eval"][sel] == 1) and np.all(((o["used_ids"] >> 24) & 0xFF) == read)
    step = min(level_shifts(keep_axes, read))
    ap = 1.0 - 0.5 ** (2 ** step)
    got = o["rgba64"][sel, 0] * 256.0 / (ap * tf.scale)
    assert np.abs(got - closed_value_aniso(x64[sel], read, keep_axes)).max() < 1e-6
    assert np.allclose(o["rgba64"][sel, 3], ap, atol=1e-15)
    # the binary32 sampling path follows the same per-axis coordinates
    assert np.abs(o["rgba32"][sel].astype(np.float64) - o["rgba64"][sel]).max() < 1e-5
    # the owner bricks of the samples are per-axis floor(x / (B 2^e_a))
    e = level_shifts(keep_axes, read)
    want_ids = {vol.brick_id(0, read, *[int(x64[i, a]) >> (5 + e[a]) for a in range(3)]) for i in sel}
    assert want_ids <= set(o["used_ids"].tolist())


@pytest.mark.parametrize("keep_axes,spacing", [([4, 0], (1.0, 1.0, 1.0)), ([4, 4], (1.0, 1.0, 4.0)),
                                               ([0, 0], (1.0, 1.0, 4.0))])
def test_anisotropic_step_sequence(keep_axes, spacing):
    """On the exact +x ray of the lod test, the step after a sample read at
    level l is 2^s with s the largest exponent such that 2^s times the
    smallest spacing is at most the smallest physical extent of a level-l
    voxel (Sec. 6.1's adaptive step), and the owner brick along x follows the
    level's x extent."""
    rng = np.random.default_rng(5)
    v0 = rng.integers(1000, 60000, (8, 8, 64)).astype(np.uint16)
    lv = synth.mean_levels(v0, 3, keep_axes)
    mn, mx = synth.leaf_ranges(v0, (8, 8, 8))
    bricks = []
    for l in range(3):
        nz, ny, nx = lv[l].shape
        bricks += [(0, l, x, y, z) for z in range(-(-nz // 32)) for y in range(-(-ny // 32)) for x in range(-(-nx // 32))]
    vol = oracle.Volume([lv], spacing, 32, (8, 8, 8), bricks, mn[None].astype(np.int64), mx[None].astype(np.int64),
                        keep_axes=keep_axes)
    sp = np.array(spacing)
    cam = synth.look_at((0.0, 4.25 * sp[1], 3.75 * sp[2]), (1.0, 4.25 * sp[1], 3.75 * sp[2]), (0.0, 0.0, 1.0), 1, 1,
                        ortho_pixel=1.0)
    lut = np.zeros((256, 4), np.float32)
    lut[:, :3] = 1.0
    lut[:, 3] = np.float32(0.001)
    tf = synth.TF(0.0, float(np.float32(255.0 / 65535.0)), lut)
    fr = synth.Frame(1, 1, cam, [tf], 0.5, [0.0, 8.0, 16.0] + [INF] * 13, [0], [2], ert=0.0)
    o = oracle.render(vol, vol.node_words(), fr)
    h, i, n = 2166136261, 0, 0
    while 0.5 * i < 64.0:
        t = 0.5 * i
        l = int(t >= 8.0) + int(t >= 16.0)
        e = level_shifts(keep_axes, l)
        ext = min(sp[a] * 2 ** e[a] for a in range(3))
        s = 0
        while 2 ** (s + 1) * sp.min() <= ext:
            s += 1
        bid = (l << 24) | (int(t) >> (5 + e[0]))
        h = fnv_words(h, [i, 0, l, bid])
        n += 1
        i += 1 << s
    assert int(o["hash"][0]) == h and int(o["n_eval"][0]) == n and int(o["i_end"][0]) == i
