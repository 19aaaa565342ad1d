"""Pins of the oracle's low-precision sampling (binary16 / bfloat16 brick
cache, lerps in the format, binary32 compositing): the rounding against
numpy's binary16 conversion and the bit-level definition of bfloat16
rounding, the lerp against exact rational arithmetic, and renders against
closed forms and error bounds."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from test_oracle_pins import all_bricks, exact_meta, frame, const_tf

FMT = {1: (11, -14), 2: (8, -126)}   # significant bits, smallest normal exponent


def rne(x: Fraction, fmt: int) -> Fraction:
    """Round-to-nearest-even of an exact rational to the format."""
    p, emin = FMT[fmt]
    if x == 0:
        return x
    sign, ax = (-1 if x < 0 else 1), abs(x)
    e = ax.numerator.bit_length() - ax.denominator.bit_length()
    if Fraction(2) ** e > ax:
        e -= 1
    q = Fraction(2) ** (max(e, emin) - (p - 1))
    r = ax / q
    n = math.floor(r)
    rest = r - n
    if rest > Fraction(1, 2) or (rest == Fraction(1, 2) and n % 2 == 1):
        n += 1
    return sign * n * q


def test_binary16_conversion_of_every_u16_and_u8_value():
    for S, top in ((16, 65536), (8, 256)):
        v = np.arange(top, dtype=np.float64) / 2.0 ** S
        want = v.astype(np.float16).astype(np.float64)
        got = np.array([oracle.round_fmt(x, 1) for x in v])
        assert np.array_equal(got, want)


def test_bfloat16_rounding_matches_the_bit_definition():
    rng = np.random.default_rng(3)
    x = rng.uniform(-1.0, 1.0, 20000).astype(np.float32)
    bits = x.view(np.uint32)
    ties = ((bits & 0xFFFF0000) | 0x8000).view(np.float32)        # exactly halfway
    x = np.concatenate([x, ties, np.float32([2.0 ** -130, 3.0 * 2.0 ** -133])])
    b = x.view(np.uint32).astype(np.uint64)
    want = (((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)).view(np.float32)
    got = np.array([oracle.round_fmt(float(v), 2) for v in x], np.float64)
    assert np.array_equal(got, want.astype(np.float64))


def fmt_values(rng, n, fmt, lo=0.0, hi=1.0):
    return [float(rne(Fraction(float(v)), fmt)) for v in rng.uniform(lo, hi, n)]


@pytest.mark.parametrize("fmt", [1, 2])
def test_lerp_is_the_exact_result_rounded_once_per_step(fmt):
    rng = np.random.default_rng(fmt)
    f = fmt_values(rng, 3000, fmt)
    a = fmt_values(rng, 3000, fmt)
    b = fmt_values(rng, 3000, fmt)
    a[:50] = [x * 2.0 ** -20 for x in a[:50]]                   # small and subnormal values
    for fi, ai, bi in zip(f, a, b):
        d = rne(Fraction(bi) - Fraction(ai), fmt)
        want = rne(Fraction(fi) * d + Fraction(ai), fmt)
        assert oracle.lerp_fmt(fi, ai, bi, fmt) == float(want)


def test_bfloat16_lerp_tie_decided_by_a_tiny_term():
    """f * d exactly halfway between two bfloat16 values, a far below a
    double's resolution of it: the exact sum lies off the tie, on a's side."""
    found = 0
    for fi in range(128, 256):
        for di in range(128, 256):
            f, d = Fraction(fi, 256), Fraction(di, 256)
            p = f * d
            if rne(p, 2) == p or rne(p + Fraction(1, 2 ** 200), 2) == rne(p - Fraction(1, 2 ** 200), 2):
                continue                                         # not a tie
            for a in (2.0 ** -90, -(2.0 ** -90)):
                want = rne(p + Fraction(a), 2)
                got = oracle.lerp_fmt(float(f), a, a + float(d), 2)
                assert got == float(want)
            found += 1
            if found > 20:
                return
    assert found > 0


def slab(value, fmt):
    a = np.full((32, 32, 32), value, np.uint16)
    lv = [[a]]
    mn, mx = exact_meta(lv, (16, 16, 16))
    return oracle.Volume(lv, (1, 1, 1), 32, (16, 16, 16), all_bricks(lv, 32, [0]), mn, mx, sample_format=fmt)


def axis_cam(cx, cy):
    return synth.look_at((cx, cy, -10.0), (cx, cy, 0.0), (0, -1, 0), 8, 8, ortho_pixel=1.0)


@pytest.mark.parametrize("fmt,sampled", [(0, 4100), (1, 4100), (2, 4096)])
def test_constant_slab_samples_the_rounded_value(fmt, sampled):
    """4100 * 2^-16 is a binary16 value (quantum 4 at 2^12) but rounds to
    4096 in bfloat16 (quantum 32): the opacity is that of the sampled value."""
    lut = np.zeros((256, 4), np.float32)
    lut[:, :3] = (0.2, 0.6, 1.0)
    lut[:, 3] = 0.01 * (1 + np.arange(256))
    tf = synth.TF(4096.0, 1.0, lut)
    vol = slab(4100, fmt)
    o = oracle.render(vol, vol.node_words(), frame(axis_cam(16.0, 16.0), 8, 8, [tf], ert=0.0))
    alpha = float(np.float32(0.01 * (1 + sampled - 4096)))
    assert np.all(o["n_eval"] == 64)
    assert np.allclose(o["rgba32"][:, 3], 1.0 - (1.0 - alpha) ** 64, rtol=0, atol=2e-6)


@pytest.mark.parametrize("fmt,bound", [(1, 8.0), (2, 64.0)])
def test_ramp_field_within_the_format_error_bound(fmt, bound):
    """Field 1000 + 90x + 10y + 40z sampled off the voxel centres (weights
    0.3 and 0.7 in x and y): every sample is within `bound` raw units of the
    binary32 path (corner and lerp roundings of a quantum of 4 (binary16) or
    32 (bfloat16) at 2^12..2^13), so with opacity slope 2.5e-6 per unit the
    opacities of 64 samples differ by at most 64 * bound * 2.5e-6 * 1.01.
    Transposing the x and y weights alone moves each sample by 32 units."""
    z, y, x = np.meshgrid(np.arange(32), np.arange(32), np.arange(32), indexing="ij")
    a = (1000 + 90 * x + 10 * y + 40 * z).astype(np.uint16)
    lv = [[a]]
    mn, mx = exact_meta(lv, (16, 16, 16))
    lut = np.zeros((256, 4), np.float32)
    lut[:, :3] = 1.0
    lut[:, 3] = 0.02 * np.arange(256) / 255.0
    tf = synth.TF(0.0, 255.0 / 8000.0, lut)                     # alpha = 2.5e-6 per raw unit
    fr = frame(axis_cam(16.3, 16.7), 8, 8, [tf], ert=0.0)
    ref = oracle.Volume(lv, (1, 1, 1), 32, (16, 16, 16), all_bricks(lv, 32, [0]), mn, mx)
    low = oracle.Volume(lv, (1, 1, 1), 32, (16, 16, 16), all_bricks(lv, 32, [0]), mn, mx, sample_format=fmt)
    o0 = oracle.render(ref, ref.node_words(), fr)
    o1 = oracle.render(low, low.node_words(), fr)
    assert np.array_equal(o0["n_eval"], o1["n_eval"])
    diff = np.abs(o1["rgba32"][:, 3].astype(np.float64) - o0["rgba32"][:, 3])
    assert diff.max() <= 64 * bound * 2.5e-6 * 1.01
    assert diff.max() > 0                                       # the format is applied
