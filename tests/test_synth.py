"""Seeded input generators: determinism, closed forms and the recipe's
statistics (CPU only)."""
import numpy as np
import pytest

import synth


def test_noise_is_deterministic_and_bounded():
    vals = [synth.noise(7, c, l, x, 3, 5, 200) for c in range(2) for l in range(2) for x in range(50)]
    assert all(0 <= v <= 200 for v in vals)
    assert vals == [synth.noise(7, c, l, x, 3, 5, 200) for c in range(2) for l in range(2) for x in range(50)]
    assert len(set(vals)) > 50


def test_downsample_rounded_mean_closed_form():
    a = np.arange(3 * 3 * 3, dtype=np.uint8).reshape(3, 3, 3)
    d = synth.downsample(a)
    assert d.shape == (2, 2, 2)
    # full 2x2x2 block at the origin: mean of {0,1,3,4,9,10,12,13} = 6.5 -> 7 (half up)
    assert d[0, 0, 0] == 7
    # corner (1,1,1) covers only voxel (2,2,2) = 26
    assert d[1, 1, 1] == 26
    # edge (0,0,1): voxels x=2, y in {0,1}, z in {0,1}: {2,5,11,14} mean 8
    assert d[0, 0, 1] == 8
    b = np.full((5, 4, 7), 60000, np.uint16)
    assert np.all(synth.downsample(b) == 60000)


def test_bricks_with_clamped_border():
    lv = np.arange(5 * 6 * 7, dtype=np.uint16).reshape(5, 6, 7)
    br = synth.bricks_from_dense(lv, 4, [(0, 0, 0), (1, 1, 1)])
    assert br.shape == (2, 6, 6, 6)
    # brick (0,0,0): slot index s holds voxel clamp(s-1)
    for z in range(6):
        for y in range(6):
            for x in range(6):
                zz, yy, xx = min(max(z - 1, 0), 4), min(max(y - 1, 0), 5), min(max(x - 1, 0), 6)
                assert br[0, z, y, x] == lv[zz, yy, xx]
                zz, yy, xx = min(max(4 + z - 1, 0), 4), min(max(4 + y - 1, 0), 5), min(max(4 + x - 1, 0), 6)
                assert br[1, z, y, x] == lv[zz, yy, xx]


def test_leaf_ranges_cover_trilinear_support_brute_force():
    rng = np.random.default_rng(3)
    vol = rng.integers(0, 255, size=(9, 10, 11), dtype=np.uint8)
    mn, mx = synth.leaf_ranges(vol, (4, 4, 2))
    nz, ny, nx = vol.shape
    for jz in range(mn.shape[0]):
        for jy in range(mn.shape[1]):
            for jx in range(mn.shape[2]):
                z0, z1 = max(jz * 2 - 1, 0), min((jz + 1) * 2, nz - 1)
                y0, y1 = max(jy * 4 - 1, 0), min((jy + 1) * 4, ny - 1)
                x0, x1 = max(jx * 4 - 1, 0), min((jx + 1) * 4, nx - 1)
                blk = vol[z0:z1 + 1, y0:y1 + 1, x0:x1 + 1]
                assert mn[jz, jy, jx] == blk.min() and mx[jz, jy, jx] == blk.max()


def test_blob_volume_matches_recipe():
    v = synth.blobs_u8((128, 128, 128), 1)
    frac = float((v < 8).mean())
    assert 0.60 <= frac <= 0.80, frac
    assert v.max() > 100
    assert np.array_equal(v, synth.blobs_u8((128, 128, 128), 1))


def test_cells_field_bricks_and_bounds():
    # the cell density of the 4 x 1024x1024x64 slab: 40 cells in 96 x 80 x 64 physical units
    cells = synth.Cells(2, 40, 3, (96, 80, 16), (1.0, 1.0, 4.0))
    assert cells.count() == 40
    assert 15 <= sum(cells.count(ch) for ch in range(3)) <= 60     # p = 0.3
    dense = cells.dense(1)
    assert dense.shape == (16, 80, 96)
    assert dense.max() > 1000 and np.median(dense) <= 200
    # a level-0 brick equals the dense volume with the clamped border
    br = cells.bricks(1, 0, 16, [(1, 2, 0)])
    ref = synth.bricks_from_dense(dense, 16, [(1, 2, 0)])
    assert np.array_equal(br, ref)
    mixed = cells.bricks_mixed(16, [(1, 0, 1, 2, 0), (2, 1, 0, 0, 0)])
    assert np.array_equal(mixed[0], br[0])
    # conservative leaf bounds contain the exact dilated ranges
    mn, mx = cells.leaf_bounds(1, (8, 8, 2))
    emn, emx = synth.leaf_ranges(dense, (8, 8, 2))
    assert np.all(mn <= emn) and np.all(mx >= emx)
    assert (mx <= 200).mean() > 0.2


def test_lod_thresholds_closed_form():
    t = synth.lod_thresholds(1.0, 1080, 90.0, 3)
    # tan(45 deg) = 1: tau_l = 2^l * 1080 / 2
    assert t[1] == pytest.approx(1080.0, rel=1e-6) and t[2] == pytest.approx(2160.0, rel=1e-6)
    assert t[3] == float("inf")


def test_voxel_source_matches_dense_field_in_the_oracle():
    """The lazily filled voxel source gives the oracle the same voxels as the
    dense field (level 0), so both march to identical results."""
    import oracle
    cells = synth.Cells(4, 60, 2, (80, 72, 20), (1.0, 1.0, 4.0))
    dense = [[cells.dense(c)] for c in range(2)]
    mins, maxs = zip(*[synth.leaf_ranges(d[0], (8, 8, 4)) for d in dense])
    mn, mx = np.stack(mins).astype(np.int64), np.stack(maxs).astype(np.int64)
    res = [(c, 0, x, y, 0) for c in range(2) for x in range(5) for y in range(5)]
    src = cells.voxel_source(16, capacity=4096)
    vd = oracle.Volume(dense, (1, 1, 4), 16, (8, 8, 4), res, mn, mx)
    vp = oracle.Volume(None, (1, 1, 4), 16, (8, 8, 4), res, mn, mx,
                       provider=(2, 1, (80, 72, 20), 2, src.fn, src.ctx))
    cam = synth.look_at((-30.0, -40.0, 150.0), (40.0, 36.0, 40.0), (0, 0, 1), 40, 32, fovy_deg=40.0)
    tfs = [synth.tf_ramp(400, 12000, rgb=(1, 0, 0), alpha_max=0.5), synth.tf_ramp(400, 12000, rgb=(0, 1, 0))]
    fr = synth.Frame(40, 32, cam, tfs, 0.5, [0.0] + [float("inf")] * 15, [0, 0], [0, 0])
    a = oracle.render(vd, vd.node_words(), fr)
    b = oracle.render(vp, vp.node_words(), fr)
    assert a["n_bs"].sum() > 1000
    for key in ("rgba32", "rgba64", "hash", "n_eval"):
        assert np.array_equal(a[key], b[key]), key
    assert src.bricks_generated() > 0
