"""Coarser-level sampling and the level choice on the GPU, on the scenes
whose oracle results are pinned by closed forms (test_oracle_levels.py):
bit-exact against the oracle, and the GPU's own image against the closed
form of the value a level-l sample reads (Sec. 6.2)."""
import numpy as np
import pytest

import oracle
import synth
from synth import recipes
from test_oracle_levels import (DIMS, INF, closed_value, first_sample_positions, fnv_words, linear_levels,
                                lod_scene, oblique_camera, value_tf)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    import torch
    assert torch.cuda.is_available(), "these tests need a CUDA GPU"
    from paper_2309_04393_gb300 import build
    build.build()
    import test_gpu_parity as tp
    return tp


@pytest.mark.parametrize("desired,resident_levels", [(1, (0, 1, 2)), (2, (0, 1, 2)), (0, (1, 2)), (1, (2,))])
def test_level_sample_value_on_gpu(gpu, desired, resident_levels):
    lv = linear_levels(3)
    mn, mx = synth.leaf_ranges(lv[0], (16, 16, 16))
    scene = recipes.Scene("linear", DIMS, (1.0, 1.0, 1.0), 1, 3, 32, (16, 16, 16), 16, levels=[lv],
                          leaf_min=mn[None].astype(np.int64), leaf_max=mx[None].astype(np.int64))
    scene.resident = scene.all_bricks(levels=list(resident_levels))
    ctx = gpu.make_ctx(scene)
    slot_to_id = gpu.load(ctx, scene)
    vol = gpu.oracle_volume(scene)
    W = H = 160
    cam = oblique_camera(W, H)
    tf = value_tf()
    fr = synth.Frame(W, H, cam, [tf], 0.5, [0.0] + [INF] * 15, [desired], [desired], ert=2.0)
    o = oracle.render(vol, vol.node_words(), fr)
    g = gpu.gpu_frame(ctx, fr, slot_to_id)
    gpu.compare(g, o)
    read = min(l for l in resident_levels if l >= desired)
    x64, inside = first_sample_positions(cam, W, H)
    sel = np.nonzero(inside)[0]
    ap = 1.0 - 0.5 ** (2 ** read)
    got = g["rgba32"][sel, 0].astype(np.float64) * 256.0 / (ap * tf.scale)
    assert np.abs(got - closed_value(x64[sel], read)).max() < 0.05
    ctx.close()


@pytest.mark.parametrize("ranges", [[(0, 2)], [(0, 2), (1, 1)]])
def test_lod_thresholds_on_gpu(gpu, ranges):
    m = len(ranges)
    vol_o = lod_scene(m)
    lv = [vol_o.levels[c] for c in range(m)]
    scene = recipes.Scene("lod", (64, 8, 8), (1.0, 1.0, 1.0), m, 3, 32, (8, 8, 8), 16, levels=lv,
                          leaf_min=vol_o.leaf_min.reshape(m, 1, 1, 8), leaf_max=vol_o.leaf_max.reshape(m, 1, 1, 8))
    scene.resident = scene.all_bricks()
    ctx = gpu.make_ctx(scene)
    slot_to_id = gpu.load(ctx, scene)
    cam = synth.look_at((0.0, 4.25, 3.75), (1.0, 4.25, 3.75), (0.0, 0.0, 1.0), 1, 1, ortho_pixel=1.0)
    lut = np.zeros((256, 4), np.float32)
    lut[:, :3] = 1.0
    lut[:, 3] = np.float32(0.001)
    tf = synth.TF(0.0, float(np.float32(255.0 / 65535.0)), lut)
    fr = synth.Frame(1, 1, cam, [tf] * m, 0.5, [0.0, 8.0, 16.0] + [INF] * 13, [r[0] for r in ranges],
                     [r[1] for r in ranges], ert=0.0)
    o = oracle.render(vol_o, vol_o.node_words(), fr)
    g = gpu.gpu_frame(ctx, fr, slot_to_id)
    gpu.compare(g, o)
    # and the hand-computed sequence of levels
    h, i = 2166136261, 0
    while 0.5 * i < 64.0:
        lod = (0.5 * i >= 8.0) + (0.5 * i >= 16.0)
        levels = [min(max(lod, lo), hi) for lo, hi in ranges]
        for c, l in enumerate(levels):
            h = fnv_words(h, [i, c, l, ((c * 3 + l) << 24) | (int(0.5 * i) // (32 << l))])
        i += 1 << min(levels)
    assert int(g["hash"][0]) == h and int(g["i_end"][0]) == i
    ctx.close()


@pytest.mark.parametrize("keep_axes,read", [([4, 0], 1), ([4, 4], 2), ([1, 6], 2)])
def test_anisotropic_level_value_on_gpu(gpu, keep_axes, read):
    """Levels that halve only some axes (Sec. 8): bit-exact against the
    oracle, every octree word included, and the GPU image against the closed
    form of the per-axis level coordinate."""
    from test_oracle_levels import closed_value_aniso, level_shifts
    lv = synth.mean_levels(linear_levels(1)[0], 3, keep_axes)
    mn, mx = synth.leaf_ranges(lv[0], (16, 16, 16))
    scene = recipes.Scene("linear_aniso", DIMS, (1.0, 1.0, 1.0), 1, 3, 32, (16, 16, 16), 16, levels=[lv],
                          leaf_min=mn[None].astype(np.int64), leaf_max=mx[None].astype(np.int64), keep_axes=keep_axes)
    scene.resident = scene.all_bricks()
    ctx = gpu.make_ctx(scene)
    slot_to_id = gpu.load(ctx, scene)
    vol = gpu.oracle_volume(scene)
    gpu.check_octree(ctx, vol)
    W = H = 160
    cam = oblique_camera(W, H)
    tf = value_tf()
    fr = synth.Frame(W, H, cam, [tf], 0.5, [0.0] + [INF] * 15, [read], [read], ert=2.0)
    o = oracle.render(vol, vol.node_words(), fr)
    g = gpu.gpu_frame(ctx, fr, slot_to_id)
    gpu.compare(g, o)
    x64, inside = first_sample_positions(cam, W, H)
    sel = np.nonzero(inside)[0]
    ap = 1.0 - 0.5 ** (2 ** min(level_shifts(keep_axes, read)))
    got = g["rgba32"][sel, 0].astype(np.float64) * 256.0 / (ap * tf.scale)
    assert np.abs(got - closed_value_aniso(x64[sel], read, keep_axes)).max() < 0.05
    ctx.close()


@pytest.mark.parametrize("keep_axes,spacing,bias", [([4, 0], (1.0, 1.0, 1.0), 0.8), ([4, 4, 0], (1.0, 1.0, 4.0), 2.0)])
def test_anisotropic_partial_residency_on_gpu(gpu, keep_axes, spacing, bias):
    """Two u8 channels over a ragged volume whose first levels halve x and y
    only, 60 % of level 0 resident (coarser substitution across anisotropic
    levels), perspective views with distance-dependent levels and two start
    depths: bit-exact against the oracle."""
    dims = (100, 90, 70)
    k = len(keep_axes) + 1
    vols = [synth.blobs_u8(dims, 61 + c, n_blobs=14) for c in range(2)]
    levels = [synth.mean_levels(v, k, keep_axes) for v in vols]
    mn, mx = recipes._exact_meta(levels, (8, 8, 8))
    scene = recipes.Scene("aniso", dims, spacing, 2, k, 32, (8, 8, 8), 8, levels=levels, leaf_min=mn, leaf_max=mx,
                          keep_axes=keep_axes)
    fine = scene.all_bricks(levels=[0])
    pick = synth.seeded_subset(9, len(fine), int(0.6 * len(fine)))
    scene.resident = scene.all_bricks(levels=list(range(1, k))) + [fine[i] for i in pick]
    ctx = gpu.make_ctx(scene)
    slot_to_id = gpu.load(ctx, scene)
    vol = gpu.oracle_volume(scene)
    gpu.check_octree(ctx, vol)
    words = vol.node_words()
    sp = np.array(spacing)
    centre = tuple(np.array(dims) * sp / 2.0)
    cam = synth.look_at(tuple(np.array(centre) + np.array([-130.0, -100.0, 90.0 * sp[2]])), centre, (0, 0, 1), 90, 70,
                        fovy_deg=40.0)
    lod = synth.lod_thresholds(float(sp.min()), 70, 40.0, k, bias=bias)
    tfs = [synth.tf_ramp(8, 255, rgb=(1, 0.4, 0.1), alpha_max=0.3), synth.tf_ramp(20, 230, rgb=(0.2, 0.6, 1))]
    for sd in (0, 2):
        fr = synth.Frame(90, 70, cam, tfs, 0.5 * float(sp.min()), lod, [0, 0], [k - 1, k - 1], start_depth=sd)
        o = oracle.render(vol, words, fr)
        g = gpu.gpu_frame(ctx, fr, slot_to_id)
        gpu.compare(g, o)
        levels_used = set(((o["used_ids"] >> 24) % k).tolist())
        assert len(levels_used) >= 2 and o["req_ids"].size > 0
    ctx.close()
