"""Homogeneous nodes on the GPU (Sec. 5.2: a node whose channel holds one
value everywhere is rendered from the node's value, Algorithm 1
isHomogeneous; exact min == max, 8-bit data only).

The scene has noise-free blobs and flat boxes above the transfer function's
threshold, each several leaves wide, so that whole subtrees hold one value.
The CPU test checks on the oracle that such nodes exist and that rays sample
them; the GPU tests compare the CUDA path with the oracle bit for bit and
check that the kernel's own counter of homogeneous channel samples equals
the oracle's.
"""
import numpy as np
import pytest

import oracle
import synth
from synth import recipes

DIMS = (96, 80, 64)
BOXES = (((8, 8, 16), (48, 40, 56), 120), ((56, 40, 8), (88, 72, 40), 200), ((60, 8, 40), (92, 32, 64), 9))


def plateau_volume(seed, noise_max=0):
    v = synth.blobs_u8(DIMS, seed, n_blobs=8, noise_max=noise_max)
    for lo, hi, val in BOXES:
        v[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] = val
    return v


def plateau_scene(m, resident_l0=1.0, seed=3):
    chans = [plateau_volume(40)] + [synth.blobs_u8(DIMS, 41 + c, n_blobs=12) for c in range(1, m)]
    levels = [synth.mean_levels(v, 3) for v in chans]
    mn, mx = recipes._exact_meta(levels, (8, 8, 8))
    s = recipes.Scene("plateaus", DIMS, (1.0, 1.0, 1.0), m, 3, 32, (8, 8, 8), 8, levels=levels,
                      leaf_min=mn, leaf_max=mx)
    fine = s.all_bricks(levels=[0])
    pick = synth.seeded_subset(seed, len(fine), int(round(resident_l0 * len(fine))))
    s.resident = s.all_bricks(levels=[1, 2]) + [fine[i] for i in pick]
    return s


def frames(m):
    tfs = [synth.tf_ramp(8, 255, rgb=(1.0, 0.5, 0.2), alpha_max=0.12)] + \
          [synth.tf_ramp(20, 230, rgb=(0.2, 0.5, 1.0), alpha_max=0.3) for _ in range(1, m)]
    ortho = synth.look_at((48.0, 40.0, -10.0), (48.0, 40.0, 32.0), (0.0, -1.0, 0.0), 120, 100, ortho_pixel=0.8)
    persp = synth.look_at((-60.0, -40.0, 110.0), (48.0, 40.0, 32.0), (0, 0, 1), 101, 77, fovy_deg=45.0)
    lod = synth.lod_thresholds(1.0, 77, 45.0, 3, bias=0.4)
    return [synth.Frame(120, 100, ortho, tfs, 0.5, [0.0] + [float("inf")] * 15, [0] * m, [0] * m),
            synth.Frame(101, 77, persp, tfs, 0.5, lod, [0] * m, [2] * m)]


def oracle_volume(scene):
    return oracle.Volume(scene.levels, scene.spacing, scene.B, scene.leaf, scene.resident, scene.leaf_min,
                         scene.leaf_max)


def homogeneous_samples(o):
    """Channel samples that took a node value: evaluated samples times the
    channels with a value, minus those read from bricks (one channel with
    every level resident has a value at each evaluated sample)."""
    return int(o["n_eval"].sum()) - int(o["n_bs"].sum())


def test_plateau_scene_has_homogeneous_nodes():
    """CPU check of the scene itself: nodes whose first channel holds a
    single value above the TF threshold exist at several depths, and the
    oracle renders samples from them without reading a brick."""
    scene = plateau_scene(1)
    vol = oracle_volume(scene)
    w = vol.node_words()[:, 0]
    mn8, mx8 = (w >> 16) & 0xFF, w >> 24
    homog = (mn8 == mx8) & (mn8 > 8)
    assert homog.sum() >= 20
    assert set(np.unique(mn8[homog]).tolist()) == {9, 120, 200}
    o = oracle.render(vol, vol.node_words(), frames(1)[0])
    assert homogeneous_samples(o) > 1000 and o["n_bs"].sum() > 1000
    # a homogeneous node adds no request and no used brick of its own
    assert o["req_ids"].size == 0


@pytest.mark.gpu
@pytest.mark.parametrize("m,resident_l0", [(1, 1.0), (2, 0.6)])
def test_homogeneous_nodes_match_oracle(m, resident_l0):
    import torch
    assert torch.cuda.is_available(), "these tests need a CUDA GPU"
    from paper_2309_04393_gb300 import build
    build.build()
    from test_gpu_parity import compare, gpu_frame, load, make_ctx, check_octree
    scene = plateau_scene(m, resident_l0)
    ctx = make_ctx(scene)
    slot_to_id = load(ctx, scene)
    vol = oracle_volume(scene)
    check_octree(ctx, vol)
    words = vol.node_words()
    for fr in frames(m):
        o = oracle.render(vol, words, fr)
        g = gpu_frame(ctx, fr, slot_to_id)
        compare(g, o)
        st = g["stats"]
        assert st[1] == o["n_eval"].sum() and st[2] == o["n_bs"].sum()
        if m == 1:
            assert st[3] == homogeneous_samples(o)
        assert st[3] > 500, "no homogeneous channel samples"
    ctx.close()
