"""Run-time channel replacement (ro_replace_channel): channel slot 1 is
given to another data-set channel.  Right after the call every node of the
slot is INVALID with an empty mask, its page tables are empty and its cache
slots are free; a frame then renders exactly what the oracle renders for a
channel without metadata or bricks (node requests for it, nothing sampled);
once the new channel's metadata and bricks arrive, frames match the oracle
for the new pair of channels bit for bit."""
import numpy as np
import pytest

import oracle
import synth
from synth import recipes
from test_gpu_parity import compare, gpu_frame, torch_cuda  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu


def two_channel_scene(second_seed):
    v0 = synth.blobs_u8((100, 90, 70), 21, n_blobs=14)
    v1 = synth.blobs_u8((100, 90, 70), second_seed, n_blobs=14)
    levels = [synth.mean_levels(v0, 3), synth.mean_levels(v1, 3)]
    mn, mx = recipes._exact_meta(levels, (8, 8, 8))
    scene = recipes.Scene("pair", (100, 90, 70), (1.0, 1.0, 1.0), 2, 3, 32, (8, 8, 8), 8, levels=levels,
                          leaf_min=mn, leaf_max=mx)
    scene.resident = scene.all_bricks()
    return scene


def test_replace_channel_then_stream_the_new_one(torch_cuda):
    from paper_2309_04393_gb300 import loader, ro
    old = two_channel_scene(22)
    new = two_channel_scene(57)                      # channel 0 identical, channel 1 another volume
    d = ro.make_desc(old.dims, old.spacing, 2, 8, 32, 3, (8, 8, 8), len(old.resident), max_upload=512)
    ctx = ro.Context(d)
    slots = loader.load_scene(ctx, old)
    slot_to_id = {s: i for i, s in slots.items()}
    W, H = 120, 100
    cam = synth.look_at((-60.0, 150.0, 120.0), (50.0, 45.0, 35.0), (0, 0, 1), W, H, fovy_deg=38.0)
    tfs = [synth.tf_ramp(8, 255, rgb=(1, 0.3, 0.1), alpha_max=0.4), synth.tf_ramp(30, 200, rgb=(0.1, 0.5, 1))]
    frame = synth.Frame(W, H, cam, tfs, 0.5, [0.0] + [float("inf")] * 15, [0, 0], [2, 2])
    vol_old = oracle.Volume(old.levels, old.spacing, 32, (8, 8, 8), old.resident, old.leaf_min, old.leaf_max)
    compare(gpu_frame(ctx, frame, slot_to_id), oracle.render(vol_old, vol_old.node_words(), frame))

    ctx.replace_channel(1)
    words = ctx.octree_words()
    # the replaced channel: INVALID everywhere with no valid ancestor (UNKNOWN)
    assert np.all(words[:, 1] == 0xFEFF0000) and np.any(words[:, 0] != 0xFEFF0000)
    pt = ctx.debug_read(1)
    n1 = [ctx.brick_index(ro.brick_id(1, l, x, y, z, 3)) for (c, l, x, y, z) in old.all_bricks() if c == 1]
    assert np.all(pt[n1] == 0)
    # the slot as the oracle sees it: no metadata and no bricks for channel 1
    none_min, none_max = new.leaf_min.copy(), new.leaf_max.copy()
    none_min[1], none_max[1] = -1, -1
    res0 = [b for b in new.resident if b[0] == 0]
    vol_gap = oracle.Volume(new.levels, new.spacing, 32, (8, 8, 8), res0, none_min, none_max)
    g = gpu_frame(ctx, frame, {s: i for i, s in slots.items() if (i >> 24) // 3 == 0})
    o = oracle.render(vol_gap, vol_gap.node_words(), frame)
    compare(g, o)
    assert g["nodes"].size > 0 and np.all(np.asarray(g["nodes"]) % 2 == 1)   # node * m + 1

    # the new channel streams in: its leaf metadata, then its bricks
    ctx.update_residency_octree(loader.meta_rows(new.leaf_min, new.leaf_max, channels=[1]))
    s1, _ = loader.upload_keys(ctx, new, [b for b in new.resident if b[0] == 1])
    ctx.update_residency_octree()
    slot_to_id = {s: i for i, s in slots.items() if (i >> 24) // 3 == 0}
    slot_to_id.update({s: i for i, s in s1.items()})
    vol_new = oracle.Volume(new.levels, new.spacing, 32, (8, 8, 8), new.resident, new.leaf_min, new.leaf_max)
    assert np.array_equal(ctx.octree_words(), vol_new.node_words())
    compare(gpu_frame(ctx, frame, slot_to_id), oracle.render(vol_new, vol_new.node_words(), frame))
