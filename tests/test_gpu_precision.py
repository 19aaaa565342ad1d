"""Low-precision sampling on the GPU (sample_format 1 = binary16, 2 =
bfloat16) against the oracle's mirror of the same arithmetic:
selection hashes, evaluated samples, final lattice indices, brick samples,
the binary32 image, requests, node requests and used bricks bit-exact.  The
error of the image against the binary64 oracle is the precision study's
number; it is bounded here by what the format's rounding allows."""
import numpy as np
import pytest

import oracle
import synth
from synth import recipes
from test_gpu_parity import gpu_frame, torch_cuda  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu

# max |dRGBA| against binary64 these formats may reach on the scenes below
BOUND = {1: 2e-2, 2: 1.5e-1}


def setup(scene, fmt, cache_slots=None):
    from paper_2309_04393_gb300 import loader, ro
    n_slots = cache_slots if cache_slots is not None else max(1, len(scene.resident))
    d = ro.make_desc(scene.dims, scene.spacing, scene.m, scene.value_bits, scene.B, scene.k, scene.leaf, n_slots,
                     max_requests=65536, max_upload=512, sample_format=fmt)
    ctx = ro.Context(d)
    slots = loader.load_scene(ctx, scene)
    vol = oracle.Volume(scene.levels, scene.spacing, scene.B, scene.leaf, scene.resident, scene.leaf_min,
                        scene.leaf_max, sample_format=fmt)
    return ctx, {s: i for i, s in slots.items()}, vol


def exact(g, o):
    for key in ("n_eval", "i_end", "n_bs", "hash", "rgba32"):
        assert np.array_equal(g[key], o[key]), f"{key} differs"
    assert np.array_equal(np.sort(g["req"]), o["req_ids"]), "request lists differ"
    assert np.array_equal(g["used"], np.sort(o["used_ids"])), "used bricks differ"
    assert np.array_equal(np.sort(g["nodes"]), np.sort(o["node_req_ids"])), "node requests differ"
    return float(np.abs(g["rgba32"].astype(np.float64) - o["rgba64"]).max())


@pytest.mark.parametrize("fmt", [1, 2])
def test_blobs128_u8(torch_cuda, fmt):
    scene = recipes.blobs128()
    ctx, slot_to_id, vol = setup(scene, fmt)
    words = vol.node_words()
    for frame in scene.frames:
        err = exact(gpu_frame(ctx, frame, slot_to_id), oracle.render(vol, words, frame))
        print(f"blobs128 fmt {fmt}: max |dRGBA| vs binary64 {err:.3e}")
        assert err <= BOUND[fmt]


@pytest.mark.parametrize("fmt", [1, 2])
def test_ragged_partial_residency_u8_two_channels(torch_cuda, fmt):
    v0 = synth.blobs_u8((100, 90, 70), 21, n_blobs=14)
    v1 = synth.blobs_u8((100, 90, 70), 22, n_blobs=14)
    levels = [synth.mean_levels(v0, 3), synth.mean_levels(v1, 3)]
    mn, mx = recipes._exact_meta(levels, (8, 8, 8))
    scene = recipes.Scene("ragged", (100, 90, 70), (1.0, 1.0, 1.0), 2, 3, 32, (8, 8, 8), 8, levels=levels,
                          leaf_min=mn, leaf_max=mx)
    fine = scene.all_bricks(levels=[0])
    pick = synth.seeded_subset(5, len(fine), int(0.6 * len(fine)))
    scene.resident = scene.all_bricks(levels=[1, 2]) + [fine[i] for i in pick]
    ctx, slot_to_id, vol = setup(scene, fmt)
    W, H = 250, 230
    cam = synth.look_at((-60.0, 150.0, 120.0), (50.0, 45.0, 35.0), (0, 0, 1), W, H, fovy_deg=38.0)
    tfs = [synth.tf_ramp(8, 255, rgb=(1, 0.3, 0.1), alpha_max=0.4), synth.tf_ramp(30, 200, rgb=(0.1, 0.5, 1))]
    frame = synth.Frame(W, H, cam, tfs, 0.5, synth.lod_thresholds(1.0, H, 38.0, 3, bias=0.35), [0, 1], [2, 2])
    o = oracle.render(vol, vol.node_words(), frame)
    err = exact(gpu_frame(ctx, frame, slot_to_id), o)
    print(f"ragged fmt {fmt}: max |dRGBA| vs binary64 {err:.3e}")
    assert o["req_ids"].size > 0 and err <= BOUND[fmt]


@pytest.mark.parametrize("fmt", [1, 2])
def test_cells_u16_four_channels_perspective(torch_cuda, fmt):
    scene = recipes.cells_slab(m=4, dims=(256, 256, 32), ncells=1250, k=5, W=160, H=128, n_views=3)
    ctx, slot_to_id, vol = setup(scene, fmt)
    words = vol.node_words()
    for frame in scene.frames:
        frame.lod_t = synth.lod_thresholds(1.0, frame.H, 40.0, scene.k, bias=1.5)
        o = oracle.render(vol, words, frame)
        err = exact(gpu_frame(ctx, frame, slot_to_id), o)
        print(f"cells4 fmt {fmt}: max |dRGBA| vs binary64 {err:.3e}")
        assert o["n_bs"].sum() > 1000 and err <= BOUND[fmt]


@pytest.mark.parametrize("fmt", [1, 2])
def test_batch_in_low_precision_equals_single_views(torch_cuda, fmt):
    from paper_2309_04393_gb300 import loader, ro
    scene = recipes.cells_slab(m=4, dims=(256, 256, 32), ncells=1250, k=5, W=120, H=90, n_views=2)
    d = ro.make_desc(scene.dims, scene.spacing, scene.m, scene.value_bits, scene.B, scene.k, scene.leaf,
                     len(scene.resident), max_batch_tiles=1024, sample_format=fmt)
    ctx = ro.Context(d)
    loader.load_scene(ctx, scene)
    singles = [ro.render_frame(ctx, f)[0].cpu().numpy() for f in scene.frames]
    ctx.read_requests()
    imgs, _ = ro.render_batch(ctx, scene.frames, tile_w=16, order=0)
    for a, b in zip(singles, imgs):
        assert np.array_equal(a, b.cpu().numpy())
