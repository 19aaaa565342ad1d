"""Degenerate and extreme cases against the oracle: a 1x1 image from a
camera inside the volume; a frame whose rays all miss the volume; rays that
reach the 2^24-sample lattice limit; the widest image the call accepts;
calls with nothing to do."""
import numpy as np
import pytest

import oracle
import synth
from synth import recipes
from test_gpu_parity import compare, gpu_frame, torch_cuda  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def blobs(torch_cuda):
    from paper_2309_04393_gb300 import loader, ro
    scene = recipes.blobs128()
    d = ro.make_desc(scene.dims, scene.spacing, 1, 8, 32, 3, (16, 16, 16), len(scene.resident))
    ctx = ro.Context(d)
    slots = loader.load_scene(ctx, scene)
    vol = oracle.Volume(scene.levels, scene.spacing, 32, (16, 16, 16), scene.resident, scene.leaf_min,
                        scene.leaf_max)
    return scene, ctx, {s: i for i, s in slots.items()}, vol


def test_single_pixel_from_inside_the_volume(blobs):
    scene, ctx, slot_to_id, vol = blobs
    cam = synth.look_at((64.3, 60.7, 50.2), (70.0, 90.0, 100.0), (0, 0, 1), 1, 1, fovy_deg=30.0)
    fr = synth.Frame(1, 1, cam, scene.frames[0].tfs, 0.5, [0.0] + [float("inf")] * 15, [0], [2])
    compare(gpu_frame(ctx, fr, slot_to_id), oracle.render(vol, vol.node_words(), fr))


def test_every_ray_misses(blobs):
    scene, ctx, slot_to_id, vol = blobs
    cam = synth.look_at((-50.0, -50.0, -50.0), (-200.0, -210.0, -190.0), (0, 0, 1), 40, 30, fovy_deg=30.0)
    fr = synth.Frame(40, 30, cam, scene.frames[0].tfs, 0.5, [0.0] + [float("inf")] * 15, [0], [2])
    g = gpu_frame(ctx, fr, slot_to_id)
    o = oracle.render(vol, vol.node_words(), fr)
    compare(g, o)
    assert not g["rgba32"].any() and g["req"].size == 0 and g["stats"][0] == 0


def test_rays_stop_at_the_lattice_limit(blobs):
    """dt = 2^-18 in a 128-voxel volume: a straight pass needs ~2^25 lattice
    samples, the march stops at 2^24 on both sides.  Bit-exact against the
    binary32 mirror; the binary64 image is not a reference here: 1 - 1e-9
    rounds to 1 in binary32, so over 2^24 steps the binary32 contract and
    binary64 arithmetic drift apart by design."""
    scene, ctx, slot_to_id, vol = blobs
    lut = np.zeros((256, 4), np.float32)
    lut[:, :3] = 1.0
    lut[:, 3] = 1e-9                                             # almost transparent, never empty
    tf = synth.TF(0.0, 1.0, lut)
    cam = synth.look_at((-5.0, 64.2, 63.9), (200.0, 64.2, 63.9), (0, 0, 1), 2, 1, ortho_pixel=0.5)
    fr = synth.Frame(2, 1, cam, [tf], 2.0 ** -18, [0.0] + [float("inf")] * 15, [0], [0], ert=0.0)
    g = gpu_frame(ctx, fr, slot_to_id)
    o = oracle.render(vol, vol.node_words(), fr)
    for key in ("hash", "n_eval", "i_end", "n_bs", "rgba32"):
        assert np.array_equal(g[key], o[key]), key
    assert np.array_equal(np.sort(g["req"]), o["req_ids"])
    assert np.all(o["i_end"] == 1 << 24)


def test_widest_image(blobs):
    scene, ctx, slot_to_id, vol = blobs
    cam = synth.look_at((64.0, -300.0, 64.0), (64.0, 64.0, 64.0), (0, 0, 1), 16384, 2, fovy_deg=10.0)
    fr = synth.Frame(16384, 2, cam, scene.frames[0].tfs, 0.5, [0.0] + [float("inf")] * 15, [0], [2])
    o_pix = np.stack([np.arange(0, 16384, 97), np.zeros(169, np.int64)], 1)
    g = gpu_frame(ctx, fr, slot_to_id)
    o = oracle.render(vol, vol.node_words(), fr, o_pix)
    idx = o_pix[:, 1] * 16384 + o_pix[:, 0]
    for key in ("hash", "n_eval", "i_end", "n_bs"):
        assert np.array_equal(g[key][idx], o[key])
    assert np.array_equal(g["rgba32"][idx], o["rgba32"])


def test_calls_with_nothing_to_do(blobs):
    from paper_2309_04393_gb300 import ro
    scene, ctx, slot_to_id, vol = blobs
    slots, ev = ctx.upload_bricks(np.zeros(0, np.uint32), np.zeros((0, 34, 34, 34), np.uint8))
    assert slots.size == 0
    ctx.update_residency_octree(np.zeros((0, 4), np.uint32))
    ids, ov, nodes = ctx.read_requests()
    assert ids.size == 0 and ov == 0
    assert np.array_equal(ctx.octree_words(), vol.node_words())
