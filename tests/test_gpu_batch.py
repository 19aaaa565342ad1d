"""Batched multi-view rendering (ro_render_batch, ro_autotune_batch).

Every view of a batch must come out exactly as ro_render renders it alone
(binary32 image, per-pixel selection hash, evaluated samples, final lattice
index, brick samples), whatever the schedule; the batch's requests, node
requests and used bricks are the union of the views', its counters the sum.
One view is also checked against the oracle directly.  Views have uneven
sizes (ragged tiles, a view smaller than one tile).
"""
import numpy as np
import pytest

import oracle
import synth
from synth import recipes

pytestmark = pytest.mark.gpu

SIZES = [(160, 128), (97, 61), (33, 200), (5, 3)]
SCHEDULES = [(8, 0), (8, 1), (4, 0), (16, 1), (32, 0), (1, 1)]


@pytest.fixture(scope="module")
def scene_ctx():
    import torch
    assert torch.cuda.is_available(), "these tests need a CUDA GPU"
    from paper_2309_04393_gb300 import build, loader, ro
    build.build()
    scene = recipes.cells_slab(m=4, dims=(256, 256, 32), ncells=1250, k=5, W=160, H=128, n_views=4)
    d = ro.make_desc(scene.dims, scene.spacing, scene.m, scene.value_bits, scene.B, scene.k, scene.leaf,
                     max(1, len(scene.resident)), max_requests=65536, max_upload=512, max_batch_tiles=4096)
    ctx = ro.Context(d)
    slots = loader.load_scene(ctx, scene)
    frames = []
    for f, (W, H) in zip(scene.frames, SIZES):
        g = synth.Frame(**{**f.__dict__, "W": W, "H": H})
        g.lod_t = synth.lod_thresholds(1.0, H, 40.0, scene.k, bias=1.5)
        frames.append(g)
    return scene, ctx, frames, {s: i for i, s in slots.items()}


def _np(t):
    return t.cpu().numpy().view(np.uint32).reshape(-1)


def singles(ctx, frames):
    """Each view rendered alone: outputs, and the union of requests/used."""
    from paper_2309_04393_gb300 import ro
    outs, req, nodes, used, stats = [], set(), set(), np.zeros(int(ctx.desc.cache_slots), bool), np.zeros(8, np.uint64)
    for f in frames:
        img, dbg = ro.render_frame(ctx, f, debug=True)
        used |= ctx.debug_read(4).astype(bool)
        r, ov, nd = ctx.read_requests()
        assert ov == 0
        req |= set(r.tolist())
        nodes |= set(nd.tolist())
        stats += ctx.stats()
        outs.append((img.cpu().numpy(), [_np(t) for t in dbg]))
    return outs, req, nodes, used, stats


def batch(ctx, frames, tile_w, order):
    from paper_2309_04393_gb300 import ro
    imgs, dbgs = ro.render_batch(ctx, frames, tile_w=tile_w, order=order, debug=True)
    used = ctx.debug_read(4).astype(bool)
    stats = ctx.stats()
    r, ov, nd = ctx.read_requests()
    assert ov == 0
    return [(i.cpu().numpy(), [_np(t) for t in d]) for i, d in zip(imgs, dbgs)], set(r.tolist()), set(nd.tolist()), \
        used, stats


def assert_same(a, b):
    for (ia, da), (ib, db) in zip(a, b):
        assert np.array_equal(ia, ib), "images differ"
        for x, y, name in zip(da, db, ("hash", "n_eval", "i_end", "n_bs")):
            assert np.array_equal(x, y), f"{name} differs"


def test_batch_equals_single_views_for_every_schedule(scene_ctx):
    scene, ctx, frames, _ = scene_ctx
    ref, req, nodes, used, stats = singles(ctx, frames)
    assert len(req) > 0 and stats[2] > 0
    for tile_w, order in SCHEDULES:
        for rep in range(2):      # the second call replays the captured graph
            got, g_req, g_nodes, g_used, g_stats = batch(ctx, frames, tile_w, order)
            assert_same(ref, got)
            assert g_req == req and g_nodes == nodes
            assert np.array_equal(g_used, used)
            assert np.array_equal(g_stats[:6], stats[:6])


def test_graph_replay_picks_up_new_cameras_and_tfs(scene_ctx):
    """Same layout (sizes, schedule): the captured graph is replayed with the
    new view table and LUTs."""
    scene, ctx, frames, _ = scene_ctx
    batch(ctx, frames, 8, 0)
    moved = []
    for f, g in zip(frames, frames[1:] + frames[:1]):
        cam = synth.look_at(tuple(np.asarray(g.camera.eye) * 1.1), (128.0, 128.0, 64.0), (0, 0, 1), f.W, f.H,
                            fovy_deg=35.0)
        tfs = [synth.tf_ramp(500.0 + 300 * c, 9000.0, rgb=(1.0, 0.5, 0.25 * c), alpha_max=0.3)
               for c in range(scene.m)]
        moved.append(synth.Frame(**{**f.__dict__, "camera": cam, "tfs": tfs}))
    ref, req, nodes, used, stats = singles(ctx, moved)
    got, g_req, g_nodes, g_used, g_stats = batch(ctx, moved, 8, 0)
    assert_same(ref, got)
    assert g_req == req and np.array_equal(g_stats[:6], stats[:6])


def test_batch_view_matches_oracle(scene_ctx):
    scene, ctx, frames, slot_to_id = scene_ctx
    vol = oracle.Volume(scene.levels, scene.spacing, scene.B, scene.leaf, scene.resident, scene.leaf_min,
                        scene.leaf_max)
    got, g_req, g_nodes, g_used, g_stats = batch(ctx, frames[:2], 16, 1)
    words = vol.node_words()
    want_req = set()
    for (img, dbg), f in zip(got, frames[:2]):
        o = oracle.render(vol, words, f)
        assert np.array_equal(dbg[0], o["hash"]) and np.array_equal(dbg[1], o["n_eval"])
        assert np.array_equal(dbg[2], o["i_end"]) and np.array_equal(dbg[3], o["n_bs"])
        assert np.array_equal(img.reshape(-1, 4), o["rgba32"])
        assert np.abs(img.reshape(-1, 4).astype(np.float64) - o["rgba64"]).max() <= 2e-3
        want_req |= set(o["req_ids"].tolist())
    assert g_req == want_req


def test_autotune_returns_a_schedule_that_renders_the_same(scene_ctx):
    scene, ctx, frames, _ = scene_ctx
    ref, req, nodes, used, stats = singles(ctx, frames)
    views = []
    from paper_2309_04393_gb300 import ro
    imgs = [ctx.torch.empty((f.H, f.W, 4), dtype=ctx.torch.float32, device=ctx.device) for f in frames]
    for f, img in zip(frames, imgs):
        views.append((ro.camera_struct(f.camera), ro.params_struct(f), img, f.W, f.H))
    (tile_w, order), ms = ctx.autotune_batch(views, [(t.lo, t.scale, t.lut) for t in frames[0].tfs])
    assert tile_w in (4, 8, 16, 32) and order in (0, 1) and ms > 0
    ctx.read_requests()
    got, g_req, _, _, g_stats = batch(ctx, frames, tile_w, order)
    assert_same(ref, got)
    assert g_req == req and np.array_equal(g_stats[:6], stats[:6])


def test_batch_errors(scene_ctx):
    from paper_2309_04393_gb300 import ro
    scene, ctx, frames, _ = scene_ctx
    with pytest.raises(ro.RoError) as e:
        ro.render_batch(ctx, frames, tile_w=3)
    assert e.value.status == 1
    with pytest.raises(ro.RoError) as e:
        ro.render_batch(ctx, [synth.Frame(**{**frames[0].__dict__, "W": 512, "H": 512})])  # 8192 tiles
    assert e.value.status == 3                                   # more tiles than max_batch_tiles
    d = ro.make_desc(scene.dims, scene.spacing, scene.m, scene.value_bits, scene.B, scene.k, scene.leaf, 8)
    plain = ro.Context(d)
    with pytest.raises(ro.RoError) as e:
        ro.render_batch(plain, frames)
    assert e.value.status == 3                                   # no batch region
    got, *_ = batch(ctx, frames, 8, 0)                            # still usable
    assert len(got) == len(frames)


def test_render_longest_first_order_changes_nothing(scene_ctx):
    """ro_render with order 1 (a one-view batch ordered by the previous
    frame's tile costs) renders what order 0 renders."""
    from paper_2309_04393_gb300 import ro
    scene, ctx, frames, _ = scene_ctx

    def one(f, order):
        img, dbg = ro.render_frame(ctx, f, debug=True, order=order)
        stats = ctx.stats()
        r, ov, nd = ctx.read_requests()
        return (img.cpu().numpy(), [_np(t) for t in dbg]), set(r.tolist()), set(nd.tolist()), stats

    for f in frames:
        ref = one(f, 0)
        for rep in range(2):                    # the second call orders by the first one's costs
            got = one(f, 1)
            assert_same([ref[0]], [got[0]])
            assert got[1] == ref[1] and got[2] == ref[2]
            assert np.array_equal(got[3][:6], ref[3][:6])
