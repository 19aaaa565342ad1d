"""INVALID node words and their pointers on the GPU (Sec. 5.2, Sec. 5.3),
through ro_update_node_metadata: every octree word bit-exact against the
oracle's (whose reading test_oracle_invalid.py pins), and frames rendered
from a partially initialised octree bit-exact against the oracle, before and
after the node requests of the first frame are answered."""
import numpy as np
import pytest

import oracle
import synth
from synth import recipes
from test_oracle_invalid import const_scene, ortho_z, random_metadata, root_only, tree

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    import torch
    assert torch.cuda.is_available(), "these tests need a CUDA GPU"
    from paper_2309_04393_gb300 import build
    build.build()
    import test_gpu_parity as tp
    return tp


def meta_rows(vol, lmin, lmax, nmin, nmax):
    """(node, channel, vmin, vmax) rows for every given range, nodes numbered
    depth-major with the leaves last (as node requests number them)."""
    first_leaf = vol.n_nodes - int(np.prod(vol.leaf_shape))
    rows = []
    for c in range(vol.m):
        li = np.nonzero(lmin[c].reshape(-1) >= 0)[0]
        rows += [(first_leaf + int(i), c, int(lmin[c].reshape(-1)[i]), int(lmax[c].reshape(-1)[i])) for i in li]
        ni = np.nonzero(nmin[c] >= 0)[0]
        rows += [(int(i), c, int(nmin[c][i]), int(nmax[c][i])) for i in ni if i < first_leaf]
    return np.array(rows, np.uint32).reshape(-1, 4)


@pytest.mark.parametrize("bpv", [1, 2])
def test_partial_metadata_matches_oracle(gpu, bpv):
    rng = np.random.default_rng(20 + bpv)
    dims, leaf = (100, 90, 70), (8, 8, 8)
    if bpv == 1:
        vols = [synth.blobs_u8(dims, 51, n_blobs=14), synth.blobs_u8(dims, 52, n_blobs=14)]
    else:
        vols = [(synth.blobs_u8(dims, 53 + c, n_blobs=14).astype(np.uint16) * 250) for c in range(2)]
    levels = [synth.mean_levels(v, 3) for v in vols]
    lmin, lmax, nmin, nmax = random_metadata(rng, vols, leaf, dims, 0.5, 0.3, bpv)
    scene = recipes.Scene("partial", dims, (1.0, 1.0, 1.0), 2, 3, 32, leaf, 8 * bpv, levels=levels,
                          leaf_min=lmin, leaf_max=lmax)
    fine = scene.all_bricks(levels=[0])
    pick = synth.seeded_subset(7, len(fine), int(0.6 * len(fine)))
    scene.resident = scene.all_bricks(levels=[1, 2]) + [fine[i] for i in pick]
    ctx = gpu.make_ctx(scene)
    from paper_2309_04393_gb300 import loader
    slots, _ = loader.upload_keys(ctx, scene, scene.resident)
    slot_to_id = {s: i for i, s in slots.items()}
    vol = oracle.Volume(levels, scene.spacing, 32, leaf, scene.resident, lmin, lmax, node_min=nmin, node_max=nmax)
    ctx.update_node_metadata(meta_rows(vol, lmin, lmax, nmin, nmax))
    gpu.check_octree(ctx, vol)
    words = vol.node_words()
    inv = ((words >> 16) & 0xFF) > (words >> 24)
    assert inv.any() and (inv & ((words >> 24) != 254)).any(), "scene lacks INVALID words with pointers"
    lo, hi = (8, 255) if bpv == 1 else (2000, 60000)
    tfs = [synth.tf_ramp(lo, hi, rgb=(1, 0.4, 0.1), alpha_max=0.3), synth.tf_ramp(lo, hi, rgb=(0.2, 0.6, 1))]
    cam = synth.look_at((-40.0, -30.0, 120.0), (50.0, 45.0, 35.0), (0, 0, 1), 88, 72, fovy_deg=42.0)
    lod = synth.lod_thresholds(1.0, 72, 42.0, 3, bias=0.5)
    node_reqs = None
    for sd in (0, 2):
        fr = synth.Frame(88, 72, cam, tfs, 0.5, lod, [0, 0], [2, 2], start_depth=sd)
        o = oracle.render(vol, words, fr)
        g = gpu.gpu_frame(ctx, fr, slot_to_id)
        gpu.compare(g, o)
        assert o["node_req_ids"].size > 0
        node_reqs = o["node_req_ids"]
    # answer the node requests with exact ranges (the data source's reply)
    D, nn, off = tree(dims, leaf)
    exact = [synth.leaf_ranges(v, leaf) for v in vols]
    first_leaf = off[D]
    for r in node_reqs:
        n, c = int(r) // 2, int(r) % 2
        d = max(i for i in range(D + 1) if off[i] <= n)
        j = n - off[d]
        jx, jy, jz = j % nn[d][0], (j // nn[d][0]) % nn[d][1], j // (nn[d][0] * nn[d][1])
        s = D - d
        sl = (slice(jz << s, (jz + 1) << s), slice(jy << s, (jy + 1) << s), slice(jx << s, (jx + 1) << s))
        a, b = int(exact[c][0][sl].min()), int(exact[c][1][sl].max())
        if n >= first_leaf:
            lmin[c].reshape(-1)[n - first_leaf], lmax[c].reshape(-1)[n - first_leaf] = a, b
        else:
            nmin[c][n], nmax[c][n] = a, b
    vol2 = oracle.Volume(levels, scene.spacing, 32, leaf, scene.resident, lmin, lmax, node_min=nmin, node_max=nmax)
    rows = [(int(r) // 2, int(r) % 2) for r in node_reqs]
    rows = [(n, c, int(lmin[c].reshape(-1)[n - first_leaf]) if n >= first_leaf else int(nmin[c][n]),
             int(lmax[c].reshape(-1)[n - first_leaf]) if n >= first_leaf else int(nmax[c][n])) for n, c in rows]
    ctx.update_node_metadata(np.array(rows, np.uint32))
    gpu.check_octree(ctx, vol2)
    fr = synth.Frame(88, 72, cam, tfs, 0.5, lod, [0, 0], [2, 2], start_depth=2)
    o = oracle.render(vol2, vol2.node_words(), fr)
    gpu.compare(gpu.gpu_frame(ctx, fr, slot_to_id), o)
    ctx.close()


def test_empty_and_homogeneous_by_ancestor_on_gpu(gpu):
    """The oracle's closed-form scenes: a root range below the TF window makes
    every INVALID node empty (nothing sampled or requested); a u8 constant
    volume with the root given [77, 77] renders from the node value."""
    from paper_2309_04393_gb300 import loader
    for value, dtype, tf in ((5, np.uint16, synth.tf_ramp(400, 12000)), (77, np.uint8, synth.tf_ramp(8, 255))):
        lv, bricks = const_scene(value, dtype)
        vol = oracle.Volume([lv], (1, 1, 1), 16, (4, 4, 4), bricks)
        root_only(vol, value, value)
        scene = recipes.Scene("const", (32, 32, 32), (1.0, 1.0, 1.0), 1, 2, 16, (4, 4, 4), 8 * np.dtype(dtype).itemsize,
                              levels=[lv], leaf_min=vol.leaf_min.reshape(1, 8, 8, 8), leaf_max=vol.leaf_max.reshape(1, 8, 8, 8))
        scene.resident = bricks
        ctx = gpu.make_ctx(scene)
        slots, _ = loader.upload_keys(ctx, scene, scene.resident)
        ctx.update_node_metadata(np.array([(0, 0, value, value)], np.uint32))
        gpu.check_octree(ctx, vol)
        for sd in (0, 2):
            fr = synth.Frame(8, 8, ortho_z(), [tf], 0.5, [0.0] + [float("inf")] * 15, [0], [0], start_depth=sd, ert=0.0)
            o = oracle.render(vol, vol.node_words(), fr)
            g = gpu.gpu_frame(ctx, fr, {s: i for i, s in slots.items()})
            gpu.compare(g, o)
            assert g["nodes"].size == 0 and g["req"].size == 0
        ctx.close()
