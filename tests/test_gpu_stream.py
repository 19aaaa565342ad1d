"""Asynchronous brick uploads (ro_upload_bricks_async, ro_upload_wait): the
ray-guided loop of Sec. 4 with each frame's requested bricks copied on a
second stream while the next frame renders.  The scatter runs after that
render on the context's stream, so every frame sees a consistent cache: the
residency, every octree word and each frame must equal the oracle's for the
resident set the page table holds, and the loop must reach the same state as
the same loop with synchronous uploads."""
import numpy as np
import pytest

import oracle
import synth
from synth import recipes

pytestmark = pytest.mark.gpu


def loop(ctx, scene, frames, image, pinned, stream, use_async, check):
    """Render frame f + 1 while frame f's requests are made and uploaded."""
    from paper_2309_04393_gb300 import ro
    from bench import decode_ids
    import test_gpu_parity as tp
    E = scene.B + 2
    maxu = int(ctx.desc.max_upload)
    dt = np.uint8 if scene.value_bits == 8 else np.uint16
    bufs = [pinned[j].numpy().view(dt)[:maxu * E ** 3].reshape(maxu, E, E, E) for j in range(2)]
    keys = scene.all_bricks()
    key_ids = np.array([ro.brick_id(c, l, x, y, z, scene.k) for (c, l, x, y, z) in keys], np.uint32)
    ro.render_frame(ctx, frames[0], image)
    ids, _, _ = ctx.read_requests()
    resident = set()
    nb = 0
    history = []
    evictions = 0
    for f in range(1, len(frames)):
        ro.render_frame(ctx, frames[f], image)          # enqueued: runs while the host makes bricks
        todo = np.array([i for i in ids.tolist() if i not in resident], np.uint32)
        for q in range(0, todo.size, maxu):
            chunk = todo[q:q + maxu]
            vox = scene.bricks(decode_ids(chunk, scene.k))
            if use_async:
                buf = bufs[nb % 2][:chunk.size]
                nb += 1
                buf[:] = vox
                _, ev = ctx.upload_bricks_async(chunk, buf, stream)
            else:
                _, ev = ctx.upload_bricks(chunk, vox)
            resident.update(chunk.tolist())
            gone = [e for e in ev.tolist() if e != 0xFFFFFFFF]
            evictions += len(gone)
            resident.difference_update(gone)
        ctx.update_residency_octree()
        ids, _, _ = ctx.read_requests()
        ctx.upload_wait()
        pt = ctx.debug_read(1)
        history.append(pt.copy())
        if check:
            res_keys = [keys[i] for i in np.nonzero(pt)[0]]
            assert {ctx.brick_index(i) for i in resident} == set(np.nonzero(pt)[0].tolist())
            vol = oracle.Volume(scene.levels, scene.spacing, scene.B, scene.leaf, res_keys, scene.leaf_min,
                                scene.leaf_max)
            tp.check_octree(ctx, vol)
            slot_to_id = {int(pt[i]) - 1: int(key_ids[i]) for i in np.nonzero(pt)[0]}
            g = tp.gpu_frame(ctx, frames[f], slot_to_id)
            o = oracle.render(vol, vol.node_words(), frames[f])
            tp.compare(g, o, exact_sets=False)
            assert np.array_equal(np.sort(g["req"]), o["req_ids"])
            ids = g["req"]
    return history, evictions


def test_async_uploads_overlap_rendering():
    import torch
    assert torch.cuda.is_available(), "this test needs a CUDA GPU"
    from paper_2309_04393_gb300 import build, loader, ro
    build.build()
    scene = recipes.cells_slab(m=2, dims=(256, 256, 64), ncells=1500, k=4, W=160, H=120, n_views=6, resident_l0=0.0)
    cam_frames = scene.frames
    E = scene.B + 2
    d = ro.make_desc(scene.dims, scene.spacing, scene.m, scene.value_bits, scene.B, scene.k, scene.leaf, 28,
                     max_upload=16)
    pinned = torch.empty((2, 16 * E * E * E * 2), dtype=torch.uint8, pin_memory=True)
    stream = torch.cuda.Stream()
    hist = {}
    for use_async in (True, False):
        ctx = ro.Context(d)
        ctx.update_residency_octree(loader.meta_rows(scene.leaf_min, scene.leaf_max))
        image = torch.empty((cam_frames[0].H, cam_frames[0].W, 4), dtype=torch.float32, device="cuda")
        hist[use_async] = loop(ctx, scene, cam_frames, image, pinned, stream, use_async, check=True)
        ctx.close()
    # the same requests, uploads, evictions and page tables either way
    (ha, ea), (hs, es) = hist[True], hist[False]
    for a, b in zip(ha, hs):
        assert np.array_equal(a, b)
    assert ea == es and ea > 0, "the loop should have evicted least recently used bricks"
    assert np.count_nonzero(ha[-1]) > 10


def test_upload_wait_without_pending_copy_returns_at_once():
    import torch
    from paper_2309_04393_gb300 import build, ro
    build.build()
    scene = recipes.blobs128()
    d = ro.make_desc(scene.dims, scene.spacing, 1, 8, 32, 3, scene.leaf, 4, max_upload=4)
    ctx = ro.Context(d)
    ctx.upload_wait()
    ctx.close()
