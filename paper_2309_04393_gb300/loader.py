"""Caller-side helpers: push a scene's bricks and leaf metadata through the
C ABI (ro_upload_bricks, ro_update_residency_octree).  The scene object
supplies k, m, B, leaf_min/leaf_max arrays and bricks(keys) -> voxels."""
from __future__ import annotations

import numpy as np

from .ro import Context, brick_id


def meta_rows(leaf_min: np.ndarray, leaf_max: np.ndarray, channels=None) -> np.ndarray:
    """(n, 4) uint32 rows (leaf, channel, vmin, vmax) for every leaf and
    channel that has metadata (entries < 0 mean none)."""
    m = leaf_min.shape[0]
    rows = []
    for c in (range(m) if channels is None else channels):
        mn = leaf_min[c].reshape(-1)
        mx = leaf_max[c].reshape(-1)
        ok = np.nonzero((mn >= 0) & (mx >= 0))[0]
        r = np.empty((ok.size, 4), np.uint32)
        r[:, 0] = ok
        r[:, 1] = c
        r[:, 2] = mn[ok]
        r[:, 3] = mx[ok]
        rows.append(r)
    return np.concatenate(rows) if rows else np.zeros((0, 4), np.uint32)


def upload_keys(ctx: Context, scene, keys, batch=None):
    """Upload the bricks (c, l, bx, by, bz) in batches; returns
    {brick_id: slot} and the list of evicted IDs."""
    keys = [tuple(int(v) for v in kk) for kk in keys]
    batch = int(ctx.desc.max_upload if batch is None else min(batch, ctx.desc.max_upload))
    slots, evicted = {}, []
    for q in range(0, len(keys), batch):
        chunk = keys[q:q + batch]
        ids = np.array([brick_id(c, l, x, y, z, scene.k) for (c, l, x, y, z) in chunk], np.uint32)
        vox = scene.bricks(chunk)
        s, ev = ctx.upload_bricks(ids, vox)
        for i, sl in zip(ids.tolist(), s.tolist()):
            slots[i] = sl
        for e in ev.tolist():
            if e != 0xFFFFFFFF:
                evicted.append(e)
                slots.pop(e, None)
    return slots, evicted


def load_scene(ctx: Context, scene, batch=None):
    """Upload the scene's resident bricks and all its leaf metadata, then
    bring the residency octree up to date."""
    slots, _ = upload_keys(ctx, scene, scene.resident, batch)
    ctx.update_residency_octree(meta_rows(scene.leaf_min, scene.leaf_max))
    return slots
