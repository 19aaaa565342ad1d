"""Error behaviour of the C ABI on a GPU: invalid arguments and capacity
errors are reported and leave the context usable; a wait whose deadline runs
out returns RO_ERR_TIMEOUT (the stream is kept busy by a finite sleep kernel,
nothing hangs or faults)."""
import ctypes

import numpy as np
import pytest

import synth
from synth import recipes

pytestmark = pytest.mark.gpu

INVALID, CAPACITY, TIMEOUT = 1, 3, 4


@pytest.fixture(scope="module")
def scene_ctx():
    import torch
    assert torch.cuda.is_available(), "this test needs a CUDA GPU"
    from paper_2309_04393_gb300 import build, loader, ro
    build.build()
    scene = recipes.blobs128()
    d = ro.make_desc(scene.dims, scene.spacing, 1, 8, 32, 3, (16, 16, 16), 40, max_requests=1024, max_upload=16)
    ctx = ro.Context(d)
    loader.upload_keys(ctx, scene, scene.resident[:30])
    ctx.update_residency_octree(loader.meta_rows(scene.leaf_min, scene.leaf_max))
    return scene, ctx


def _status(fn, *a):
    from paper_2309_04393_gb300 import ro
    with pytest.raises(ro.RoError) as e:
        fn(*a)
    return e.value.status


def test_invalid_uploads_are_rejected_and_context_survives(scene_ctx):
    from paper_2309_04393_gb300 import ro
    scene, ctx = scene_ctx
    E = 34
    vox = np.zeros((2, E, E, E), np.uint8)
    good = ro.brick_id(0, 0, 3, 3, 3, 3)
    assert _status(ctx.upload_bricks, [good, good], vox) == INVALID            # duplicate ID
    assert _status(ctx.upload_bricks, [ro.brick_id(0, 0, 4, 0, 0, 3)], vox[:1]) == INVALID   # outside
    assert _status(ctx.upload_bricks, [ro.brick_id(1, 0, 0, 0, 0, 3)], vox[:1]) == INVALID   # channel 1 of 1
    many = np.zeros((17, E, E, E), np.uint8)
    ids = [ro.brick_id(0, 0, x, y, z, 3) for x in range(4) for y in range(4) for z in range(2)][:17]
    assert _status(ctx.upload_bricks, ids, many) == CAPACITY                    # > max_upload
    assert _status(ctx.update_residency_octree, np.array([[10 ** 6, 0, 1, 2]], np.uint32)) == INVALID
    slots, ev = ctx.upload_bricks([good], vox[:1])                              # still usable
    assert slots[0] < 40


def test_invalid_render_parameters(scene_ctx):
    from paper_2309_04393_gb300 import ro
    scene, ctx = scene_ctx
    f = scene.frames[0]
    bad = synth.Frame(**{**f.__dict__, "lmax": [3]})                           # lmax >= levels
    assert _status(ro.render_frame, ctx, bad) == INVALID
    bad = synth.Frame(**{**f.__dict__, "dt": 0.0})
    assert _status(ro.render_frame, ctx, bad) == INVALID
    bad = synth.Frame(**{**f.__dict__, "start_depth": 9})
    assert _status(ro.render_frame, ctx, bad) == INVALID
    assert _status(ctx.set_timeout, 0) == INVALID
    img, _ = ro.render_frame(ctx, f)                                            # still usable
    ctx.read_requests()
    assert float(img[..., 3].max()) > 0


def test_wait_deadline_returns_timeout_and_context_survives(scene_ctx):
    import torch
    from paper_2309_04393_gb300 import ro
    scene, ctx = scene_ctx
    ctx.set_timeout(5)                       # 5 ms
    with torch.cuda.stream(ctx.stream):
        torch.cuda._sleep(2_000_000_000)     # about a second of spinning, then it ends by itself
    assert _status(ctx.read_requests) == TIMEOUT
    torch.cuda.synchronize()
    ctx.set_timeout(30000)
    ro.render_frame(ctx, scene.frames[0])
    ids, ov, _ = ctx.read_requests()         # not latched: the context works again
    assert ov == 0
