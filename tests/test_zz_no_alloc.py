"""The allocation-free flag compaction (ro_compact_flags_noalloc).

Some callers of this library cannot allocate device memory: a plugin whose
host application owns all GPU memory and gives it no allocator, or a frame
loop in which a device allocation would stall the GPU.  The entry point keeps
its scratch in a static device array instead.  Here it is checked against
the request readback of ro_read_requests on two frames in a row: after each
render the context's request flags are copied into a caller-owned device
buffer and compacted by ro_compact_flags_noalloc, and both lists must name
the same bricks (integer results: exact)."""
import ctypes

import numpy as np
import pytest

import synth
from synth import recipes

pytestmark = pytest.mark.gpu


def test_noalloc_compaction_matches_request_readback():
    import torch
    assert torch.cuda.is_available(), "this test needs a CUDA GPU"
    from paper_2309_04393_gb300 import build, loader, ro
    build.build()
    scene = recipes.blobs128()
    fine = scene.all_bricks(levels=[0])
    pick = synth.seeded_subset(9, len(fine), len(fine) // 2)
    scene.resident = scene.all_bricks(levels=[1, 2]) + [fine[i] for i in pick]
    desc = ro.make_desc(scene.dims, scene.spacing, scene.m, scene.value_bits, scene.B, scene.k, scene.leaf,
                        len(scene.resident), max_upload=128)
    ctx = ro.Context(desc)
    loader.load_scene(ctx, scene)
    n = int(ctx.sizes.n_bricks)
    pad = (n + 15) // 16 * 16
    flags = torch.zeros(pad, dtype=torch.uint8, device="cuda")
    ids = torch.full((pad,), -1, dtype=torch.int32, device="cuda")
    total = torch.zeros(1, dtype=torch.int32, device="cuda")
    frames = [synth.Frame(**{**scene.frames[0].__dict__, "skip": False}), scene.frames[1]]
    for frame in frames:                       # two calls in a row share the static scratch
        ro.render_frame(ctx, frame)
        host_flags = ctx.debug_read(3)         # this frame's request flags
        flags[:n].copy_(torch.from_numpy(host_flags).to("cuda"))
        ro.compact_flags_noalloc(flags, ids, total)
        torch.cuda.synchronize()
        count = int(total.item())
        got = ids[:count].cpu().numpy().astype(np.uint32)
        req, overflow, _ = ctx.read_requests()
        want = np.sort(np.array([ctx.brick_index(int(i)) for i in req], np.uint32))
        assert overflow == 0 and count > 0
        assert count == int((host_flags != 0).sum()) == req.size
        assert np.array_equal(got, want)
        assert int(flags.sum().item()) == 0    # every flag cleared
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_2309_04393_gb300 import ro
    L = ro.load()
    flags = torch.zeros(16, dtype=torch.uint8, device="cuda")
    total = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # more flags than 2^28: refused before any device work
    rc = L.ro_compact_flags_noalloc(ctypes.c_void_p(flags.data_ptr()), (1 << 28) + 16, None, 0,
                                    ctypes.c_void_p(total.data_ptr()), stream)
    assert rc == 3  # RO_ERR_CAPACITY
    rc = L.ro_compact_flags_noalloc(ctypes.c_void_p(flags.data_ptr()), 15, None, 0,
                                    ctypes.c_void_p(total.data_ptr()), stream)
    assert rc == 1  # RO_ERR_INVALID_ARG: not a multiple of 16


@pytest.mark.parametrize("n,cap", [(4096 * 3 + 16 * 37, 100), (16 * 5, 3), (4096 * 70 + 48, 0)])
def test_noalloc_ragged_counts_and_truncation(n, cap):
    """Flag counts that are not a multiple of the 4096-flag tile, and an
    output capacity below the number of set flags: the ids are the first
    `cap` set indices in ascending order, total counts them all, and every
    flag is cleared; two calls in a row reuse the static scratch."""
    import torch
    from paper_2309_04393_gb300 import ro
    rng = np.random.default_rng(n)
    for rep in range(2):
        density = 0.02 * (rep + 1) if n > 1000 else 0.4 + 0.2 * rep
        host = (rng.random(n) < density).astype(np.uint8) * rng.integers(1, 256, n).astype(np.uint8)
        flags = torch.from_numpy(host).to("cuda")
        ids = torch.full((max(cap, 1),), -1, dtype=torch.int32, device="cuda")
        total = torch.zeros(1, dtype=torch.int32, device="cuda")
        ro.compact_flags_noalloc(flags, ids[:cap] if cap else ids[:0], total)
        torch.cuda.synchronize()
        want = np.nonzero(host)[0]
        assert want.size > cap
        assert int(total.item()) == want.size
        got = ids.cpu().numpy()
        assert np.array_equal(got[:cap], want[:cap].astype(np.int32))
        if cap == 0:
            assert got[0] == -1
        assert int(flags.sum().item()) == 0
