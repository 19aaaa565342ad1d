"""The compensator's CUDA kernels against its binary64 oracle: upsample,
forward pass and gradients within the binary32 tolerance of their sums (the
weights enter both sides as bfloat16 values), and training steps lowering
the loss."""
import numpy as np
import pytest

from oracle import compensator as omc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mc():
    import torch
    assert torch.cuda.is_available(), "these tests need a CUDA GPU"
    from paper_2309_04393_gb300 import build, mc as mcmod
    build.build()
    return mcmod, mcmod.Compensator(4)


def rounded(params):
    return [(omc.bf16(W), b) for W, b in params]


def test_upsample_matches_oracle(mc):
    import torch
    mcmod, m = mc
    rng = np.random.default_rng(1)
    slots = rng.integers(0, 65536, (3, 34, 34, 34)).astype(np.uint16)
    octs = [(0, 0, 0), (1, 0, 1), (1, 1, 1)]
    codes = np.array([o[0] | (o[1] << 1) | (o[2] << 2) for o in octs], np.int32)
    x0 = m.upsample(torch.from_numpy(slots.view(np.int16)).cuda(), torch.from_numpy(codes).cuda()).cpu().numpy()
    for k, o in enumerate(octs):
        want = omc.upsample(slots[k], o) / 65536.0
        assert np.abs(x0[k] - want).max() <= 2e-7


def test_forward_and_gradients_match_oracle(mc):
    import torch
    mcmod, m = mc
    rng = np.random.default_rng(2)
    params = [(W * 3.0, rng.normal(0, 0.05, b.shape)) for W, b in omc.init_params(4)]
    m.set_params(params)
    x0 = rng.uniform(0.0, 1.0, (2, 34, 34, 34))
    target = np.clip(x0 + rng.normal(0.0, 0.05, x0.shape), 0, 1)
    tx, tt = torch.from_numpy(x0.astype(np.float32)).cuda(), torch.from_numpy(target.astype(np.float32)).cuda()
    y = m.forward(tx).cpu().numpy()
    q = rounded([(W.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64))
                 for W, b in params])
    x0f = x0.astype(np.float32).astype(np.float64)
    for k in range(2):
        want, _ = omc.forward(q, x0f[k], bf16_inputs=(0, 1, 2, 3))
        err = np.abs(y[k] - want)
        # binary32 sums agree to ~1e-7; where an activation lies within a
        # binary32 step of a bfloat16 rounding boundary the two sides round
        # it one bfloat16 step apart, which moves the 27 neighbours of the
        # next layer by about |w| * |a| * 2^-8 and spreads from there (the
        # last layer's input is rounded too, so a flip there reaches y
        # directly).  The oracle against itself with binary32-sized noise
        # (2^-23) on every layer input gives median 0, 99 % 3.8e-4, 99.9 %
        # 1.0e-3, max 2.5e-3 on these inputs (and 99 % 4.7e-4, max 3.6e-3 on
        # the 32-grid test's): the bounds below sit about 2x above that
        assert np.median(err) <= 1e-6
        assert np.quantile(err, 0.99) <= 1e-3
        assert err.max() <= 7.5e-3 * max(1.0, np.abs(want).max())
    g, loss = m.gradients(tx, tt)
    g = g.cpu().numpy()
    tf = target.astype(np.float32).astype(np.float64)
    # the oracle's loss over both grids: the mean of the per-grid means
    losses, grads = zip(*[omc.loss_and_grads(q, x0f[k], tf[k], bf16_inputs=(0, 1, 2, 3)) for k in range(2)])
    want_loss = sum(losses) / 2
    assert abs(float(loss.item()) - want_loss) <= 1e-4 * want_loss
    # the oracle mirrors the GPU's rounding of the output gradients entering
    # every layer's tensor-core weight- and input-gradient products
    losses, grads = zip(*[omc.loss_and_grads(q, x0f[k], tf[k], bf16_inputs=(0, 1, 2, 3), bf16_grads=(0, 1, 2, 3))
                          for k in range(2)])
    want = [(sum(gr[i][0] for gr in grads) / 2, sum(gr[i][1] for gr in grads) / 2) for i in range(4)]
    got = mcmod.unflatten(g.astype(np.float64))
    # per layer, weights and biases apart: binary32 sums in another order,
    # and the rare bfloat16 flips of the forward pass, stay far below 1e-3 of
    # each part's largest gradient (a dropped tap or term does not)
    for i in range(4):
        for part in (0, 1):
            scale = np.abs(want[i][part]).max()
            rel = np.abs(got[i][part] - want[i][part]).max() / scale
            assert rel <= 1e-3, f"layer {i} {'weights' if part == 0 else 'biases'}: {rel:.2e} of the largest"


def test_adam_steps_match_oracle(mc):
    """Three Adam steps on fixed gradients (ro_mc_apply_gradients) against
    the oracle's Algorithm 1 in binary64: parameters and both moment
    estimates element by element, within the rounding of binary32 updates."""
    import torch
    mcmod, m = mc
    rng = np.random.default_rng(12)
    p0 = rng.normal(0.0, 0.1, mcmod.PARAMS).astype(np.float32)
    m.set_params(p0)
    lr = 1e-3
    P, M, V = p0.astype(np.float64), np.zeros(mcmod.PARAMS), np.zeros(mcmod.PARAMS)
    S = np.zeros(mcmod.PARAMS)   # the first moment's recursion on magnitudes: its terms' size
    for t in range(1, 4):
        g = (rng.normal(0.0, 1.0, mcmod.PARAMS) * 10.0 ** rng.uniform(-6, 1, mcmod.PARAMS)).astype(np.float32)
        g[rng.integers(0, mcmod.PARAMS, 100)] = 0.0
        m.apply_gradients(torch.from_numpy(g).cuda(), lr)
        P, M, V = omc.adam_step(P, g.astype(np.float64), M, V, t, lr)
        S = 0.9 * S + 0.1 * np.abs(g.astype(np.float64))
        gp = m.get_params().astype(np.float64)
        gm, gv, step = m.get_moments()
        assert step == t
        # m can cancel (gradients of opposite signs): bound it by its terms
        assert np.all(np.abs(gm - M) <= 1e-6 * S + 1e-30)
        assert np.all(np.abs(gv - V) <= 1e-6 * np.abs(V) + 1e-30)
        assert np.all(np.abs(gp - P) <= 4e-7 * np.abs(P) + 1e-5 * lr)
    # train_step takes the same path after its own gradients: the step count goes on
    x0 = torch.rand((1, 34, 34, 34), device="cuda")
    m.train_step(x0, x0, lr)
    assert m.get_moments()[2] == 4


def test_training_lowers_the_loss(mc):
    import torch
    mcmod, m = mc
    rng = np.random.default_rng(3)
    m.set_params(omc.init_params(5))
    z, y, x = np.meshgrid(np.arange(34), np.arange(34), np.arange(34), indexing="ij")
    base = 0.3 + 0.2 * np.sin(x / 5.0) * np.cos(y / 7.0) + 0.1 * np.sin(z / 3.0)
    x0 = np.stack([base + 0.02 * rng.normal(size=base.shape) for _ in range(4)])
    target = 0.8 * x0 + 0.1                     # a function of the input the network can learn
    tx, tt = torch.from_numpy(x0.astype(np.float32)).cuda(), torch.from_numpy(target.astype(np.float32)).cuda()
    loss = torch.zeros(1, device="cuda")
    first = None
    for step in range(40):
        m.train_step(tx, tt, 2e-3, loss)
        if first is None:
            first = float(loss.item())
    last = float(loss.item())
    assert last < 0.5 * first


def test_compensate_bricks_writes_the_predictions_into_the_cache(mc):
    import torch
    from paper_2309_04393_gb300 import loader, ro
    from synth import recipes
    mcmod, m = mc
    m.set_params(omc.init_params(7))
    scene = recipes.cells_slab(m=2, dims=(128, 128, 64), ncells=300, k=3, W=64, H=64, n_views=1, resident_l0=0.5)
    d = ro.make_desc(scene.dims, scene.spacing, scene.m, scene.value_bits, scene.B, scene.k, scene.leaf,
                     len(scene.all_bricks()), max_upload=64)
    ctx = ro.Context(d)
    loader.load_scene(ctx, scene)
    res = set(scene.resident)
    missing = [b for b in scene.all_bricks(levels=[0]) if b not in res][:4]
    assert len(missing) == 4
    ids = [ro.brick_id(c, 0, bx, by, bz, scene.k) for (c, l, bx, by, bz) in missing]
    slots = mcmod.compensate_bricks(ctx, m, ids)
    pt = ctx.debug_read(1)
    for i, s in zip(ids, slots):
        assert pt[ctx.brick_index(i)] == s + 1
    cache = ctx.debug_read(5).reshape(int(d.cache_slots), -1)
    # expected: the network on the parents' upsampled slots, to raw values
    parents = np.stack([scene.bricks(np.array([[c, 1, bx // 2, by // 2, bz // 2]], np.int32))[0]
                        for (c, l, bx, by, bz) in missing])
    octs = np.array([(bx & 1) | ((by & 1) << 1) | ((bz & 1) << 2) for (c, l, bx, by, bz) in missing], np.int32)
    x0 = m.upsample(torch.from_numpy(parents.view(np.int16)).cuda(), torch.from_numpy(octs).cuda())
    y = m.forward(x0).cpu().numpy()
    want = np.clip(np.rint(y * 65536.0), 0, 65535).astype(np.uint16)
    for k, s in enumerate(slots):
        got = cache[s, :34 ** 3 * 2].view(np.uint16).reshape(34, 34, 34)
        assert np.array_equal(got, want[k])
    with pytest.raises(ro.RoError):                              # already resident now
        mcmod.compensate_bricks(ctx, m, ids[:1])
    with pytest.raises(ro.RoError):                              # a level-1 id
        mcmod.compensate_bricks(ctx, m, [ro.brick_id(0, 1, 0, 0, 0, scene.k)])
    img, _ = ro.render_frame(ctx, scene.frames[0])               # the context still renders
    assert float(img[..., 3].max()) > 0


def test_full_batch_matches_oracle_samples_and_per_grid_gradients(mc):
    """The training batch of the bench (32 grids, the launch configuration
    it times): sampled grids of the forward pass against the oracle, and the
    batch gradient against the mean of the 32 one-grid gradients (the loss
    is a mean over the batch, so this holds at any size; it checks how the
    weight-gradient kernels share a batch between blocks)."""
    import torch
    mcmod, _ = mc
    n = 32
    big = mcmod.Compensator(n)
    try:
        rng = np.random.default_rng(11)
        params = [(W * 3.0, rng.normal(0, 0.05, b.shape)) for W, b in omc.init_params(6)]
        big.set_params(params)
        x0 = rng.uniform(0.0, 1.0, (n, 34, 34, 34))
        target = np.clip(x0 + rng.normal(0.0, 0.05, x0.shape), 0, 1)
        tx = torch.from_numpy(x0.astype(np.float32)).cuda()
        tt = torch.from_numpy(target.astype(np.float32)).cuda()
        y = big.forward(tx).cpu().numpy()
        q = rounded([(W.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64))
                     for W, b in params])
        x0f = x0.astype(np.float32).astype(np.float64)
        for k in (0, 17, n - 1):
            want, _ = omc.forward(q, x0f[k], bf16_inputs=(0, 1, 2, 3))
            err = np.abs(y[k] - want)
            # bounds of the two-grid forward test (bfloat16 rounding flips)
            assert np.median(err) <= 1e-6
            assert np.quantile(err, 0.99) <= 1e-3
            assert err.max() <= 7.5e-3 * max(1.0, np.abs(want).max())
        g, loss = big.gradients(tx, tt)
        g = g.cpu().numpy().astype(np.float64)
        mean_g = np.zeros_like(g)
        mean_loss = 0.0
        for k in range(n):
            gk, lk = big.gradients(tx[k:k + 1], tt[k:k + 1])
            mean_g += gk.cpu().numpy().astype(np.float64) / n
            mean_loss += float(lk.item()) / n
        # the per-grid terms are the same binary32 / bfloat16 values scaled by
        # 2^-5 (exact); only the order of the binary32 sums differs
        assert abs(float(loss.item()) - mean_loss) <= 1e-5 * mean_loss
        assert np.abs(g - mean_g).max() <= 1e-4 * np.abs(mean_g).max()
    finally:
        big.close()
