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
        want, _ = omc.forward(q, x0f[k])
        assert np.abs(y[k] - want).max() <= 2e-4 * max(1.0, np.abs(want).max())
    g, loss = m.gradients(tx, tt)
    g = g.cpu().numpy()
    tf = target.astype(np.float32).astype(np.float64)
    # the oracle's loss over both grids: the mean of the per-grid means
    losses, grads = zip(*[omc.loss_and_grads(q, x0f[k], tf[k]) for k in range(2)])
    want_loss = sum(losses) / 2
    assert abs(float(loss.item()) - want_loss) <= 1e-4 * want_loss
    want_g = mcmod.flatten([(sum(gr[i][0] for gr in grads) / 2, sum(gr[i][1] for gr in grads) / 2)
                            for i in range(4)]).astype(np.float64)
    scale = np.abs(want_g).max()
    assert np.abs(g - want_g).max() <= 1e-3 * scale


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
