"""Pins of the compensator oracle: the upsample reproduces linear fields
exactly (trilinear interpolation is exact on them) and constants; the
convolution of an identity or a one-tap shift kernel is the input itself or
the shifted input with zero fill; the hand-written gradients match finite
differences of the loss; random asymmetric weights match scipy's
cross-correlation and the input gradient is the convolution's adjoint;
bfloat16 rounding at exact ties goes to even."""
import numpy as np
import pytest

from oracle import compensator as mc


@pytest.mark.parametrize("octant", [(0, 0, 0), (1, 0, 1), (1, 1, 1)])
def test_upsample_reproduces_linear_fields(octant):
    z, y, x = np.meshgrid(np.arange(34), np.arange(34), np.arange(34), indexing="ij")
    a, bx, by, bz = 1000.0, 3.0, -2.0, 5.0
    slot = a + bx * (x - 1) + by * (y - 1) + bz * (z - 1)          # level-1 voxel u = slot index - 1
    up = mc.upsample(slot, octant)
    X = np.arange(34) - 1 + 32 * np.array(octant)[:, None]          # per axis (x, y, z)
    u = (X + 0.5) / 2 - 0.5
    want = a + bx * u[0][None, None, :] + by * u[1][None, :, None] + bz * u[2][:, None, None]
    assert np.allclose(up, want, rtol=0, atol=1e-9)
    assert np.allclose(mc.upsample(np.full((34, 34, 34), 77.0), octant), 77.0, atol=0)


def test_conv_identity_and_shift_kernels():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(5, 6, 7, 3))
    W = np.zeros((27, 3, 3))
    W[13] = np.eye(3)                                               # centre tap
    b = np.array([0.5, -1.0, 2.0])
    assert np.allclose(mc.conv3(x, W, b), x + b, atol=1e-12)
    W = np.zeros((27, 3, 3))
    W[(2 * 3 + 1) * 3 + 1] = np.eye(3)                              # tap dz = +1: out[z] = x[z + 1]
    out = mc.conv3(x, W, np.zeros(3))
    assert np.allclose(out[:-1], x[1:], atol=1e-12) and np.all(out[-1] == 0)


def test_conv_matches_scipy_correlate_for_asymmetric_weights():
    """Random, non-symmetric weights against scipy's n-d cross-correlation
    with zero fill: a transposed weight index or a swapped tap axis fails
    here (the identity and shift kernels above are symmetric in both)."""
    from scipy import ndimage
    rng = np.random.default_rng(4)
    x = rng.normal(size=(5, 6, 7, 2))
    W = rng.normal(size=(27, 2, 3))
    b = rng.normal(size=3)
    out = mc.conv3(x, W, b)
    for co in range(3):
        want = np.full(x.shape[:3], b[co])
        for ci in range(2):
            # tap (dz * 3 + dy) * 3 + dx reads the input at offset (dz-1, dy-1, dx-1)
            K = W[:, ci, co].reshape(3, 3, 3)
            want += ndimage.correlate(x[..., ci], K, mode="constant", cval=0.0)
        assert np.allclose(out[..., co], want, rtol=0, atol=1e-12)
    # the input gradient is the adjoint of the convolution: <conv(x), g> = <x, conv^T(g)>
    g = rng.normal(size=(5, 6, 7, 3))
    dx, dW, db = mc.conv3_backward(x, W, g)
    lhs = float(np.sum((mc.conv3(x, W, np.zeros(3))) * g))
    assert abs(lhs - float(np.sum(x * dx))) <= 1e-9 * max(1.0, abs(lhs))
    assert np.allclose(db, g.sum(axis=(0, 1, 2)), atol=1e-12)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(2)
    params = [(W * 30.0, rng.normal(0, 0.05, b.shape)) for W, b in mc.init_params(3)]
    x0 = rng.uniform(0.0, 1.0, (4, 5, 4))
    target = x0 + rng.normal(0.0, 0.1, x0.shape)
    loss, grads = mc.loss_and_grads(params, x0, target)
    h = 1e-6
    for li in range(4):
        W, b = params[li]
        for _ in range(6):
            t, ci, co = rng.integers(27), rng.integers(W.shape[1]), rng.integers(W.shape[2])
            for s in (+1, -1):
                Wp = W.copy()
                Wp[t, ci, co] += s * h
                p2 = list(params)
                p2[li] = (Wp, b)
                if s > 0:
                    lp = mc.loss_and_grads(p2, x0, target)[0]
                else:
                    lm = mc.loss_and_grads(p2, x0, target)[0]
            num = (lp - lm) / (2 * h)
            assert abs(num - grads[li][0][t, ci, co]) <= 1e-6 + 1e-4 * abs(num)
        co = rng.integers(b.shape[0])
        bp, bm = b.copy(), b.copy()
        bp[co] += h
        bm[co] -= h
        p2, p3 = list(params), list(params)
        p2[li], p3[li] = (W, bp), (W, bm)
        num = (mc.loss_and_grads(p2, x0, target)[0] - mc.loss_and_grads(p3, x0, target)[0]) / (2 * h)
        assert abs(num - grads[li][1][co]) <= 1e-6 + 1e-4 * abs(num)


def test_bf16_ties_to_even():
    assert mc.bf16(1.0 + 2.0 ** -8) == 1.0                         # halfway, to even
    assert mc.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6          # halfway, to even (up)
    assert mc.bf16(1.0 + 2.0 ** -8 + 2.0 ** -20) == 1.0 + 2.0 ** -7  # above halfway


def test_bf16_gradient_rounding_bound():
    """The bfloat16 rounding of the output gradients of layers 1 and 2 moves
    each of their weight gradients by at most the unit roundoff 2^-8 times
    sum(|input| * |gradient|) over the voxels and taps that enter it; the
    bias gradients and the first and last layers' gradients only change
    through the rounded gradient that flows further down."""
    rng = np.random.default_rng(6)
    params = [(W * 3.0, rng.normal(0, 0.05, b.shape)) for W, b in mc.init_params(5)]
    params = [(mc.bf16(W), b) for W, b in params]
    x0 = rng.uniform(0.0, 1.0, (6, 5, 7))
    target = np.clip(x0 + rng.normal(0.0, 0.05, x0.shape), 0, 1)
    _, exact = mc.loss_and_grads(params, x0, target, bf16_inputs=(1, 2))
    _, rounded = mc.loss_and_grads(params, x0, target, bf16_inputs=(1, 2), bf16_grads=(2,))
    # only layer 2's own products use the rounded gradient: its bias
    # gradient and layer 3's gradients are unchanged
    assert np.array_equal(rounded[3][0], exact[3][0]) and np.array_equal(rounded[3][1], exact[3][1])
    assert np.array_equal(rounded[2][1], exact[2][1])
    # bound for layer 2's weight gradient from |bf16(g) - g| <= 2^-8 |g|
    y, acts = mc.forward(params, x0, bf16_inputs=(1, 2))
    g = (2.0 / y.size) * (y - target)[..., None]
    for i in (2,):
        g = mc.conv3_backward(acts[i + 1], params[i + 1][0], g)[0] * (acts[i + 1] > 0.0)
    _, bound, _ = mc.conv3_backward(np.abs(acts[2]), np.abs(params[2][0]), np.abs(g))
    diff = np.abs(rounded[2][0] - exact[2][0])
    assert np.all(diff <= 2.0 ** -8 * bound + 1e-18)
    assert diff.max() > 0.0
    _, both = mc.loss_and_grads(params, x0, target, bf16_inputs=(1, 2), bf16_grads=(1, 2))
    assert not np.array_equal(both[1][0], rounded[1][0]) and np.array_equal(both[2][0], rounded[2][0])


@pytest.mark.parametrize("g", [0.3, -2.0e3, 1.0e-9])
def test_adam_constant_gradient_closed_form(g):
    """With one constant gradient g the bias-corrected moments are exactly g
    and g^2 at every step, so every step moves the parameter by
    -lr * g / (|g| + eps): lr * sign(g) for |g| >> eps, lr / 11 at g = 1e-9
    (eps = 1e-8 added to the root, not under it)."""
    lr, eps = 0.01, 1e-8
    p, m, v = np.array([0.25]), np.zeros(1), np.zeros(1)
    for t in range(1, 11):
        p_new, m, v = mc.adam_step(p, np.array([g]), m, v, t, lr)
        step = lr * g / (abs(g) + eps)
        assert abs((p - p_new)[0] - step) <= 1e-12 * max(1.0, abs(step))
        p = p_new
    if g == 1.0e-9:
        assert abs(step - lr / 11.0) < 1e-15


def test_adam_weighted_average_form():
    """After t steps the bias-corrected moments are weighted means of the
    gradients so far, m_hat = sum beta1^(t-i) g_i / sum beta1^(t-i) (and v_hat
    of g_i^2 with beta2): the parameter trajectory written from that explicit
    form equals the recursion's."""
    rng = np.random.default_rng(8)
    lr, b1, b2, eps = 0.003, 0.9, 0.999, 1e-8
    G = rng.normal(0.0, 1.0, (7, 5)) * np.array([1e-3, 1.0, 50.0, 1e-6, 3.0])
    p0 = rng.normal(size=5)
    p, m, v = p0.copy(), np.zeros(5), np.zeros(5)
    want = p0.copy()
    for t in range(1, 8):
        p, m, v = mc.adam_step(p, G[t - 1], m, v, t, lr)
        w1 = b1 ** np.arange(t - 1, -1, -1)
        w2 = b2 ** np.arange(t - 1, -1, -1)
        m_hat = (w1[:, None] * G[:t]).sum(0) / w1.sum()
        v_hat = (w2[:, None] * G[:t] ** 2).sum(0) / w2.sum()
        want = want - lr * m_hat / (np.sqrt(v_hat) + eps)
        assert np.allclose(p, want, rtol=0, atol=1e-12)
        # the moments themselves are the unnormalised sums
        assert np.allclose(m, (1 - b1) * (w1[:, None] * G[:t]).sum(0), rtol=1e-12, atol=0)
        assert np.allclose(v, (1 - b2) * (w2[:, None] * G[:t] ** 2).sum(0), rtol=1e-12, atol=0)


def test_adam_is_invariant_to_gradient_scale():
    rng = np.random.default_rng(9)
    G = rng.normal(size=(5, 4))
    runs = []
    for scale in (1.0, 1000.0):
        p, m, v = np.ones(4), np.zeros(4), np.zeros(4)
        for t in range(1, 6):
            p, m, v = mc.adam_step(p, scale * G[t - 1], m, v, t, 0.01)
        runs.append(p)
    assert np.allclose(runs[0], runs[1], rtol=0, atol=1e-9)
