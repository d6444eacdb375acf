"""Pins of the FP64 surrogate oracle (oracle/surrogate.py) to facts outside
itself: torch's bfloat16 conversion, scipy's 2-D correlation, a hand-built
network with a closed-form output, central finite differences, the adjoint
identity of a convolution, Adam's closed form under a constant gradient, and
the AOS step (Eq. 4) that the training pairs must reproduce."""
import numpy as np
import pytest

from oracle import surrogate as so


def _rng(seed):
    return np.random.default_rng(seed)


def test_param_count_and_layout():
    # widths 5-32-32-32-1 with 3x3 kernels and biases
    assert so.PARAM_COUNT == 32 * 9 * 5 + 32 + 32 * 9 * 32 + 32 + 32 * 9 * 32 + 32 + 1 * 9 * 32 + 1
    p = np.arange(so.PARAM_COUNT, dtype=np.float64)
    np.testing.assert_array_equal(so.pack(so.unpack(p)), p)
    (W1, b1), *_ = so.unpack(p)
    assert W1.shape == (32, 3, 3, 5) and b1[0] == 32 * 9 * 5


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    r = _rng(1)
    x = np.concatenate([
        r.standard_normal(20000) * np.exp(r.uniform(-30, 30, 20000)),
        # exact ties: 8 significant bits plus a half unit of the 9th
        (256 + np.arange(-64, 64) * 2 + 1) / 512.0 * 2.0 ** r.integers(-20, 20, 128),
        [0.0, -0.0, 1.0, -1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, 65504.0],
    ]).astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    got = so.bf16_round(x.astype(np.float64))
    np.testing.assert_array_equal(got, want)


def test_conv3x3_matches_scipy_correlation():
    signal = pytest.importorskip("scipy.signal")
    r = _rng(2)
    x = r.standard_normal((2, 5, 7, 3))
    W = r.standard_normal((4, 3, 3, 3))
    b = r.standard_normal(4)
    got = so.conv3x3(x, W, b)
    for n in range(2):
        for o in range(4):
            want = b[o] + sum(
                signal.correlate2d(x[n, :, :, i], W[o, :, :, i], mode="same", boundary="fill", fillvalue=0)
                for i in range(3))
            np.testing.assert_allclose(got[n, :, :, o], want, rtol=0, atol=1e-12)


def test_conv_backward_is_the_adjoint():
    r = _rng(3)
    x = r.standard_normal((2, 6, 5, 3))
    W = r.standard_normal((4, 3, 3, 3))
    dz = r.standard_normal((2, 6, 5, 4))
    zero = np.zeros(4)
    # <conv(x), dz> = <x, conv_dx(dz)>
    lhs = np.sum(so.conv3x3(x, W, zero) * dz)
    assert abs(lhs - np.sum(x * so.conv3x3_dx(dz, W))) < 1e-10 * max(1.0, abs(lhs))
    # the map is linear in W: its derivative along a unit weight is exact
    dW, db = so.conv3x3_dw(dz, x)
    for (o, ky, kx, i) in [(0, 0, 0, 0), (3, 2, 1, 2), (1, 1, 2, 0), (2, 0, 2, 1)]:
        E = np.zeros_like(W)
        E[o, ky, kx, i] = 1.0
        assert abs(np.sum(so.conv3x3(x, E, zero) * dz) - dW[o, ky, kx, i]) < 1e-10
    np.testing.assert_allclose(db, dz.sum(axis=(0, 1, 2)), atol=1e-12)


def _hand_built_params(alpha, beta, gamma, delta, eps, bias):
    """A network whose raw output is z = alpha dx(y, x+1) - beta dy(y-1, x)
    + gamma g + delta s + eps c + bias, with zero outside the image: the
    signed differences pass the ReLUs as positive and negative parts."""
    layers = [(np.zeros(ws), np.zeros(bs)) for ws, bs in so.layer_shapes()]
    W1 = layers[0][0]
    W1[0, 1, 1, 0], W1[1, 1, 1, 0] = 1.0, -1.0   # dx+, dx-
    W1[2, 1, 1, 1], W1[3, 1, 1, 1] = 1.0, -1.0   # dy+, dy-
    W1[4, 1, 1, 2] = W1[5, 1, 1, 3] = W1[6, 1, 1, 4] = 1.0  # g, s, c
    for l in (1, 2):
        for ch in range(7):
            layers[l][0][ch, 1, 1, ch] = 1.0
    W4, b4 = layers[3]
    W4[0, 1, 2, 0], W4[0, 1, 2, 1] = alpha, -alpha     # tap (dy, dx) = (0, +1)
    W4[0, 0, 1, 2], W4[0, 0, 1, 3] = -beta, beta       # tap (dy, dx) = (-1, 0)
    W4[0, 1, 1, 4] = gamma
    W4[0, 1, 1, 5] = delta
    W4[0, 1, 1, 6] = eps
    b4[0] = bias
    return so.pack(layers)


@pytest.mark.parametrize("bf16", [False, True])
def test_forward_matches_closed_form(bf16):
    r = _rng(4)
    n, h, w = 2, 6, 9
    L = r.uniform(0, 1, (n, h, w))
    g = r.uniform(0.05, 1, (n, h, w))
    tau = np.array([0.7, 12.5])
    a, b_, c, d, e, bias = 0.5, 0.25, 0.125, 2.0, -0.75, 0.0625
    p = _hand_built_params(a, b_, c, d, e, bias)
    got, _ = so.forward(p, L, g, tau, bf16=bf16)
    q = so.bf16_round if bf16 else (lambda v: v)
    dx = np.zeros_like(L)
    dx[:, :, :-1] = q(16.0 * (L[:, :, 1:] - L[:, :, :-1]))
    dy = np.zeros_like(L)
    dy[:, :-1, :] = q(16.0 * (L[:, 1:, :] - L[:, :-1, :]))
    gq, sq = q(g), q(np.log1p(tau) / 5.0)
    right = np.zeros_like(L)          # dx at (y, x + 1)
    right[:, :, :-1] = dx[:, :, 1:]
    up = np.zeros_like(L)             # dy at (y - 1, x)
    up[:, 1:, :] = dy[:, :-1, :]
    z = a * right - b_ * up + c * gq + d * sq[:, None, None] + e + bias
    np.testing.assert_allclose(got, L + z / 256.0, rtol=0, atol=1e-14)


def test_constant_offset_leaves_the_step_unchanged():
    # the inputs see L only through its differences, like the AOS step
    r = _rng(9)
    L = r.uniform(0, 0.5, (2, 7, 8))
    g = r.uniform(0.1, 1, (2, 7, 8))
    p = _random_params(10)
    a, _ = so.forward(p, L, g, [1.0, 3.0], bf16=False)
    b, _ = so.forward(p, L + 0.25, g, [1.0, 3.0], bf16=False)
    np.testing.assert_allclose(b - 0.25, a, rtol=0, atol=1e-13)


def _random_params(seed, scale=1.0):
    r = _rng(seed)
    layers = []
    for ws, bs in so.layer_shapes():
        fan_in = ws[1] * ws[2] * ws[3]
        layers.append((r.standard_normal(ws) * scale * np.sqrt(2.0 / fan_in), r.standard_normal(bs) * 0.1))
    return so.pack(layers)


def test_backward_matches_finite_differences():
    r = _rng(5)
    n, h, w = 2, 5, 6
    L = r.uniform(0, 1, (n, h, w))
    g = r.uniform(0.05, 1, (n, h, w))
    tau = np.array([1.5, 30.0])
    T = L + 0.1 * r.standard_normal((n, h, w))
    p = _random_params(6)
    f0, grad = so.backward(p, L, g, tau, T, bf16=False)
    assert abs(f0 - so.loss(so.forward(p, L, g, tau, bf16=False)[0], T)) < 1e-15
    # sample entries of every weight and bias block
    idx, o = [], 0
    for ws, bs in so.layer_shapes():
        nw, nb = int(np.prod(ws)), int(np.prod(bs))
        idx += list(o + r.choice(nw, 12, replace=False)) + list(o + nw + r.choice(nb, min(nb, 4), replace=False))
        o += nw + nb
    hstep = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += hstep
        pm[i] -= hstep
        fd = (so.loss(so.forward(pp, L, g, tau, bf16=False)[0], T)
              - so.loss(so.forward(pm, L, g, tau, bf16=False)[0], T)) / (2 * hstep)
        assert abs(fd - grad[i]) <= 1e-6 * max(1e-3, abs(grad[i])), (i, fd, grad[i])


def test_loss_is_the_mean_square():
    r = _rng(7)
    a = r.standard_normal((2, 3, 4))
    b = r.standard_normal((2, 3, 4))
    s = 0.0
    for i in range(2):
        for y in range(3):
            for x in range(4):
                s += (a[i, y, x] - b[i, y, x]) ** 2
    assert abs(so.loss(a, b) - s / 24) < 1e-15
    assert so.loss(a, a) == 0.0


def test_adam_closed_form_under_constant_gradient():
    r = _rng(8)
    p0 = r.standard_normal(50)
    g = r.standard_normal(50)
    lr, eps = 1e-2, 1e-8
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    for k in range(1, 6):
        p, m, v = so.adam(p, g, m, v, k, lr, eps=eps)
        # bias-corrected moments equal g and g^2 exactly: each step moves
        # every parameter by lr g / (|g| + eps)
        np.testing.assert_allclose(p, p0 - k * lr * g / (np.abs(g) + eps), rtol=0, atol=1e-12)


def test_training_pairs_reproduce_the_aos_step(oracle_mod):
    from paper_1706_06750_gb300 import synth
    img = synth.image(48, 40, 5000)
    opt = oracle_mod.Options.make(octaves=2, sublevels=2)
    levels, k = oracle_mod.build_scale_space(img, opt)
    _, t = oracle_mod.scale_table(2, 2, 1.6)
    g = [oracle_mod.conductance(levels[i], k) for i in range(len(levels) - 1)]
    pairs = so.training_pairs(levels, g, np.diff(t))
    assert len(pairs) == 3
    for Li, gi, taui, Lj in pairs:
        np.testing.assert_allclose(oracle_mod.aos_step(Li, gi, taui)[2], Lj, rtol=0, atol=1e-13)
