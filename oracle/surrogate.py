"""FP64 oracle of the learned AOS surrogate.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU legs of ``bench.py`` may import it; the CUDA library never does.  It shares
no code with the CUDA kernels.

The surrogate is not part of the paper.  It stands in for one semi-implicit
AOS step (Eq. 4, Sec. II-B): given the previous level L, its conductance g
(Eq. 2-3) and the step tau = t_i - t_{i-1}, it predicts the next level.

Network contract (every choice below is a reading of the surrogate's
one-line specification -- four 3x3 convolutions, 32 channels, BF16 weights,
FP32 accumulation -- made concrete):

* per-pixel inputs x0 = (dx, dy, g, s, c):
  dx = 16 (L[y, x+1] - L[y, x]) (0 in the last column),
  dy = 16 (L[y+1, x] - L[y, x]) (0 in the last row),
  s = log(1 + tau) / 5 and c = 1; outside the image every input is zero, so
  c marks where the image ends.  The level enters through its differences
  only: the AOS step commutes with adding a constant to L (every row of the
  operator A_l of Eq. 4 sums to zero), and BF16 holds small differences
  precisely where it cannot resolve the step's changes on L itself;
* h1 = relu(conv(x0; W1, b1)), h2 = relu(conv(h1; W2, b2)),
  h3 = relu(conv(h2; W3, b3)), z = conv(h3; W4, b4), widths 5-32-32-32-1;
* conv(x; W, b)[p, o] = b[o] + sum_{dy,dx in -1..1} sum_i
  W[o, dy+1, dx+1, i] x[p + (dy, dx), i], with x = 0 outside the image;
* L_next = L + z / 256;
* loss = mean over all pixels of all samples of (L_next - T)^2.

Storage precision (``bf16=True``): the weights, every layer input (x0, h1,
h2, h3) and every back-propagated layer-output gradient (dz, dh3, dh2, dh1,
taken after the ReLU mask) are rounded to bfloat16, round to nearest even;
biases stay FP32.  Sums are exact here (FP64); the kernels accumulate in FP32.

Parameter vector layout (``PARAM_COUNT`` floats): for each layer in order,
W[out][3][3][in] then b[out].

Parity: pinned -- tests/test_oracle_surrogate.py checks bf16_round against
the bfloat16 conversion of torch, conv3x3 against scipy's 2-D correlation, the
forward pass against a hand-built network with a closed-form output, backward
against central finite differences, and adam against its closed form under a
constant gradient.
"""
from __future__ import annotations

import numpy as np

WIDTHS = (5, 32, 32, 32, 1)
OUT_SCALE = 1.0 / 256.0   # L_next = L + OUT_SCALE z
DIFF_SCALE = 16.0         # dx, dy = DIFF_SCALE x forward differences
LAYERS = 4


def layer_shapes():
    """[(W shape, b shape)] per layer."""
    return [((WIDTHS[l + 1], 3, 3, WIDTHS[l]), (WIDTHS[l + 1],)) for l in range(LAYERS)]


PARAM_COUNT = sum(int(np.prod(ws)) + int(np.prod(bs)) for ws, bs in layer_shapes())


def unpack(params):
    """Flat parameter vector -> [(W, b)] views in the contract's layout."""
    params = np.asarray(params, dtype=np.float64)
    if params.shape != (PARAM_COUNT,):
        raise ValueError("expected %d parameters" % PARAM_COUNT)
    out, o = [], 0
    for ws, bs in layer_shapes():
        nw, nb = int(np.prod(ws)), int(np.prod(bs))
        out.append((params[o:o + nw].reshape(ws), params[o + nw:o + nw + nb]))
        o += nw + nb
    return out


def pack(layers):
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in layers]).astype(np.float64)


def bf16_round(x):
    """Rounds to the nearest bfloat16 value (8 significant bits, ties to
    even); values stay float64."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)                       # x = m 2^e, 0.5 <= |m| < 1
    return np.ldexp(np.rint(m * 256.0), e - 8)  # np.rint rounds half to even


def conv3x3(x, W, b):
    """conv(x; W, b) of the contract.  x [n, h, w, in], W [out, 3, 3, in],
    b [out] -> [n, h, w, out]; zero padding."""
    n, h, w, _ = x.shape
    xp = np.zeros((n, h + 2, w + 2, x.shape[3]))
    xp[:, 1:h + 1, 1:w + 1, :] = x
    out = np.broadcast_to(np.asarray(b, dtype=np.float64), (n, h, w, W.shape[0])).copy()
    for ky in range(3):
        for kx in range(3):
            # tap (ky, kx) reads x at p + (ky - 1, kx - 1)
            out += np.einsum("nhwi,oi->nhwo", xp[:, ky:ky + h, kx:kx + w, :], W[:, ky, kx, :])
    return out


def conv3x3_dx(dz, W):
    """Gradient of sum(conv(x) * dz) with respect to x: every output pixel q
    sends W[:, tap] dz[q] back to x at q + offset(tap)."""
    n, h, w, _ = dz.shape
    dxp = np.zeros((n, h + 2, w + 2, W.shape[3]))
    for ky in range(3):
        for kx in range(3):
            dxp[:, ky:ky + h, kx:kx + w, :] += np.einsum("nhwo,oi->nhwi", dz, W[:, ky, kx, :])
    return dxp[:, 1:h + 1, 1:w + 1, :]


def conv3x3_dw(dz, x):
    """Gradients of sum(conv(x) * dz) with respect to W and b."""
    n, h, w, _ = x.shape
    xp = np.zeros((n, h + 2, w + 2, x.shape[3]))
    xp[:, 1:h + 1, 1:w + 1, :] = x
    dW = np.zeros((dz.shape[3], 3, 3, x.shape[3]))
    for ky in range(3):
        for kx in range(3):
            dW[:, ky, kx, :] = np.einsum("nhwo,nhwi->oi", dz, xp[:, ky:ky + h, kx:kx + w, :])
    return dW, dz.sum(axis=(0, 1, 2))


def features(L, g, tau):
    """x0 [n, h, w, 5] from L, g [n, h, w] and tau [n]."""
    L = np.asarray(L, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    s = np.log1p(np.asarray(tau, dtype=np.float64)) / 5.0
    x0 = np.zeros(L.shape + (5,))
    x0[:, :, :-1, 0] = DIFF_SCALE * (L[:, :, 1:] - L[:, :, :-1])
    x0[:, :-1, :, 1] = DIFF_SCALE * (L[:, 1:, :] - L[:, :-1, :])
    x0[..., 2] = g
    x0[..., 3] = s[:, None, None]
    x0[..., 4] = 1.0
    return x0


def forward(params, L, g, tau, bf16=True):
    """Returns (L_next [n, h, w], cache for backward)."""
    rnd = bf16_round if bf16 else (lambda a: a)
    layers = [(rnd(W), b) for W, b in unpack(params)]
    L = np.asarray(L, dtype=np.float64)
    a = rnd(features(L, g, tau))
    acts = [a]
    for l in range(LAYERS):
        W, b = layers[l]
        z = conv3x3(a, W, b)
        if l < LAYERS - 1:
            a = rnd(np.maximum(z, 0.0))
            acts.append(a)
        else:
            y = z[..., 0]
    return L + OUT_SCALE * y, {"layers": layers, "acts": acts, "bf16": bf16}


def loss(L_next, T):
    e = np.asarray(L_next, dtype=np.float64) - np.asarray(T, dtype=np.float64)
    return float(np.mean(e * e))


def backward(params, L, g, tau, T, bf16=True):
    """Returns (loss, gradient vector) of the contract's loss."""
    L_next, cache = forward(params, L, g, tau, bf16)
    rnd = bf16_round if bf16 else (lambda a: a)
    layers, acts = cache["layers"], cache["acts"]
    e = L_next - np.asarray(T, dtype=np.float64)
    dz = rnd((OUT_SCALE * 2.0 / e.size) * e)[..., None]   # dloss/dz, one channel
    grads = [None] * LAYERS
    for l in range(LAYERS - 1, -1, -1):
        W, _ = layers[l]
        grads[l] = conv3x3_dw(dz, acts[l])
        if l > 0:
            da = conv3x3_dx(dz, W)
            dz = rnd(da * (acts[l] > 0.0))       # ReLU of the layer below
    return float(np.mean(e * e)), pack(grads)


def adam(params, grad, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, 2015) with bias correction; step
    counts from 1.  Returns (params, m, v)."""
    m = b1 * np.asarray(m, dtype=np.float64) + (1.0 - b1) * grad
    v = b2 * np.asarray(v, dtype=np.float64) + (1.0 - b2) * grad * grad
    mhat = m / (1.0 - b1 ** step)
    vhat = v / (1.0 - b2 ** step)
    return np.asarray(params, dtype=np.float64) - lr * mhat / (np.sqrt(vhat) + eps), m, v


def training_pairs(levels, g_levels, taus):
    """(L_i, g_i, tau_i, L_{i+1}) for i = 0 .. N-2 of one evolved scale
    space: g_levels[i] is the conductance used to step levels[i] to
    levels[i+1] with step taus[i]."""
    return [(levels[i], g_levels[i], float(taus[i]), levels[i + 1]) for i in range(len(levels) - 1)]
