"""Pins of the oracle's Thomas solver and AOS step (CPU only).

What the method fixes, independent of the oracle's code: the solve equals a
dense library solve of the system built from its definition; constant images
are fixed points; Neumann borders preserve the mean; constant conductance is
linear implicit diffusion with a DCT-II closed form; the maximum principle;
and the first-order agreement with one explicit diffusion step.
"""
import numpy as np
import pytest
from scipy import fft as sfft


def _random_tridiag(rng, n):
    a = -rng.random(n)
    c = -rng.random(n)
    a[0] = 0.0
    c[-1] = 0.0
    b = 1.0 + np.abs(a) + np.abs(c) + rng.random(n)
    return a, b, c


@pytest.mark.parametrize("n", [1, 2, 3, 17, 64])
def test_thomas_matches_dense_solve(oracle_mod, n):
    rng = np.random.default_rng(n)
    a, b, c = _random_tridiag(rng, n)
    d = rng.standard_normal(n)
    M = np.diag(b) + np.diag(a[1:], -1) + np.diag(c[:-1], 1)
    ref = np.linalg.solve(M, d)
    got = oracle_mod.thomas(a, b, c, d)
    assert np.max(np.abs(got - ref)) < 1e-12


def _aos_dense(L, g, tau):
    """AOS from its definition with dense matrices and numpy.linalg.solve."""
    h, w = L.shape

    def line(gl, dl):
        n = gl.size
        B = np.eye(n)
        for j in range(n - 1):
            wgt = 0.5 * (gl[j] + gl[j + 1])
            B[j, j + 1] -= 2 * tau * wgt
            B[j + 1, j] -= 2 * tau * wgt
            B[j, j] += 2 * tau * wgt
            B[j + 1, j + 1] += 2 * tau * wgt
        return np.linalg.solve(B, dl)

    ux = np.stack([line(g[y], L[y]) for y in range(h)])
    uy = np.stack([line(g[:, x], L[:, x]) for x in range(w)], axis=1)
    return ux, uy, 0.5 * (ux + uy)


@pytest.mark.parametrize("shape", [(8, 6), (5, 9), (1, 7), (6, 1)])
def test_aos_matches_dense_brute_force(oracle_mod, shape):
    rng = np.random.default_rng(7)
    L = rng.random(shape)
    g = 0.05 + rng.random(shape)
    for tau in (0.1, 3.7, 60.0):
        ux, uy, ln = oracle_mod.aos_step(L, g, tau)
        rx, ry, rl = _aos_dense(L, g, tau)
        assert np.max(np.abs(ux - rx)) < 1e-12
        assert np.max(np.abs(uy - ry)) < 1e-12
        assert np.max(np.abs(ln - rl)) < 1e-12


def test_aos_constant_image_is_fixed_point(oracle_mod):
    rng = np.random.default_rng(8)
    L = np.full((12, 15), 0.42)
    g = rng.random((12, 15))
    _, _, ln = oracle_mod.aos_step(L, g, 25.0)
    assert np.max(np.abs(ln - 0.42)) < 1e-14


def test_aos_preserves_line_sums_and_mean(oracle_mod):
    rng = np.random.default_rng(9)
    L = rng.random((20, 31))
    g = rng.random((20, 31))
    ux, uy, ln = oracle_mod.aos_step(L, g, 12.0)
    assert np.max(np.abs(ux.sum(axis=1) - L.sum(axis=1))) < 1e-11
    assert np.max(np.abs(uy.sum(axis=0) - L.sum(axis=0))) < 1e-11
    assert abs(ln.sum() - L.sum()) < 1e-10 * L.size


def test_aos_constant_conductance_is_linear_implicit_diffusion(oracle_mod):
    # With g = gamma everywhere each line operator is I - 2 tau gamma Lap_N,
    # diagonalised by the DCT-II with eigenvalues 1 + 8 tau gamma sin^2(pi k/2n).
    rng = np.random.default_rng(10)
    h, w, gamma, tau = 16, 23, 0.7, 5.0
    L = rng.random((h, w))
    g = np.full((h, w), gamma)

    def solve_lines(X, axis):
        n = X.shape[axis]
        k = np.arange(n)
        lam = 1.0 + 8.0 * tau * gamma * np.sin(np.pi * k / (2 * n)) ** 2
        Xh = sfft.dct(X, type=2, norm="ortho", axis=axis)
        Xh = Xh / (lam[None, :] if axis == 1 else lam[:, None])
        return sfft.idct(Xh, type=2, norm="ortho", axis=axis)

    ref = 0.5 * (solve_lines(L, 1) + solve_lines(L, 0))
    _, _, ln = oracle_mod.aos_step(L, g, tau)
    assert np.max(np.abs(ln - ref)) < 1e-12


def test_aos_maximum_principle(oracle_mod):
    rng = np.random.default_rng(11)
    L = rng.random((25, 18))
    g = rng.random((25, 18))
    _, _, ln = oracle_mod.aos_step(L, g, 40.0)
    assert ln.min() >= L.min() - 1e-14
    assert ln.max() <= L.max() + 1e-14


def test_aos_small_tau_matches_explicit_step(oracle_mod):
    # (L_next - L) / tau -> sum over neighbours of (g_i+g_j)/2 (L_j - L_i)
    rng = np.random.default_rng(12)
    L = rng.random((14, 19))
    g = 0.2 + rng.random((14, 19))
    tau = 1e-5
    _, _, ln = oracle_mod.aos_step(L, g, tau)
    div = np.zeros_like(L)
    h, w = L.shape
    for y in range(h):
        for x in range(w):
            for (yy, xx) in ((y, x - 1), (y, x + 1), (y - 1, x), (y + 1, x)):
                if 0 <= yy < h and 0 <= xx < w:
                    div[y, x] += 0.5 * (g[y, x] + g[yy, xx]) * (L[yy, xx] - L[y, x])
    rate = (ln - L) / tau
    assert np.max(np.abs(rate - div)) < 1e-3 * (1 + np.max(np.abs(div)))


def test_scale_space_invariants(oracle_mod):
    rng = np.random.default_rng(13)
    img = rng.random((24, 40))
    opt = oracle_mod.Options.make(octaves=2, sublevels=4)
    lv, k = oracle_mod.build_scale_space(img, opt)
    assert lv.shape == (8, 24, 40)
    assert k > 0
    # L_0 is the presmoothed image
    assert np.max(np.abs(lv[0] - oracle_mod.gaussian(img, 1.6))) < 1e-15
    # every level keeps the mean of L_0 and stays inside its range
    for i in range(1, 8):
        assert abs(lv[i].mean() - lv[0].mean()) < 1e-12
        assert lv[i].min() >= lv[i - 1].min() - 1e-14
        assert lv[i].max() <= lv[i - 1].max() + 1e-14
    # a constant image stays constant through the whole scale space
    lv, k = oracle_mod.build_scale_space(np.full((9, 11), 0.25), opt)
    assert np.max(np.abs(lv - 0.25)) < 1e-14
    assert k == 0.03


def test_oracle_results_do_not_depend_on_the_thread_count(oracle_mod):
    """The loops over independent pixels and lines may run on several host
    threads; every output is computed by the same operations either way."""
    from paper_1706_06750_gb300 import synth
    img = synth.image(97, 61, 77).astype(np.float64)
    opt = oracle_mod.Options.make(octaves=2, sublevels=4)
    n0 = oracle_mod.threads()
    try:
        oracle_mod.set_threads(1)
        lv1, D1, kp1, k1 = oracle_mod.kaze_detect(img, opt)
        oracle_mod.set_threads(max(4, n0))
        lv4, D4, kp4, k4 = oracle_mod.kaze_detect(img, opt)
    finally:
        oracle_mod.set_threads(n0)
    assert k1 == k4 and np.array_equal(lv1, lv4) and np.array_equal(D1, D4)
    assert np.array_equal(kp1, kp4)
