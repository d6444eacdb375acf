"""Pins of the FED oracle (Eq. 5, Sec. II-A) against facts fixed by the
mathematics: the stopping-time identity of a FED cycle, closed-form step
sizes, minimal cycle length, conservation, the DCT-II closed form of linear
diffusion with constant conductance, one explicit step computed
independently, l2 stability, and agreement with AOS to second order."""
import math

import numpy as np
import pytest

import oracle


def cycle_time(n, tau_max=0.25):
    # sum_j 1 / (2 cos^2(pi (2j+1) / (4n+2))) = (n^2 + n) / 3 (Grewenig,
    # Weickert & Bruhn 2010)
    return tau_max * (n * n + n) / 3.0


def test_step_sizes_closed_forms():
    # dt equal to a cycle's own stopping time: no rescaling
    t1 = oracle.fed_tau(cycle_time(1))
    assert len(t1) == 1 and t1[0] == pytest.approx(0.25 * 2.0 / 3.0, rel=1e-14)  # 1 / (2 cos^2(pi/6))
    t2 = oracle.fed_tau(cycle_time(2))
    c1 = math.sqrt((5 + math.sqrt(5)) / 8)       # cos(pi/10)
    c3 = math.sqrt((5 - math.sqrt(5)) / 8)       # cos(3 pi/10)
    assert np.allclose(t2, [0.25 / (2 * c1 * c1), 0.25 / (2 * c3 * c3)], rtol=1e-13)
    for n in range(1, 60):
        t = oracle.fed_tau(cycle_time(n))
        assert len(t) == n
        assert t.sum() == pytest.approx(cycle_time(n), rel=1e-12)
        assert t.max() > 0.25 * (n > 1)          # single steps beyond the explicit limit
        assert np.all(np.diff(t) > 0)             # increasing within the cycle


@pytest.mark.parametrize("dt", [1e-4, 0.1, 0.53, 1.0, 3.3, 17.0, 67.9, 231.0])
def test_cycle_is_minimal_and_reaches_dt(dt):
    t = oracle.fed_tau(dt)
    n = len(t)
    assert cycle_time(n) >= dt * (1 - 1e-12)
    assert n == 1 or cycle_time(n - 1) < dt
    assert t.sum() == pytest.approx(dt, rel=1e-12)


def test_no_step_for_zero_time():
    assert len(oracle.fed_tau(0.0)) == 0
    L = np.random.default_rng(1).random((5, 6))
    assert np.array_equal(oracle.fed_evolve(L, np.ones_like(L), 0.0), L)


def test_constant_image_and_conservation():
    rng = np.random.default_rng(2)
    g = rng.uniform(0.05, 1.0, (23, 31))
    C = np.full((23, 31), 0.37)
    assert np.allclose(oracle.fed_evolve(C, g, 9.0), 0.37, atol=1e-14)
    L = rng.random((23, 31))
    out = oracle.fed_evolve(L, g, 9.0)
    assert abs(out.sum() - L.sum()) <= 1e-10 * L.size


def _dct_diffusion(L, gamma, taus):
    from scipy.fft import dctn, idctn
    h, w = L.shape
    lx = 4 * np.sin(np.pi * np.arange(w) / (2 * w)) ** 2
    ly = 4 * np.sin(np.pi * np.arange(h) / (2 * h)) ** 2
    lam = gamma * (ly[:, None] + lx[None, :])
    amp = np.ones_like(lam)
    for t in taus:
        amp *= 1.0 - t * lam
    return idctn(dctn(L, type=2, norm="ortho") * amp, type=2, norm="ortho")


@pytest.mark.parametrize("shape,dt", [((16, 20), 2.0), ((9, 33), 20.0), ((1, 40), 7.0)])
def test_constant_conductance_equals_dct_product(shape, dt):
    # with g = gamma the step is gamma times the Neumann 5-point Laplacian,
    # diagonal in the DCT-II basis with eigenvalues -4 (sin^2(pi kx/2w) +
    # sin^2(pi ky/2h)): the cycle multiplies each mode by prod_j (1 - tau_j lam)
    rng = np.random.default_rng(3)
    L = rng.random(shape)
    gamma = 0.8
    out = oracle.fed_evolve(L, np.full(shape, gamma), dt)
    ref = _dct_diffusion(L, gamma, oracle.fed_tau(dt))
    assert np.allclose(out, ref, atol=1e-10)


def test_one_step_is_the_explicit_divergence():
    rng = np.random.default_rng(4)
    L = rng.random((12, 17))
    g = rng.uniform(0.1, 1.0, (12, 17))
    dt = 0.05                                     # one step of size dt
    assert len(oracle.fed_tau(dt)) == 1
    # flux form written with array slices: no flux through the border
    div = np.zeros_like(L)
    fx = 0.5 * (g[:, 1:] + g[:, :-1]) * (L[:, 1:] - L[:, :-1])
    fy = 0.5 * (g[1:, :] + g[:-1, :]) * (L[1:, :] - L[:-1, :])
    div[:, :-1] += fx
    div[:, 1:] -= fx
    div[:-1, :] += fy
    div[1:, :] -= fy
    assert np.allclose(oracle.fed_evolve(L, g, dt), L + dt * div, atol=1e-15)
    assert np.allclose(oracle.fed_step(L, g, dt), L + dt * div, atol=1e-15)


def test_l2_stable_for_long_cycles():
    rng = np.random.default_rng(5)
    L = rng.random((40, 50)) - 0.5
    g = rng.uniform(0.0, 1.0, (40, 50))
    out = oracle.fed_evolve(L, g, 68.0)
    assert np.linalg.norm(out) <= np.linalg.norm(L) * (1 + 1e-12)


def test_agrees_with_aos_to_second_order():
    # both approximate the same diffusion: their difference shrinks like dt^2
    rng = np.random.default_rng(6)
    from scipy import ndimage
    L = ndimage.gaussian_filter(rng.random((30, 30)), 2.0)
    g = rng.uniform(0.3, 1.0, (30, 30))
    errs = []
    for dt in (0.04, 0.02):
        _, _, aos = oracle.aos_step(L, g, dt)
        errs.append(np.max(np.abs(oracle.fed_evolve(L, g, dt) - aos)))
    assert errs[1] < errs[0] / 3.0


def test_scale_space_with_fed():
    img = np.random.default_rng(7).random((40, 48))
    opt = oracle.Options.make(octaves=2, sublevels=3, scheme=oracle.SCHEME_FED)
    lv, k = oracle.build_scale_space(img, opt)
    m = lv.reshape(lv.shape[0], -1).mean(axis=1)
    assert np.allclose(m, m[0], atol=1e-12)
    const, _ = oracle.build_scale_space(np.full((20, 24), 0.5), opt)
    assert np.allclose(const, 0.5, atol=1e-14)
    # AOS and FED levels are close (same diffusion, different discretisation)
    lv_a, _ = oracle.build_scale_space(img, oracle.Options.make(octaves=2, sublevels=3))
    assert np.max(np.abs(lv - lv_a)) < 0.05


def _amplification(t, lam=np.linspace(0.0, 8.0, 4001)):
    f = [np.abs(1.0 - tk * lam) for tk in t]
    b = 0.0
    for j in range(len(t)):
        head = np.prod(f[: j + 1], axis=0).max()
        tail = np.prod(f[j + 1:], axis=0).max() if j + 1 < len(t) else 1.0
        b += head * tail
    return b


def test_kappa_cycle_order():
    # hand-worked kappa cycle: n = 4, p = 5, kappa = 2 gives 1, 3, 0, 2
    t = oracle.fed_tau(cycle_time(4))
    order, kappa = oracle.fed_order(cycle_time(4))
    assert sorted(order) == [0, 1, 2, 3]
    p = 5
    seq = [((l + 1) * kappa) % p - 1 for l in range(p - 1)]
    assert list(order) == [i for i in seq if 0 <= i < 4]
    # long cycles: the chosen order keeps FP32 rounding bounded where the
    # natural (increasing) order would amplify it beyond any use
    for dt in (5.0, 20.0, 67.9):
        t = oracle.fed_tau(dt)
        order, _ = oracle.fed_order(dt)
        assert sorted(order) == list(range(len(t)))
        b_nat, b_ord = _amplification(t), _amplification(t[order])
        assert b_ord < 1e3 and b_ord < b_nat, (dt, b_nat, b_ord)
        assert len(t) < 15 or b_ord < b_nat / 1e4, (dt, b_nat, b_ord)
