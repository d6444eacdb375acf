"""Pins of the oracle's contrast factor k and conductance (CPU only)."""
import numpy as np
import pytest


def _cosine_image(w, h, amp, period_cycles):
    # A cosine that is even about x = -1/2 and x = W - 1/2 is its own
    # half-sample symmetric extension, so every linear filter acts on it as
    # on the infinite signal and the smoothed gradient has a closed form.
    x = np.arange(w, dtype=np.float64)
    omega = np.pi * period_cycles / w
    row = amp * np.cos(omega * (x + 0.5))
    return np.tile(row, (h, 1)), omega


def test_contrast_k_closed_form_cosine(oracle_mod):
    w, h, amp = 512, 24, 0.2
    img, omega = _cosine_image(w, h, amp, 3)
    k, hmax, hist, n = oracle_mod.contrast_k(img, sigma_d=1.0, pct=0.7, nbins=300)
    # closed form of |grad| of G_1 * img with the Scharr x-derivative:
    # Gaussian gain sum_j w_j cos(omega j), central difference gain sin(omega)
    wts = oracle_mod.gaussian_weights(1.0)
    r = (len(wts) - 1) // 2
    gain = float(np.sum(wts * np.cos(omega * np.arange(-r, r + 1))))
    x = np.arange(1, w - 1, dtype=np.float64)
    m = np.abs(amp * gain * np.sin(omega) * np.sin(omega * (x + 0.5)))
    m_all = np.tile(m, h - 2)
    assert hmax == pytest.approx(m.max(), rel=1e-12)
    nz = m_all[m_all > 0]
    assert n == nz.size
    # independent histogram and percentile of the closed-form magnitudes
    bins = np.minimum(np.floor(300 * nz / m.max()).astype(int), 299)
    ref_hist = np.bincount(bins, minlength=300)
    assert np.array_equal(hist, ref_hist)
    cum = np.cumsum(ref_hist)
    b = int(np.argmax(cum >= 0.7 * nz.size))
    assert k == pytest.approx(m.max() * (b + 1) / 300, rel=1e-12)
    # and k brackets the empirical 70th percentile of |grad| within one bin
    q = np.quantile(nz, 0.7)
    assert q <= k + 1e-15 and k - q <= m.max() / 300 + 1e-15


def test_contrast_k_fallback_constant_image(oracle_mod):
    k, hmax, hist, n = oracle_mod.contrast_k(np.full((20, 30), 0.4))
    assert n == 0 and hmax == 0.0 and k == 0.03


def test_conductance_values(oracle_mod):
    rng = np.random.default_rng(3)
    img = rng.random((9, 14))
    k = 0.05
    g2 = oracle_mod.conductance(img, k, diffusivity=oracle_mod.G2)
    g1 = oracle_mod.conductance(img, k, diffusivity=oracle_mod.G1)
    assert np.all(g2 > 0) and np.all(g2 <= 1)
    assert np.all(g1 >= 0) and np.all(g1 <= 1)
    # on a constant image there is no gradient: g == 1
    assert np.all(oracle_mod.conductance(np.full((5, 6), 0.3), k) == 1.0)
    # Eq. 3 on the closed-form gradient of the cosine image
    img, omega = _cosine_image(256, 8, 0.2, 2)
    wts = oracle_mod.gaussian_weights(1.0)
    r = (len(wts) - 1) // 2
    gain = float(np.sum(wts * np.cos(omega * np.arange(-r, r + 1))))
    x = np.arange(256, dtype=np.float64)
    m2 = (0.2 * gain * np.sin(omega) * np.sin(omega * (x + 0.5))) ** 2
    g = oracle_mod.conductance(img, k)
    assert np.max(np.abs(g - 1.0 / (1.0 + m2 / k ** 2))) < 1e-12
    g = oracle_mod.conductance(img, k, diffusivity=oracle_mod.G1)
    assert np.max(np.abs(g - np.exp(-m2 / k ** 2))) < 1e-12
