"""Pins of the oracle's linear filters and scale table (CPU only).

Each check compares the oracle with something other than itself: a library
routine (numpy / scipy) doing the same linear filtering, a closed form, or an
invariant the method fixes.
"""
import numpy as np
import pytest
from scipy import ndimage

pytestmark = pytest.mark.filterwarnings("ignore")


def test_reflect_matches_numpy_symmetric_pad(oracle_mod):
    # Half-sample symmetric extension == numpy 'symmetric' padding, including
    # repeated reflection for pads wider than the signal.
    for n in (1, 2, 3, 7):
        base = np.arange(n)
        padded = np.pad(base, 3 * n + 2, mode="symmetric")
        for i in range(-(3 * n + 2), n + 3 * n + 2):
            assert oracle_mod.reflect(i, n) == padded[i + 3 * n + 2]


@pytest.mark.parametrize("sigma", [0.8, 1.0, 1.6, 2.3])
def test_gaussian_weights_properties(oracle_mod, sigma):
    w = oracle_mod.gaussian_weights(sigma)
    r = (len(w) - 1) // 2
    j = np.arange(-r, r + 1)
    assert abs(w.sum() - 1.0) < 1e-14
    assert np.allclose(w, w[::-1], atol=0, rtol=0)
    assert np.all(np.diff(w[: r + 1]) > 0)  # unimodal
    # the sampled kernel's variance is sigma^2 up to truncation at 3 sigma
    var = float((w * j * j).sum())
    assert abs(var - sigma * sigma) / (sigma * sigma) < 0.05
    assert r >= 3 * sigma - 1e-12 and r < 3 * sigma + 1


@pytest.mark.parametrize("sigma", [1.0, 1.6])
def test_gaussian_matches_scipy_reflect(oracle_mod, sigma):
    rng = np.random.default_rng(1)
    img = rng.random((13, 21))
    w = oracle_mod.gaussian_weights(sigma)
    # scipy mode='reflect' is the half-sample symmetric extension
    ref = ndimage.correlate1d(img, w, axis=1, mode="reflect")
    ref = ndimage.correlate1d(ref, w, axis=0, mode="reflect")
    got = oracle_mod.gaussian(img, sigma)
    assert np.max(np.abs(got - ref)) < 1e-14


def test_gaussian_tiny_image_and_invariants(oracle_mod):
    # constant preserved exactly (up to rounding) even when 2r+1 > n
    c = np.full((2, 3), 0.37)
    assert np.max(np.abs(oracle_mod.gaussian(c, 1.6) - 0.37)) < 1e-15
    # a linear ramp is preserved away from the borders (symmetric kernel)
    x = np.arange(40, dtype=np.float64)
    ramp = np.tile(0.01 * x + 0.2, (20, 1))
    out = oracle_mod.gaussian(ramp, 1.6)
    assert np.max(np.abs(out[:, 6:-6] - ramp[:, 6:-6])) < 1e-14


def test_scharr_matches_scipy_and_ramps(oracle_mod):
    rng = np.random.default_rng(2)
    img = rng.random((11, 17))
    kx = np.array([[-3, 0, 3], [-10, 0, 10], [-3, 0, 3]], dtype=np.float64) / 32.0
    lx, ly = oracle_mod.scharr(img)
    assert np.max(np.abs(lx - ndimage.correlate(img, kx, mode="reflect"))) < 1e-15
    assert np.max(np.abs(ly - ndimage.correlate(img, kx.T, mode="reflect"))) < 1e-15
    # exact gradient of a plane in the interior
    yy, xx = np.mgrid[0:9, 0:12].astype(np.float64)
    plane = 0.3 * xx - 0.7 * yy + 2.0
    lx, ly = oracle_mod.scharr(plane)
    assert np.max(np.abs(lx[1:-1, 1:-1] - 0.3)) < 1e-14
    assert np.max(np.abs(ly[1:-1, 1:-1] + 0.7)) < 1e-14
    # derivative of x^2 is 2x in the interior (central differences are exact)
    sq = xx ** 2
    lx, _ = oracle_mod.scharr(sq)
    assert np.max(np.abs(lx[1:-1, 1:-1] - 2 * xx[1:-1, 1:-1])) < 1e-12


def test_scale_table_octave_structure(oracle_mod):
    O, S, s0 = 4, 4, 1.6
    sig, t = oracle_mod.scale_table(O, S, s0)
    assert sig.shape == (O * S,)
    assert sig[0] == pytest.approx(s0, rel=1e-15)
    # one octave doubles the scale, sub-levels are equally spaced in log scale
    assert np.allclose(sig[S:] / sig[:-S], 2.0, rtol=1e-14)
    assert np.allclose(sig[1:] / sig[:-1], 2.0 ** (1.0 / S), rtol=1e-14)
    assert np.all(np.diff(t) > 0)


def test_scale_time_relation_is_linear_diffusion_variance(oracle_mod):
    """Eq. 7: diffusing for time t spreads a point to variance 2t = sigma^2.

    Checked with an explicit 1-D heat-equation run, independent of the
    formula: the variance of the diffused delta must equal sigma_i^2.
    """
    sig, t = oracle_mod.scale_table(1, 4, 1.6)
    n = 401
    for i in (0, 3):
        u = np.zeros(n)
        u[n // 2] = 1.0
        dt = 0.01
        steps = int(round(t[i] / dt))
        for _ in range(steps):
            u = u + dt * (np.roll(u, 1) - 2 * u + np.roll(u, -1))
        x = np.arange(n) - n // 2
        var = float((u * x * x).sum())
        assert var == pytest.approx(sig[i] ** 2, rel=2e-3)
