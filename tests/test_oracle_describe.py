"""Pins of the description oracle (orientation + 64-D M-SURF, Sec. II-C)
against facts fixed by the mathematics: closed forms on polynomial images,
exact covariance under 90-degree rotation and mirroring, invariance to
intensity scale and offset, planted response clusters."""
import math
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
from oracle import describe as od  # noqa: E402
from paper_1706_06750_gb300 import synth  # noqa: E402


def _grid(W, H):
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    return x, y


def _circ(a, b):
    d = abs(a - b) % (2 * math.pi)
    return min(d, 2 * math.pi - d)


def test_derivatives_closed_forms():
    # interior pixels (>= s from the border): the step-s Scharr pair of a
    # cubic is 3 u^2 + s^2, of x*y it is (v, u), of a ramp its slopes
    W, H = 40, 36
    x, y = _grid(W, H)
    for s in (1, 2, 3):
        sl = np.s_[s:H - s, s:W - s]
        Lx, Ly = od.first_derivatives(x ** 3, s)
        assert np.allclose(Lx[sl], 3 * x[sl] ** 2 + s * s, atol=1e-9)
        assert np.allclose(Ly[sl], 0.0, atol=1e-9)
        Lx, Ly = od.first_derivatives(x * y, s)
        assert np.allclose(Lx[sl], y[sl], atol=1e-12) and np.allclose(Ly[sl], x[sl], atol=1e-12)
        Lx, Ly = od.first_derivatives(0.3 * x - 0.7 * y + 2.0, s)
        assert np.allclose(Lx[sl], 0.3, atol=1e-12) and np.allclose(Ly[sl], -0.7, atol=1e-12)
    # at the border the symmetric extension makes the normal derivative of a
    # ramp vanish at the reflected taps: column 0 sees L(-1) = L(0)
    Lx, _ = od.first_derivatives(x, 1)
    assert np.allclose(Lx[:, 0], 0.5)


def test_bilinear_brute_force():
    rng = np.random.default_rng(3)
    img = rng.random((5, 7))
    assert od.bilinear(img, np.array([2.0]), np.array([3.0]))[0] == img[3, 2]
    v = od.bilinear(img, np.array([2.5]), np.array([3.5]))[0]
    assert v == pytest.approx(img[3:5, 2:4].mean(), abs=1e-15)
    v = od.bilinear(img, np.array([1.25]), np.array([0.0]))[0]
    assert v == pytest.approx(0.75 * img[0, 1] + 0.25 * img[0, 2], abs=1e-15)
    # taps clamp into the image
    assert od.bilinear(img, np.array([-3.0]), np.array([9.0]))[0] == img[4, 0]


def test_orientation_sample_set():
    a, b, w = od.orientation_samples()
    assert len(a) == 109                       # lattice points strictly inside radius 6
    assert np.all(a * a + b * b < 36) and w.max() == 1.0


@pytest.mark.parametrize("gx,gy", [(0.003, -0.002), (-0.004, 0.001), (-0.001, -0.002), (0.0, 0.002)])
def test_ramp_orientation_and_descriptor_closed_form(gx, gy):
    W, H = 160, 150
    x, y = _grid(W, H)
    L = gx * x + gy * y + 0.4
    kx, ky, sigma = 80.3, 74.6, 2.0
    ang, desc = od.describe_level(L, sigma, [(kx, ky)])
    # every response points along the gradient, so the orientation is its angle
    assert _circ(ang[0], math.atan2(gy, gx) % (2 * math.pi)) < 1e-12
    # in the keypoint frame the gradient lies on x': components (w2 c, 0, w2 c, 0)
    w2 = np.array([[math.exp(-((p - 1.5) ** 2 + (q - 1.5) ** 2) / 4.5) for p in range(4)] for q in range(4)])
    exp = np.zeros(64)
    for q in range(4):
        for p in range(4):
            exp[4 * (4 * q + p) + 0] = w2[q, p]
            exp[4 * (4 * q + p) + 2] = w2[q, p]
    exp /= np.linalg.norm(exp)
    assert np.allclose(desc[0], exp, atol=1e-12)


def test_parabola_descriptor_closed_form():
    # L = c x^2: L_x = 2 c x exactly, so with theta = 0 every subregion sums
    # 2 c (x + sigma c_p) times the sum of its sample weights (odd moments
    # cancel): the entries follow the subregion centres c_p = -7.5 .. 7.5
    W, H = 300, 200
    x, y = _grid(W, H)
    kx, ky, sigma = 150.0, 100.0, 3.0
    ang, desc = od.describe_level(1e-4 * x * x, sigma, [(kx, ky)])
    assert _circ(ang[0], 0.0) < 1e-12
    cp = np.array([-7.5, -2.5, 2.5, 7.5])
    exp = np.zeros(64)
    for q in range(4):
        for p in range(4):
            w2 = math.exp(-((p - 1.5) ** 2 + (q - 1.5) ** 2) / 4.5)
            exp[4 * (4 * q + p) + 0] = w2 * (kx + sigma * cp[p])
            exp[4 * (4 * q + p) + 2] = w2 * (kx + sigma * cp[p])
    exp /= np.linalg.norm(exp)
    assert np.allclose(desc[0], exp, atol=1e-12)
    # the same along y: the orientation turns to +90 degrees and x' = +y, so
    # the subregion index p (along x') again carries the centre offsets
    ang, desc = od.describe_level(1e-4 * y * y, sigma, [(100.0, 100.0)])
    assert _circ(ang[0], math.pi / 2) < 1e-12
    exp = np.zeros(64)
    for q in range(4):
        for p in range(4):
            w2 = math.exp(-((p - 1.5) ** 2 + (q - 1.5) ** 2) / 4.5)
            exp[4 * (4 * q + p) + 0] = w2 * (100.0 + sigma * cp[p])
            exp[4 * (4 * q + p) + 2] = w2 * (100.0 + sigma * cp[p])
    exp /= np.linalg.norm(exp)
    assert np.allclose(desc[0], exp, atol=1e-12)


def _random_points(rng, W, H, n, margin):
    return [(rng.uniform(margin, W - 1 - margin), rng.uniform(margin, H - 1 - margin)) for _ in range(n)]


def test_rotation_by_90_degrees_is_exact():
    L = synth.image(96, 80, 11).astype(np.float64)
    H, W = L.shape
    rng = np.random.default_rng(12)
    pts = _random_points(rng, W, H, 12, 2.0)
    for sigma in (1.6, 2.7):
        a0, d0 = od.describe_level(L, sigma, pts)
        R = np.rot90(L)          # R[i, j] = L[j, W - 1 - i]: (x, y) -> (y, W - 1 - x)
        a1, d1 = od.describe_level(R, sigma, [(y, W - 1 - x) for x, y in pts])
        for t0, t1 in zip(a0, a1):
            assert _circ(t1, (t0 - math.pi / 2) % (2 * math.pi)) < 1e-9
        assert np.allclose(d0, d1, atol=1e-9)


def test_mirror_flips_the_frame():
    L = synth.image(90, 70, 21).astype(np.float64)
    H, W = L.shape
    rng = np.random.default_rng(22)
    pts = _random_points(rng, W, H, 12, 1.0)
    sigma = 2.2
    a0, d0 = od.describe_level(L, sigma, pts)
    a1, d1 = od.describe_level(L[:, ::-1], sigma, [(W - 1 - x, y) for x, y in pts])
    for k in range(len(pts)):
        assert _circ(a1[k], (math.pi - a0[k]) % (2 * math.pi)) < 1e-9
        e = np.zeros(64)
        for q in range(4):
            for p in range(4):
                src = 4 * (4 * (3 - q) + p)
                dst = 4 * (4 * q + p)
                e[dst:dst + 4] = d0[k, src:src + 4] * np.array([1.0, -1.0, 1.0, 1.0])
        assert np.allclose(d1[k], e, atol=1e-9)


def test_intensity_scale_and_offset_do_not_matter():
    L = synth.image(70, 64, 31).astype(np.float64)
    pts = _random_points(np.random.default_rng(32), 70, 64, 6, 0.0)
    a0, d0 = od.describe_level(L, 1.6, pts)
    a1, d1 = od.describe_level(3.0 * L + 7.0, 1.6, pts)
    assert np.allclose(a0, a1, atol=1e-12) and np.allclose(d0, d1, atol=1e-12)
    assert np.allclose(np.linalg.norm(d0, axis=1), 1.0, atol=1e-12)


def test_dominant_orientation_of_planted_clusters():
    # a cluster of five unit vectors within 40 degrees around 200 degrees and
    # three longer ones at 30 degrees: the pi/3 window holding the first wins
    ang = np.deg2rad([182.0, 191.0, 200.0, 209.0, 218.0])
    rx = list(np.cos(ang)) + [1.2 * math.cos(math.radians(30))] * 3
    ry = list(np.sin(ang)) + [1.2 * math.sin(math.radians(30))] * 3
    want = math.atan2(np.sin(ang).sum(), np.cos(ang).sum()) % (2 * math.pi)
    assert _circ(od.dominant_orientation(np.array(rx), np.array(ry)), want) < 1e-12
    # a window cannot hold two clusters 90 degrees apart: the longer one wins
    rx = [1.0, 1.0, 0.0]
    ry = [0.0, 0.0, 1.5]
    assert _circ(od.dominant_orientation(np.array(rx), np.array(ry)), 0.0) < 1e-12
    # no response at all
    assert od.dominant_orientation(np.zeros(4), np.zeros(4)) == 0.0


def test_upright_and_given_angles():
    L = synth.image(64, 64, 41).astype(np.float64)
    pts = [(31.5, 30.25)]
    a, d = od.describe_level(L, 1.6, pts, upright=True)
    assert a[0] == 0.0
    a2, d2 = od.describe_level(L, 1.6, pts, thetas=[0.0])
    assert np.array_equal(d, d2)


def test_absolute_components_on_a_centred_parabola():
    # L = c (x - x_k)^2 at the keypoint's own column, frame fixed at theta = 0:
    # r_x' = 2 c sigma (c_p + u) changes sign inside the inner subregions, so
    # the signed sums follow c_p alone while the absolute sums weigh |c_p + u|
    W, H = 200, 160
    x, y = _grid(W, H)
    kx, ky, sigma, c = 100.0, 80.0, 2.0, 1e-4
    _, desc = od.describe_level(c * (x - kx) ** 2, sigma, [(kx, ky)], thetas=[0.0])
    u, v = np.meshgrid(np.arange(-4, 5), np.arange(-4, 5), indexing="xy")
    w1 = np.exp(-(u * u + v * v) / 12.5)
    exp = np.zeros(64)
    for q in range(4):
        for p in range(4):
            cp = (p - 1.5) * 5.0
            w2 = math.exp(-((p - 1.5) ** 2 + (q - 1.5) ** 2) / 4.5)
            exp[4 * (4 * q + p) + 0] = w2 * 2 * c * sigma * cp * w1.sum()
            exp[4 * (4 * q + p) + 2] = w2 * 2 * c * sigma * np.sum(w1 * np.abs(cp + u))
    exp /= np.linalg.norm(exp)
    assert np.allclose(desc[0], exp, atol=1e-12)


def test_equal_windows_take_the_first():
    # two equal clusters at 90 and 270 degrees: windows starting at 35 .. 90
    # degrees and at 215 .. 270 degrees tie; the first window wins
    rx = np.array([0.0, 0.0])
    ry = np.array([1.0, -1.0])
    assert _circ(od.dominant_orientation(rx, ry), math.pi / 2) < 1e-12
