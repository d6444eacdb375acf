"""Pins of the oracle's multiscale derivatives, detector response and
extrema (CPU only)."""
import numpy as np
import pytest
from scipy import ndimage


def test_step_size_rounding(oracle_mod):
    assert oracle_mod.step_size(0.3) == 1
    assert oracle_mod.step_size(1.49) == 1
    assert oracle_mod.step_size(2.5) == 3
    assert oracle_mod.step_size(21.53) == 22
    sig, _ = oracle_mod.scale_table(4, 4, 1.6)
    # hand-rounded steps of 1.6 * 2^(i/4), i = 0..15
    expect = [2, 2, 2, 3, 3, 4, 5, 5, 6, 8, 9, 11, 13, 15, 18, 22]
    assert [oracle_mod.step_size(s) for s in sig] == expect


def _dilated(k5, s):
    """5x5 tap kernel spread onto the lattice {-2s..2s}^2."""
    out = np.zeros((4 * s + 1, 4 * s + 1))
    out[::s, ::s] = k5
    return out


@pytest.mark.parametrize("s", [1, 2, 3])
def test_hessian_matches_scipy_with_hand_composed_stencils(oracle_mod, s):
    # Hand composition of two step-s Scharr derivatives:
    #   [-1 0 1] * [-1 0 1] = [1 0 -2 0 1];  [3 10 3] * [3 10 3] = [9 60 118 60 9];
    #   [-1 0 1] * [3 10 3] = [-3 -10 0 10 3]
    dd = np.array([1, 0, -2, 0, 1]) / (4.0 * s * s)
    ss = np.array([9, 60, 118, 60, 9]) / 256.0
    ds = np.array([-3, -10, 0, 10, 3]) / (32.0 * s)
    rng = np.random.default_rng(20 + s)
    L = rng.random((17, 23))
    xx, yy, xy = oracle_mod.hessian(L, s)
    kxx = _dilated(np.outer(ss, dd), s)  # rows index y, columns index x
    kyy = _dilated(np.outer(dd, ss), s)
    kxy = _dilated(np.outer(ds, ds), s)
    for got, k in ((xx, kxx), (yy, kyy), (xy, kxy)):
        ref = ndimage.correlate(L, k, mode="reflect")
        assert np.max(np.abs(got - ref)) < 1e-13


@pytest.mark.parametrize("s", [1, 2, 5])
def test_doh_of_analytic_quadratic(oracle_mod, s):
    a, b, c, d, e = 0.003, -0.0017, 0.0021, 0.4, -0.2
    h, w = 8 * s + 9, 8 * s + 11
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    f = a * xx ** 2 + b * xx * yy + c * yy ** 2 + d * xx + e * yy
    lxx, lyy, lxy = oracle_mod.hessian(f, s)
    m = 2 * s
    sl = (slice(m, h - m), slice(m, w - m))
    assert np.max(np.abs(lxx[sl] - 2 * a)) < 1e-12
    assert np.max(np.abs(lyy[sl] - 2 * c)) < 1e-12
    assert np.max(np.abs(lxy[sl] - b)) < 1e-12
    sigma = float(s)  # step_size(sigma) == s
    D = oracle_mod.doh(f, sigma, 0)
    assert np.max(np.abs(D[sl] - s ** 4 * (4 * a * c - b * b))) < 1e-12 * s ** 4
    # literal normalisation of Eq. 8: (sigma / 2^o)^2
    D = oracle_mod.doh(f, sigma, 1, doh_norm=oracle_mod.DOH_PAPER_LITERAL)
    assert np.max(np.abs(D[sl] - (sigma / 2) ** 2 * (4 * a * c - b * b))) < 1e-12


def test_doh_rotation_covariance(oracle_mod):
    rng = np.random.default_rng(30)
    L = ndimage.gaussian_filter(rng.random((26, 26)), 2.0)
    D = oracle_mod.doh(L, 2.3, 0)
    Dr = oracle_mod.doh(np.rot90(L).copy(), 2.3, 0)
    assert np.max(np.abs(np.rot90(D) - Dr)) < 1e-15
    # transposing the image swaps Lxx and Lyy and keeps Lxy
    xx, yy, xy = oracle_mod.hessian(L, 2)
    txx, tyy, txy = oracle_mod.hessian(L.T.copy(), 2)
    assert np.max(np.abs(txx - yy.T)) < 1e-16
    assert np.max(np.abs(tyy - xx.T)) < 1e-16
    assert np.max(np.abs(txy - xy.T)) < 1e-16


def _strict_maxima(D, thr):
    """Brute force: strict 3x3x3 maxima above thr, levels 1..N-2, 1-px border."""
    n, h, w = D.shape
    out = []
    for i in range(1, n - 1):
        for y in range(1, h - 1):
            for x in range(1, w - 1):
                v = D[i, y, x]
                if v <= thr:
                    continue
                cube = D[i - 1:i + 2, y - 1:y + 2, x - 1:x + 2].copy()
                cube[1, 1, 1] = -np.inf
                if v > cube.max():
                    out.append((i, y, x))
    return out


def test_extrema_brute_force_on_random_stack(oracle_mod):
    rng = np.random.default_rng(40)
    D = rng.random((5, 14, 17)) * 0.01
    opt = oracle_mod.Options.make(octaves=1, sublevels=5, edge_r=0.0)
    kp = oracle_mod.find_extrema(D, opt)
    got = {(int(k["level"]), int(k["iy"]), int(k["ix"])) for k in kp}
    brute = _strict_maxima(D, 0.001)
    assert got <= set(brute)
    # every brute-force maximum that was dropped fails the quadratic fit:
    # offset -H^-1 g (solved with numpy) leaves the pixel or H is singular
    for (i, y, x) in brute:
        P = D[i, y - 1:y + 2, x - 1:x + 2]
        g = np.array([(P[1, 2] - P[1, 0]) / 2, (P[2, 1] - P[0, 1]) / 2])
        Hm = np.array([[P[1, 2] - 2 * P[1, 1] + P[1, 0],
                        (P[2, 2] - P[2, 0] - P[0, 2] + P[0, 0]) / 4],
                       [(P[2, 2] - P[2, 0] - P[0, 2] + P[0, 0]) / 4,
                        P[2, 1] - 2 * P[1, 1] + P[0, 1]]])
        off = -np.linalg.solve(Hm, g)
        kept = (i, y, x) in got
        assert kept == bool(np.all(np.abs(off) <= 1.0))
    # ties are not maxima
    D2 = np.zeros((3, 5, 5))
    D2[1, 2, 2] = D2[1, 2, 3] = 0.5
    assert len(oracle_mod.find_extrema(D2, opt)) == 0


def test_subpixel_recovers_quadratic_vertex(oracle_mod):
    x0, y0 = 7.3, 5.8
    yy, xx = np.mgrid[0:12, 0:15].astype(np.float64)
    peak = 0.5 - 0.01 * ((xx - x0) ** 2 + 1.5 * (yy - y0) ** 2) + 0.002 * (xx - x0) * (yy - y0)
    D = np.stack([peak * 0.5, peak, peak * 0.5])
    opt = oracle_mod.Options.make(octaves=1, sublevels=3, edge_r=10.0)
    kp = oracle_mod.find_extrema(D, opt)
    assert len(kp) == 1
    assert kp[0]["x"] == pytest.approx(x0, abs=1e-12)
    assert kp[0]["y"] == pytest.approx(y0, abs=1e-12)
    assert (kp[0]["ix"], kp[0]["iy"]) == (7, 6)


def test_edge_test_rejects_ridges_keeps_blobs(oracle_mod):
    yy, xx = np.mgrid[0:21, 0:21].astype(np.float64)

    def stack(sx, sy):
        p = np.exp(-((xx - 10) ** 2 / (2 * sx * sx) + (yy - 10) ** 2 / (2 * sy * sy)))
        return np.stack([0.5 * p, p, 0.5 * p])

    opt = oracle_mod.Options.make(octaves=1, sublevels=3, edge_r=10.0)
    assert len(oracle_mod.find_extrema(stack(2.0, 2.0), opt)) == 1
    # principal curvature ratio 400 >> r = 10: rejected
    assert len(oracle_mod.find_extrema(stack(1.0, 20.0), opt)) == 0
    # with the test disabled the ridge peak is a keypoint
    opt0 = oracle_mod.Options.make(octaves=1, sublevels=3, edge_r=0.0)
    assert len(oracle_mod.find_extrema(stack(1.0, 20.0), opt0)) == 1


def test_planted_blob_found_at_its_centre_and_scale(oracle_mod):
    # one bright isotropic blob of std 4 on a flat background
    h, w = 64, 72
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    cx, cy, sd = 35.4, 30.7, 4.0
    img = 0.3 + 0.5 * np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2 * sd * sd))
    opt = oracle_mod.Options.make(octaves=3, sublevels=4)
    lv, D, kp, k = oracle_mod.kaze_detect(img, opt)
    assert len(kp) >= 1
    best = kp[np.argmax(kp["response"])]
    assert abs(best["x"] - cx) < 1.0 and abs(best["y"] - cy) < 1.0
    # selected scale within a factor 2 of the blob's own
    assert sd / 2 <= best["sigma"] <= sd * 2


@pytest.mark.parametrize("ratio,kept", [(9.0, True), (11.0, False), (1.0 / 11.0, False)])
def test_edge_test_threshold_uses_trace_of_both_curvatures(oracle_mod, ratio, kept):
    # D = 1 - p x^2 - q y^2: the discrete Hessian is exact (Dxx = -2p,
    # Dyy = -2q, Dxy = 0), so Tr^2/Det = (1 + p/q)^2 / (p/q) against
    # (r+1)^2/r = 12.1 for r = 10: a curvature ratio of 9 passes, 11 fails.
    yy, xx = np.mgrid[0:9, 0:9].astype(np.float64)
    q = 0.004
    p = ratio * q
    peak = 1.0 - p * (xx - 4) ** 2 - q * (yy - 4) ** 2
    D = np.stack([0.5 * peak, peak, 0.5 * peak])
    opt = oracle_mod.Options.make(octaves=1, sublevels=3, edge_r=10.0)
    assert (len(oracle_mod.find_extrema(D, opt)) == 1) == kept


# --- the sigma x sigma cross-level window (reading W1) ----------------------

def _stack(seed, n=8, h=40, w=44):
    from scipy import ndimage
    rng = np.random.default_rng(seed)
    return np.stack([ndimage.gaussian_filter(rng.random((h, w)), 1.2) * 0.01 for _ in range(n)])


def test_sigma_window_is_the_3x3_test_when_windows_are_3x3(oracle_mod):
    oracle = oracle_mod
    # s_i <= 3 on every level (sigma0 = 0.5): r_i = 1, the two tests coincide
    D = _stack(41)
    o3 = oracle.Options.make(octaves=2, sublevels=4, sigma0=0.5, dthreshold=0.0, edge_r=0.0)
    ow = oracle.Options.make(octaves=2, sublevels=4, sigma0=0.5, dthreshold=0.0, edge_r=0.0,
                             extrema_window=oracle.EXTREMA_SIGMA_WINDOW)
    a, b = oracle.find_extrema(D, o3), oracle.find_extrema(D, ow)
    assert len(a) > 10 and np.array_equal(a, b)


def test_sigma_window_keeps_a_subset(oracle_mod):
    oracle = oracle_mod
    D = _stack(42)
    o3 = oracle.Options.make(octaves=2, sublevels=4, dthreshold=0.0, edge_r=0.0)
    ow = oracle.Options.make(octaves=2, sublevels=4, dthreshold=0.0, edge_r=0.0,
                             extrema_window=oracle.EXTREMA_SIGMA_WINDOW)
    a, b = oracle.find_extrema(D, o3), oracle.find_extrema(D, ow)
    ka = {(int(k["level"]), int(k["ix"]), int(k["iy"])) for k in a}
    kb = {(int(k["level"]), int(k["ix"]), int(k["iy"])) for k in b}
    assert kb <= ka and len(kb) < len(ka)


def test_sigma_window_planted(oracle_mod):
    oracle = oracle_mod
    # level 6 of 4 x 4 levels: sigma = 1.6 * 2^1.5 = 4.53, s = 5, r = 2.  A
    # peak at (20, 20) with a larger value two pixels away one level up is
    # a 3x3x3 maximum but not a sigma-window maximum; three pixels away it
    # is outside the window and the peak survives both tests
    N, h, w = 16, 41, 41
    for off, keep in ((2, False), (3, True)):
        D = np.zeros((N, h, w))
        D[6, 20, 20] = 1.0
        D[7, 20, 20 + off] = 2.0
        o3 = oracle.Options.make(dthreshold=0.5, edge_r=0.0)
        ow = oracle.Options.make(dthreshold=0.5, edge_r=0.0, extrema_window=oracle.EXTREMA_SIGMA_WINDOW)
        at = lambda kp: any(int(k["level"]) == 6 and int(k["ix"]) == 20 and int(k["iy"]) == 20 for k in kp)
        assert at(oracle.find_extrema(D, o3))
        assert at(oracle.find_extrema(D, ow)) == keep
