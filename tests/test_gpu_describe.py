"""Parity of the CUDA description path (orientation + 64-D M-SURF, Sec. II-C)
with the FP64 oracle, through the C ABI.

Inputs are seeded synthetic images used directly as a level, or the FP64
oracle's own scale space and keypoints; nothing the CUDA path computes is
fed to the oracle.

Tolerances (FP32 kernel vs FP64 oracle on the same FP32 level):
  * descriptor entries (unit vectors): max |diff| <= 1e-4 on images up to
    256 px, 2e-4 at 1920 px -- the FP32 sample positions carry ~ulp(x)
    (1.2e-4 px at x ~ 1920) into the bilinear weights, the 81-sample sums
    ~1e-6 relative;
  * orientation: |diff| <= 1e-4 rad (window sums of 109 samples, ~1e-5
    relative).  A response within rounding of a sector boundary may fall
    into the neighbouring sector on one side and shift the winning window's
    sum: at most max(1, 3 %) of the keypoints may differ by more, and the
    descriptor of EVERY keypoint is also checked against the oracle
    evaluated at the GPU's own angle.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import describe as od  # noqa: E402
from paper_1706_06750_gb300 import synth  # noqa: E402

DESC_TOL = 1e-4
DESC_TOL_FULL = 2e-4
ANGLE_TOL = 1e-4


@pytest.fixture(scope="module")
def kz():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1706_06750_gb300 import build, kaze
    build.build()
    oracle.build()
    return kaze


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def circ(a, b):
    d = np.abs(np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64)) % (2 * math.pi)
    return np.minimum(d, 2 * math.pi - d)


def check_against_oracle(L32, sigma, pts, ang_g, desc_g, desc_tol, upright=False):
    """Angles within ANGLE_TOL (a few boundary flips allowed), every
    descriptor within desc_tol of the oracle's at the GPU's angle."""
    L = L32.astype(np.float64)
    ang_o, desc_o = od.describe_level(L, float(np.float32(sigma)), pts, upright=upright)
    bad = int(np.sum(circ(ang_g, ang_o) > ANGLE_TOL))
    assert bad <= max(1, int(0.03 * len(pts))), (bad, len(pts))
    _, desc_at = od.describe_level(L, float(np.float32(sigma)), pts, thetas=ang_g.astype(np.float64))
    err = float(np.max(np.abs(desc_g - desc_at))) if len(pts) else 0.0
    assert err <= desc_tol, err
    # (not compared with desc_o directly: an angle 1e-4 rad off turns sample
    # positions up to ~17 sigma away by that angle, which the descriptor
    # follows)
    return bad


def seeded_points(rng, w, h, n, pad=0.0):
    return [(float(np.float32(rng.uniform(-pad, w - 1 + pad))), float(np.float32(rng.uniform(-pad, h - 1 + pad))))
            for _ in range(n)]


@pytest.mark.parametrize("shape,sigma", [((130, 150), 1.6), ((97, 120), 2.69), ((150, 131), 6.4), ((64, 200), 12.8)])
def test_op_describe_matches_oracle(kz, shape, sigma):
    h, w = shape
    L = synth.image(w, h, 700 + h).astype(np.float32)
    pts = seeded_points(np.random.default_rng(h + w), w, h, 60)
    with kz.Kaze(w, h) as k:
        ang, desc = k.op_describe(dev(L), sigma, pts)
        assert k.last_launch_count() == 1
    assert np.allclose(np.linalg.norm(desc, axis=1), 1.0, atol=1e-5)
    check_against_oracle(L, sigma, pts, ang, desc, DESC_TOL)


def test_upright_and_edge_positions(kz):
    h, w = 90, 110
    L = synth.image(w, h, 801).astype(np.float32)
    # near and beyond the border: bilinear taps clamp on both sides
    pts = [(0.0, 0.0), (w - 1.0, h - 1.0), (-40.5, 3.25), (w + 17.0, h + 30.0), (55.5, -8.0), (0.49, 88.51)]
    with kz.Kaze(w, h) as k:
        ang, desc = k.op_describe(dev(L), 2.0, pts, upright=True)
    assert np.all(ang == 0.0)
    check_against_oracle(L, 2.0, pts, ang, desc, DESC_TOL, upright=True)
    with kz.Kaze(w, h) as k:
        ang, desc = k.op_describe(dev(L), 2.0, pts)
    check_against_oracle(L, 2.0, pts, ang, desc, DESC_TOL)


def test_degenerate_images(kz):
    # a constant level: no response at all -> angle 0 and a zero descriptor
    with kz.Kaze(40, 30) as k:
        ang, desc = k.op_describe(dev(np.full((30, 40), 0.37, np.float32)), 1.6, [(20.0, 15.0), (3.3, 2.2)])
    assert np.all(ang == 0.0) and np.all(desc == 0.0)
    # a 3 x 3 image with steps far beyond its size: repeated reflection
    L = np.array([[0.1, 0.5, 0.2], [0.9, 0.3, 0.4], [0.6, 0.8, 0.0]], np.float32)
    pts = [(1.0, 1.0), (0.25, 1.75)]
    with kz.Kaze(3, 3) as k:
        ang, desc = k.op_describe(dev(L), 9.0, pts)
    check_against_oracle(L, 9.0, pts, ang, desc, DESC_TOL)


def test_pipeline_describe_on_oracle_scale_space(kz):
    """The handle's levels against the oracle's FP64 scale space of the same
    image, at the oracle's keypoints: levels differ by FP32 rounding
    (<= 2e-5), so the tolerance here is looser (5e-3), and 90 % of the
    orientations must agree to 1e-3 rad."""
    img = synth.workload_image("256x256")
    h, w = img.shape
    s0 = float(np.float32(1.6))
    opt = oracle.Options.make(octaves=2, sublevels=4, sigma0=s0)
    lv_o, _, kp_o, _ = oracle.kaze_detect(img.astype(np.float64), opt)
    assert len(kp_o) >= 10
    kps = np.zeros(len(kp_o), dtype=kz.KEYPOINT_DTYPE)
    for i, p in enumerate(kp_o):
        kps[i]["x"], kps[i]["y"], kps[i]["level"] = p["x"], p["y"], p["level"]
    with kz.Kaze(w, h, octaves=2, sublevels=4) as k:
        k.build_scale_space(dev(img))
        out, desc = k.describe(kps)
        assert k.last_launch_count() == 1
        # the same kernel on one level at a time gives the same bits
        for lev in sorted(set(int(v) for v in kps["level"])):
            sel = kps["level"] == lev
            a1, d1 = k.op_describe(k.level(lev, copy=False), k.level_sigma(lev), kps[sel])
            assert np.array_equal(d1, desc[sel]) and np.array_equal(a1, out["angle"][sel].astype(np.float64))
    sig, t = oracle.scale_table(2, 4, s0)
    with kz.Kaze(w, h, octaves=2, sublevels=4) as k:
        # the scale table the library reports (Eq. 6-7) is the oracle's, rounded once to FP32
        for lev in range(8):
            assert k.level_sigma(lev) == float(np.float32(sig[lev]))
    agree, n = 0, 0
    for lev in sorted(set(int(v) for v in kps["level"])):
        sel = np.nonzero(kps["level"] == lev)[0]
        pts = [(float(kps[i]["x"]), float(kps[i]["y"])) for i in sel]
        ang_o, desc_o = od.describe_level(lv_o[lev], float(np.float32(sig[lev])), pts)
        d = circ(out["angle"][sel], ang_o)
        agree += int(np.sum(d <= 1e-3))
        n += len(sel)
        ok = d <= 1e-3
        if np.any(ok):
            assert np.max(np.abs(desc[sel][ok] - desc_o[ok])) <= 5e-3
    assert agree >= 0.9 * n


def test_describe_device_and_invalid_levels(kz):
    img = synth.image(120, 100, 901)
    with kz.Kaze(120, 100, octaves=2, sublevels=3) as k:
        k.build_scale_space(dev(img))
        kps = np.zeros(5, dtype=kz.KEYPOINT_DTYPE)
        kps["x"] = [10.5, 60.0, 100.25, 30.0, 5.0]
        kps["y"] = [20.0, 50.5, 80.0, 10.0, 90.0]
        kps["level"] = [0, 3, 5, 7, -1]          # the last two are not levels of this handle
        d_kp = k.keypoints_to_device(kps)
        d_desc = torch.full((5, 64), 7.0, device="cuda")
        k.describe_device(d_kp, d_desc, 5)
        torch.cuda.synchronize()
        got = k.keypoints_from_device(d_kp, 5)
        hd = d_desc.cpu().numpy()
        valid = kps[:3]
        ref_kp, ref_desc = k.describe(valid)
        assert np.array_equal(hd[:3], ref_desc) and np.array_equal(got["angle"][:3], ref_kp["angle"])
        assert np.all(hd[3:] == 0.0) and np.all(got["angle"][3:] == 0.0)
        # the host entry point refuses them
        with pytest.raises(kz.KazeError) as e:
            k.describe(kps)
        assert e.value.status == kz.ERR_INVALID_ARG
        bad = valid.copy()
        bad[1]["x"] = np.nan
        with pytest.raises(kz.KazeError) as e:
            k.describe(bad)
        assert e.value.status == kz.ERR_INVALID_ARG
        # nothing to do is fine
        kp0, d0 = k.describe(kps[:0])
        assert d0.shape == (0, 64)
    with kz.Kaze(64, 64, max_keypoints=4) as k:
        with pytest.raises(kz.KazeError) as e:
            k.describe(kps[:1])
        assert e.value.status == kz.ERR_STATE
        k.build_scale_space(dev(synth.image(64, 64, 3)))
        many = np.zeros(5, dtype=kz.KEYPOINT_DTYPE)
        with pytest.raises(kz.KazeError) as e:
            k.describe(many)
        assert e.value.status == kz.ERR_CAPACITY


def test_deterministic(kz):
    L = synth.image(200, 160, 77).astype(np.float32)
    pts = seeded_points(np.random.default_rng(78), 200, 160, 100)
    with kz.Kaze(200, 160) as k:
        x = dev(L)
        a1, d1 = k.op_describe(x, 3.2, pts)
        a2, d2 = k.op_describe(x, 3.2, pts)
    assert np.array_equal(a1, a2) and np.array_equal(d1, d2)


def test_full_size_sampled(kz):
    """1920 x 1200 seeded level, 400 keypoints over the 16 scales of the
    detector; the oracle recomputes a sample of 48 of them."""
    w, h = 1920, 1200
    L = synth.workload_image("1920x1200").astype(np.float32)
    sig, _ = oracle.scale_table(4, 4, float(np.float32(1.6)))
    rng = np.random.default_rng(1920)
    pts = seeded_points(rng, w, h, 400)
    levels = rng.integers(0, 16, size=400)
    with kz.Kaze(w, h) as k:
        x = dev(L)
        res = {}
        for lev in range(16):
            sel = np.nonzero(levels == lev)[0]
            if len(sel):
                res[lev] = (sel, k.op_describe(x, float(sig[lev]), [pts[i] for i in sel]))
    sample = rng.choice(400, size=48, replace=False)
    for lev, (sel, (ang, desc)) in res.items():
        pick = [j for j, i in enumerate(sel) if i in set(sample)]
        if not pick:
            continue
        check_against_oracle(L, float(sig[lev]), [pts[sel[j]] for j in pick], ang[pick], desc[pick], DESC_TOL_FULL)


def test_full_size_rotation_covariance(kz):
    """A property at full size: detecting and describing the image turned by
    90 degrees gives the same keypoints turned, with the angle lowered by
    pi/2 and the same descriptor (up to the FP32 differences of the two
    scale spaces; 90 % of matched keypoints within 2e-3)."""
    img = synth.workload_image("1920x1200")
    h, w = img.shape
    rot = np.ascontiguousarray(np.rot90(img))          # (x, y) -> (y, w - 1 - x)
    with kz.Kaze(1920, 1920) as k:
        kp0 = k.detect(dev(img))
        kp0, d0 = k.describe(kp0)
        kp1 = k.detect(dev(rot))
        kp1, d1 = k.describe(kp1)
    assert len(kp0) >= 100
    # a pixel (ix, iy) of the image sits at (iy, w - 1 - ix) of the turned one
    index = {(int(q["level"]), w - 1 - int(q["iy"]), int(q["ix"])): j for j, q in enumerate(kp1)}
    matched, good = 0, 0
    for i, p in enumerate(kp0):
        j = index.get((int(p["level"]), int(p["ix"]), int(p["iy"])))
        if j is None:
            continue
        matched += 1
        da = circ(kp1[j]["angle"], (float(p["angle"]) - math.pi / 2) % (2 * math.pi))
        if da <= 2e-3 and np.max(np.abs(d0[i] - d1[j])) <= 2e-3:
            good += 1
    assert matched >= 0.9 * len(kp0)
    assert good >= 0.9 * matched
