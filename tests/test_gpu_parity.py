"""Parity of the CUDA path with the FP64 oracle (needs a GB300 / sm_103a).

Every call goes through the C ABI of libkaze.so via the ctypes binding.
Tolerances (FP32 kernels vs FP64 oracle):
  * scale-space pixels: max |diff| <= 2e-5 (images in [0, 1]);
  * detector response: max |diff| <= 1e-4 * max |DoH| of the level;
  * keypoints: same level within 0.5 px, overlap >= 99.5 % after removing
    keypoints whose admitting decision is within rounding of its boundary;
  * contrast factor: the same histogram bin or the adjacent one.
Single-step checks feed both sides the same FP32 input, so they isolate the
arithmetic of one kernel.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1706_06750_gb300 import synth  # noqa: E402

from kp_match import compare  # noqa: E402

SCALE_TOL = 2e-5
DOH_REL_TOL = 1e-4
KP_OVERLAP = 0.995


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


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def options(kz, **kw):
    return kz.default_options(**kw)


def oracle_options(gpu_opt, k_override=0.0):
    return oracle.Options.make(
        octaves=gpu_opt.octaves, sublevels=gpu_opt.sublevels, sigma0=float(gpu_opt.sigma0),
        sigma_d=float(gpu_opt.sigma_d), k_percentile=gpu_opt.k_percentile, nbins=gpu_opt.nbins,
        diffusivity=gpu_opt.diffusivity, dthreshold=float(np.float32(gpu_opt.dthreshold)),
        edge_r=float(gpu_opt.edge_r), doh_norm=gpu_opt.doh_norm, k_override=k_override)


def random_smooth(rng, h, w, sigma=1.5):
    from scipy import ndimage
    return np.clip(ndimage.gaussian_filter(rng.random((h, w)), sigma) * 1.5 - 0.25, 0, 1)


# ------------------------------------------------------------ single steps --

@pytest.mark.parametrize("shape", [(256, 256), (131, 257), (3, 3), (40, 2100), (2100, 40)])
def test_gaussian_step(kz, shape):
    rng = np.random.default_rng(1)
    img = rng.random(shape).astype(np.float32)
    h, w = shape
    with kz.Kaze(w, h) as k:
        src = dev(img)
        out = torch.empty_like(src)
        k.op_gaussian(src, out, 1.6)
        torch.cuda.synchronize()
    ref = oracle.gaussian(img.astype(np.float64), 1.6)
    assert np.max(np.abs(host(out) - ref)) < 1e-6


@pytest.mark.parametrize("shape", [(256, 256), (131, 257), (1200, 1920)])
def test_contrast_step(kz, shape):
    h, w = shape
    img = synth.image(w, h, 77)
    L0 = oracle.gaussian(img.astype(np.float64), 1.6).astype(np.float32)
    with kz.Kaze(w, h) as k:
        kg, hmax_g, hist_g = k.op_contrast(dev(L0))
    kr, hmax_r, hist_r, n_r = oracle.contrast_k(L0.astype(np.float64), 1.0, 0.7, 300)
    assert hmax_g == pytest.approx(hmax_r, rel=1e-5)
    # A pixel may land in a neighbouring bin only if its FP64 magnitude lies
    # within FP32 reach of a bin edge; each such pixel moves at most one count
    # out of one bin and into another.
    lx, ly = oracle.scharr(oracle.gaussian(L0.astype(np.float64), 1.0))
    m = np.hypot(lx, ly)[1:-1, 1:-1]
    u = 300 * m[m > 0] / hmax_r
    near = int(np.sum(np.abs(u - np.round(u)) < 1e-4)) + int(np.sum(m == 0))
    assert abs(int(hist_g.sum()) - n_r) <= near
    assert np.abs(hist_g - hist_r).sum() <= 2 * near
    width = hmax_r / 300
    assert abs(kg - kr) <= width * 1.0001 + 1e-7


def test_contrast_constant_image_fallback(kz):
    with kz.Kaze(64, 48) as k:
        kg, hmax, hist = k.op_contrast(torch.full((48, 64), 0.3, device="cuda"))
    assert kg == pytest.approx(0.03) and hmax == 0.0 and hist.sum() == 0


@pytest.mark.parametrize("shape", [(256, 256), (131, 257), (3, 5)])
@pytest.mark.parametrize("diff", [2, 1])
def test_conductance_step(kz, shape, diff):
    rng = np.random.default_rng(2)
    h, w = shape
    L = random_smooth(rng, h, w).astype(np.float32)
    kval = 0.02
    with kz.Kaze(w, h, diffusivity=diff) as k:
        g = torch.empty((h, w), device="cuda")
        k.op_conductance(dev(L), g, kval)
        torch.cuda.synchronize()
    ref = oracle.conductance(L.astype(np.float64), kval, 1.0, diff)
    # FP32 gradients of values in [0, 1] carry an absolute error of ~5e-7;
    # |dg/d|grad|| is at most 0.86/k for g1 and 0.65/k for g2, so with
    # k = 0.02 the conductance may differ by up to ~2e-5.
    assert np.max(np.abs(host(g) - ref)) < 2e-5


def misaligned(a, pitch):
    """A [h, w] view with row pitch `pitch` whose first element is 4 bytes past
    a 16-byte boundary (the library then takes its one-column-a-lane
    gradient kernel instead of the four-column one)."""
    h, w = a.shape
    base = torch.zeros(h * pitch + 8, device="cuda")
    v = base[1:1 + h * pitch].view(h, pitch)[:, :w]
    v.copy_(torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)))
    assert v.data_ptr() % 16 == 4
    return v


@pytest.mark.parametrize("shape", [(256, 256), (131, 257), (3, 5), (40, 483), (1200, 1920)])
@pytest.mark.parametrize("diff", [2, 1])
def test_conductance_kernels_agree_bitwise(kz, shape, diff):
    """The four-column gradient kernel (aligned planes) and the one-column
    kernel (any alignment) form the conductance with the same operations in
    the same order: equal bit for bit, also at ragged widths and borders."""
    rng = np.random.default_rng(12)
    h, w = shape
    L = random_smooth(rng, h, w).astype(np.float32)
    pitch = (w + 3) // 4 * 4
    with kz.Kaze(w, h, diffusivity=diff) as k:
        buf = torch.zeros((h, pitch), device="cuda")
        a = buf[:, :w]
        a.copy_(torch.from_numpy(L))
        ga = torch.zeros((h, pitch), device="cuda")[:, :w]
        k.op_conductance(a, ga, 0.02)
        b = misaligned(L, pitch + 4)
        gb = misaligned(np.zeros_like(L), pitch + 4)
        k.op_conductance(b, gb, 0.02)
        torch.cuda.synchronize()
        assert torch.equal(ga, gb)
        # the maximum pass of the contrast factor, both ways
        assert k.op_contrast(a)[:2] == k.op_contrast(b)[:2]


@pytest.mark.parametrize("shape", [(256, 256), (131, 257), (3, 3), (4, 61), (61, 4),
                                   (40, 2100), (2100, 40), (1200, 1920)])
@pytest.mark.parametrize("tau", [0.53, 67.9])
def test_aos_step(kz, shape, tau):
    rng = np.random.default_rng(3)
    h, w = shape
    pitch = (w + 31) // 32 * 32
    L = random_smooth(rng, h, w).astype(np.float32)
    g = (0.02 + 0.98 * rng.random((h, w))).astype(np.float32)
    with kz.Kaze(w, h) as k:
        Lp = torch.zeros((h, pitch), device="cuda")[:, :w]
        Gp = torch.zeros((h, pitch), device="cuda")[:, :w]
        Lp.copy_(dev(L))
        Gp.copy_(dev(g))
        ux = torch.zeros((h, pitch), device="cuda")[:, :w]
        ln = torch.zeros((h, pitch), device="cuda")[:, :w]
        k.op_aos_step(Lp, Gp, ux, ln, tau)
        torch.cuda.synchronize()
    rx, ry, rl = oracle.aos_step(L.astype(np.float64), g.astype(np.float64), tau)
    assert np.max(np.abs(host(ux) - rx)) < 5e-6
    assert np.max(np.abs(host(ln) - rl)) < 5e-6


@pytest.mark.parametrize("s_sigma", [(1.6, 0), (2.69, 0), (9.05, 2), (21.5, 3)])
def test_doh_step(kz, s_sigma):
    sigma, octave = s_sigma
    rng = np.random.default_rng(4)
    h, w = 131, 257
    L = random_smooth(rng, h, w, 3.0).astype(np.float32)
    for norm in (kz.DOH_SIGMA4, kz.DOH_PAPER_LITERAL):
        with kz.Kaze(w, h, doh_norm=norm) as k:
            D = torch.empty((h, w), device="cuda")
            k.op_doh(dev(L), D, sigma, octave)
            torch.cuda.synchronize()
        ref = oracle.doh(L.astype(np.float64), sigma, octave, norm)
        assert np.max(np.abs(host(D) - ref)) <= DOH_REL_TOL * np.max(np.abs(ref))


def test_extrema_step_on_identical_responses(kz):
    # both sides read the same FP32 responses: comparisons are exact, so the
    # sets agree except for decisions sitting on a sub-pixel/edge boundary
    img = synth.workload_image("256x256")
    opt = oracle.Options.make(octaves=2, sublevels=4)
    lv, _ = oracle.build_scale_space(img, opt)
    D = oracle.detector_response(lv, opt).astype(np.float32)
    sig, _ = oracle.scale_table(2, 4, 1.6)
    with kz.Kaze(256, 256, octaves=2, sublevels=4) as k:
        kp_g = k.op_extrema(dev(D.reshape(-1, 256)).reshape(8, 256, 256), sig)
    kp_r = oracle.find_extrema(D.astype(np.float64), oracle.Options.make(
        octaves=2, sublevels=4, dthreshold=float(np.float32(0.001))))
    ov, m, ur, ug, md = compare(kp_r, kp_g, D.astype(np.float64))
    assert not ur and not ug
    assert len(kp_r) > 20 and ov == 1.0
    assert md < 1e-4


@pytest.mark.parametrize("thr", [0.001, 1e-9])
def test_listed_extrema_equal_the_full_scan(kz, thr):
    """After the response launch the extremum launch visits only the pixels it
    listed (above the threshold, one pixel inside, levels 1 .. N-2); with a
    threshold so low that the list overflows (over 65536 entries here) it
    scans every pixel.  Either way the keypoints are exactly those of the full
    scan of the same responses (kaze_op_extrema)."""
    img = synth.workload_image("256x256")
    with kz.Kaze(256, 256, octaves=2, sublevels=4, dthreshold=thr, max_keypoints=1 << 16) as k:
        kp = k.detect(dev(img))
        D = k.responses().clone()
        sig = [k.level_sigma(i) for i in range(8)]
        kp_full = k.op_extrema(D, sig)
        if thr < 1e-6:
            assert int((D[1:7, 1:-1, 1:-1] > thr).sum()) > 65536
    assert len(kp) > 20 and np.array_equal(kp, kp_full)


# -------------------------------------------------------------- pipeline --

def run_pipeline(kz, img, octaves, sublevels, k_override=0.0, **kw):
    h, w = img.shape
    with kz.Kaze(w, h, octaves=octaves, sublevels=sublevels, k_override=k_override, **kw) as k:
        x = dev(img)
        k.build_scale_space(x)
        kg = k.contrast()
        levels = host(k.levels())
        k.detector_response()
        D = host(k.responses())
        kp = k.find_extrema()
    return levels, D, kp, kg


def check_pipeline(kz, img, octaves, sublevels, check_k=True, **kw):
    opt0 = oracle.Options.make(octaves=octaves, sublevels=sublevels)
    L0 = oracle.gaussian(img.astype(np.float64), 1.6)
    k_ref, hmax_ref, _, _ = oracle.contrast_k(L0)
    if check_k:
        _, _, _, k_gpu = run_pipeline(kz, img, octaves, sublevels)
        assert abs(k_gpu - k_ref) <= hmax_ref / 300 * 1.0001 + 1e-7
    # compare the rest with the same k on both sides
    kf = float(np.float32(k_ref))
    lv_g, D_g, kp_g, _ = run_pipeline(kz, img, octaves, sublevels, k_override=kf, **kw)
    opt = oracle.Options.make(octaves=octaves, sublevels=sublevels, k_override=kf,
                              dthreshold=float(np.float32(0.001)))
    lv_r, D_r, kp_r, _ = oracle.kaze_detect(img.astype(np.float64), opt)
    err = np.max(np.abs(lv_g - lv_r), axis=(1, 2))
    assert np.all(err <= SCALE_TOL), err
    dmax = np.max(np.abs(D_r), axis=(1, 2))
    derr = np.max(np.abs(D_g - D_r), axis=(1, 2))
    assert np.all(derr <= DOH_REL_TOL * dmax + 1e-12), derr / dmax
    ov, m, ur, ug, md = compare(kp_r, kp_g, D_r)
    assert ov >= KP_OVERLAP, (ov, len(kp_r), len(kp_g), ur[:3], ug[:3])
    return lv_g, kp_g, kp_r


def test_pipeline_256(kz):
    img = synth.workload_image("256x256")
    _, kp_g, kp_r = check_pipeline(kz, img, 2, 4)
    assert len(kp_r) >= 30


def test_pipeline_ragged(kz):
    img = synth.image(257, 131, 11)
    check_pipeline(kz, img, 2, 4)


def test_pipeline_tiny_and_thin(kz):
    rng = np.random.default_rng(5)
    for shape in ((3, 3), (5, 40), (40, 5)):
        img = rng.random(shape).astype(np.float32)
        check_pipeline(kz, img, 1, 3)


def test_pipeline_g1_and_literal_norm(kz):
    img = synth.image(200, 150, 12)
    L0 = oracle.gaussian(img.astype(np.float64), 1.6)
    k_ref = float(np.float32(oracle.contrast_k(L0)[0]))
    lv_g, D_g, kp_g, _ = run_pipeline(kz, img, 2, 4, k_override=k_ref, diffusivity=1,
                                      doh_norm=kz.DOH_PAPER_LITERAL)
    opt = oracle.Options.make(octaves=2, sublevels=4, k_override=k_ref, diffusivity=1,
                              doh_norm=oracle.DOH_PAPER_LITERAL, dthreshold=float(np.float32(0.001)))
    lv_r, D_r, kp_r, _ = oracle.kaze_detect(img.astype(np.float64), opt)
    assert np.max(np.abs(lv_g - lv_r)) <= SCALE_TOL
    dmax = np.max(np.abs(D_r), axis=(1, 2))
    assert np.all(np.max(np.abs(D_g - D_r), axis=(1, 2)) <= DOH_REL_TOL * dmax + 1e-12)
    ov = compare(kp_r, kp_g, D_r)[0]
    assert ov >= KP_OVERLAP


def test_constant_image(kz):
    img = np.full((64, 80), 0.42, dtype=np.float32)
    lv, D, kp, k = run_pipeline(kz, img, 2, 4)
    assert k == pytest.approx(0.03)
    assert np.max(np.abs(lv - 0.42)) < 1e-6
    assert len(kp) == 0


def test_mean_preserved_and_max_principle(kz):
    img = synth.workload_image("256x256")
    lv, _, _, _ = run_pipeline(kz, img, 2, 4)
    m0 = lv[0].mean()
    for i in range(1, lv.shape[0]):
        assert abs(lv[i].mean() - m0) < 2e-6
        assert lv[i].min() >= lv[i - 1].min() - 1e-6 and lv[i].max() <= lv[i - 1].max() + 1e-6


def test_detect_graph_equals_eager_and_host_path(kz):
    img = synth.workload_image("256x256")
    with kz.Kaze(256, 256, octaves=2, sublevels=4) as k:
        x = dev(img)
        k.build_scale_space(x)
        k.detector_response()
        eager = k.find_extrema()
        g1 = k.detect(x)
        g2 = k.detect(x)  # replay
        hst = k.detect_host(img)
        pinned = torch.from_numpy(img).pin_memory()
        hp = k.detect_host(pinned)
    for other in (g1, g2, hst, hp):
        assert np.array_equal(eager, other)


def test_detect_host_next_streams_images(kz):
    """A stream of host images with the next one copied ahead (two input
    planes, two recorded graphs): every result equals the image detected on
    its own, also when a copied-ahead image is skipped, a device detection
    comes in between, or the size of the next image differs (rejected)."""
    imgs = [synth.image(320, 240, 50 + j) for j in range(4)]
    pinned = [torch.from_numpy(a).pin_memory() for a in imgs]
    with kz.Kaze(320, 240, octaves=2, sublevels=4) as k:
        alone = [k.detect_host(a) for a in imgs]
        assert all(len(r) > 0 for r in alone)
        got = [k.detect_host(pinned[0], next_image=pinned[1]),
               k.detect_host(pinned[1], next_image=pinned[2]),
               k.detect_host(pinned[2], next_image=pinned[3]),
               k.detect_host(pinned[3])]
        for a, b in zip(alone, got):
            assert np.array_equal(a, b)
        # copy ahead of 1, then detect 3 instead, then a device image, then 1
        r1 = k.detect_host(pinned[0], next_image=pinned[1])
        r3 = k.detect_host(pinned[3], next_image=pinned[2])
        rd = k.detect(dev(imgs[2]))
        r2 = k.detect_host(pinned[2], next_image=pinned[1])
        r4 = k.detect_host(pinned[1])
        for a, b in ((alone[0], r1), (alone[3], r3), (alone[2], rd), (alone[2], r2), (alone[1], r4)):
            assert np.array_equal(a, b)
        with pytest.raises(kz.KazeError):
            k.detect_host(pinned[0], next_image=torch.zeros((240, 300)).pin_memory())


def test_capacity_overflow_reports_true_count(kz):
    img = synth.workload_image("256x256")
    with kz.Kaze(256, 256, octaves=2, sublevels=4) as k:
        full = k.detect(dev(img))
        n = len(full)
        assert n > 5
        part = k.detect(dev(img), capacity=3)
        assert k.last_status == kz.ERR_CAPACITY and k.last_count == n
        assert np.array_equal(part, full[:3])
    with kz.Kaze(256, 256, octaves=2, sublevels=4, max_keypoints=4) as k:
        part = k.detect(dev(img))
        assert k.last_status == kz.ERR_CAPACITY and k.last_count == n and len(part) == 4


def test_invalid_arguments(kz):
    with kz.Kaze(64, 64) as k:
        with pytest.raises(kz.KazeError) as e:
            k.build_scale_space(torch.zeros((2, 64), device="cuda"))
        assert e.value.status == kz.ERR_INVALID_ARG
        with pytest.raises(kz.KazeError) as e:
            k.build_scale_space(torch.zeros((65, 64), device="cuda"))
        assert e.value.status == kz.ERR_INVALID_ARG
    with kz.Kaze(64, 64) as k:
        with pytest.raises(kz.KazeError) as e:
            k.detector_response()
        assert e.value.status == kz.ERR_STATE


# ------------------------------------------------------------- full size --

def test_full_size_1920x1200_against_oracle(kz):
    img = synth.workload_image("1920x1200")
    lv_g, kp_g, kp_r = check_pipeline(kz, img, 4, 4)
    assert len(kp_r) >= 100


def test_full_size_4096x3072_sampled_steps(kz):
    """4096x3072 (12.6 Mpx): the GPU pipeline end to end (every level keeps
    the mean of L_0, keypoints are found), and single steps at full size on
    inputs the oracle makes itself: the oracle's presmoothed image and its
    conductance feed two AOS steps (the step sizes of levels 1 and 15) and
    the response of level 9 on both sides."""
    img = synth.workload_image("4096x3072")
    h, w = img.shape
    sig, t = oracle.scale_table(4, 4, 1.6)
    L0 = oracle.gaussian(img.astype(np.float64), 1.6).astype(np.float32)
    kref = oracle.contrast_k(L0.astype(np.float64))[0]
    g = oracle.conductance(L0.astype(np.float64), kref, 1.0, oracle.G2).astype(np.float32)
    with kz.Kaze(w, h, octaves=4, sublevels=4) as k:
        x = dev(img)
        k.build_scale_space(x)
        k.detector_response()
        kp = k.find_extrema()
        means = [float(k.level(i, copy=False).double().mean()) for i in range(16)]
        L0d, gd = dev(L0), dev(g)
        ux, Ln, D = torch.empty_like(L0d), torch.empty_like(L0d), torch.empty_like(L0d)
        for i in (1, 15):
            tau = float(np.float32(t[i] - t[i - 1]))
            k.op_aos_step(L0d, gd, ux, Ln, tau)
            _, _, ref = oracle.aos_step(L0.astype(np.float64), g.astype(np.float64), tau)
            assert np.max(np.abs(host(Ln) - ref)) <= SCALE_TOL
        k.op_doh(L0d, D, float(np.float32(sig[9])), 2)
        ref = oracle.doh(L0.astype(np.float64), float(np.float32(sig[9])), 2)
        assert np.max(np.abs(host(D) - ref)) <= DOH_REL_TOL * np.max(np.abs(ref))
    assert max(abs(m - means[0]) for m in means) < 1e-5
    assert len(kp) >= 100


# ------------------------------------------------- sigma x sigma window --

def test_sigma_window_extrema_on_identical_responses(kz):
    """The exact cross-level window (reading W1) on the oracle's own FP32
    responses: comparisons are exact, so the keypoint sets agree up to
    decisions on a sub-pixel / edge boundary; the window keeps a subset of
    the 3x3x3 keypoints."""
    img = synth.workload_image("256x256")
    opt = oracle.Options.make(octaves=4, sublevels=4)
    lv, _ = oracle.build_scale_space(img, opt)
    D = oracle.detector_response(lv, opt).astype(np.float32)
    sig, _ = oracle.scale_table(4, 4, 1.6)
    with kz.Kaze(256, 256, octaves=4, sublevels=4, extrema_window=kz.EXTREMA_SIGMA_WINDOW) as k:
        kp_g = k.op_extrema(dev(D.reshape(-1, 256)).reshape(16, 256, 256), sig)
    with kz.Kaze(256, 256, octaves=4, sublevels=4) as k:
        kp_3 = k.op_extrema(dev(D.reshape(-1, 256)).reshape(16, 256, 256), sig)
    kp_r = oracle.find_extrema(D.astype(np.float64), oracle.Options.make(
        octaves=4, sublevels=4, dthreshold=float(np.float32(0.001)),
        extrema_window=oracle.EXTREMA_SIGMA_WINDOW))
    ov, m, ur, ug, md = compare(kp_r, kp_g, D.astype(np.float64))
    assert not ur and not ug
    assert len(kp_r) > 10 and ov == 1.0 and md < 1e-4
    key = lambda kp: {(int(p["level"]), int(p["ix"]), int(p["iy"])) for p in kp}
    assert key(kp_g) <= key(kp_3) and len(kp_g) < len(kp_3)


def test_sigma_window_pipeline_1920x1200(kz):
    img = synth.workload_image("1920x1200")
    with kz.Kaze(1920, 1200, extrema_window=kz.EXTREMA_SIGMA_WINDOW) as k:
        kp_w = k.detect(dev(img))
        D = host(k.responses())
    with kz.Kaze(1920, 1200) as k:
        kp_3 = k.detect(dev(img))
    key = lambda kp: {(int(p["level"]), int(p["ix"]), int(p["iy"])) for p in kp}
    assert key(kp_w) <= key(kp_3) and 0 < len(kp_w) < len(kp_3)
    # every kept keypoint is above its window one level below and above
    sig, _ = oracle.scale_table(4, 4, 1.6)
    for p in kp_w[:200]:
        i, x, y = int(p["level"]), int(p["ix"]), int(p["iy"])
        r = max(1, oracle.step_size(sig[i]) // 2)
        for l in (i - 1, i + 1):
            win = D[l, max(0, y - r):y + r + 1, max(0, x - r):x + r + 1]
            assert D[i, y, x] > win.max()


def test_batch_refuses_fed_and_window(kz):
    for bad in (dict(scheme=kz.SCHEME_FED), dict(extrema_window=kz.EXTREMA_SIGMA_WINDOW)):
        with pytest.raises(kz.KazeError):
            kz.Batch([(64, 64), (80, 48)], **bad)
