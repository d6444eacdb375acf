"""Parity of the CUDA FED evolution (Eq. 5, scheme KAZE_SCHEME_FED) with the
FP64 oracle, through the C ABI.

Single cycles run on oracle-made inputs (the oracle's presmoothed image and
its conductance, rounded to FP32).  Tolerance: a cycle's FP32 rounding is
amplified by at most B = sum_j max|head_j| max|tail_j| (the worst-case bound
the step order is chosen by, computed here independently); each step rounds
a handful of times, so |gpu - oracle| <= 8 * 2^-24 * B * max|L| + 2^-22.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1706_06750_gb300 import synth  # noqa: E402

from kp_match import compare  # noqa: E402


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


def padded(a):
    """Device copy whose rows start on 16-byte boundaries (pitch % 4 == 0)."""
    h, w = a.shape
    buf = torch.zeros((h, (w + 3) // 4 * 4), device="cuda")
    v = buf[:, :w]
    v.copy_(torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)))
    return v


def amplification(t, lam=np.linspace(0.0, 8.0, 2001)):
    f = [np.abs(1.0 - tk * lam) for tk in t]
    b = 0.0
    for j in range(len(t)):
        head = np.prod(f[: j + 1], axis=0).max()
        tail = np.prod(f[j + 1:], axis=0).max() if j + 1 < len(t) else 1.0
        b += head * tail
    return b


def oracle_inputs(w, h, seed):
    img = synth.image(w, h, seed).astype(np.float64)
    L0 = oracle.gaussian(img, 1.6).astype(np.float32)
    k = oracle.contrast_k(L0.astype(np.float64))[0]
    g = oracle.conductance(L0.astype(np.float64), k, 1.0, oracle.G2).astype(np.float32)
    return L0, g


@pytest.mark.parametrize("shape", [(97, 131), (256, 256), (5, 64), (1200, 1920)])
@pytest.mark.parametrize("dt", [0.53, 5.0, 67.9])
def test_fed_cycle_matches_oracle(kz, shape, dt):
    h, w = shape
    if h * w > 1e6 and dt < 67:
        pytest.skip("full size only for the longest cycle")
    L0, g = oracle_inputs(w, h, 900 + h)
    with kz.Kaze(w, h) as k:
        x, gd = padded(L0), padded(g)
        scratch, out = padded(np.zeros_like(L0)), padded(np.zeros_like(L0))
        n = k.op_fed_cycle(x, gd, scratch, out, dt)
        assert k.last_launch_count() == n
        got = out.cpu().numpy().astype(np.float64)
    ref = oracle.fed_evolve(L0.astype(np.float64), g.astype(np.float64), dt)
    t = oracle.fed_tau(dt)
    assert n == len(t)
    order, _ = oracle.fed_order(dt)
    tol = 8 * 2.0 ** -24 * amplification(t[order]) * np.abs(L0).max() + 2.0 ** -22
    err = np.max(np.abs(got - ref))
    assert err <= tol, (err, tol)


def test_fed_zero_time_copies(kz):
    L0, g = oracle_inputs(40, 30, 5)
    with kz.Kaze(40, 30) as k:
        x, gd = padded(L0), padded(g)
        scratch, out = padded(np.zeros_like(L0)), padded(np.full_like(L0, 9.0))
        assert k.op_fed_cycle(x, gd, scratch, out, 0.0) == 0
        assert torch.equal(out, x)


def test_pipeline_fed_256(kz):
    """The whole detection with FED levels against the oracle's FED scale
    space (same k on both sides): levels within 1e-4, responses within
    1e-4 of each level's max |DoH| plus the level error propagated, and
    the keypoints agree (>= 99 %)."""
    img = synth.workload_image("256x256")
    s0 = float(np.float32(1.6))
    L0 = oracle.gaussian(img.astype(np.float64), s0)
    kref = oracle.contrast_k(L0)[0]
    kf = float(np.float32(kref))
    opt = oracle.Options.make(octaves=2, sublevels=4, sigma0=s0, k_override=kf, scheme=oracle.SCHEME_FED,
                              dthreshold=float(np.float32(0.001)))
    lv_r, D_r, kp_r, _ = oracle.kaze_detect(img.astype(np.float64), opt)
    with kz.Kaze(256, 256, octaves=2, sublevels=4, k_override=kf, scheme=kz.SCHEME_FED) as k:
        kp_g = k.detect(dev(img))
        launches = k.last_launch_count()
        lv_g = k.levels().cpu().numpy().astype(np.float64)
        D_g = k.responses().cpu().numpy().astype(np.float64)
    sig, t = oracle.scale_table(2, 4, s0)
    steps = sum(len(oracle.fed_tau(t[i] - t[i - 1])) for i in range(1, 8))
    assert launches == 1 + 1 + 7 + steps + 1 + 1      # presmooth, set k, conductances, steps, doh, extrema
    err = np.max(np.abs(lv_g - lv_r), axis=(1, 2))
    assert np.all(err <= 1e-4), err
    dmax = np.max(np.abs(D_r), axis=(1, 2))
    derr = np.max(np.abs(D_g - D_r), axis=(1, 2))
    assert np.all(derr <= 1e-3 * dmax + 1e-9), derr / dmax
    ov, m, ur, ug, md = compare(kp_r, kp_g, D_r)
    assert len(kp_r) >= 10 and ov >= 0.99, (ov, len(kp_r), len(kp_g))


def test_fed_full_size_invariants(kz):
    img = synth.workload_image("1920x1200")
    with kz.Kaze(1920, 1200, scheme=kz.SCHEME_FED) as k:
        kp = k.detect(dev(img))
        means = [float(k.level(i, copy=False).double().mean()) for i in range(16)]
        lo = min(float(k.level(i, copy=False).min()) for i in range(16))
        hi = max(float(k.level(i, copy=False).max()) for i in range(16))
    assert max(abs(m - means[0]) for m in means) < 1e-5
    assert -1e-3 <= lo and hi <= 1.0 + 1e-3
    assert len(kp) >= 100
    with kz.Kaze(64, 48, scheme=kz.SCHEME_FED) as k:
        k.detect(dev(np.full((48, 64), 0.25, np.float32)))
        assert float((k.levels() - 0.25).abs().max()) < 1e-6


def test_fed_options_validated(kz):
    for bad in (dict(scheme=2), dict(scheme=kz.SCHEME_FED, fed_tau_max=0.3), dict(fed_tau_max=0.0)):
        with pytest.raises(kz.KazeError):
            kz.Kaze(64, 64, **bad)
