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


def launches_for(n):
    """A cycle of n steps runs as ceil(n / 4) launches of up to four steps."""
    return -(-n // 4)


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
        assert k.last_launch_count() == launches_for(n)
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
    space (same k on both sides), at the tolerances of the AOS pipeline:
    levels within 2e-5, responses within 1e-4 of each level's max |DoH|,
    keypoints >= 99.5 % (the cycle order keeps the FP32 rounding of a
    cycle to a few ulp times its amplification bound; measured errors stay
    below 1e-6 at 1920x1200, test_gpu_fullsize)."""
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
    steps = sum(launches_for(len(oracle.fed_tau(t[i] - t[i - 1]))) for i in range(1, 8))
    assert launches == 1 + 1 + 7 + steps + 1 + 1      # presmooth, set k, conductances, steps, doh, extrema
    err = np.max(np.abs(lv_g - lv_r), axis=(1, 2))
    assert np.all(err <= 2e-5), err
    dmax = np.max(np.abs(D_r), axis=(1, 2))
    derr = np.max(np.abs(D_g - D_r), axis=(1, 2))
    assert np.all(derr <= 1e-4 * dmax + 1e-12), derr / dmax
    ov, m, ur, ug, md = compare(kp_r, kp_g, D_r)
    assert len(kp_r) >= 10 and ov >= 0.995, (ov, len(kp_r), len(kp_g))


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


# ---- several explicit steps in one launch --------------------------------------

def cycle_head(dt, k):
    """The first k step sizes of the FED cycle reaching dt, in its step order."""
    t = oracle.fed_tau(dt)
    order, _ = oracle.fed_order(dt)
    return [float(np.float32(v)) for v in t[order][:k]]


@pytest.mark.parametrize("shape", [(3, 3), (5, 121), (97, 131), (33, 250), (40, 483), (1200, 1920)])
@pytest.mark.parametrize("k", [2, 3, 4])
def test_fused_steps_equal_single_steps(kz, shape, k):
    """k steps in one launch give, bit for bit, what k one-step launches give
    (the wavefront sums in the same order); the shapes cover one column of
    warps, a warp's ragged last lane, several warps and CTAs, and images
    shorter than a warp's rows."""
    h, w = shape
    L0, g = oracle_inputs(w, h, 40 + k + h)
    taus = cycle_head(67.9, k)
    with kz.Kaze(w, h) as kk:
        x, gd = padded(L0), padded(g)
        fused = padded(np.zeros_like(L0))
        kk.op_fed_steps(x, gd, fused, taus)
        assert kk.last_launch_count() == 1
        a, b = padded(np.zeros_like(L0)), padded(np.zeros_like(L0))
        src = x
        for j, t in enumerate(taus):
            dst = a if j % 2 == 0 else b
            kk.op_fed_steps(src, gd, dst, [t])
            src = dst
        torch.cuda.synchronize()
        assert torch.equal(fused, src)


@pytest.mark.parametrize("shape", [(97, 131), (256, 256)])
def test_fused_steps_match_oracle(kz, shape):
    h, w = shape
    L0, g = oracle_inputs(w, h, 7 + h)
    taus = cycle_head(30.0, 4)
    with kz.Kaze(w, h) as kk:
        x, gd, out = padded(L0), padded(g), padded(np.zeros_like(L0))
        kk.op_fed_steps(x, gd, out, taus)
        got = out.cpu().numpy().astype(np.float64)
    ref = L0.astype(np.float64)
    for t in taus:
        ref = oracle.fed_step(ref, g.astype(np.float64), t)
    tol = 8 * 2.0 ** -24 * amplification(np.array(taus)) * np.abs(L0).max() + 2.0 ** -22
    assert np.max(np.abs(got - ref)) <= tol


def test_fused_steps_ignore_row_padding(kz):
    """Whatever the padding columns beyond w hold (here NaN), the image's
    columns do not see it."""
    h, w = 20, 130
    L0, g = oracle_inputs(w, h, 3)
    with kz.Kaze(w, h) as kk:
        bufs = []
        for a in (L0, g):
            buf = torch.full((h, 132), float("nan"), device="cuda")
            buf[:, :w].copy_(torch.from_numpy(a))
            bufs.append(buf[:, :w])
        out = padded(np.zeros_like(L0))
        ref = padded(np.zeros_like(L0))
        taus = cycle_head(67.9, 4)
        kk.op_fed_steps(bufs[0], bufs[1], out, taus)
        kk.op_fed_steps(padded(L0), padded(g), ref, taus)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all() and torch.equal(out, ref)


def test_fused_steps_arguments_checked(kz):
    L0, g = oracle_inputs(64, 32, 1)
    with kz.Kaze(64, 32) as kk:
        x, gd, out = padded(L0), padded(g), padded(np.zeros_like(L0))
        for bad in ([], [0.1] * 5):
            with pytest.raises(kz.KazeError):
                kk.op_fed_steps(x, gd, out, bad)
        with pytest.raises(kz.KazeError):
            kk.op_fed_steps(x, gd, x, [0.1, 0.2])
        with pytest.raises(kz.KazeError):
            kk.op_fed_steps(x, gd, out, [0.1, float("inf")])
