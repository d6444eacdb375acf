"""The resident AOS evolution (kaze_options.aos_solver = KAZE_AOS_AUTO: all
N-1 steps of Eq. 4 in one cooperative launch, 128 x 120 tiles held in shared
memory, lines solved in chunks coupled through their end values) against the
FP64 oracle, on sizes that exercise one tile, ragged tiles, lines shorter than
a chunk and the full 1920x1200 workload; against the line kernels
(KAZE_AOS_LINES); and its bounded grid-barrier waits."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1706_06750_gb300 import synth  # noqa: E402

SCALE_TOL = 2e-5


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


def gpu_levels(kz, img, octaves, sublevels, k, **kw):
    h, w = img.shape
    with kz.Kaze(w, h, octaves=octaves, sublevels=sublevels, k_override=k, **kw) as kh:
        kh.build_scale_space(dev(img))
        lv = kh.levels().cpu().numpy().astype(np.float64)
        prof = kh.profile(dev(img))
    return lv, prof


def oracle_levels(img, octaves, sublevels, k, **kw):
    opt = oracle.Options.make(octaves=octaves, sublevels=sublevels, k_override=k, **kw)
    lv, _ = oracle.build_scale_space(img.astype(np.float64), opt)
    return lv


def k_of(img):
    L0 = oracle.gaussian(img.astype(np.float64), 1.6)
    return float(np.float32(oracle.contrast_k(L0)[0]))


@pytest.mark.parametrize("shape", [(120, 128), (121, 129), (131, 257), (240, 384), (3, 3), (7, 300),
                                   (300, 7), (16, 17)])
def test_resident_scale_space_against_oracle(kz, shape):
    h, w = shape
    img = synth.image(w, h, 40 + h + w) if min(h, w) >= 16 else \
        np.random.default_rng(h * 1000 + w).random(shape).astype(np.float32)
    k = k_of(img)
    lv_g, prof = gpu_levels(kz, img, 2, 4, k)
    # presmoothing, the contrast factor and every step in one launch
    assert prof["front_evolve"][1] == 1, prof
    for kind in ("presmooth", "grad_max", "grad_hist", "aos_rows", "aos_cols", "conductance", "aos_evolve"):
        assert prof[kind][1] == 0, (kind, prof)
    lv_r = oracle_levels(img, 2, 4, k)
    err = np.max(np.abs(lv_g - lv_r), axis=(1, 2))
    assert np.all(err <= SCALE_TOL), err


def test_resident_g1_against_oracle(kz):
    img = synth.image(250, 190, 77)
    k = k_of(img)
    lv_g, prof = gpu_levels(kz, img, 2, 4, k, diffusivity=kz.G1)
    assert prof["front_evolve"][1] == 1
    lv_r = oracle_levels(img, 2, 4, k, diffusivity=oracle.G1)
    assert np.max(np.abs(lv_g - lv_r)) <= SCALE_TOL


def test_resident_and_line_kernels_at_1920x1200(kz):
    """Both solvers of the same method against the oracle on the workload
    image (4 x 4 levels, 150 tiles): each within the scale-space tolerance."""
    img = synth.workload_image("1920x1200")
    k = k_of(img)
    lv_a, prof = gpu_levels(kz, img, 4, 4, k)
    assert prof["front_evolve"][1] == 1
    lv_l, prof_l = gpu_levels(kz, img, 4, 4, k, aos_solver=kz.AOS_LINES)
    assert prof_l["front_evolve"][1] == 0 and prof_l["aos_rows"][1] == 15
    lv_r = oracle_levels(img, 4, 4, k)
    ea = np.max(np.abs(lv_a - lv_r), axis=(1, 2))
    el = np.max(np.abs(lv_l - lv_r), axis=(1, 2))
    assert np.all(ea <= SCALE_TOL), ea
    assert np.all(el <= SCALE_TOL), el
    # mean preserved (Neumann lines, symmetric operators)
    m = lv_a.reshape(16, -1).mean(axis=1)
    assert np.max(np.abs(m - m[0])) < 2e-6


def test_resident_too_large_falls_back_to_lines(kz):
    # 32 x 26 tiles do not fit one per SM: the line kernels run; the streamed
    # tile passes (three launches a step) when asked for
    x = torch.rand(3072, 4096, device="cuda")
    with kz.Kaze(4096, 3072, octaves=1, sublevels=2) as kh:
        prof = kh.profile(x)
    assert prof["front_evolve"][1] == 0 and prof["stream_a"][1] == 0 and prof["aos_rows"][1] == 1
    with kz.Kaze(4096, 3072, octaves=1, sublevels=2, aos_solver=kz.AOS_STREAMED) as kh:
        prof = kh.profile(x)
    assert prof["aos_rows"][1] == 0
    assert prof["stream_a"][1] == 1 and prof["stream_x"][1] == 1 and prof["stream_b"][1] == 1


@pytest.mark.parametrize("shape", [(120, 128), (121, 129), (131, 257), (240, 384), (3, 3), (7, 300),
                                   (300, 7), (16, 17)])
def test_streamed_scale_space_against_oracle(kz, shape):
    """The streamed tile passes (forced) against the oracle: one tile, ragged
    tiles, lines shorter than a chunk."""
    h, w = shape
    img = synth.image(w, h, 40 + h + w) if min(h, w) >= 16 else \
        np.random.default_rng(h * 1000 + w).random(shape).astype(np.float32)
    k = k_of(img)
    lv_g, prof = gpu_levels(kz, img, 2, 4, k, aos_solver=kz.AOS_STREAMED)
    assert prof["stream_b"][1] == 7 and prof["front_evolve"][1] == 0, prof
    lv_r = oracle_levels(img, 2, 4, k)
    err = np.max(np.abs(lv_g - lv_r), axis=(1, 2))
    assert np.all(err <= SCALE_TOL), err


def test_streamed_g1_and_1920x1200_against_oracle(kz):
    img = synth.image(250, 190, 77)
    k = k_of(img)
    lv_g, _ = gpu_levels(kz, img, 2, 4, k, diffusivity=kz.G1, aos_solver=kz.AOS_STREAMED)
    lv_r = oracle_levels(img, 2, 4, k, diffusivity=oracle.G1)
    assert np.max(np.abs(lv_g - lv_r)) <= SCALE_TOL
    img = synth.workload_image("1920x1200")
    k = k_of(img)
    lv_g, _ = gpu_levels(kz, img, 4, 4, k, aos_solver=kz.AOS_STREAMED)
    lv_r = oracle_levels(img, 4, 4, k)
    err = np.max(np.abs(lv_g - lv_r), axis=(1, 2))
    assert np.all(err <= SCALE_TOL), err


def test_stalled_barrier_times_out_and_the_handle_recovers(kz):
    img = synth.image(400, 300, 5)
    x = dev(img)
    with kz.Kaze(400, 300, octaves=2, sublevels=4) as kh:
        ref = kh.detect(x)
        kh.set_evolve_wait_limit(1 << 22, stall_tile=1)
        with pytest.raises(kz.KazeError) as e:
            kh.detect(x)
        assert e.value.status == kz.ERR_TIMEOUT
        kh.set_evolve_wait_limit(0, -1)
        again = kh.detect(x)
    assert np.array_equal(ref, again)


@pytest.mark.parametrize("shape", [(1200, 1920), (131, 257), (7, 300)])
def test_resident_front_matches_the_separate_kernels(kz, shape):
    """With the presmoothing and the contrast factor inside the resident
    launch, L_0 and the histogram's percentile are those of the presmoothing
    and contrast kernels (the same operations in the same order): L_0 and k
    are equal bit for bit, and every later level within FP32 rounding of the
    line kernels' (which start from the same L_0 and k)."""
    h, w = shape
    img = synth.image(w, h, 21 + h) if min(shape) >= 16 else \
        np.random.default_rng(3).random(shape).astype(np.float32)
    x = dev(img)
    with kz.Kaze(w, h, octaves=2, sublevels=4) as a, kz.Kaze(w, h, octaves=2, sublevels=4,
                                                           aos_solver=kz.AOS_LINES) as b:
        a.build_scale_space(x)
        b.build_scale_space(x)
        assert a.contrast() == b.contrast()
        la, lb = a.levels(), b.levels()
        assert torch.equal(la[0], lb[0])
        assert (la - lb).abs().max().item() <= 2 * SCALE_TOL
        pa = a.profile(x)
    assert pa["front_evolve"][1] == 1 and pa["presmooth"][1] == 0 and pa["grad_max"][1] == 0
