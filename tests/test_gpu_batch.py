"""The batched persistent path (kaze_batch_*) against the single-image path
and the oracle, its solve-tile shapes and its bounded waits (needs a GPU)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1706_06750_gb300 import synth  # noqa: E402

from kp_match import compare  # noqa: E402

SIZES = [(160, 120), (257, 131), (96, 96), (64, 200), (300, 40), (130, 130)]


@pytest.fixture(scope="module")
def kz():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1706_06750_gb300 import build, kaze
    build.build()
    oracle.build()
    return kaze


def images(sizes, seed0=500):
    return [synth.image(w, h, seed0 + j) for j, (w, h) in enumerate(sizes)]


def single_path(kz, img, **kw):
    h, w = img.shape
    with kz.Kaze(w, h, octaves=2, sublevels=4, **kw) as k:
        x = torch.from_numpy(img).cuda()
        k.build_scale_space(x)
        kval = k.contrast()
        lv = k.levels().cpu().numpy()
        k.detector_response()
        D = k.responses().cpu().numpy()
        kp = k.find_extrema()
    return lv, D, kp, kval


def test_batch_matches_single_image_path(kz):
    """The default batch execution (the resident evolution: the same tile
    code as the single-image launch) against the single-image path."""
    imgs = images(SIZES)
    xs = [torch.from_numpy(a).cuda() for a in imgs]
    with kz.Batch(SIZES, octaves=2, sublevels=4) as b:
        assert b.tuning()[0] == kz.BATCH_RESIDENT
        kps = b.detect(xs)
        for i, img in enumerate(imgs):
            lv, D, kp, _ = single_path(kz, img)
            for l in range(8):
                assert np.max(np.abs(b.level(i, l).cpu().numpy() - lv[l])) <= 2e-6, (i, l)
                dm = np.max(np.abs(D[l]))
                assert np.max(np.abs(b.response(i, l).cpu().numpy() - D[l])) <= 1e-5 * dm + 1e-12, (i, l)
            ov = compare(kp, kps[i], D.astype(np.float64))[0]
            assert ov >= 0.995, (i, len(kp), len(kps[i]))


@pytest.mark.parametrize("tuning", [(0, 4, 1, 8), (0, 4, 2, 8), (0, 8, 1, 8), (0, 8, 2, 8),
                                    (1, 4, 2, 2), (1, 4, 2, 16), (2, 4, 1, 8)])
def test_every_execution_shape_gives_the_same_result(kz, tuning):
    """Against the work-queue launch with 4-column strips: the other shapes
    of the line solvers within FP32 rounding of one another (2e-6); the
    resident evolution (chunked spike solves) within twice the oracle
    tolerance, as two solvers each within 2e-5 of the oracle."""
    imgs = images(SIZES, 700)
    xs = [torch.from_numpy(a).cuda() for a in imgs]
    ltol, dtol = (4e-5, 2e-4) if tuning[0] == kz.BATCH_RESIDENT else (2e-6, 1e-5)
    with kz.Batch(SIZES, octaves=2, sublevels=4) as b:
        b.set_tuning(kz.BATCH_PERSISTENT, 4, 2, 8)
        ref = b.detect(xs)
        L7 = [b.level(i, 7).cpu().numpy() for i in range(len(SIZES))]
        D5 = [b.response(i, 5).cpu().numpy() for i in range(len(SIZES))]
        b.set_tuning(*tuning)
        assert b.tuning() == tuning
        got = b.detect(xs)
        for i in range(len(SIZES)):
            assert np.max(np.abs(b.level(i, 7).cpu().numpy() - L7[i])) <= ltol
            assert np.max(np.abs(b.response(i, 5).cpu().numpy() - D5[i])) <= dtol * np.max(np.abs(D5[i]))
            a = {(int(r["level"]), int(r["iy"]), int(r["ix"])) for r in got[i]}
            e = {(int(r["level"]), int(r["iy"]), int(r["ix"])) for r in ref[i]}
            assert len(a & e) >= 0.995 * max(len(a), len(e), 1)


def test_batch_against_oracle(kz):
    img = synth.image(200, 150, 901)
    L0 = oracle.gaussian(img.astype(np.float64), 1.6)
    kf = float(np.float32(oracle.contrast_k(L0)[0]))
    x = torch.from_numpy(img).cuda()
    with kz.Batch([(200, 150), (96, 64)], octaves=2, sublevels=4, k_override=kf) as b:
        kps = b.detect([x, torch.rand(64, 96, device="cuda")])
        lv = np.stack([b.level(0, l).cpu().numpy() for l in range(8)]).astype(np.float64)
        D = np.stack([b.response(0, l).cpu().numpy() for l in range(8)]).astype(np.float64)
    opt = oracle.Options.make(octaves=2, sublevels=4, k_override=kf, dthreshold=float(np.float32(0.001)))
    lv_r, D_r, kp_r, _ = oracle.kaze_detect(img.astype(np.float64), opt)
    assert np.max(np.abs(lv - lv_r)) <= 2e-5
    dmax = np.max(np.abs(D_r), axis=(1, 2))
    assert np.all(np.max(np.abs(D - D_r), axis=(1, 2)) <= 1e-4 * dmax + 1e-12)
    assert compare(kp_r, kps[0], D_r)[0] >= 0.995


def test_stalled_dependency_times_out_and_the_handle_recovers(kz):
    imgs = images(SIZES[:3], 800)
    xs = [torch.from_numpy(a).cuda() for a in imgs]
    with kz.Batch(SIZES[:3], octaves=2, sublevels=4) as b:
        ref = b.detect(xs)
        b.set_wait_limit(1 << 24, stall_image=1)  # ~10 ms per wait
        with pytest.raises(kz.KazeError) as e:
            b.detect(xs)
        assert e.value.status == kz.ERR_TIMEOUT
        b.set_wait_limit(1 << 31, stall_image=-1)
        again = b.detect(xs)
        for i in range(3):
            assert np.array_equal(again[i], ref[i])


def test_mixed_size_workload_sample(kz):
    """The 64-image mixed-size workload: the default execution (the resident
    evolution) against the concurrent one (line solvers): two FP32 solvers,
    each held to 99.5 % keypoint overlap with the oracle, so at least 99 %
    with each other; three images against the single-image path (the same
    arithmetic: no keypoint off a decision boundary may differ); keypoint
    counts sane for all."""
    sizes = synth.batch_sizes(64)
    imgs = synth.batch_images(64)
    xs = [torch.from_numpy(a).cuda() for a in imgs]
    with kz.Batch(sizes) as b:
        kps = b.detect(xs)
        D = {i: np.stack([b.response(i, l).cpu().numpy() for l in range(16)]).astype(np.float64)
             for i in (0, 17, 63)}
        b.set_tuning(kz.BATCH_CONCURRENT, 4, 2, 8)
        kpc = b.detect(xs)
    assert all(len(k) > 10 for k in kps)
    total = sum(len(k) for k in kps)
    common = 0
    for a, c in zip(kps, kpc):
        sa = {(int(r["level"]), int(r["iy"]), int(r["ix"])) for r in a}
        sc = {(int(r["level"]), int(r["iy"]), int(r["ix"])) for r in c}
        common += len(sa & sc)
    assert common >= 0.99 * total
    # three images against the single-image path; keypoints that differ
    # must sit on a decision boundary of the response
    for i in (0, 17, 63):
        h, w = imgs[i].shape
        with kz.Kaze(w, h) as k:
            ref = k.detect(xs[i])
        ov, m, ur, ug, md = compare(ref, kps[i], D[i])
        assert ov >= 0.995 and not ur and not ug, (i, ov, ur[:2], ug[:2])


def test_handle_build_batch_equals_batch_object(kz):
    """kaze_build_batch on a handle runs the same batch as kaze_batch_* and
    keeps it while the size list repeats."""
    sizes = SIZES[:3]
    imgs = images(sizes, 950)
    xs = [torch.from_numpy(a).cuda() for a in imgs]
    with kz.Batch(sizes, octaves=2, sublevels=4) as b:
        ref = b.detect(xs)
    with kz.Kaze(4096, 4096, octaves=2, sublevels=4) as k:
        got = k.build_batch(xs)
        again = k.build_batch(xs)
        for a, r, g in zip(got, ref, again):
            assert np.array_equal(a, r) and np.array_equal(g, r)
        with pytest.raises(kz.KazeError):
            k.build_batch([torch.zeros((2, 64), device="cuda")])
    with kz.Kaze(256, 256, scheme=kz.SCHEME_FED) as k:
        with pytest.raises(kz.KazeError):
            k.build_batch(xs)


def test_resident_mode_needs_every_image_to_fit(kz):
    """A batch with an image of more tiles than SMs (4096x3072: 32 x 26 tiles
    of 128 x 120) starts in the work-queue execution, refuses the resident
    one (and keeps its tuning), and detects; a batch of small images starts
    resident."""
    sizes = [(4096, 3072), (640, 480)]
    xs = [torch.rand(h, w, device="cuda") for w, h in sizes]
    with kz.Batch(sizes, octaves=1, sublevels=3) as b:
        assert b.tuning()[0] == kz.BATCH_PERSISTENT
        with pytest.raises(kz.KazeError):
            b.set_tuning(kz.BATCH_RESIDENT, 4, 1, 8)
        assert b.tuning()[0] == kz.BATCH_PERSISTENT
        kps = b.detect(xs)
        assert len(kps) == 2
    with kz.Batch(SIZES, octaves=1, sublevels=3) as b:
        assert b.tuning()[0] == kz.BATCH_RESIDENT
