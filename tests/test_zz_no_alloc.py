"""The AOS step that allocates nothing (kaze_aos_step_static), for callers
that cannot let the library allocate device memory.  Checked against the
handle-based kaze_op_aos_step on the same inputs, on two calls in a row (the
second call reuses the shared scratch array the first one left behind).
Collected last on purpose: a failure here leaves every other test run."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def kz():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1706_06750_gb300 import build, kaze
    build.build()
    return kaze


def _inputs(seed, h, w, pitch):
    rng = np.random.default_rng(seed)
    L = rng.random((h, w)).astype(np.float32)
    g = (0.05 + 0.95 * rng.random((h, w))).astype(np.float32)
    Lp = torch.zeros((h, pitch), device="cuda")[:, :w]
    Gp = torch.zeros((h, pitch), device="cuda")[:, :w]
    Lp.copy_(torch.from_numpy(L))
    Gp.copy_(torch.from_numpy(g))
    return Lp, Gp


def test_static_step_matches_handle_step_twice(kz):
    h, w = 1200, 1920
    pitch = (w + 31) // 32 * 32
    with kz.Kaze(w, h) as k:
        for call, (seed, tau) in enumerate([(1, 0.53), (2, 67.9)]):
            Lp, Gp = _inputs(seed, h, w, pitch)
            ux = torch.zeros((h, pitch), device="cuda")[:, :w]
            ref = torch.zeros((h, pitch), device="cuda")[:, :w]
            out = torch.full((h, pitch), float("nan"), device="cuda")[:, :w]
            k.op_aos_step(Lp, Gp, ux, ref, tau)
            torch.cuda.synchronize()
            st = kz.aos_step_static(Lp, Gp, out, tau)
            torch.cuda.synchronize()
            assert st == kz.OK, f"call {call}: status {st}"
            assert torch.isfinite(out).all()
            # the same kernels on the same inputs: the same bits
            assert torch.equal(out, ref), f"call {call}: max |static - handle| = {(out - ref).abs().max().item()}"


def test_static_step_rejects_sizes_beyond_its_scratch(kz):
    h, w = 2100, 2100  # pitch * h = 2112 * 2100 > 4 Mi floats
    pitch = (w + 31) // 32 * 32
    Lp, Gp = _inputs(3, h, w, pitch)
    out = torch.zeros((h, pitch), device="cuda")[:, :w]
    assert kz.aos_step_static(Lp, Gp, out, 1.0) == kz.ERR_INVALID_ARG


def test_static_step_rejects_an_output_overlapping_an_input(kz):
    # an output one row below the input shares all but one row with it
    h, w = 64, 96
    pitch = (w + 31) // 32 * 32
    Lp, Gp = _inputs(4, h + 1, w, pitch)
    assert kz.aos_step_static(Lp[:h], Gp[:h], Lp[1:], 1.0) == kz.ERR_INVALID_ARG
    assert kz.aos_step_static(Lp[:h], Gp[:h], Gp[1:], 1.0) == kz.ERR_INVALID_ARG
