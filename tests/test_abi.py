"""CPU checks of the C ABI: the library builds for sm_103a, loads without a
GPU, exports every entry point include/kaze.h declares, and the host-side
struct layouts seen by the binding match the C header."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "kaze.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kaze_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libkaze():
    from paper_1706_06750_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(libkaze):
    names = declared_functions()
    assert "kaze_create" in names and "kaze_find_extrema" in names
    for n in names:
        assert hasattr(libkaze, n), n


def test_only_the_abi_is_exported():
    from paper_1706_06750_gb300 import build
    out = subprocess.check_output(["nm", "-D", "--defined-only", build.build()], text=True)
    syms = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert syms == set(declared_functions())


def test_struct_layout_matches_header(tmp_path):
    from paper_1706_06750_gb300 import kaze
    prog = tmp_path / "layout.c"
    prog.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "kaze.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu\\n\", sizeof(kaze_options),"
        " offsetof(kaze_options, k_percentile), offsetof(kaze_options, max_keypoints),"
        " sizeof(kaze_keypoint), offsetof(kaze_keypoint, iy)); return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    vals = [int(v) for v in subprocess.check_output([str(exe)], text=True).split()]
    assert vals == [ctypes.sizeof(kaze.Options), kaze.Options.k_percentile.offset,
                    kaze.Options.max_keypoints.offset, ctypes.sizeof(kaze.Keypoint),
                    kaze.Keypoint.iy.offset]


def test_host_only_entry_points_without_gpu(libkaze):
    from paper_1706_06750_gb300 import kaze
    o = kaze.default_options()
    assert (o.octaves, o.sublevels, o.nbins, o.diffusivity) == (4, 4, 300, kaze.G2)
    assert abs(o.sigma0 - 1.6) < 1e-6 and abs(o.k_percentile - 0.7) < 1e-15
    L = kaze.lib()
    assert L.kaze_status_string(kaze.ERR_CAPACITY) == b"keypoint capacity exceeded"
    # argument validation happens before any CUDA call
    h = ctypes.c_void_p()
    bad = kaze.default_options(octaves=0)
    assert L.kaze_create(ctypes.byref(bad), 64, 64, None, ctypes.byref(h)) == kaze.ERR_INVALID_ARG
    assert h.value is None
    assert b"octaves" in L.kaze_last_error(None)
    good = kaze.default_options()
    assert L.kaze_create(ctypes.byref(good), 2, 64, None, ctypes.byref(h)) == kaze.ERR_INVALID_ARG
    L.kaze_destroy(None)


def test_null_handles_are_rejected_without_gpu(libkaze):
    """Every entry point that takes a handle returns KAZE_ERR_INVALID_ARG for a
    NULL handle before touching the device (checked here on a machine with
    no GPU): the streaming host detection, the fused FED steps, the FED
    cycle and the single-step operators."""
    from paper_1706_06750_gb300 import kaze
    L = kaze.lib()
    n = ctypes.c_int()
    buf = (kaze.Keypoint * 4)()
    taus = (ctypes.c_float * 2)(0.1, 0.2)
    assert L.kaze_detect_host_next(None, None, None, 64, 64, 64, buf, 4, ctypes.byref(n)) == kaze.ERR_INVALID_ARG
    assert L.kaze_detect_host(None, None, 64, 64, 64, buf, 4, ctypes.byref(n)) == kaze.ERR_INVALID_ARG
    assert L.kaze_op_fed_steps(None, None, None, None, 64, 64, 64, taus, 2) == kaze.ERR_INVALID_ARG
    assert L.kaze_op_fed_cycle(None, None, None, None, None, 64, 64, 64, 1.0, ctypes.byref(n)) == kaze.ERR_INVALID_ARG
    assert L.kaze_op_conductance(None, None, None, 64, 64, 64, 0.02) == kaze.ERR_INVALID_ARG
