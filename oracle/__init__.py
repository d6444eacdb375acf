"""FP64 CPU oracle of the KAZE nonlinear scale space and detector.

TEST INFRASTRUCTURE ONLY.  The oracle is the plain, slow restatement of the
method (arXiv 1706.06750, Sec. II and III) that the CUDA path is checked
against.  Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it.  It shares no code with the CUDA library.

The arithmetic lives in ``kaze_oracle.c`` (compiled with gcc into
``oracle/_build/libkaze_oracle.so``); this module only marshals numpy arrays.
Images are 2-D arrays indexed ``[y, x]``; every floating-point value is
float64.

Parity status per function (which external facts pin it is listed in the
test files ``tests/test_oracle_*.py``): every function here is pinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kaze_oracle.c")
_HDR = os.path.join(_HERE, "kaze_oracle.h")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libkaze_oracle.so")
_lock = threading.Lock()
_lib = None

G1 = 1
G2 = 2
DOH_SIGMA4 = 0
DOH_PAPER_LITERAL = 1
SCHEME_AOS = 0
SCHEME_FED = 1
EXTREMA_3X3 = 0
EXTREMA_SIGMA_WINDOW = 1


class Options(ctypes.Structure):
    """Mirror of ``ko_options``; defaults are the workloads' settings."""

    _fields_ = [
        ("octaves", ctypes.c_int),
        ("sublevels", ctypes.c_int),
        ("sigma0", ctypes.c_double),
        ("sigma_d", ctypes.c_double),
        ("k_percentile", ctypes.c_double),
        ("nbins", ctypes.c_int),
        ("diffusivity", ctypes.c_int),
        ("dthreshold", ctypes.c_double),
        ("edge_r", ctypes.c_double),
        ("doh_norm", ctypes.c_int),
        ("k_override", ctypes.c_double),
        ("scheme", ctypes.c_int),
        ("fed_tau_max", ctypes.c_double),
        ("extrema_window", ctypes.c_int),
    ]

    @classmethod
    def make(cls, octaves=4, sublevels=4, sigma0=1.6, sigma_d=1.0,
             k_percentile=0.7, nbins=300, diffusivity=G2, dthreshold=0.001,
             edge_r=10.0, doh_norm=DOH_SIGMA4, k_override=0.0, scheme=0, fed_tau_max=0.25, extrema_window=0):
        return cls(octaves, sublevels, sigma0, sigma_d, k_percentile, nbins,
                   diffusivity, dthreshold, edge_r, doh_norm, k_override, scheme, fed_tau_max,
                   extrema_window)


class Keypoint(ctypes.Structure):
    _fields_ = [
        ("x", ctypes.c_double),
        ("y", ctypes.c_double),
        ("sigma", ctypes.c_double),
        ("response", ctypes.c_double),
        ("level", ctypes.c_int),
        ("octave", ctypes.c_int),
        ("sublevel", ctypes.c_int),
        ("ix", ctypes.c_int),
        ("iy", ctypes.c_int),
    ]


KEYPOINT_DTYPE = np.dtype([
    ("x", np.float64), ("y", np.float64), ("sigma", np.float64),
    ("response", np.float64), ("level", np.int32), ("octave", np.int32),
    ("sublevel", np.int32), ("ix", np.int32), ("iy", np.int32),
], align=True)
assert KEYPOINT_DTYPE.itemsize == ctypes.sizeof(Keypoint)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, no architecture flags)."""
    with _lock:
        fresh = (os.path.exists(_LIB_PATH)
                 and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)
                 and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_HDR))
        if fresh and not force:
            return _LIB_PATH
        os.makedirs(_BUILD_DIR, exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        # loops over independent pixels and lines on every host core where
        # gcc offers OpenMP (the same results with any thread count)
        try:
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                                   "-o", tmp, _SRC, "-lm"], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                                   "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    dp = ctypes.POINTER(ctypes.c_double)
    i = ctypes.c_int
    d = ctypes.c_double
    sig = {
        "ko_reflect": (ctypes.c_long, [ctypes.c_long, ctypes.c_long]),
        "ko_set_threads": (None, [i]),
        "ko_threads": (i, []),
        "ko_scale_table": (None, [i, i, d, dp, dp]),
        "ko_gaussian_weights": (i, [d, dp, i]),
        "ko_gaussian": (None, [dp, dp, i, i, d]),
        "ko_scharr": (None, [dp, dp, dp, i, i]),
        "ko_contrast_k": (d, [dp, i, i, d, d, i, dp,
                              ctypes.POINTER(ctypes.c_longlong),
                              ctypes.POINTER(ctypes.c_longlong)]),
        "ko_conductance": (None, [dp, i, i, d, d, i, dp]),
        "ko_thomas": (None, [i, dp, dp, dp, dp, dp]),
        "ko_aos_step": (None, [dp, dp, i, i, d, dp, dp, dp]),
        "ko_fed_tau": (i, [d, d, dp, i]),
        "ko_fed_order": (i, [i, dp, ctypes.POINTER(ctypes.c_int)]),
        "ko_fed_step": (None, [dp, dp, i, i, d, dp]),
        "ko_fed_evolve": (i, [dp, dp, i, i, d, d, dp]),
        "ko_build_scale_space": (i, [dp, i, i, ctypes.POINTER(Options), dp, dp]),
        "ko_step_size": (i, [d]),
        "ko_hessian": (None, [dp, i, i, i, dp, dp, dp]),
        "ko_doh": (None, [dp, i, i, d, i, i, dp]),
        "ko_find_extrema": (i, [dp, i, i, i, i, dp, d, d, i,
                                ctypes.POINTER(Keypoint), i]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _c(a):
    """C-contiguous float64 copy/view and its pointer."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _out(shape):
    a = np.empty(shape, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def reflect(i: int, n: int) -> int:
    return int(_load().ko_reflect(i, n))


def set_threads(n: int) -> None:
    """Host threads for the oracle's loops over independent pixels and lines
    (the results do not depend on it)."""
    _load().ko_set_threads(int(n))


def threads() -> int:
    return int(_load().ko_threads())


def scale_table(octaves: int, sublevels: int, sigma0: float = 1.6):
    """Eq. 6 (reading: sigma0 * 2^(o + s/S)) and Eq. 7 (t = sigma^2 / 2)."""
    n = octaves * sublevels
    s, sp = _out(n)
    t, tp = _out(n)
    _load().ko_scale_table(octaves, sublevels, sigma0, sp, tp)
    return s, t


def gaussian_weights(sigma: float) -> np.ndarray:
    w, wp = _out(1024)
    r = _load().ko_gaussian_weights(sigma, wp, 1024)
    if r < 0:
        raise ValueError("sigma too large")
    return w[: 2 * r + 1].copy()


def gaussian(img, sigma: float) -> np.ndarray:
    img, ip = _c(img)
    h, w = img.shape
    out, op = _out((h, w))
    _load().ko_gaussian(ip, op, w, h, sigma)
    return out


def scharr(img):
    img, ip = _c(img)
    h, w = img.shape
    lx, xp = _out((h, w))
    ly, yp = _out((h, w))
    _load().ko_scharr(ip, xp, yp, w, h)
    return lx, ly


def contrast_k(L0, sigma_d=1.0, pct=0.7, nbins=300):
    """Returns (k, hmax, histogram, number of binned pixels)."""
    L0, lp = _c(L0)
    h, w = L0.shape
    hmax = ctypes.c_double(0.0)
    hist = np.zeros(nbins, dtype=np.int64)
    n = ctypes.c_longlong(0)
    k = _load().ko_contrast_k(
        lp, w, h, sigma_d, pct, nbins, ctypes.byref(hmax),
        hist.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), ctypes.byref(n))
    return float(k), float(hmax.value), hist, int(n.value)


def conductance(L, k: float, sigma_d=1.0, diffusivity=G2) -> np.ndarray:
    L, lp = _c(L)
    h, w = L.shape
    g, gp = _out((h, w))
    _load().ko_conductance(lp, w, h, sigma_d, k, diffusivity, gp)
    return g


def thomas(a, b, c, d) -> np.ndarray:
    a, ap = _c(a)
    b, bp = _c(b)
    c, cp = _c(c)
    d, dp = _c(d)
    n = d.shape[0]
    x, xp = _out(n)
    _load().ko_thomas(n, ap, bp, cp, dp, xp)
    return x


def aos_step(Lprev, g, tau: float):
    """Returns (ux, uy, Lnext) of one AOS step."""
    Lprev, lp = _c(Lprev)
    g, gp = _c(g)
    h, w = Lprev.shape
    ux, uxp = _out((h, w))
    uy, uyp = _out((h, w))
    ln, lnp = _out((h, w))
    _load().ko_aos_step(lp, gp, w, h, tau, uxp, uyp, lnp)
    return ux, uy, ln


def fed_tau(dt: float, tau_max: float = 0.25) -> np.ndarray:
    """Step sizes of one FED cycle reaching stopping time dt (Eq. 5)."""
    n = _load().ko_fed_tau(dt, tau_max, None, 0)
    t, tp = _out((max(n, 1),))
    _load().ko_fed_tau(dt, tau_max, tp, n)
    return t[:n]


def fed_order(dt: float, tau_max: float = 0.25):
    """(order, kappa): the step order of the FED cycle reaching dt (reading F5)."""
    t = fed_tau(dt, tau_max)
    n = len(t)
    order = (ctypes.c_int * max(n, 1))()
    tt, tp = _c(t if n else np.zeros(1))
    kappa = _load().ko_fed_order(n, tp, order)
    return np.array(order[:n], dtype=np.int64), int(kappa)


def fed_step(L, g, tau: float) -> np.ndarray:
    """One explicit step with fixed conductance (flux form, no flux through the border)."""
    L, lp = _c(L)
    g, gp = _c(g)
    h, w = L.shape
    out, op = _out((h, w))
    _load().ko_fed_step(lp, gp, w, h, tau, op)
    return out


def fed_evolve(L, g, dt: float, tau_max: float = 0.25) -> np.ndarray:
    """One FED cycle from L to stopping time dt with fixed conductance g."""
    L, lp = _c(L)
    g, gp = _c(g)
    h, w = L.shape
    out, op = _out((h, w))
    _load().ko_fed_evolve(lp, gp, w, h, dt, tau_max, op)
    return out


def build_scale_space(img, opt: Options | None = None):
    """Returns (levels [N, H, W], k)."""
    opt = opt or Options.make()
    img, ip = _c(img)
    h, w = img.shape
    n = opt.octaves * opt.sublevels
    lv, lvp = _out((n, h, w))
    k = ctypes.c_double(0.0)
    rc = _load().ko_build_scale_space(ip, w, h, ctypes.byref(opt), lvp, ctypes.byref(k))
    if rc != 0:
        raise ValueError("ko_build_scale_space failed")
    return lv, float(k.value)


def step_size(sigma: float) -> int:
    return int(_load().ko_step_size(sigma))


def hessian(L, s: int):
    L, lp = _c(L)
    h, w = L.shape
    xx, xxp = _out((h, w))
    yy, yyp = _out((h, w))
    xy, xyp = _out((h, w))
    _load().ko_hessian(lp, w, h, s, xxp, yyp, xyp)
    return xx, yy, xy


def doh(L, sigma_i: float, octave: int, doh_norm=DOH_SIGMA4) -> np.ndarray:
    L, lp = _c(L)
    h, w = L.shape
    D, Dp = _out((h, w))
    _load().ko_doh(lp, w, h, sigma_i, octave, doh_norm, Dp)
    return D


def detector_response(levels, opt: Options | None = None) -> np.ndarray:
    """DoH of every level, [N, H, W]."""
    opt = opt or Options.make()
    sig, _ = scale_table(opt.octaves, opt.sublevels, opt.sigma0)
    return np.stack([doh(levels[i], sig[i], i // opt.sublevels, opt.doh_norm)
                     for i in range(levels.shape[0])])


def find_extrema(D, opt: Options | None = None, cap: int = 1 << 20) -> np.ndarray:
    """Keypoints (structured array, KEYPOINT_DTYPE) sorted by (level, iy, ix)."""
    opt = opt or Options.make()
    D, dp = _c(D)
    n, h, w = D.shape
    sig, _ = scale_table(opt.octaves, opt.sublevels, opt.sigma0)
    sig, sp = _c(sig[:n])
    out = (Keypoint * max(cap, 1))()
    cnt = _load().ko_find_extrema(dp, w, h, n, opt.sublevels, sp, opt.dthreshold,
                                  opt.edge_r, opt.extrema_window, out, cap)
    if cnt > cap:
        raise ValueError(f"{cnt} keypoints exceed cap {cap}")
    arr = np.frombuffer(out, dtype=KEYPOINT_DTYPE, count=cnt).copy()
    return np.sort(arr, order=["level", "iy", "ix"])


def kaze_detect(img, opt: Options | None = None):
    """Scale space + detector response + extrema of one image.

    Returns (levels, DoH, keypoints, k)."""
    opt = opt or Options.make()
    lv, k = build_scale_space(img, opt)
    D = detector_response(lv, opt)
    kp = find_extrema(D, opt)
    return lv, D, kp, k
