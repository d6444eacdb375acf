"""FP64 oracle of keypoint description (Sec. II-C): the dominant orientation
and the 64-D M-SURF descriptor of a keypoint on its nonlinear scale level.

TEST INFRASTRUCTURE ONLY.  This is the plain, slow restatement of the
description step that the CUDA path is checked against.  Only the test
suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import it.  It shares no code with the CUDA library.

Readings of the paper (which leaves these details open or prints them
garbled), in the order the computation uses them:

D1  First derivatives of level L_i at pixel (u, v): the step-s Scharr pair
    of the detector (s = s_i = max(1, round(sigma_i))), on the half-sample
    symmetric extension of L_i:
        L_x = sum_b c_b (L(u+s, v+b s) - L(u-s, v+b s)) / (2 s),
        c = (3, 10, 3) / 16 for b = -1, 0, 1;  L_y is the transpose.
D2  Values between pixels by bilinear interpolation of the pixel values;
    each of the four taps is clamped into the image.
D3  Orientation samples at (x + a sigma_i, y + b sigma_i) for integers a, b
    with a^2 + b^2 < 36 (radius 6 sigma_i, step sigma_i), each weighted by a
    Gaussian of std 2.5 sigma_i centred on the keypoint.
D4  Dominant orientation: the response angles fall into 72 sectors of 5
    degrees; a window of 12 consecutive sectors (pi / 3) slides over the 72
    start sectors; the window whose summed response is longest wins (the
    first on ties) and its summed vector gives the angle, in [0, 2 pi); no
    response at all gives 0.
D5  Descriptor geometry: 4 x 4 subregions in the keypoint's frame (x' along
    the orientation, y' = x' turned by +90 degrees); subregion (p, q) is
    centred at ((p - 1.5) 5, (q - 1.5) 5) sigma_i and holds 9 x 9 samples
    spaced sigma_i (offsets -4 .. 4), i.e. 9 sigma_i wide, overlapping its
    neighbours by 2 sigma_i; the window spans 24 sigma_i.
D6  Sample weight: Gaussian of std 2.5 sigma_i around the subregion centre;
    responses are turned into the keypoint's frame
        r_x' = L_x cos(theta) + L_y sin(theta),
        r_y' = -L_x sin(theta) + L_y cos(theta);
    subregion vector (sum r_x', sum r_y', sum |r_x'|, sum |r_y'|), weighted
    by a Gaussian of std 1.5 in units of the 4 x 4 subregion grid, centred
    on the keypoint (std 1.5 sigma_i in pixels would leave the outer ring at
    ~1e-11 of the inner one).
D7  Layout: entry 4 (4 q + p) + c for component c of subregion (p, q); the
    64 entries are divided by their Euclidean norm (left at 0 if it is 0).
D8  Upright mode (no rotation invariance): theta = 0.

Parity status: pinned (tests/test_oracle_describe.py: ramp and parabola
closed forms, 90-degree rotation covariance, mirror symmetry, intensity
invariance, orientation of planted response clusters).
"""
from __future__ import annotations

import math

import numpy as np

ORI_RADIUS2 = 36      # a^2 + b^2 < 36
ORI_STD = 2.5
SECTORS = 72
WINDOW = 12           # sectors per window: 12 * 5 degrees = pi / 3
SUB_SPACING = 5.0
SUB_HALF = 4
SUB_STD = 2.5
GRID_STD = 1.5
DESC_LEN = 64


def step_size(sigma: float) -> int:
    """s_i = max(1, round(sigma_i)), half away from zero (the detector's step)."""
    s = int(math.floor(sigma + 0.5))
    return max(1, s)


def reflect(i: np.ndarray, n: int) -> np.ndarray:
    """Half-sample symmetric reflection into [0, n), repeated as often as needed."""
    i = np.asarray(i, dtype=np.int64)
    period = 2 * n
    m = np.mod(i, period)
    return np.where(m < n, m, period - 1 - m)


def first_derivatives(L: np.ndarray, s: int):
    """D1: L_x, L_y of the whole level (float64 arrays [H, W])."""
    L = np.asarray(L, dtype=np.float64)
    H, W = L.shape
    xs = np.arange(W)
    ys = np.arange(H)
    c = (3.0 / 16.0, 10.0 / 16.0, 3.0 / 16.0)

    def at(dx, dy):
        return L[np.ix_(reflect(ys + dy, H), reflect(xs + dx, W))]

    Lx = np.zeros((H, W))
    Ly = np.zeros((H, W))
    for k, b in enumerate((-1, 0, 1)):
        Lx += c[k] * (at(s, b * s) - at(-s, b * s)) / (2.0 * s)
        Ly += c[k] * (at(b * s, s) - at(b * s, -s)) / (2.0 * s)
    return Lx, Ly


def bilinear(img: np.ndarray, px: np.ndarray, py: np.ndarray) -> np.ndarray:
    """D2: bilinear interpolation at real positions, taps clamped into the image."""
    H, W = img.shape
    x0 = np.floor(px)
    y0 = np.floor(py)
    fx = px - x0
    fy = py - y0
    x0 = x0.astype(np.int64)
    y0 = y0.astype(np.int64)
    xa = np.clip(x0, 0, W - 1)
    xb = np.clip(x0 + 1, 0, W - 1)
    ya = np.clip(y0, 0, H - 1)
    yb = np.clip(y0 + 1, 0, H - 1)
    return ((1.0 - fx) * (1.0 - fy) * img[ya, xa] + fx * (1.0 - fy) * img[ya, xb]
            + (1.0 - fx) * fy * img[yb, xa] + fx * fy * img[yb, xb])


def orientation_samples():
    """D3: the integer offsets (a, b) of the orientation samples and their weights."""
    a, b = np.meshgrid(np.arange(-6, 7), np.arange(-6, 7), indexing="xy")
    keep = a * a + b * b < ORI_RADIUS2
    a = a[keep].astype(np.float64)
    b = b[keep].astype(np.float64)
    w = np.exp(-(a * a + b * b) / (2.0 * ORI_STD * ORI_STD))
    return a, b, w


def dominant_orientation(rx: np.ndarray, ry: np.ndarray) -> float:
    """D4: angle of the longest summed response over the pi/3 windows."""
    rx = np.asarray(rx, dtype=np.float64)
    ry = np.asarray(ry, dtype=np.float64)
    phi = np.arctan2(ry, rx)
    phi = np.where(phi < 0.0, phi + 2.0 * math.pi, phi)
    q = np.floor(phi * (SECTORS / (2.0 * math.pi))).astype(np.int64)
    q = np.clip(q, 0, SECTORS - 1)
    sx = np.bincount(q, weights=rx, minlength=SECTORS)
    sy = np.bincount(q, weights=ry, minlength=SECTORS)
    best, bx, by = -1.0, 0.0, 0.0
    for k in range(SECTORS):
        idx = [(k + m) % SECTORS for m in range(WINDOW)]
        wx = float(np.sum(sx[idx]))
        wy = float(np.sum(sy[idx]))
        n2 = wx * wx + wy * wy
        if n2 > best:
            best, bx, by = n2, wx, wy
    if best <= 0.0:
        return 0.0
    t = math.atan2(by, bx)
    return t + 2.0 * math.pi if t < 0.0 else t


def orientation(Lx, Ly, x: float, y: float, sigma: float) -> float:
    """D3 + D4 for a keypoint at (x, y) on a level of scale sigma."""
    a, b, w = orientation_samples()
    px = x + a * sigma
    py = y + b * sigma
    return dominant_orientation(w * bilinear(Lx, px, py), w * bilinear(Ly, px, py))


def descriptor(Lx, Ly, x: float, y: float, sigma: float, theta: float) -> np.ndarray:
    """D5 - D7: the 64-D M-SURF vector for orientation theta."""
    co, si = math.cos(theta), math.sin(theta)
    u, v = np.meshgrid(np.arange(-SUB_HALF, SUB_HALF + 1), np.arange(-SUB_HALF, SUB_HALF + 1), indexing="xy")
    u = u.ravel().astype(np.float64)
    v = v.ravel().astype(np.float64)
    w1 = np.exp(-(u * u + v * v) / (2.0 * SUB_STD * SUB_STD))
    out = np.zeros(DESC_LEN)
    for q in range(4):
        for p in range(4):
            cp = (p - 1.5) * SUB_SPACING
            cq = (q - 1.5) * SUB_SPACING
            du = cp + u                      # offsets in the keypoint frame, units of sigma
            dv = cq + v
            px = x + sigma * (du * co - dv * si)
            py = y + sigma * (du * si + dv * co)
            gx = bilinear(Lx, px, py)
            gy = bilinear(Ly, px, py)
            rxp = gx * co + gy * si
            ryp = -gx * si + gy * co
            w2 = math.exp(-((p - 1.5) ** 2 + (q - 1.5) ** 2) / (2.0 * GRID_STD * GRID_STD))
            base = 4 * (4 * q + p)
            out[base + 0] = w2 * np.sum(w1 * rxp)
            out[base + 1] = w2 * np.sum(w1 * ryp)
            out[base + 2] = w2 * np.sum(w1 * np.abs(rxp))
            out[base + 3] = w2 * np.sum(w1 * np.abs(ryp))
    n = math.sqrt(float(np.sum(out * out)))
    return out / n if n > 0.0 else out


def describe_level(L: np.ndarray, sigma: float, points, upright: bool = False, thetas=None):
    """Orientation and descriptor of every (x, y) in ``points`` on one level.

    ``thetas``, if given, replaces the orientation step (the descriptor is then
    evaluated at those angles).  Returns (angles [n], descriptors [n, 64])."""
    Lx, Ly = first_derivatives(L, step_size(sigma))
    n = len(points)
    ang = np.zeros(n)
    desc = np.zeros((n, DESC_LEN))
    for i, (x, y) in enumerate(points):
        if thetas is not None:
            t = float(thetas[i])
        elif upright:
            t = 0.0
        else:
            t = orientation(Lx, Ly, float(x), float(y), sigma)
        ang[i] = t
        desc[i] = descriptor(Lx, Ly, float(x), float(y), sigma, t)
    return ang, desc
