"""Seeded synthetic grayscale images shaped like the paper's workloads.

The paper times KAZE on photographs of 8 sizes from 240x400 to 1920x1200
(Sec. IV); that image set is not available, so these seeded images stand in
for it.  This module holds no part of the method's arithmetic: it only draws
pixels, and both the CUDA path and the CPU oracle consume its output.

Recipe (all draws from ``numpy.random.default_rng(seed)``):
  1. a constant 0.5 background;
  2. 40 Gaussian blobs: centre uniform over the image, standard deviation
     log-uniform in [1.5, min(W, H)/16], amplitude uniform in [-0.45, 0.45];
  3. 10 axis-aligned rectangles: corner uniform, sides uniform in
     [0.05, 0.3] x the image dimension, added value uniform in [-0.3, 0.3];
  4. optionally (the 4096x3072 workload) 4 plane sinusoids of amplitude 0.05,
     period log-uniform in [4, 64] px, orientation uniform in [0, pi), phase
     uniform in [0, 2 pi);
  5. Gaussian noise of standard deviation 0.01;
  6. clipped to [0, 1] and stored as float32.
"""
from __future__ import annotations

import numpy as np

# Sizes of the batched workload, (W, H).
BATCH_SIZES = ((640, 480), (1280, 720), (1920, 1080), (1920, 1200))


def image(w: int, h: int, seed: int, n_blobs: int = 40, n_rects: int = 10,
          sinusoids: bool = False, noise_std: float = 0.01) -> np.ndarray:
    """One seeded float32 image of shape (h, w) with values in [0, 1]."""
    rng = np.random.default_rng(seed)
    img = np.full((h, w), 0.5, dtype=np.float64)
    ys = np.arange(h, dtype=np.float64)[:, None]
    xs = np.arange(w, dtype=np.float64)[None, :]

    smax = max(min(w, h) / 16.0, 1.5)
    for _ in range(n_blobs):
        cx = rng.uniform(0, w)
        cy = rng.uniform(0, h)
        sd = float(np.exp(rng.uniform(np.log(1.5), np.log(smax))))
        amp = rng.uniform(-0.45, 0.45)
        # Only a window of +-5 std is touched; beyond it the blob is < 4e-6.
        r = int(np.ceil(5 * sd))
        x0, x1 = max(0, int(cx) - r), min(w, int(cx) + r + 1)
        y0, y1 = max(0, int(cy) - r), min(h, int(cy) + r + 1)
        if x0 >= x1 or y0 >= y1:
            continue
        dx2 = (xs[:, x0:x1] - cx) ** 2
        dy2 = (ys[y0:y1, :] - cy) ** 2
        img[y0:y1, x0:x1] += amp * np.exp(-(dx2 + dy2) / (2 * sd * sd))

    for _ in range(n_rects):
        rw = max(1, int(rng.uniform(0.05, 0.3) * w))
        rh = max(1, int(rng.uniform(0.05, 0.3) * h))
        x0 = int(rng.uniform(0, w))
        y0 = int(rng.uniform(0, h))
        val = rng.uniform(-0.3, 0.3)
        img[y0:y0 + rh, x0:x0 + rw] += val

    if sinusoids:
        for _ in range(4):
            period = float(np.exp(rng.uniform(np.log(4.0), np.log(64.0))))
            theta = rng.uniform(0, np.pi)
            phase = rng.uniform(0, 2 * np.pi)
            img += 0.05 * np.sin(2 * np.pi * (xs * np.cos(theta) + ys * np.sin(theta))
                                 / period + phase)

    img += rng.normal(0.0, noise_std, size=(h, w))
    return np.clip(img, 0.0, 1.0).astype(np.float32)


def workload_image(name: str, j: int = 0) -> np.ndarray:
    """Image j of a named workload (seed = 1000 * workload number + j)."""
    if name == "256x256":
        return image(256, 256, 1000 + j)
    if name == "1920x1200":
        return image(1920, 1200, 2000 + j)
    if name == "4096x3072":
        return image(4096, 3072, 3000 + j, sinusoids=True)
    raise KeyError(name)


def batch_sizes(n: int = 64, seed: int = 4000):
    """Sizes (W, H) of the mixed-size batch, drawn uniformly from BATCH_SIZES."""
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, len(BATCH_SIZES), size=n)
    return [BATCH_SIZES[i] for i in idx]


def batch_images(n: int = 64, seed: int = 4000):
    """The mixed-size batch: image j has seed 4000 + j."""
    return [image(w, h, seed + j) for j, (w, h) in enumerate(batch_sizes(n, seed))]


def training_crop(j: int, size: int = 512) -> np.ndarray:
    """Crop j of the learned surrogate's training set: a size x size window
    of a 1920x1200 image of the recipe above (seed 5000 + j), at a position
    drawn from ``default_rng(100000 + j)``."""
    img = image(1920, 1200, 5000 + j)
    rng = np.random.default_rng(100000 + j)
    x0 = int(rng.integers(0, 1920 - size + 1))
    y0 = int(rng.integers(0, 1200 - size + 1))
    return np.ascontiguousarray(img[y0:y0 + size, x0:x0 + size])
