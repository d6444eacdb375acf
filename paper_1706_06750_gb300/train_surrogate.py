"""Trains the learned AOS surrogate on the GPU with the library's own
forward, backward and Adam kernels (kaze_surrogate_train_step).

Training data: the pair set that ``oracle/make_surrogate_pairs.py`` writes
(levels.npy, cond.npy, meta.json).  Pair (j, i) asks the network to map
(L_i, g_i, tau_i) of crop j to L_{i+1}; the first ``meta["pairs"]`` pairs in
(crop, level) order form the training set.  The arrays are uploaded to the
GPU once; each step draws ``--batch`` pairs from a seeded permutation
(reshuffled every epoch) and passes their device planes to the library.
The learning rate follows a cosine from ``--lr`` down to ``--lr / 20``.
Every ``--log-every`` steps the loss of a fixed probe batch (pairs spread
evenly over the set) is logged beside the batch loss.

    python -m paper_1706_06750_gb300.train_surrogate --pairs DIR --out CKPT \\
        [--steps 20000] [--batch 8] [--lr 1e-3] [--seed 0] [--resume CKPT] \\
        [--checkpoint-every 1000]

Prints one JSON line per ``--log-every`` steps and a final summary line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np


def load_pairs(d):
    with open(os.path.join(d, "meta.json")) as f:
        meta = json.load(f)
    levels = np.load(os.path.join(d, "levels.npy"), mmap_mode="r")
    cond = np.load(os.path.join(d, "cond.npy"), mmap_mode="r")
    n_lv = meta["levels"]
    index = [(j, i) for j in range(meta["crops"]) for i in range(n_lv - 1)][: meta["pairs"]]
    return meta, levels, cond, index


def lr_at(step, steps, lr):
    """Cosine from lr (step 0) to lr / 20 (last step)."""
    c = 0.5 * (1.0 + math.cos(math.pi * min(step, steps) / max(1, steps)))
    return lr / 20.0 + (lr - lr / 20.0) * c


def train(pairs_dir, out, steps=20000, batch=8, lr=1e-3, seed=0, resume=None, checkpoint_every=1000,
          log_every=100, log=print):
    import torch

    from . import kaze
    meta, levels_np, cond_np, index = load_pairs(pairs_dir)
    size = meta["size"]
    taus = np.asarray(meta["taus"], dtype=np.float32)
    levels = torch.from_numpy(np.array(levels_np)).cuda()
    cond = torch.from_numpy(np.array(cond_np)).cuda()
    s = kaze.Surrogate(size, size, batch, train=True, seed=seed)
    if resume:
        s.load(resume)
    start = s.steps_taken()
    # a fixed probe batch (spread over crops and levels) whose loss is
    # logged beside the noisy per-batch loss
    probe = [index[k] for k in np.linspace(0, len(index) - 1, batch).astype(int)]
    pL = [levels[j, i] for j, i in probe]
    pg = [cond[j, i] for j, i in probe]
    pT = [levels[j, i + 1] for j, i in probe]
    ptau = [float(taus[i]) for _, i in probe]
    rng = np.random.default_rng(seed)
    order = np.concatenate([rng.permutation(len(index)) for _ in range((steps * batch) // len(index) + 2)])
    t0 = time.time()
    hist = []
    for step in range(start, steps):
        pick = [index[k] for k in order[step * batch:(step + 1) * batch]]
        L = [levels[j, i] for j, i in pick]
        g = [cond[j, i] for j, i in pick]
        T = [levels[j, i + 1] for j, i in pick]
        tau = [float(taus[i]) for _, i in pick]
        want = (step + 1) % log_every == 0 or step == start or step + 1 == steps
        loss = s.train_step(L, g, tau, T, lr_at(step, steps, lr), want_loss=want)
        if want:
            probe_loss, _ = s.gradients(pL, pg, ptau, pT)
            hist.append((step + 1, probe_loss))
            log(json.dumps({"step": step + 1, "loss": loss, "probe_loss": probe_loss,
                            "lr": lr_at(step, steps, lr), "seconds": round(time.time() - t0, 2)}))
        if checkpoint_every and (step + 1) % checkpoint_every == 0 and step + 1 < steps:
            s.save(out)
    torch.cuda.synchronize()
    s.save(out)
    return {"steps": steps, "batch": batch, "pairs": len(index), "seconds": time.time() - t0,
            "first_probe_loss": hist[0][1] if hist else None, "final_probe_loss": hist[-1][1] if hist else None,
            "checkpoint": out}


def main(argv=None):
    ap = argparse.ArgumentParser(description="Train the learned AOS surrogate on oracle pairs.")
    ap.add_argument("--pairs", required=True)
    ap.add_argument("--out", required=True)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--resume", default=None)
    ap.add_argument("--checkpoint-every", type=int, default=1000)
    ap.add_argument("--log-every", type=int, default=100)
    a = ap.parse_args(argv)
    from . import build
    build.build()
    r = train(a.pairs, a.out, a.steps, a.batch, a.lr, a.seed, a.resume, a.checkpoint_every, a.log_every)
    print(json.dumps(r))
    return 0


if __name__ == "__main__":
    sys.exit(main())
