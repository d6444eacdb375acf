"""Writes the learned surrogate's training pairs, computed by the FP64 oracle
alone (no CUDA code is involved).

Pair (j, i), i = 0 .. N-2, of crop j (``synth.training_crop(j)``): the level
L_i of the crop's nonlinear scale space (Sec. II-A), its conductance g_i
(Eq. 2-3 with the crop's contrast factor k), the step tau_i = t_{i+1} - t_i
(Eq. 7) and the next level L_{i+1}, the AOS step of Eq. 4 from (L_i, g_i,
tau_i).  Crops are added until `--pairs` pairs exist.

Output, float32 in DIR:
  levels.npy  [crops, N, S, S]   L_0 .. L_{N-1}
  cond.npy    [crops, N-1, S, S] g_0 .. g_{N-2}
  meta.json   sizes, taus, the k of every crop, the pair count

    python oracle/make_surrogate_pairs.py --out DIR [--pairs 2000] [--size 512]
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def one_crop(args):
    j, size, octaves, sublevels = args
    import oracle
    from paper_1706_06750_gb300 import synth
    img = synth.training_crop(j, size)
    opt = oracle.Options.make(octaves=octaves, sublevels=sublevels)
    levels, k = oracle.build_scale_space(img, opt)
    cond = np.stack([oracle.conductance(levels[i], k) for i in range(len(levels) - 1)])
    return j, levels.astype(np.float32), cond.astype(np.float32), k


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--out", required=True)
    ap.add_argument("--pairs", type=int, default=2000)
    ap.add_argument("--size", type=int, default=512)
    ap.add_argument("--octaves", type=int, default=4)
    ap.add_argument("--sublevels", type=int, default=4)
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 1)
    a = ap.parse_args(argv)
    import oracle
    oracle.build()
    n_levels = a.octaves * a.sublevels
    crops = -(-a.pairs // (n_levels - 1))
    os.makedirs(a.out, exist_ok=True)
    levels = np.lib.format.open_memmap(os.path.join(a.out, "levels.npy"), mode="w+", dtype=np.float32,
                                       shape=(crops, n_levels, a.size, a.size))
    cond = np.lib.format.open_memmap(os.path.join(a.out, "cond.npy"), mode="w+", dtype=np.float32,
                                     shape=(crops, n_levels - 1, a.size, a.size))
    ks = [0.0] * crops
    t0 = time.time()
    jobs = [(j, a.size, a.octaves, a.sublevels) for j in range(crops)]
    with mp.get_context("spawn").Pool(max(1, min(a.workers, crops))) as pool:
        for j, lv, cd, k in pool.imap_unordered(one_crop, jobs):
            levels[j] = lv
            cond[j] = cd
            ks[j] = k
    levels.flush()
    cond.flush()
    _, t = oracle.scale_table(a.octaves, a.sublevels, 1.6)
    meta = {"crops": crops, "size": a.size, "octaves": a.octaves, "sublevels": a.sublevels,
            "levels": n_levels, "pairs": a.pairs, "taus": np.diff(t).tolist(), "k": ks,
            "crop_seeds": [5000 + j for j in range(crops)], "seconds": time.time() - t0}
    with open(os.path.join(a.out, "meta.json"), "w") as f:
        json.dump(meta, f, indent=1)
    print(json.dumps({k: meta[k] for k in ("crops", "pairs", "seconds")}))


if __name__ == "__main__":
    main()
