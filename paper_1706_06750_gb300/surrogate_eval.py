"""Judges the learned AOS surrogate against the plain GPU AOS path.

For every image, the same handle options run twice: once with AOS (the
method) and once with the surrogate standing in for every AOS step.  Reported:

* one-step error: the surrogate applied to AOS level L_{i-1} (with its
  conductance) against AOS level L_i, beside the error of skipping the step
  (L_{i-1} against L_i), RMS over pixels, per level;
* rollout error: the surrogate's own scale space against AOS, max |.| and RMS
  per level;
* keypoint repeatability: the share of AOS keypoints that the surrogate's
  detection reproduces on the same level within 1 and 2.5 pixels, and the
  share of surrogate keypoints that AOS confirms within 2.5 pixels;
* time: the scale space of one detection (presmoothing, contrast factor,
  conductances and the evolution; the resident AOS evolution takes them in
  one launch, the surrogate path in separate ones), with CUDA events from
  ``kaze_profile``, and a batched step of all images in one fused launch
  against one AOS step per image.

Only the library is used; the FP64 oracle plays no part here.
"""
from __future__ import annotations

import numpy as np


def match_share(a, b, radius):
    """Share of keypoints of `a` that have a keypoint of `b` on the same
    level within `radius` pixels (1.0 when `a` is empty)."""
    if len(a) == 0:
        return 1.0
    hit = 0
    for lv in np.unique(a["level"]):
        pa = a[a["level"] == lv]
        pb = b[b["level"] == lv]
        if len(pb) == 0:
            continue
        ax = pa["x"].astype(np.float64)[:, None]
        ay = pa["y"].astype(np.float64)[:, None]
        for s in range(0, len(pb), 4096):
            q = pb[s:s + 4096]
            d2 = (ax - q["x"][None, :]) ** 2 + (ay - q["y"][None, :]) ** 2
            near = (d2 <= radius * radius).any(axis=1)
            if s == 0:
                found = near
            else:
                found |= near
        hit += int(found.sum())
    return hit / len(a)




def evaluate(surrogate, images, octaves=4, sublevels=4, batch_reps=5):
    """`surrogate`: a kaze.Surrogate; `images`: 2-D float32 CUDA tensors of
    one size.  Returns a dict of the measurements listed above."""
    import torch

    from . import kaze
    h, w = images[0].shape
    aos = kaze.Kaze(w, h, octaves=octaves, sublevels=sublevels)
    sgk = kaze.Kaze(w, h, octaves=octaves, sublevels=sublevels)
    sgk.set_surrogate(surrogate)
    N = aos.n_levels
    one_step = np.zeros((len(images), N - 1))
    skip = np.zeros((len(images), N - 1))
    roll_max = np.zeros((len(images), N))
    roll_rms = np.zeros((len(images), N))
    rep1, rep25, conf25, n_aos, n_sg = [], [], [], [], []
    t_aos, t_sg = [], []
    prev_all, g_all, taus = [], [], None
    for j, img in enumerate(images):
        kp_a = aos.detect(img)
        lv_a = aos.levels()
        k = aos.contrast()
        kp_s = sgk.detect(img)
        lv_s = sgk.levels()
        t = [aos.level_time(i) for i in range(N)]
        taus = [t[i] - t[i - 1] for i in range(1, N)]
        for i in range(1, N):
            prev = lv_a[i - 1]
            g = torch.empty_like(prev)
            aos.op_conductance(prev, g, k)
            pred = torch.empty_like(prev)
            surrogate.step(prev, g, [taus[i - 1]], pred)
            torch.cuda.synchronize()
            one_step[j, i - 1] = float(torch.sqrt(torch.mean((pred.double() - lv_a[i].double()) ** 2)))
            skip[j, i - 1] = float(torch.sqrt(torch.mean((prev.double() - lv_a[i].double()) ** 2)))
            if i == 1:
                prev_all.append(prev)
                g_all.append(g)
        for i in range(N):
            d = (lv_s[i].double() - lv_a[i].double()).abs()
            roll_max[j, i] = float(d.max())
            roll_rms[j, i] = float(torch.sqrt(torch.mean(d * d)))
        rep1.append(match_share(kp_a, kp_s, 1.0))
        rep25.append(match_share(kp_a, kp_s, 2.5))
        conf25.append(match_share(kp_s, kp_a, 2.5))
        n_aos.append(len(kp_a))
        n_sg.append(len(kp_s))
        pa = aos.profile(img)
        ps = sgk.profile(img)
        # the scale space of one detection: everything but the response and extrema
        t_aos.append(sum(ms for kind, (ms, n) in pa.items() if kind not in ("doh", "extrema")))
        t_sg.append(sum(ms for kind, (ms, n) in ps.items() if kind not in ("doh", "extrema")))

    # batched step: every image's first step (L_0 and its conductance) in
    # one fused launch, against one AOS step per image (kaze_op_aos_step)
    n = len(images)
    Ls = prev_all
    gs = g_all
    outs = [torch.empty_like(Ls[0]) for _ in range(n)]
    ux = torch.empty_like(Ls[0])
    tau = taus[0]
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    for _ in range(2):
        surrogate.step(Ls, gs, [tau] * n, outs)
    st = surrogate.stream
    best_sg, best_aos = float("inf"), float("inf")
    for _ in range(batch_reps):
        torch.cuda.synchronize()
        ev[0].record(st)
        surrogate.step(Ls, gs, [tau] * n, outs)
        ev[1].record(st)
        st.synchronize()
        best_sg = min(best_sg, ev[0].elapsed_time(ev[1]))
        ev[2].record(aos.stream)
        for i in range(n):
            aos.op_aos_step(Ls[i], gs[i], ux, outs[i], tau)
        ev[3].record(aos.stream)
        aos.stream.synchronize()
        best_aos = min(best_aos, ev[2].elapsed_time(ev[3]))
    aos.close()
    sgk.close()
    return {
        "images": n, "size": [w, h], "levels": N,
        "one_step_rms": one_step.mean(axis=0).tolist(),
        "skip_step_rms": skip.mean(axis=0).tolist(),
        "one_step_gain": float(1.0 - one_step.mean() / skip.mean()),
        "rollout_max": roll_max.max(axis=0).tolist(),
        "rollout_rms": roll_rms.mean(axis=0).tolist(),
        "repeatability_1px": float(np.mean(rep1)),
        "repeatability_2_5px": float(np.mean(rep25)),
        "confirmed_2_5px": float(np.mean(conf25)),
        "keypoints_aos": int(np.sum(n_aos)), "keypoints_surrogate": int(np.sum(n_sg)),
        "evolution_ms_aos": float(np.mean(t_aos)), "evolution_ms_surrogate": float(np.mean(t_sg)),
        "batched_step_ms_surrogate": best_sg, "batched_step_ms_aos": best_aos,
    }


def time_step(w, h, n, path="fused", reps=10, warmup=3, checkpoint=None, seed=0):
    """Device time of one surrogate step over n seeded w x h planes (one
    launch for the fused paths), CUDA events on the surrogate's stream;
    returns ms per step and the rate in logical TFLOP/s of the 5-32-32-32-1
    network (2 x 9 x 2208 FLOP per pixel)."""
    import torch
    from . import kaze
    paths = {"fused": kaze.SURROGATE_FUSED, "fused_sync": kaze.SURROGATE_FUSED_SYNC,
             "layered": kaze.SURROGATE_LAYERED}
    s = kaze.Surrogate(max_w=w, max_h=h, max_samples=n, seed=seed)
    if checkpoint:
        s.load(checkpoint)
    gen = torch.Generator(device="cpu").manual_seed(seed)
    L = torch.rand(n, h, w, generator=gen).cuda()
    g = torch.rand(n, h, w, generator=gen).cuda()
    out = torch.empty_like(L)
    tau = [4.0] * n
    for _ in range(warmup):
        s.step(L, g, tau, out, path=paths[path])
    s.sync()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s.stream)
    for _ in range(reps):
        s.step(L, g, tau, out, path=paths[path])
    e1.record(s.stream)
    s.sync()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    s.close()
    flops = 2.0 * 9 * (5 * 32 + 32 * 32 + 32 * 32 + 32 * 1) * w * h * n
    return {"path": path, "images": n, "size": [w, h], "ms": ms, "tflops": flops / ms * 1e-9}


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser(description="Time one surrogate step on seeded planes.")
    ap.add_argument("--size", type=int, nargs=2, default=[1920, 1200], metavar=("W", "H"))
    ap.add_argument("--images", type=int, default=1)
    ap.add_argument("--path", choices=["fused", "fused_sync", "layered"], default="fused")
    ap.add_argument("--reps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--checkpoint", default=None)
    a = ap.parse_args()
    print(json.dumps(time_step(a.size[0], a.size[1], a.images, a.path, a.reps, a.warmup, a.checkpoint)))
