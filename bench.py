"""Throughput of the KAZE scale space + detector on GB300.

One step = one whole detection of one 1920x1200 float32 image (4 octaves x 4
sublevels): presmoothing, contrast factor, 15 AOS steps, the detector
response of all 16 levels and the 3x3x3 extrema with the keypoint count and
slots copied to the host -- kaze_detect_enqueue through the C ABI, replaying
its recorded CUDA graph (kaze_detect_collect, the host's wait and sort,
follows each step's end event).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line on rank 0.  `value` (Mpixel/s) comes from CUDA events
around each step with the input already in HBM; L2 is flushed (a 256 MiB
memset) before every step, outside the events.  `e2e` is the same metric
through kaze_detect_host_next on a stream of pinned host images: every
step copies an image to the device (the next step's, on a second stream
while this one is detected; two input planes) and reads the keypoints
back, all inside the events; `e2e.single` is kaze_detect_host, one image
copied and detected after the other.  `roofline` takes the kernel with the
largest share of device time, measured with per-launch CUDA events
(kaze_profile) right after the timed region.  `cpu_baseline` times the FP64
CPU oracle on a bounded sample of the same workload.
Under torchrun (N > 1) every rank detects its own images (independent
replicas, no collective on the data path) and the slowest rank's time sets
the whole-job throughput.
Two sections ride along on the same line: `batched` (64 mixed-size images:
the autotuned batch execution against image-after-image detection) and
`surrogate` (the learned AOS stand-in judged by AOS on 16 images, with the
tensor-core roofline of its fused kernel).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpixel/s KAZE scale-space+detector at 1920x1200"
UNIT = "Mpixel/s"
W_IMG, H_IMG = 1920, 1200
OCTAVES, SUBLEVELS = 4, 4
WORKLOAD = "1920x1200 float32 image, 4 octaves x 4 sublevels, scale space + detector response + extrema"
L2_FLUSH_BYTES = 256 << 20
KEYPOINT_SLOTS = 4096  # keypoints a detection copies to the host with the count
FALLBACK_HBM_GBS = 6800.0


def env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


# ------------------------------------------------------------------ clocks --

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------- roofline --

def algorithmic_bytes(kind, pixels, n_levels, nbins=300):
    """Minimum bytes a kernel kind must move in one detection (FP32 planes,
    P pixels, N levels), from the method's data flow:
      presmoothing       read I, write L_0                          8 P
      contrast factor    two reads of L_0 (maximum, histogram)      8 P  (4 + 4)
      each AOS step      pass A: read L_i-1, write g, write u_x    12 P
                         pass B: read L_i-1, g, u_x, write L_i     16 P
      detector response  read L_i, write DoH_i per level            8 P
      extrema            read DoH_i once per level                  4 P
    in all P (40 N - 12) bytes (628 P for N = 16).  The line kernels split
    pass A into the conductance launch (read L, write g: 8 P) and the row
    half (write u_x: 4 P); the column half is pass B (16 P); the resident
    evolution takes all N - 1 steps in one launch (28 P each), and with the
    presmoothing and the contrast factor inside it (front_evolve) also their
    8 P + 8 P.  The streamed tile passes are pass A (stream_a, 12 P a step)
    and pass B (stream_b, 16 P), the line pass between them (stream_x)
    moving only the segment records."""
    steps = n_levels - 1
    table = {
        "presmooth": 8, "grad_max": 4, "grad_hist": 4, "conductance": 8 * steps,
        "aos_rows": 4 * steps, "aos_cols": 16 * steps, "aos_evolve": 28 * steps,
        "front_evolve": 8 + 8 + 28 * steps,
        "stream_a": 12 * steps, "stream_b": 16 * steps,
        "doh": 8 * n_levels, "extrema": 4 * n_levels,
    }
    if kind in table:
        return table[kind] * pixels
    if kind == "percentile":
        return 4 * nbins
    return 4


def detection_bytes(pixels, n_levels):
    """Algorithmic bytes of one whole detection: P (40 N - 12)."""
    return pixels * (40 * n_levels - 12)


# multiply-adds per pixel of the surrogate network: 3x3 taps x (5*32 + 32*32
# + 32*32 + 32*1); the kernels execute more (16 input and 8 output channels
# stored, halo recomputation), but the roofline counts the network's own
SURROGATE_MACS_PER_PIXEL = 9 * (5 * 32 + 32 * 32 + 32 * 32 + 32 * 1)
SURROGATE_CKPT = os.path.join(ROOT, "paper_1706_06750_gb300", "weights", "surrogate.ckpt")


def measured_bf16_peak():
    """The sustained bf16 peak (the surrogate's batched step runs for
    milliseconds under the power cap), else the burst one."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        if "bf16_tflops_sustained" in d:
            return float(d["bf16_tflops_sustained"]), "measured (sustained)"
        return float(d["bf16_tflops"]), "measured (burst)"
    except (OSError, KeyError, ValueError):
        return 1700.0, "fallback (sustained)"


def measured_hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


# source files of each kernel kind (with the helpers they include)
KIND_SOURCES = {
    "presmooth": ["k_filters.cu"], "grad_max": ["k_filters.cu"], "grad_hist": ["k_filters.cu"],
    "percentile": ["k_filters.cu"], "conductance": ["k_filters.cu"],
    "aos_rows": ["aos_solver.cuh", "k_aos.cu", "k_aos_va.cu", "k_aos_vb.cu", "k_aos_vc.cu", "k_aos_vd.cu"],
    "aos_cols": ["aos_solver.cuh", "k_aos.cu", "k_aos_va.cu", "k_aos_vb.cu", "k_aos_vc.cu", "k_aos_vd.cu"],
    "aos_evolve": ["k_evolve.cu"],
    "front_evolve": ["k_evolve.cu"],
    "stream_a": ["k_evolve.cu"], "stream_x": ["k_evolve.cu"], "stream_b": ["k_evolve.cu"],
    "doh": ["k_detector.cu", "doh_walk.cuh"], "extrema": ["k_detector.cu"], "describe": ["k_describe.cu"],
    "fed": ["k_fed.cu"],
}


def kernel_source_digest(kind):
    """Digest of the sources a kernel kind is built from (its files and the
    shared internal header)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1706_06750_gb300", "csrc")
    for name in sorted(set(KIND_SOURCES.get(kind, [])) | {"kaze_internal.h"}):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kind):
    """DRAM bytes per launch of `kind` from the committed ncu summary, if it was
    taken on the kind's current sources (else None).  The summary's table rows
    read | kind | kernel | bytes per launch | source digest | ..."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    m = re.search(rf"^\|\s*{re.escape(kind)}\s*\|[^|]*\|\s*([0-9.eE+]+)\s*\|\s*([0-9a-f]+)\s*\|", text, re.M)
    if not m or m.group(2) != kernel_source_digest(kind):
        return None
    return float(m.group(1))


# ------------------------------------------------------------------ oracle --

def oracle_full_rate(img, threads, octaves=OCTAVES, sublevels=SUBLEVELS):
    """Times the FP64 oracle on the whole image with `threads` host threads
    (its loops over independent pixels and lines); returns (Mpixel/s,
    seconds)."""
    import numpy as np

    import oracle
    oracle.build()
    oracle.set_threads(threads)
    opt = oracle.Options.make(octaves=octaves, sublevels=sublevels)
    t0 = time.perf_counter()
    oracle.kaze_detect(np.ascontiguousarray(img, dtype=np.float64), opt)
    dt = time.perf_counter() - t0
    return img.size / dt / 1e6, dt


def oracle_sample_rate(img, seconds_budget, octaves=OCTAVES, sublevels=SUBLEVELS, threads=1):
    """Times the FP64 oracle with `threads` host threads on a centred crop
    sized to the budget; returns (Mpixel/s, crop w, crop h, seconds)."""
    import numpy as np

    import oracle
    oracle.build()
    oracle.set_threads(threads)
    h, w = img.shape
    sec_per_px = 9e-6 / max(1, threads)  # rough FP64 oracle cost per pixel for 16 levels
    area = max(64 * 64, min(w * h, int(seconds_budget / sec_per_px)))
    scale = min(1.0, (area / (w * h)) ** 0.5)
    cw, ch = max(32, int(w * scale)), max(32, int(h * scale))
    x0, y0 = (w - cw) // 2, (h - ch) // 2
    crop = np.ascontiguousarray(img[y0:y0 + ch, x0:x0 + cw], dtype=np.float64)
    opt = oracle.Options.make(octaves=octaves, sublevels=sublevels)
    t0 = time.perf_counter()
    oracle.kaze_detect(crop, opt)
    dt = time.perf_counter() - t0
    return cw * ch / dt / 1e6, cw, ch, dt


def _oracle_worker_init():
    import oracle
    oracle.build()


def _oracle_crop_job(args):
    crop, octaves, sublevels = args
    import oracle
    oracle.kaze_detect(crop, oracle.Options.make(octaves=octaves, sublevels=sublevels))
    return crop.size


def oracle_all_cores_rate(img, seconds_budget, octaves=OCTAVES, sublevels=SUBLEVELS):
    """The FP64 oracle as it stands on every host core at once: one process
    per core (spawned), each detecting its own copy of a centred crop; the
    pool is started before the clock.  Returns (Mpixel/s, cores, crop w,
    crop h, seconds)."""
    import multiprocessing as mp

    import numpy as np
    cores = os.cpu_count() or 1
    h, w = img.shape
    sec_per_px = 4e-6
    area = max(64 * 64, min(w * h, int(seconds_budget / sec_per_px)))
    scale = min(1.0, (area / (w * h)) ** 0.5)
    cw, ch = max(32, int(w * scale)), max(32, int(h * scale))
    x0, y0 = (w - cw) // 2, (h - ch) // 2
    crop = np.ascontiguousarray(img[y0:y0 + ch, x0:x0 + cw], dtype=np.float64)
    with mp.get_context("spawn").Pool(cores, initializer=_oracle_worker_init) as pool:
        pool.map(_oracle_worker_init_probe, range(cores))  # every worker is up
        t0 = time.perf_counter()
        px = sum(pool.map(_oracle_crop_job, [(crop, octaves, sublevels)] * cores, chunksize=1))
        dt = time.perf_counter() - t0
    return px / dt / 1e6, cores, cw, ch, dt


def _oracle_worker_init_probe(_):
    return 0


# ------------------------------------------------------------ multi-rank --

def replica_seed(rank):
    """Seed of the workload image of `rank` (independent replicas)."""
    return 2000 + rank


def max_over_ranks(v, dist=None, device="cpu"):
    """The slowest rank's value (every rank receives it); v itself when not
    distributed.  device: where the reduction tensor lives (cuda for NCCL,
    cpu for gloo)."""
    if dist is None:
        return v
    import torch
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, steps, units_per_step, t_ms):
    """Units processed by all ranks per second (in millions), from the
    slowest rank's summed step time."""
    return world * steps * units_per_step / (t_ms * 1e-3) / 1e6


# -------------------------------------------------------------- reference --

def run_reference(args, rank, world):
    """Reference arm: the FP64 CPU oracle, as it stands, on the host cores,
    each step a bounded crop of the workload; rank 0 alone runs and prints."""
    if rank != 0:
        return 0
    from paper_1706_06750_gb300 import synth
    img = synth.workload_image("1920x1200")
    cores = os.cpu_count() or 1
    budget = max(0.05, 120.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        oracle_sample_rate(img, budget, threads=cores)
    rates, secs = [], 0.0
    cw = ch = 0
    for _ in range(args.steps):
        r, cw, ch, dt = oracle_sample_rate(img, budget, threads=cores)
        rates.append(r)
        secs += dt
    value = args.steps * cw * ch / secs / 1e6
    part = ("the whole 1920x1200 workload image" if (cw, ch) == (W_IMG, H_IMG)
            else f"centred {cw}x{ch} crop of the 1920x1200 workload image")
    sample = (f"{part} per step, {OCTAVES}x{SUBLEVELS} levels, scale space + response + extrema, "
              f"FP64 oracle on {cores} host threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------- ours --

def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_1706_06750_gb300 import build, kaze, synth

    build.build()
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", rank=rank, world_size=world)

    img = synth.image(W_IMG, H_IMG, replica_seed(rank))
    pixels = W_IMG * H_IMG
    k = kaze.Kaze(W_IMG, H_IMG, octaves=OCTAVES, sublevels=SUBLEVELS)
    x = torch.from_numpy(img).cuda()
    pinned = torch.from_numpy(img).pin_memory()
    pinned2 = torch.from_numpy(img.copy()).pin_memory()  # the stream alternates two host buffers
    stream_bufs = (pinned, pinned2)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    stream = k.stream  # the stream the library launches on; events go there

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for i in range(args.warmup):
        k.detect(x)
        k.detect_host(pinned)
        k.detect_host(stream_bufs[i % 2], next_image=stream_bufs[(i + 1) % 2])
    n_kp = len(k.detect(x))
    launches = k.last_launch_count()

    def timed(fn, after=None):
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        with torch.cuda.stream(stream):
            for i in range(args.steps):
                flush.zero_()
                starts[i].record(stream)
                fn()
                ends[i].record(stream)
                if after is not None:
                    after()
        torch.cuda.synchronize()
        return sum(s.elapsed_time(e) for s, e in zip(starts, ends))

    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.3)
    barrier()
    # the device's time for a whole detection: the recorded detection with
    # the count and keypoint slots copied to the host; the host's wait and
    # sort (kaze_detect_collect) follow the end event
    t_dev_ms = timed(lambda: k.detect_enqueue(x), after=k.detect_collect)
    barrier()
    t_single_ms = timed(lambda: k.detect_host(pinned))
    barrier()
    # the stream: the first timed image is copied ahead by this call
    k.detect_host(stream_bufs[1], next_image=stream_bufs[0])
    step = [0]

    def stream_step():
        i = step[0]
        step[0] += 1
        k.detect_host(stream_bufs[i % 2], next_image=stream_bufs[(i + 1) % 2])

    t_e2e_ms = timed(stream_step)
    barrier()
    clk = clocks.stop()

    def slowest(v):
        return max_over_ranks(v, dist, "cuda")

    t_dev_ms = slowest(t_dev_ms)
    t_e2e_ms = slowest(t_e2e_ms)
    t_single_ms = slowest(t_single_ms)

    # per-kernel device time with events around every launch
    prof_steps = max(3, min(20, args.steps))
    acc = {}
    for _ in range(prof_steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        for name, (ms, n) in k.profile(x).items():
            a = acc.setdefault(name, [0.0, 0])
            a[0] += ms
            a[1] += n
    total_ms = sum(v[0] for v in acc.values()) or 1.0
    kernels = {}
    for name, (ms, n) in acc.items():
        if n == 0:
            continue
        per = ms / n
        per_step = n // prof_steps
        ab = algorithmic_bytes(name, pixels, OCTAVES * SUBLEVELS) / max(1, per_step)
        kernels[name] = {"ms_per_launch": per, "launches_per_step": per_step, "share": ms / total_ms,
                         "algorithmic_bytes_per_launch": ab, "algorithmic_gbs": ab / (per * 1e-3) / 1e9}
    dom = max(kernels, key=lambda n: kernels[n]["share"])
    peak, peak_kind = measured_hbm_peak()
    dom_bytes = kernels[dom]["algorithmic_bytes_per_launch"]
    achieved = kernels[dom]["algorithmic_gbs"]
    traffic = ncu_traffic(dom)

    large = None if args.no_large else run_large(args, kaze, synth, torch, flush, slowest, barrier, peak)
    describe = run_describe(args, k, torch, stream, flush, k.detect(x), slowest, barrier)
    fed = run_fed(args, kaze, torch, img, flush, slowest, barrier, t_dev_ms / args.steps)
    batched = None if args.no_batch else run_batched(args, kaze, synth, torch, stream, world, rank,
                                                        slowest, barrier)
    surrogate = None if args.no_surrogate else run_surrogate(args, kaze, synth, torch, rank)

    if dist is not None:
        dist.barrier()
    if rank != 0:
        dist.destroy_process_group()
        return 0

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        rate, secs = oracle_full_rate(img, 1)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"the whole 1920x1200 workload image, {OCTAVES}x{SUBLEVELS} levels, scale space + "
                         f"response + extrema, FP64 oracle on one host thread, {secs:.1f} s"}
        cores = os.cpu_count() or 1
        arate, asecs = oracle_full_rate(img, cores)
        cpu["all_cores"] = {"value": arate, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"the whole image, the oracle's independent loops on {cores} host "
                                      f"threads, {asecs:.2f} s"}

    whole_bytes = detection_bytes(pixels, OCTAVES * SUBLEVELS)
    whole_gbs = whole_bytes / (t_dev_ms / args.steps * 1e-3) / 1e9
    value = whole_job_rate(world, args.steps, pixels, t_dev_ms)
    e2e = whole_job_rate(world, args.steps, pixels, t_e2e_ms)
    e2e_single = whole_job_rate(world, args.steps, pixels, t_single_ms)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_dev_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded blobs + rectangles + noise, one image per rank)",
        "config": {"workload": WORKLOAD, "width": W_IMG, "height": H_IMG, "octaves": OCTAVES,
                   "sublevels": SUBLEVELS, "keypoints": n_kp,
                   "l2": "flushed before every step (256 MiB memset outside the timed events)",
                   "parallelism": f"replicas x{world}"},
        "clocks": clk,
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": pixels * 4,
                # count and status, the keypoint slots copied with them, and
                # a second copy only when there are more keypoints than slots
                "d2h_bytes_per_step": 8 + 40 * KEYPOINT_SLOTS + (40 * n_kp if n_kp > KEYPOINT_SLOTS else 0),
                "api": "kaze_detect_host_next (pinned host images; each step copies the next step's image "
                       "during its detection and reads its keypoints back)",
                "single": {"value": e2e_single, "unit": UNIT, "api": "kaze_detect_host (copy, then detect)"}},
        "gpu_launches": launches * args.steps,
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                     "peak_source": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic,
                     "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum per launch, one "
                                        "single-kernel capture with cold caches (profiles/ncu_traffic.md); "
                                        "null when the kernel changed since"),
                     "algorithmic_bytes_per_launch": dom_bytes,
                     "whole": {"algorithmic_bytes": whole_bytes, "ms": t_dev_ms / args.steps,
                               "achieved": whole_gbs, "frac": whole_gbs / peak,
                               "model": "P (40 N - 12) bytes: 628 B/px at N = 16"}},
        "kernels": kernels,
        # compact scalars of the side sections, beside their full records
        "whole_frac": whole_gbs / peak,
        "large_mpix_per_s": large["mpix_per_s"] if large else None,
        "large_frac": large["roofline_whole"]["frac"] if large else None,
        "batched_img_per_s": batched["img_per_s"] if batched else None,
        "batched_plain_img_per_s": batched["plain_img_per_s"] if batched else None,
        "batched_resident_img_per_s": batched["resident_img_per_s"] if batched else None,
        "batched_queue_img_per_s": batched["queue_img_per_s"] if batched else None,
        "batched_frac": batched["roofline_whole"]["frac"] if batched else None,
        "large": large,
        "describe": describe,
        "fed": fed,
        "batched": batched,
        "surrogate": surrogate,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    k.close()
    return 0


def run_large(args, kaze, synth, torch, flush, max_over_ranks, barrier, peak):
    """The 4096x3072 workload image with its sinusoidal texture (4 x 4
    levels, scale space + detector, the keypoints copied back): Mpixel/s
    device-resident, timed like the main line, and the whole-detection
    fraction of the HBM roofline for its P (40 N - 12) bytes."""
    W, H = 4096, 3072
    img = synth.workload_image("4096x3072")
    k = kaze.Kaze(W, H, octaves=OCTAVES, sublevels=SUBLEVELS)
    x = torch.from_numpy(img).cuda()
    for _ in range(max(3, min(args.warmup, 5))):
        k.detect(x)
    n_kp = len(k.detect(x))
    reps = max(3, min(args.steps, 20))
    st = k.stream
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
    barrier()
    with torch.cuda.stream(st):
        for i in range(reps):
            flush.zero_()
            starts[i].record(st)
            k.detect_enqueue(x)
            ends[i].record(st)
            k.detect_collect()
    torch.cuda.synchronize()
    ms = max_over_ranks(sum(s.elapsed_time(e) for s, e in zip(starts, ends)) / reps)
    launches = k.last_launch_count()
    kinds = {name: n for name, (t, n) in k.profile(x).items() if n}
    k.close()
    byts = detection_bytes(W * H, OCTAVES * SUBLEVELS)
    gbs = byts / (ms * 1e-3) / 1e9
    return {"workload": "4096x3072 float32 image with sinusoidal texture, 4 octaves x 4 sublevels",
            "ms_per_step": ms, "mpix_per_s": W * H / (ms * 1e-3) / 1e6, "keypoints": n_kp,
            "launches_per_step": launches, "kernels": kinds,
            "roofline_whole": {"algorithmic_bytes": byts, "achieved": gbs, "peak": peak, "unit": "GB/s",
                               "frac": gbs / peak},
            "l2": "flushed before every step"}


def run_fed(args, kaze, torch, img, flush, max_over_ranks, barrier, aos_ms):
    """The same detection with the FED evolution of Eq. 5 (the paper's own
    GPU scheme: one cycle of explicit steps per level) instead of AOS,
    graph-replayed, L2 flushed before every step."""
    k = kaze.Kaze(W_IMG, H_IMG, octaves=OCTAVES, sublevels=SUBLEVELS, scheme=kaze.SCHEME_FED)
    x = torch.from_numpy(img).cuda()
    for _ in range(args.warmup):
        k.detect(x)
    n_kp = len(k.detect(x))
    launches = k.last_launch_count()
    reps = max(3, min(args.steps, 50))
    st = k.stream
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
    barrier()
    with torch.cuda.stream(st):
        for i in range(reps):
            flush.zero_()
            starts[i].record(st)
            k.detect(x)
            ends[i].record(st)
    torch.cuda.synchronize()
    ms = max_over_ranks(sum(s.elapsed_time(e) for s, e in zip(starts, ends)) / reps)
    prof = k.profile(x)
    t = [k.level_time(i) for i in range(OCTAVES * SUBLEVELS)]
    k.close()
    steps = sum(fed_cycle_length(b - a) for a, b in zip(t, t[1:]))
    fed_ms, fed_n = prof.get("fed", (0.0, 0))
    # a launch takes up to four explicit steps and moves 12 bytes a pixel (read L, g; write L)
    return {"ms_per_step": ms, "mpix_per_s": W_IMG * H_IMG / (ms * 1e-3) / 1e6, "keypoints": n_kp,
            "launches_per_step": launches, "explicit_steps": steps, "fed_launches": fed_n,
            "ms_per_fed_launch": fed_ms / fed_n if fed_n else None,
            "ms_per_explicit_step": fed_ms / steps if steps else None,
            "fed_launch_algorithmic_gbs": (12 * W_IMG * H_IMG / (fed_ms / fed_n * 1e-3) / 1e9) if fed_n else None,
            "aos_ms_per_step": aos_ms, "aos_over_fed_speed": ms / aos_ms}


def fed_cycle_length(dt, tau_max=0.25):
    """Explicit steps of the FED cycle reaching dt: the least n with
    tau_max (n^2 + n) / 3 >= dt (Eq. 5)."""
    n = 1
    while tau_max * (n * n + n) / 3.0 < dt:
        n += 1
    return n


def run_only(args, local_rank):
    """One side section (description or FED detection) on the workload
    image, printed as a JSON line of its own."""
    import torch

    from paper_1706_06750_gb300 import build, kaze, synth
    build.build()
    torch.cuda.set_device(local_rank)
    img = synth.image(W_IMG, H_IMG, replica_seed(0))
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def barrier():
        torch.cuda.synchronize()

    if args.only == "fed":
        k = kaze.Kaze(W_IMG, H_IMG, octaves=OCTAVES, sublevels=SUBLEVELS)
        x = torch.from_numpy(img).cuda()
        k.detect(x)
        st = k.stream
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(st):
            e0.record(st)
            k.detect(x)
            e1.record(st)
        torch.cuda.synchronize()
        aos_ms = e0.elapsed_time(e1)
        k.close()
        out = run_fed(args, kaze, torch, img, flush, max_over_ranks, barrier, aos_ms)
    else:
        k = kaze.Kaze(W_IMG, H_IMG, octaves=OCTAVES, sublevels=SUBLEVELS)
        x = torch.from_numpy(img).cuda()
        out = run_describe(args, k, torch, k.stream, flush, k.detect(x), max_over_ranks, barrier)
        k.close()
    print(json.dumps({"section": args.only, "workload": WORKLOAD, **out}), flush=True)
    return 0


def run_describe(args, k, torch, stream, flush, kp, max_over_ranks, barrier):
    """Orientation + 64-D M-SURF descriptor (Sec. II-C) of the workload
    image's keypoints on its device-resident levels: one launch per step, the
    keypoints already on the device, L2 flushed before every step."""
    n = len(kp)
    if n == 0:
        return {"keypoints": 0}
    d_kp = k.keypoints_to_device(kp)
    d_desc = torch.empty((n, 64), device="cuda")
    for _ in range(args.warmup):
        k.describe_device(d_kp, d_desc, n)
    reps = max(3, min(args.steps, 50))
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
    barrier()
    with torch.cuda.stream(stream):
        for i in range(reps):
            flush.zero_()
            starts[i].record(stream)
            k.describe_device(d_kp, d_desc, n)
            ends[i].record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(sum(s.elapsed_time(e) for s, e in zip(starts, ends)) / reps)
    return {"keypoints": n, "ms_per_step": ms, "us_per_keypoint": ms * 1e3 / n,
            "keypoints_per_s": n / (ms * 1e-3), "launches_per_step": k.last_launch_count(),
            "l2": "flushed before every step"}


def run_batched(args, kaze, synth, torch, stream, world, rank, max_over_ranks, barrier):
    """64 mixed-size images (each rank its own set): the batched persistent
    path (autotuned solve tiles, cached) against the plain single-image path
    run image after image.  The 64 inputs (~360 MB) exceed L2."""
    sizes = synth.batch_sizes(64, seed=4000 + 100 * rank)
    imgs = [torch.from_numpy(a).cuda() for a in synth.batch_images(64, seed=4000 + 100 * rank)]
    mpx = sum(w * h for w, h in sizes) / 1e6
    reps = max(2, min(args.steps, 10))
    cache = os.path.join(ROOT, "paper_1706_06750_gb300", "_build", "batch_tuning.json")
    def time_batch(b):
        for _ in range(2):
            b.detect(imgs)
        barrier()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        with torch.cuda.stream(b.stream):
            ev[0].record(b.stream)
            for _ in range(reps):
                b.detect(imgs)
            ev[1].record(b.stream)
        torch.cuda.synchronize()
        return max_over_ranks(ev[0].elapsed_time(ev[1]))

    with kaze.Batch(sizes) as b:
        tuning, tune_ms = b.autotune(imgs, reps=2, cache=cache)
        t_batch = time_batch(b)
        counts = [len(k) for k in b.detect(imgs)]
        # the resident evolution of the whole batch in one launch, and the
        # work-queue launch of the whole detection (its best shape)
        b.set_tuning(kaze.BATCH_RESIDENT, 4, 1, 8)
        t_res = time_batch(b)
        t_queue, queue_shape = None, None
        for shape in ((kaze.BATCH_PERSISTENT, 4, 2, 8), (kaze.BATCH_PERSISTENT, 8, 1, 8)):
            b.set_tuning(*shape)
            t = time_batch(b)
            if t_queue is None or t < t_queue:
                t_queue, queue_shape = t, shape
        b.set_tuning(*tuning)
    n_levels = OCTAVES * SUBLEVELS
    launches = {kaze.BATCH_PERSISTENT: 1, kaze.BATCH_RESIDENT: 1 + 2 * 64}.get(
        tuning[0], 64 * (3 * (n_levels - 1) + 4 + 3 + 1))
    mw = max(w for w, _ in sizes)
    mh = max(h for _, h in sizes)
    with kaze.Kaze(mw, mh) as k:
        for x in imgs[:4]:
            k.detect(x)
        barrier()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        with torch.cuda.stream(k.stream):
            ev[0].record(k.stream)
            for x in imgs:
                k.detect(x)
            ev[1].record(k.stream)
        torch.cuda.synchronize()
        t_plain = max_over_ranks(ev[0].elapsed_time(ev[1]))
    img_s = world * 64 * reps / (t_batch * 1e-3)
    plain_s = world * 64 / (t_plain * 1e-3)
    mode = {kaze.BATCH_PERSISTENT: "work-queue", kaze.BATCH_RESIDENT: "resident"}.get(tuning[0], "concurrent")
    batch_bytes = sum(detection_bytes(w * h, n_levels) for w, h in sizes)
    return {"images": 64, "megapixels": round(mpx, 3), "img_per_s": img_s,
            "roofline_whole": {"algorithmic_bytes": batch_bytes,
                               "achieved": batch_bytes / (t_batch / reps * 1e-3) / 1e9,
                               "frac": batch_bytes / (t_batch / reps * 1e-3) / 1e9 / measured_hbm_peak()[0]},
            "mpix_per_s": img_s * mpx / 64, "ms_per_batch": t_batch / reps,
            "plain_img_per_s": plain_s, "plain_ms_per_64": t_plain,
            "speedup_vs_plain": img_s / plain_s,
            "tuning": {"mode": mode, "cols_per_strip": tuning[1], "ctas_per_sm": tuning[2],
                       "streams": tuning[3]},
            "autotune_best_ms": tune_ms, "keypoints": int(sum(counts)),
            "kernel_launches_per_batch": launches,
            "resident_ms_per_batch": t_res / reps,
            "resident_img_per_s": world * 64 * reps / (t_res * 1e-3),
            "queue_ms_per_batch": t_queue / reps,
            "queue_img_per_s": world * 64 * reps / (t_queue * 1e-3),
            "queue_shape": {"cols_per_strip": queue_shape[1], "ctas_per_sm": queue_shape[2]},
            "note": ("autotuned execution of the batch (graph-replayed); plain = kaze_detect image "
                     "after image on one stream; resident = every image's evolution in one persistent "
                     "cooperative launch (images packed into waves of one tile per SM), then each image's "
                     "response and extrema launch; work-queue = the whole detection of the batch as one "
                     "persistent work-queue launch")}


def run_surrogate(args, kaze, synth, torch, rank):
    """The learned AOS surrogate judged by plain GPU AOS on 16 seeded 1920x1200
    images (seeds 2000 + 16 rank + j): pixel error, keypoint repeatability and
    time (surrogate_eval), plus the roofline of the fused surrogate kernel on
    the batched step (all 16 images in one launch)."""
    from paper_1706_06750_gb300 import surrogate_eval
    if not os.path.exists(SURROGATE_CKPT):
        return {"unavailable": "no trained checkpoint at paper_1706_06750_gb300/weights/surrogate.ckpt"}
    s = kaze.Surrogate(seed=0)
    s.load(SURROGATE_CKPT)
    imgs = [torch.from_numpy(synth.image(W_IMG, H_IMG, 2000 + 16 * rank + j)).cuda() for j in range(16)]
    r = surrogate_eval.evaluate(s, imgs, OCTAVES, SUBLEVELS, batch_reps=max(3, min(args.steps, 10)))
    flops = 2.0 * SURROGATE_MACS_PER_PIXEL * W_IMG * H_IMG * len(imgs)
    achieved = flops / (r["batched_step_ms_surrogate"] * 1e-3) / 1e12
    peak, src = measured_bf16_peak()
    r["roofline"] = {"bound": "tensor", "kernel": "surrogate (fused)", "achieved": achieved, "peak": peak,
                     "peak_source": src, "unit": "TFLOP/s", "frac": achieved / peak,
                     "flops_per_launch": flops, "traffic": None}
    r["speedup_vs_aos_batched_step"] = r["batched_step_ms_aos"] / r["batched_step_ms_surrogate"]
    r["checkpoint"] = os.path.relpath(SURROGATE_CKPT, ROOT)
    s.close()
    return r


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--no-large", action="store_true", help="skip the 4096x3072 section")
    ap.add_argument("--only", choices=["describe", "fed"], default=None,
                    help="run one side section alone on the workload image (profiling cases)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank = env_int("RANK", 0)
    world = env_int("WORLD_SIZE", 1)
    local_rank = env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.only:
        return run_only(args, local_rank)
    return run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
