#!/usr/bin/env python
"""Benchmark: 1080p 8-level Oriented FAST, frames/s and Mpix/s on GB300.

Workload (one step): a batch of B synthetic 1920x1080 uint8 frames (1/f-noise
background, 200 rectangles, 30 checkerboards, blur sigma 1, noise sigma 3),
each through the whole chain -- 8-level bilinear pyramid at scale 1.2 (border
19), FAST-9 score with t=20 and fallback t=7 per 30x30 cell, strict 3x3 NMS,
Harris 7x7 with k=0.04, top 1000 per frame split by level area, centroid
orientation with radius 15.

Reported:
  value        batched path, frames/s (inputs resident in HBM, one
               of_detect_batch call per step, B frames)
  plain        per-frame path (one of_detect_batch call per frame), frames/s
  mixed        64 frames of uneven sizes (720x540 .. 1920x1080, 8 levels each)
               in one batched call vs one call per frame, frames/s
  e2e          batched path with host buffers: pinned H2D of the frames and
               D2H of keypoints + counts inside the timed region (double
               buffered: the next step's upload overlaps this step's detection)
  roofline     dominant stage: algorithmic bytes per launch / its mean
               CUDA-event duration over the timed region, vs measured HBM peak
  cpu_baseline the CPU oracle on a bounded sample, all host cores (N=1, rank 0)

--impl reference runs the CPU oracle as the reference arm (bounded samples).
Multi-GPU (torchrun): replicas only, each rank runs the same per-GPU workload.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

W_, H_, LEVELS, SCALE, FAST_T, FAST_T_LO, HARRIS_K, NFEAT = 1920, 1080, 8, 1.2, 20, 7, 0.04, 1000
BORDER = 19
WORKLOAD = ("1920x1080 u8 frames, 8-level bilinear pyramid scale 1.2, FAST-9 t=20 (fallback t=7 "
            "per 30x30 cell), strict 3x3 NMS, Harris 7x7 k=0.04, top 1000 per frame by level "
            "area, centroid r=15")
METRIC = "1080p 8-level Oriented FAST frames/s"


def _gen(seed: int):
    import synth

    return synth.scene(W_, H_, seed, background="pink")


def _oracle_detect(img):
    import oracle

    return len(oracle.detect(img, levels=LEVELS, scale=SCALE, fast_t=FAST_T, fast_t_lo=FAST_T_LO,
                             harris_k=HARRIS_K, n_features=NFEAT))


SERVE_SIZES = [(640, 480), (1280, 720), (1920, 1080), (3840, 2160)]
DISPARITIES = (4, 9, 14, 19)  # stereo pairs of the serving mix: right view = left shifted by one of these
# The uneven-size batch: 64 frames drawn uniformly from these sizes, 8 levels each (~512 images).
MIXED_SIZES = [(720, 540), (1080, 720), (1440, 1080), (1920, 1080)]
MIXED_FRAMES = 64


def mixed_frames(pool, n: int, seed: int = 3):
    import numpy as np

    picks = np.random.default_rng(seed).integers(0, len(MIXED_SIZES), n)
    return pool.map(_gen_sized, [(MIXED_SIZES[k][0], MIXED_SIZES[k][1], 5000 + i) for i, k in enumerate(picks)])


def _gen_sized(args):
    import synth

    w, h, seed = args
    return synth.scene(w, h, seed, background="pink")


def serving_leg(pool, seconds: float, rate: float, seed: int = 0, clients: int = 1, max_outstanding: int = 0):
    """Poisson arrivals at `rate` frames/s of the mixed-size workload (split
    over `clients` submitting threads), through the continuous-batching
    server; returns latency percentiles and throughput.  max_outstanding > 0:
    a client waits while that many frames are submitted and not yet returned
    (a bounded backlog when the offered rate exceeds what the server serves)."""
    import threading

    import numpy as np

    import paper_2506_07164_gb300 as ofg

    frames = {sz: pool.map(_gen_sized, [(sz[0], sz[1], 500 + 10 * i + k) for k in range(3)])
              for i, sz in enumerate(SERVE_SIZES)}

    def shifted(img, d):  # right view: the left one shifted by disparity d, last column repeated
        right = np.empty_like(img)
        right[:, : img.shape[1] - d] = img[:, d:]
        right[:, img.shape[1] - d:] = img[:, -1:]
        return right

    # Right views made before timing, so the submitting threads only submit.
    rights = {sz: [[shifted(img, d) for d in DISPARITIES] for img in frames[sz]] for sz in SERVE_SIZES}
    srv = ofg.of_server_create(max_w=3840, max_h=2160, levels=LEVELS, scale=SCALE, fast_t=FAST_T,
                               fast_t_lo=FAST_T_LO, harris_k=HARRIS_K, n_features=NFEAT, slots=4,
                               max_batch=16, memory_budget=12 << 30)
    done = []
    submitted = [0] * clients
    crate = rate / clients

    def client(c):
        rng = np.random.default_rng(seed + 1000 * c)
        t0 = time.perf_counter()
        t_next = t0
        while t_next - t0 < seconds:
            now = time.perf_counter()
            if t_next > now:
                time.sleep(t_next - now)
            while max_outstanding and sum(submitted) - len(done) > max_outstanding:
                time.sleep(0.001)
            if time.perf_counter() - t0 >= seconds:
                break  # a backlog-bound client stops at the leg's end, not at its schedule's
            sz = SERVE_SIZES[int(rng.integers(0, len(SERVE_SIZES)))]
            if rng.random() < 0.2:  # stereo pair: right view = left shifted by a seeded disparity
                k = int(rng.integers(0, 3))
                right = rights[sz][k][int(rng.integers(0, len(DISPARITIES)))]
                ofg.of_server_submit(srv, frames[sz][k], tag=1)
                ofg.of_server_submit(srv, right, tag=2)
                submitted[c] += 2
                t_next += float(rng.exponential(2.0 / crate))
            else:
                ofg.of_server_submit(srv, frames[sz][int(rng.integers(0, 3))], tag=0)
                submitted[c] += 1
                t_next += float(rng.exponential(1.0 / crate))

    # Warm the plans of each size class (first use captures a graph) before timing.
    for sz in SERVE_SIZES:
        for k in range(2):
            ofg.of_server_submit(srv, frames[sz][0], tag=-1)
    got = 0
    while got < 2 * len(SERVE_SIZES):
        got += len(ofg.of_server_poll(srv, 64, NFEAT, wait_ms=100))
    ths = [threading.Thread(target=client, args=(c,)) for c in range(clients)]
    wall0 = time.perf_counter()
    for th in ths:
        th.start()
    while any(th.is_alive() for th in ths) or len(done) < sum(submitted):
        for r, _ in ofg.of_server_poll(srv, 256, NFEAT, wait_ms=20, keypoints=False):
            done.append((r.t_submit, r.t_done, r.count, r.batch_frames, r.w * r.h))
        if not any(th.is_alive() for th in ths) and time.perf_counter() - wall0 > seconds + 60:
            break
    for th in ths:
        th.join()
    stats = ofg.of_server_stats(srv)
    ofg.of_server_destroy(srv)
    lat = np.array([b - a for a, b, *_ in done]) * 1000.0
    first = min(a for a, *_ in done)
    last = max(b for _, b, *_ in done)
    ok = sum(1 for d in done if d[2] >= 0)
    return {"offered_rate_fps": round(rate, 1), "submitted_fps": round(sum(submitted) / seconds, 1),
            "client_threads": clients,
            "frames": len(done), "ok": ok,
            "frames_per_s": round(len(done) / (last - first), 1),
            "mpix_per_s": round(sum(d[4] for d in done) / (last - first) / 1e6, 1),
            "p50_ms": round(float(np.percentile(lat, 50)), 3), "p99_ms": round(float(np.percentile(lat, 99)), 3),
            "mean_ms": round(float(lat.mean()), 3), "mean_batch_frames": round(float(np.mean([d[3] for d in done])), 2),
            "batches": stats["batches"], "slots": 4, "memory_budget_bytes": 12 << 30,
            "max_outstanding": max_outstanding or None,
            "mix": "uniform over 640x480/1280x720/1920x1080/3840x2160; 20% of arrivals are stereo pairs "
                   "(right view shifted by 4, 9, 14 or 19 px)",
            "seconds": seconds}


TUNING_FIELDS = ("resize_tile_h", "fast_blocks_per_sm", "nms_blocks_per_sm", "fast_order", "nms_order", "resize_tma",
                 "stream_groups", "fast_cell_tiles", "nms_tile_h", "fast_tile_h")

# The paper's variant pipelines (Table 2; Figs. 8-9 order them by runtime, slowest first).
ABLATION_PIPELINES = [("Baseline_ORB", 0, 0), ("Binary_ORB", 1, 0), ("SM_ORB", 3, 0), ("Sep_ORB", 3, 1),
                      ("Para-Sep_ORB", 3, 2), ("Semi-Sep_ORB", 3, 3)]
ABLATION_FAST = [("Baseline(FAST)", 0), ("BinaryFAST", 1), ("SMFAST", 2), ("SM-BinaryFAST", 3)]
ABLATION_SIZES = [(720, 540), (1080, 720), (1440, 1080), (1920, 1080)]


def ablation_leg(pool, det, stream, reps: int = 20):
    """Time each paper variant (FAST + Harris of every FAST point at t = 20, no NMS) on one synthetic scene of
    each of the paper's image sizes, on 1 and 4 pyramid layers (the detector's own levels)."""
    import torch

    import paper_2506_07164_gb300 as ofg

    imgs = pool.map(_gen_sized, [(w, h, 7000 + i) for i, (w, h) in enumerate(ABLATION_SIZES)])
    out = {"unit": "ms per image (CUDA events, mean of %d calls after 3 warm-ups)" % reps, "fast_t": FAST_T,
           "border": 19, "sizes": {}}
    holds = []
    for (w, h), img in zip(ABLATION_SIZES, imgs):
        dev0 = torch.from_numpy(img).cuda()
        det.detect_batch([dev0], levels=4, scale=SCALE, fast_t=FAST_T, n_features=NFEAT)
        torch.cuda.synchronize()
        levels = []
        for lv in range(4):
            a, dims = det.inspect(ofg.OF_BUF_LEVEL, 0, lv)
            lw, lh = int(dims[0]), int(dims[1])
            levels.append((torch.from_numpy(a.reshape(lh, lw).copy()).cuda(), lw, lh))
        cap = w * h
        pts = torch.empty(cap * 32, dtype=torch.uint8, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int32, device="cuda")

        def call(fv, hv, n_layers):
            for t_img, lw, lh in levels[:n_layers]:
                ofg.of_variant_detect(fv, hv, t_img, lw, lh, lw, FAST_T, 19, HARRIS_K, pts, cnt, cap, stream)

        def time_it(fv, hv, n_layers):
            with torch.cuda.stream(stream):
                for _ in range(3):
                    call(fv, hv, n_layers)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(reps):
                    call(fv, hv, n_layers)
                e1.record(stream)
                e1.synchronize()
            return e0.elapsed_time(e1) / reps

        entry = {}
        for n_layers in (1, 4):
            pipes = {name: round(time_it(fv, hv, n_layers), 4) for name, fv, hv in ABLATION_PIPELINES}
            fast = {name: round(time_it(fv, -1, n_layers), 4) for name, fv in ABLATION_FAST}
            call(3, -1, 1)
            torch.cuda.synchronize()
            times = [pipes[name] for name, _, _ in ABLATION_PIPELINES]
            order = all(a >= b for a, b in zip(times, times[1:]))
            holds.append(order)
            entry[f"layers{n_layers}"] = {"pipelines": pipes, "fast_only": fast,
                                          "paper_order_holds": order}
        entry["fast_points_layer0"] = int(cnt.item())
        out["sizes"][f"{w}x{h}"] = entry
    out["paper_order"] = " > ".join(name for name, _, _ in ABLATION_PIPELINES) + " (runtime, paper Figs. 8-9)"
    out["paper_order_holds_everywhere"] = all(holds)
    return out


def make_frames(n: int, pool=None):
    seeds = list(range(n))
    if pool is not None:
        return pool.map(_gen, seeds)
    return [_gen(s) for s in seeds]


def cpu_baseline(pool, cores: int, frames, n_frames: int):
    """The oracle as it stands, frame-parallel over `cores` processes (detect only)."""
    import oracle

    oracle.build()
    work = [frames[i % len(frames)] for i in range(n_frames)]
    pool.map(_oracle_detect, work[:cores])  # warm the workers
    t0 = time.perf_counter()
    pool.map(_oracle_detect, work)
    wall = time.perf_counter() - t0
    return {"value": round(n_frames / wall, 4), "unit": "frames/s", "cores": cores, "kind": "oracle",
            "sample": f"{n_frames} frames of the timed workload ({len(frames)} distinct), one oracle "
                      f"process per core, wall {wall:.1f} s"}


def sample_clocks(stop_path: str, out_path: str):
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        return subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                 "-lms", "100", "-i", os.environ.get("LOCAL_RANK", "0")],
                                stdout=open(out_path, "w"), stderr=subprocess.DEVNULL)
    except (OSError, FileNotFoundError):
        return None


def summarize_clocks(path: str):
    sm, mx, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    try:
        for line in open(path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
    except OSError:
        pass
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": ["unsampled"]}
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
            "samples": len(sm)}


# ALU roofline of the FAST score.  The integer ALU pipe (min/max, logic,
# permutes, shifts) takes 16 lanes per clock in each of the 4 sub-partitions
# of an SM: 64 lane-ops per clock per SM.  Algorithmic work of the score: per
# pixel pair, 2 x (16 + 16 + 8) three-input packed min/max operations of the
# arc network plus 1 for the final score = 81, i.e. 40.5 per pixel of the
# detect regions (tile padding is not work the method asks for).
ALU_LANES_PER_SM_CLK = 64
FAST_OPS_PER_PX = 40.5
# L2 (lts__t_bytes.sum) and DRAM (dram__bytes_read.sum + dram__bytes_write.sum)
# bytes per frame of each stage's kernels, from one ncu capture of the
# per-stage launches (of_time_stages) over a batch of 1080p frames with 8
# levels, divided by the frames.  Valid while the kernels' code
# (kernels_sha1) and the per-stage launch choices below are the ones captured;
# otherwise the line reports null.
STAGE_TRAFFIC = {"code_sha1": "15beeae98e4bf634d86ea749ce057c562c4ff06e", "frames": 64, "tuning": {"resize_tma": 1, "resize_tile_h": 64, "fast_cell_tiles": 4, "fast_tile_h": 32, "nms_tile_h": 32}, "l2_bytes_per_frame": {"pyramid": 24196450, "fast": 30250878, "nms_harris": 37334777, "select": 2605176, "orient": 2479839}, "dram_bytes_per_frame": {"pyramid": 7743236, "fast": 12241556, "nms_harris": 14609800, "select": 1026060, "orient": 533236}}


def code_sha1(path):
    """SHA-1 of a source file's code: '//' comments and blank lines removed, so
    that edits to comments leave a capture of the same code valid."""
    import hashlib
    import re

    with open(path) as f:
        lines = [re.sub(r"//.*$", "", l).rstrip() for l in f.read().splitlines()]
    return hashlib.sha1("\n".join(l for l in lines if l.strip()).encode()).hexdigest()


def kernels_sha1():
    """SHA-1 over the code (comments and blank lines removed) of every kernel
    source and header of the library."""
    import glob
    import hashlib

    csrc = os.path.join(ROOT, "paper_2506_07164_gb300", "csrc")
    files = sorted(glob.glob(os.path.join(csrc, "k_*.cu")) + glob.glob(os.path.join(csrc, "*.cuh")) +
                   [os.path.join(csrc, "of_internal.h")])
    return hashlib.sha1("".join(code_sha1(f) for f in files).encode()).hexdigest()


STAGE_TUNING_FIELDS = ("resize_tma", "resize_tile_h", "fast_cell_tiles", "fast_tile_h", "nms_tile_h")


def traffic_ok(tuning):
    """STAGE_TRAFFIC describes these kernels and launch choices."""
    return (STAGE_TRAFFIC is not None and STAGE_TRAFFIC["code_sha1"] == kernels_sha1() and
            all(int(tuning.get(k, -1)) == STAGE_TRAFFIC["tuning"][k] for k in STAGE_TUNING_FIELDS))


def detect_region_pixels(lw, lh):
    """Pixels whose FAST score the method needs per frame: the detect regions of all levels."""
    return sum(max(0, w - 2 * BORDER) * max(0, h - 2 * BORDER) for w, h in zip(lw, lh))


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def measure_read_peaks(ofg, torch, stream, reps: int = 3):
    """Read bandwidth with the library's probe: L2 (buffers of 8..48 MB, read
    many times; best) and HBM (a 4 GiB buffer).  GB/s of bytes read."""
    sink = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = {}
    for name, sizes, total in (("l2", [8 << 20, 16 << 20, 32 << 20, 48 << 20], 24e9), ("hbm", [4 << 30], 16e9)):
        best = 0.0
        for nb in sizes:
            buf = torch.ones(nb, dtype=torch.uint8, device="cuda")
            r = max(1, int(total / nb))
            with torch.cuda.stream(stream):
                ofg.of_probe_read(buf, nb, r, sink, stream)  # warm (and load the buffer into L2)
                for _ in range(reps):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    ofg.of_probe_read(buf, nb, r, sink, stream)
                    e1.record(stream)
                    e1.synchronize()
                    best = max(best, nb * r / (e0.elapsed_time(e1) / 1000.0) / 1e9)
            del buf
        out[name] = round(best, 1)
    torch.cuda.synchronize()
    return out


def floor_bytes_per_frame(levels_w, levels_h, kept):
    """Least HBM traffic of one frame with every level kept resident: read the
    input, write levels 1..L-1, read every level once for detection, write
    the keypoint records."""
    px = [w * h for w, h in zip(levels_w, levels_h)]
    return px[0] + sum(px[1:]) + sum(px) + 64 * kept


def stage_bytes(levels_w, levels_h, cand_counts, kept_counts):
    """Algorithmic HBM bytes per frame for each stage (see the design notes)."""
    lw, lh = levels_w, levels_h
    px = [w * h for w, h in zip(lw, lh)]
    det = [max(0, w - 2 * BORDER) * max(0, h - 2 * BORDER) for w, h in zip(lw, lh)]
    pyr = sum(px[:-1]) + sum(px[1:])                      # read l-1, write l
    fast = sum(px) + sum(det)                             # read levels, write score maps
    nmsh = sum(det) + sum(px) + 12 * sum(cand_counts)     # read scores + levels, write candidates
    sel = 12 * sum(cand_counts) + 12 * sum(kept_counts)   # read candidates, write kept
    orient = (709 + 81 + 12 + 64) * sum(kept_counts)      # disc + footprint + kept + record
    return [pyr, fast, nmsh, sel, orient]


def reduce_max_over_ranks(values, dist=None, device="cpu"):
    """Element-wise maximum of per-rank timings (replicas: the slowest rank sets the job time)."""
    import torch

    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def replicas_value(frames_per_rank: int, world: int, ms_max: float) -> float:
    """Whole-job frames/s: every rank processed frames_per_rank frames within ms_max."""
    return frames_per_rank * world / (ms_max / 1000.0)


def run_reference(args, rank: int, world: int):
    """Reference arm: the CPU oracle, bounded sample per step."""
    if rank != 0:
        return 0
    import multiprocessing as mp

    cores = min(os.cpu_count() or 1, 16)
    ctx = mp.get_context("spawn")
    frames_per_step = cores
    with ctx.Pool(cores) as pool:
        import oracle

        oracle.build()
        frames = make_frames(frames_per_step, pool)
        for _ in range(args.warmup):
            pool.map(_oracle_detect, frames)
        per_step = []
        for k in range(args.steps):
            t0 = time.perf_counter()
            pool.map(_oracle_detect, frames)
            per_step.append(time.perf_counter() - t0)
    tot = sum(per_step)
    value = frames_per_step * args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "frames/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1000 * tot / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": WORKLOAD, "frames_per_step": frames_per_step},
            "cpu_baseline": {"value": round(value, 4), "unit": "frames/s", "cores": cores, "kind": "oracle",
                             "sample": f"{frames_per_step} distinct 1920x1080 frames per step, one "
                                       "oracle process per core"},
            "e2e": {"value": round(value, 4), "unit": "frames/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def parse_tuning(text):
    """--tuning: a JSON object holding every field of TUNING_FIELDS as an integer.

    The bench line's own "autotune" object is accepted as it is: the search
    statistics it also holds (candidates, stage times) are dropped.  Other keys
    and missing fields are errors; the library validates the values."""
    stats = ("candidates_tried", "resize_ms", "fast_ms", "nms_ms")
    try:
        obj = json.loads(text)
    except ValueError as e:
        raise SystemExit(f"--tuning: not JSON ({e})")
    if not isinstance(obj, dict):
        raise SystemExit("--tuning: expected a JSON object")
    unknown = sorted(set(obj) - set(TUNING_FIELDS) - set(stats))
    missing = [k for k in TUNING_FIELDS if k not in obj]
    if unknown or missing:
        raise SystemExit(f"--tuning: unknown fields {unknown}, missing fields {missing}")
    bad = [k for k in TUNING_FIELDS if isinstance(obj[k], bool) or not isinstance(obj[k], int)]
    if bad:
        raise SystemExit(f"--tuning: fields {bad} must be integers")
    return {k: obj[k] for k in TUNING_FIELDS}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--batch", type=int, default=128, help="frames per step")
    ap.add_argument("--plain-frames", type=int, default=32, help="frames per step of the per-frame leg")
    ap.add_argument("--distinct", type=int, default=16, help="distinct synthetic frames")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-frames", type=int, default=0, help="oracle sample size (0: 2 x cores)")
    ap.add_argument("--skip-plain", action="store_true", help="skip the per-frame path (profiling)")
    ap.add_argument("--serve-seconds", type=float, default=4.0, help="serving leg duration (0: skip)")
    ap.add_argument("--serve-rate", type=float, default=500.0, help="Poisson arrival rate, frames/s")
    ap.add_argument("--serve-sat-rate", type=float, default=20000.0,
                    help="offered rate of the saturated serving leg, frames/s, with at most 512 frames "
                         "outstanding (0: skip)")
    ap.add_argument("--skip-e2e", action="store_true", help="skip the host-buffer path (profiling)")
    ap.add_argument("--skip-learned", action="store_true", help="skip the learned tile-proposal leg")
    ap.add_argument("--skip-ablation", action="store_true", help="skip the paper-variant ablation leg")
    ap.add_argument("--skip-mixed", action="store_true", help="skip the uneven-size batch leg")
    ap.add_argument("--tuning", type=str, default=None,
                    help="JSON object of every launch-configuration field (%s): installed with of_set_tuning "
                         "instead of the autotuner's search, so that a profiling run launches what a timed "
                         "run chose" % ", ".join(TUNING_FIELDS))
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    fixed_tuning = parse_tuning(args.tuning) if args.tuning else None

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import multiprocessing as mp

    cores = os.cpu_count() or 1
    pool = mp.get_context("spawn").Pool(min(cores, 16))
    frames_np = make_frames(args.distinct, pool)

    import numpy as np
    import torch

    import paper_2506_07164_gb300 as ofg

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    ofg.build()
    ofg.load()
    B = args.batch
    stream = torch.cuda.Stream()
    dev_frames = [torch.from_numpy(frames_np[i % len(frames_np)]).cuda() for i in range(B)]
    torch.cuda.synchronize()
    batched = ofg.Detector(W_, H_, max_levels=LEVELS, max_features=NFEAT, max_batch=B, fast_t_lo=FAST_T_LO,
                           stream=stream)
    plain = ofg.Detector(W_, H_, max_levels=LEVELS, max_features=NFEAT, max_batch=1, fast_t_lo=FAST_T_LO,
                         stream=stream)
    frames = [(t, W_, H_, W_) for t in dev_frames]
    # Autotune the batched plan once (launch configuration per stage), or install the
    # given one, then time it.
    with torch.cuda.stream(stream):
        if fixed_tuning is None:
            tuning = ofg.of_autotune(batched.h, frames, LEVELS, SCALE, FAST_T, HARRIS_K, NFEAT, batched.out,
                                     batched.counts, reps=3).as_dict()
        else:
            ofg.of_set_tuning(batched.h, frames, LEVELS, SCALE, FAST_T, HARRIS_K, NFEAT, batched.out,
                              batched.counts, ofg.OfTuning(**fixed_tuning))
            tuning = dict(fixed_tuning)
    torch.cuda.synchronize()

    def step_batched(events=None):
        if events is not None:
            ofg.of_time_stages(batched.h, events)
        ofg.of_detect_batch(batched.h, frames, LEVELS, SCALE, FAST_T, HARRIS_K, NFEAT, batched.out,
                            batched.counts)

    def step_plain():
        for f in frames[: args.plain_frames]:
            ofg.of_detect_batch(plain.h, [f], LEVELS, SCALE, FAST_T, HARRIS_K, NFEAT, plain.out, plain.counts)

    def timed(fn, steps, warmup, per_step_events=False, nvtx_name="timed"):
        for _ in range(warmup):
            fn() if not per_step_events else fn(None)
        barrier()
        evs = None
        if per_step_events:
            evs = [[torch.cuda.Event(enable_timing=True) for _ in range(ofg.OF_N_STAGES + 1)]
                   for _ in range(steps)]
            for row in evs:
                for e in row:
                    e.record(stream)
        barrier()
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push(nvtx_name)
        start.record(stream)
        for k in range(steps):
            fn(evs[k]) if per_step_events else fn()
        end.record(stream)
        torch.cuda.nvtx.range_pop()
        end.synchronize()
        barrier()
        ms = start.elapsed_time(end)
        stage_ms = None
        if evs:
            stage_ms = [statistics.mean(row[i].elapsed_time(row[i + 1]) for row in evs)
                        for i in range(ofg.OF_N_STAGES)]
        return ms, stage_ms

    # Clock samples go to $OFAST_CLOCKS_DIR when that directory exists (to keep them), else to /tmp.
    clock_dir = os.environ.get("OFAST_CLOCKS_DIR", "")
    clock_file = (os.path.join(clock_dir, f"clocks_rank{rank}.csv") if clock_dir and os.path.isdir(clock_dir)
                  else f"/tmp/ofast_clocks_{os.getpid()}.csv")
    smi = sample_clocks("", clock_file)
    time.sleep(0.3)
    ms_b, _ = timed(step_batched, args.steps, args.warmup, nvtx_name="batched_timed")
    if smi is not None:
        smi.terminate()
        smi.wait()
    clocks = summarize_clocks(clock_file)
    # Stage times: the same kernels run stage by stage (the per-stage graphs of
    # of_time_stages, one launch per stage over the whole batch), with events
    # between the stages; the timed graph above may run two frame groups on
    # two branches whose stages overlap.
    ms_stages, stage_ms = timed(step_batched, args.steps, 1, per_step_events=True, nvtx_name="stages_timed")
    plain_steps = max(2, args.steps // 4)
    plain_frames = min(args.plain_frames, B)
    ms_p = float("nan")
    if not args.skip_plain:
        ms_p, _ = timed(step_plain, plain_steps, 2, nvtx_name="plain_timed")

    # Uneven sizes: one batched call over 64 frames of four sizes (its own
    # autotuned plan) against one call per frame on the same frames.
    mixed = None
    ms_m = ms_mp = float("nan")
    if not args.skip_mixed:
        mdev = [torch.from_numpy(a).cuda() for a in mixed_frames(pool, MIXED_FRAMES)]
        mframes = [(t, t.shape[1], t.shape[0], t.shape[1]) for t in mdev]
        mdet = ofg.Detector(W_, H_, max_levels=LEVELS, max_features=NFEAT, max_batch=MIXED_FRAMES,
                            fast_t_lo=FAST_T_LO, stream=stream)
        with torch.cuda.stream(stream):
            mtun = ofg.of_autotune(mdet.h, mframes, LEVELS, SCALE, FAST_T, HARRIS_K, NFEAT, mdet.out,
                                   mdet.counts, reps=3).as_dict()

        def step_mixed():
            ofg.of_detect_batch(mdet.h, mframes, LEVELS, SCALE, FAST_T, HARRIS_K, NFEAT, mdet.out, mdet.counts)

        def step_mixed_plain():
            for f in mframes:
                ofg.of_detect_batch(plain.h, [f], LEVELS, SCALE, FAST_T, HARRIS_K, NFEAT, plain.out, plain.counts)

        ms_m, _ = timed(step_mixed, args.steps, args.warmup, nvtx_name="mixed_timed")
        ms_mp, _ = timed(step_mixed_plain, plain_steps, 2, nvtx_name="mixed_plain_timed")
        # The per-frame path's last call is the batch's last frame: same records.
        last = MIXED_FRAMES - 1
        nb, npl = int(mdet.counts[last].item()), int(plain.counts[0].item())
        same = nb == npl and torch.equal(mdet.out[last * NFEAT * 64:(last * NFEAT + nb) * 64],
                                         plain.out[: npl * 64])
        mpx_m = sum(w * h for (_, w, h, _) in mframes) / 1e6
        mixed = {"frames_per_step": MIXED_FRAMES, "sizes": [f"{w}x{h}" for w, h in MIXED_SIZES],
                 "base_mpix_per_step": round(mpx_m, 2), "steps": args.steps, "plain_steps": plain_steps,
                 "last_frame_identical_to_per_frame": bool(same),
                 "autotune": {k: mtun[k] for k in TUNING_FIELDS}}
        mdet.close()

    # End to end through the public API with host buffers: every step copies
    # its B frames from one pinned host batch to the device (one copy), detects
    # and copies the keypoint records and counts back.  Two device input sets,
    # each with its own handle, let step k+1's upload (copy stream) overlap
    # step k's detection (compute stream); the timed region ends with a full
    # synchronize, so every step's copies are inside it.
    host_batch = torch.empty((B, H_, W_), dtype=torch.uint8).pin_memory()
    for i in range(B):
        host_batch[i].copy_(torch.from_numpy(frames_np[i % len(frames_np)]))
    dev_sets = [torch.empty((B, H_, W_), dtype=torch.uint8, device="cuda") for _ in range(2)]
    e2e_dets = [batched]
    copy_stream = torch.cuda.Stream()
    out_host = [torch.empty(B * NFEAT * 64, dtype=torch.uint8).pin_memory() for _ in range(2)]
    cnt_host = [torch.empty(B, dtype=torch.int32).pin_memory() for _ in range(2)]
    e2e_frames = [[(dev_sets[k][i], W_, H_, W_) for i in range(B)] for k in range(2)]

    def e2e_steps_run(n):
        ready = [torch.cuda.Event() for _ in range(2)]
        done = [torch.cuda.Event() for _ in range(2)]
        for k in range(n):
            c = k % 2
            det = e2e_dets[c]
            with torch.cuda.stream(copy_stream):
                if k >= 2:
                    copy_stream.wait_event(done[c])  # the detect that last read set c
                dev_sets[c].copy_(host_batch, non_blocking=True)
                ready[c].record(copy_stream)
            with torch.cuda.stream(stream):
                stream.wait_event(ready[c])
                ofg.of_detect_batch(det.h, e2e_frames[c], LEVELS, SCALE, FAST_T, HARRIS_K, NFEAT, det.out,
                                    det.counts)
                done[c].record(stream)
                cnt_host[c].copy_(det.counts[:B], non_blocking=True)
                out_host[c].copy_(det.out[: B * NFEAT * 64], non_blocking=True)
        torch.cuda.synchronize()

    e2e_steps = max(4, args.steps)
    e2e_s = float("nan")
    if not args.skip_e2e:
        e2e_dets.append(ofg.Detector(W_, H_, max_levels=LEVELS, max_features=NFEAT, max_batch=B,
                                     fast_t_lo=FAST_T_LO, stream=stream))
        with torch.cuda.stream(stream):
            ofg.of_set_tuning(e2e_dets[1].h, e2e_frames[1], LEVELS, SCALE, FAST_T, HARRIS_K, NFEAT, e2e_dets[1].out,
                              e2e_dets[1].counts, ofg.OfTuning(**{k: tuning[k] for k in TUNING_FIELDS}))
        e2e_steps_run(2)
        barrier()
        t0 = time.perf_counter()
        e2e_steps_run(e2e_steps)
        barrier()
        e2e_s = time.perf_counter() - t0
        # The last step's records are the same frames' records as the timed batched path.
        assert np.array_equal(cnt_host[(e2e_steps - 1) % 2].numpy(), batched.counts[:B].cpu().numpy())

    # Correctness spot check of the timed configuration: frame 0 vs frame 0 of a single call.
    torch.cuda.synchronize()
    counts = batched.counts[:B].cpu().numpy()

    # Plan geometry and candidate counts for the algorithmic byte model.
    lw, lh, _ = ofg.of_plan_levels(W_, H_, LEVELS, SCALE, NFEAT)
    cand = []
    kept = []
    for l in range(LEVELS):
        _, dims = ofg.of_inspect(batched.h, ofg.OF_BUF_CAND, 0, l)
        cand.append(dims[2])
    recs = ofg.keypoints_to_numpy(batched.out[: NFEAT * 64])[: int(counts[0])]
    for l in range(LEVELS):
        kept.append(int((recs["level"] == l).sum()))
    per_frame = stage_bytes(lw, lh, cand, kept)

    # Max over ranks.
    ms_b, ms_p, e2e_s, ms_m, ms_mp = reduce_max_over_ranks([ms_b, ms_p, e2e_s, ms_m, ms_mp], dist, device="cuda")

    value = replicas_value(B * args.steps, world, ms_b)
    plain_fps = replicas_value(plain_frames * plain_steps, world, ms_p)
    e2e_fps = replicas_value(B * e2e_steps, world, e2e_s * 1000.0)
    if mixed is not None:
        m_fps = replicas_value(MIXED_FRAMES * args.steps, world, ms_m)
        mp_fps = replicas_value(MIXED_FRAMES * plain_steps, world, ms_mp)
        per_frame_mpix = mixed["base_mpix_per_step"] / MIXED_FRAMES
        mixed.update({"value": round(m_fps, 2), "unit": "frames/s", "mpix_per_s": round(m_fps * per_frame_mpix, 1),
                      "plain": round(mp_fps, 2), "plain_mpix_per_s": round(mp_fps * per_frame_mpix, 1),
                      "batched_vs_plain": round(m_fps / mp_fps, 3)})
    mpix = W_ * H_ / 1e6

    peak, peak_kind = measured_peaks()
    shares = [m / sum(stage_ms) for m in stage_ms]
    dom = int(np.argmax(stage_ms))
    stage_hbm = {n: round(per_frame[i] * B / (stage_ms[i] / 1000.0) / 1e9 / peak, 4)
                 for i, n in enumerate(ofg.STAGE_NAMES)}
    n_sms = torch.cuda.get_device_properties(local).multi_processor_count
    sm_max = float(clocks.get("sm_max_mhz") or 2070.0)
    if ofg.STAGE_NAMES[dom] == "fast":
        # The dominant stage is integer-ALU bound: report it against the ALU pipe.
        ops = FAST_OPS_PER_PX * detect_region_pixels(lw, lh) * B
        achieved = ops / (stage_ms[dom] / 1000.0) / 1e9
        peak_alu = n_sms * ALU_LANES_PER_SM_CLK * sm_max * 1e6 / 1e9
        kname = {0: "k_fast", 1: "k_fast_cells", 2: "k_fast_aligned", 3: "k_fast_warp",
                 4: "k_fast_cstrip"}[int(tuning.get("fast_cell_tiles", 0))]
        roofline = {"bound": "alu", "kernel": kname, "achieved": round(achieved, 1), "peak": round(peak_alu, 1),
                    "peak_kind": f"derived: {n_sms} SMs x {ALU_LANES_PER_SM_CLK} ALU lanes/clk x {sm_max:.0f} MHz",
                    "unit": "Gop/s", "frac": round(achieved / peak_alu, 4),
                    "traffic": round(STAGE_TRAFFIC["dram_bytes_per_frame"]["fast"] * B) if traffic_ok(tuning) else None,
                    "algorithmic_bytes": per_frame[1] * B,
                    "hbm_frac_of_measured": stage_hbm["fast"], "hbm_peak_gbs": peak}
    else:
        achieved = per_frame[dom] * B / (stage_ms[dom] / 1000.0) / 1e9
        roofline = {"bound": "hbm", "kernel": ofg.STAGE_NAMES[dom], "achieved": round(achieved, 1), "peak": peak,
                    "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": None}
    roofline.update({"stage_ms_per_step": {n: round(m, 4) for n, m in zip(ofg.STAGE_NAMES, stage_ms)},
                     "stage_share": {n: round(x, 4) for n, x in zip(ofg.STAGE_NAMES, shares)},
                     "stage_frac_of_hbm": stage_hbm,
                     "algorithmic_bytes_per_frame": dict(zip(ofg.STAGE_NAMES, per_frame))})
    # L2 beside HBM: measured read peaks (library probe), and each stage's
    # captured L2 and DRAM bytes over its live stage time.
    peaks_rd = measure_read_peaks(ofg, torch, stream)
    roofline["read_peaks_gbs"] = {"l2": peaks_rd["l2"], "hbm": peaks_rd["hbm"],
                                  "how": "of_probe_read: 16-byte L2-only loads, 8x256 threads per SM; L2: best "
                                         "of 8..48 MB buffers read repeatedly; HBM: a 4 GiB buffer"}
    if traffic_ok(tuning):
        l2b, drb = STAGE_TRAFFIC["l2_bytes_per_frame"], STAGE_TRAFFIC["dram_bytes_per_frame"]
        roofline["stage_l2_gbs"] = {n: round(l2b[n] * B / (stage_ms[i] / 1000.0) / 1e9, 1)
                                    for i, n in enumerate(ofg.STAGE_NAMES)}
        roofline["stage_frac_of_l2"] = {n: round(v / peaks_rd["l2"], 4) for n, v in roofline["stage_l2_gbs"].items()}
        roofline["stage_dram_gbs"] = {n: round(drb[n] * B / (stage_ms[i] / 1000.0) / 1e9, 1)
                                      for i, n in enumerate(ofg.STAGE_NAMES)}
        roofline["stage_dram_frac_of_hbm"] = {n: round(v / peak, 4) for n, v in roofline["stage_dram_gbs"].items()}
    else:
        roofline["stage_l2_gbs"] = roofline["stage_frac_of_l2"] = None
        roofline["stage_traffic_note"] = "kernels or launch choices differ from the captured ones"
    # The whole step against the memory roofline: least HBM bytes per frame
    # (input, resident levels written once and read once, records) at the
    # measured frame rate.
    floor = floor_bytes_per_frame(lw, lh, float(np.mean(counts)))

    # Learned tile proposal on the same batch: committed network and threshold.
    learned_out = None
    if not args.skip_learned:
        from paper_2506_07164_gb300 import learned as lrn

        meta = json.load(open(lrn.DEFAULT_META))
        net = lrn.TileNet(0).load(lrn.DEFAULT_WEIGHTS)
        thr, dil, mc = meta["threshold"], meta["dilate"], meta["min_confidence"]
        plain_recs = ofg.keypoints_to_numpy(batched.out[: B * NFEAT * 64]).copy()
        plain_cnt = batched.counts[:B].cpu().numpy().copy()

        def step_learned():
            ofg.of_detect_learned(batched.h, frames, LEVELS, SCALE, FAST_T, HARRIS_K, NFEAT, net.net, thr, mc, dil,
                                  batched.out, batched.counts, want_stats=False)

        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                step_learned()
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.nvtx.range_push("learned_timed")
            e0.record(stream)
            for _ in range(args.steps):
                step_learned()
            e1.record(stream)
            torch.cuda.nvtx.range_pop()
            e1.synchronize()
            ms_l = e0.elapsed_time(e1)
            st = ofg.of_detect_learned(batched.h, frames, LEVELS, SCALE, FAST_T, HARRIS_K, NFEAT, net.net, thr, mc,
                                       dil, batched.out, batched.counts, want_stats=True)
        torch.cuda.synchronize()
        lrec = ofg.keypoints_to_numpy(batched.out[: B * NFEAT * 64])
        lcnt = batched.counts[:B].cpu().numpy()
        inter = union = tot = same = 0
        for f in range(B):
            a = plain_recs[f * NFEAT: f * NFEAT + plain_cnt[f]]
            b = lrec[f * NFEAT: f * NFEAT + lcnt[f]]
            A = {(int(l), int(y), int(x)) for l, y, x in zip(a["level"], a["y_l"], a["x_l"])}
            Bs = {(int(l), int(y), int(x)) for l, y, x in zip(b["level"], b["y_l"], b["x_l"])}
            inter += len(A & Bs)
            union += len(A | Bs)
            tot += len(A)
            same += int(len(a) == len(b) and np.array_equal(a.view(np.uint8), b.view(np.uint8)))
        lfps = B * args.steps * world / (ms_l / 1000.0)
        learned_out = {"value": round(lfps, 2), "unit": "frames/s", "ms_per_step": round(ms_l / args.steps, 4),
                       "vs_plain_batched": round(lfps / value, 3), "recall": round(inter / max(1, tot), 5),
                       "jaccard": round(inter / max(1, union), 5), "identical_frames": same, "frames": B,
                       "proposed_fraction": round(st["proposed"] / max(1, st["tiles"]), 4),
                       "fallback_images": st["fallback_images"], "threshold": thr, "dilate": dil,
                       "network": "3x conv3x3 s2 (8/16/16) + GAP + linear, bf16 weights, fp32 accumulate; "
                                  f"trained on {meta['train_frames']} synthetic 1080p frames "
                                  f"({meta['train_tiles']} tiles, {meta['steps']} Adam steps)"}
        net.close()

    ablation = None
    if not args.skip_ablation and rank == 0:
        ablation = ablation_leg(pool, batched, stream)

    serving = serving_sat = None
    if args.serve_seconds > 0:
        serving = serving_leg(pool, args.serve_seconds, args.serve_rate)
        if args.serve_sat_rate > 0:
            serving_sat = serving_leg(pool, args.serve_seconds, args.serve_sat_rate, seed=1, clients=8,
                                      max_outstanding=512)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n = args.cpu_frames or 2 * min(cores, 16)
        cpu = cpu_baseline(pool, min(cores, 16), frames_np, n)
    pool.close()

    # Per frame group: one resize per level after the first, FAST, the threshold
    # pass (FAST forms 0, 3, 4; after the per-warp NMS kernel, which applies the
    # thresholds itself, only where the FAST form leaves the flags to it: forms
    # 0 and 3), NMS + Harris, top-N, orientation.
    form = int(tuning.get("fast_cell_tiles", 0))
    has_pass = form in (0, 3) or (form == 4 and int(tuning.get("nms_tile_h", 64)) != 32)
    per_group = (LEVELS - 1) + 4 + (1 if has_pass else 0)
    kernels_per_step = per_group * int(tuning.get("stream_groups", 1))
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "frames/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_b / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "frames_per_step": B, "distinct_frames": len(frames_np),
                   "parallelism": f"replicas x{world}",
                   "l2": f"inputs larger than L2: {B} frames x {W_ * H_ / 1e6:.2f} MB per step"},
        "mpix_per_s": round(value * mpix, 1),
        "memory_roofline": {"floor_bytes_per_frame": round(floor), "achieved_gbs": round(floor * value / 1e9, 1),
                            "peak_gbs": peak, "peak_kind": peak_kind, "frac": round(floor * value / 1e9 / peak, 4),
                            "floor": "input + levels 1..7 written + all levels read once + 64 B records"},
        "staged_ms_per_step": round(ms_stages / args.steps, 4),
        "plain": {"value": round(plain_fps, 2), "unit": "frames/s", "mpix_per_s": round(plain_fps * mpix, 1),
                  "steps": plain_steps, "frames_per_step": plain_frames,
                  "launch": "one of_detect_batch call (one graph) per frame"},
        "batched_vs_plain": round(value / plain_fps, 3),
        "e2e": {"value": round(e2e_fps, 2), "unit": "frames/s", "h2d_bytes_per_step": B * W_ * H_,
                "d2h_bytes_per_step": B * NFEAT * 64 + 4 * B, "steps": e2e_steps,
                "pipelining": "two device input sets and handles; step k+1's H2D (copy stream) overlaps "
                              "step k's detection"},
        "autotune": {k: (round(v, 4) if isinstance(v, float) else v) for k, v in tuning.items()},
        "tuning_source": "autotuned" if fixed_tuning is None else "fixed (--tuning)",
        "roofline": roofline,
        "mixed": mixed,
        "learned": learned_out,
        "ablation": ablation,
        "serving": serving,
        "serving_saturated": serving_sat,
        "cpu_baseline": cpu,
        "clocks": clocks,
        "gpu_launches": kernels_per_step * args.steps,
        "keypoints_per_frame": float(np.mean(counts)),
        "candidates_frame0": cand,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    for d in e2e_dets[1:]:
        d.close()
    batched.close()
    plain.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
