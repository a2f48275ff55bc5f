"""Benchmark of the box-tracking hot path on the batched multi-stream workload.

Workload (one step): 32 independent video streams, resolutions drawn from
{720x576, 1280x720, 1920x1080}, each with a target of 2,000-20,000 points
(log-uniform) as Shi-Tomasi corners over an 8x8 grid of boxes, and a smooth
displacement field of at most 12 px between its two frames.  A step runs the
whole hot path for every stream: the pyramid of the new frame, the corners of
frame t inside the boxes, pyramidal LK (4 levels, 21x21 window, 30
iterations, eps 0.01) and the per-box median update.  Frames alternate
between each stream's two renders, so every step tracks a real pair.

Headline (`value`): LK tracked points/s (OK points only) of the batched path
(one omt_batch_step per step for all streams, FP16-stored pyramids by
default, replayed as a CUDA graph), with every input resident on the device.
Beside it, in `config`: the plain per-stream FP32 path (five C-ABI calls per
stream and step) on the same streams, the ratio of the two, stream-frames/s
and per-step latency percentiles.  `e2e` copies every step's frames host ->
device from pinned memory and reads every box back.

Beside the step: `served` runs the serving loop (workload 5: 64 streams of
mixed resolution, Poisson arrivals, 40 GB admission budget) and searches the
highest arrival rate each path serves with p99 frame latency <= 40 ms, for
the batched FP16 path and the plain per-stream FP32 path; `roofline` divides
the LK kernel's algorithmic flops by a measured FP32 multiply-add peak
(probe/fma_peak.cu, timed in the same run); `cpu_baseline` times the FP64
oracle on the host cores, one thread and all, on workloads 1-4.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl omt|reference]
                    [--storage f16|f32] [--streams S] [--no-graph] [--no-tune]
                    [--no-serve] [--no-cpu-baseline]
    python bench.py --flow | --match | --overlap | --working-level
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = ("32 streams {720x576,1280x720,1920x1080}, 2k-20k points/stream (8x8 box grid), "
            "|d|<=12 px, 4 levels, 21x21 window, 30 iterations, eps 0.01")
METRIC = "LK tracked points/s"
LEVELS, WIN, MAX_ITER, EPS, MIN_DIST = 4, 21, 30, 0.01, 3.0
GRID = (8, 8)
FALLBACK_PEAKS = {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}
SMS, FP32_LANES = 148, 128


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return dict(FALLBACK_PEAKS), "fallback"


def source_digest(files) -> str:
    """sha256 over kernel source files (paths relative to the repository)."""
    import hashlib
    h = hashlib.sha256()
    for rel in files:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def dram_traffic(kernel: str):
    """DRAM bytes of one ncu capture of `kernel` (profiles/traffic.json), or
    None when the kernel's sources changed since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f).get(kernel)
    if not rec or source_digest(rec["sources"]) != rec["sha256"]:
        return None
    return rec


def combine_ranks(times, counts, device):
    """Whole-job figures of a multi-rank run: the slowest rank's times (max)
    and the points of all ranks (sum), over the initialised process group."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(list(times), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor(list(counts), dtype=torch.float64, device=device)
    dist.all_reduce(c)
    return [float(x) for x in t], [float(x) for x in c]


def dist_env():
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        import tempfile
        self.dev = device_index
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix="omt_clocks_", suffix=".csv")
        os.close(fd)

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


def make_streams(n_streams: int, rank: int):
    from paper_1910_06017_b300 import synth
    return [synth.stream_pair(rank * n_streams + s) for s in range(n_streams)]


def cap_of(sp) -> int:
    return int(math.ceil(sp.n_target / (GRID[0] * GRID[1])))


def lk_flops(iters: np.ndarray, status: np.ndarray, levels: int, win: int) -> float:
    """Algorithmic FP32 flops of the LK kernel for these points.

    Per point and level reached: the frame-t window costs 27 N flops (three
    bilinear samples at 7 flops each plus three multiply-adds) and each
    iteration 12 N (one bilinear sample, a subtraction, two multiply-adds),
    N = win^2; the 2x2 solves are ignored.  A level is reached down to the
    last level with iterations, plus the level where a point was lost on
    its eigenvalue."""
    N = win * win
    it = iters.astype(np.int64)
    reached = np.zeros(len(it), np.int64)
    nz = it > 0
    for L in range(levels):
        reached += np.any(nz[:, :L + 1], axis=1)
    reached += ((status & 2) > 0).astype(np.int64)
    return float(27 * N * reached.sum() + 12 * N * it.sum())


def pyramid_bytes_per_px(storage: str, levels: int) -> float:
    """Compulsory DRAM bytes of the pyramid per level-0 pixel: read the u8
    frame, write its u8 copy, write every level >= 1 once and every level's
    gradient pair once (level L holds 4^-L of the pixels)."""
    esz = 2.0 if storage == "f16" else 4.0
    frac = [4.0 ** -L for L in range(levels)]
    return 1.0 + 1.0 + esz * sum(frac[1:]) + 2 * esz * sum(frac)


def params_for(omt, storage, max_corners):
    return omt.default_params(levels=LEVELS, win=WIN, max_iter=MAX_ITER, eps=EPS,
                              max_corners=max_corners, storage=storage, min_dist=MIN_DIST)


def measure_plain(omt, torch, streams, dev, steps, warmup):
    """Plain per-stream FP32 path: ms per step (CUDA events) and OK points."""
    trackers, frames, boxes = [], [], []
    for sp in streams:
        w, h = sp.size
        T = omt.StreamTracker(w, h, params_for(omt, omt.F32, cap_of(sp)), len(sp.boxes), dev)
        f0, f1 = torch.from_numpy(sp.frame0).to(dev), torch.from_numpy(sp.frame1).to(dev)
        T.prime(f0)
        trackers.append(T)
        frames.append((f0, f1))
        boxes.append(torch.from_numpy(sp.boxes).to(dev))

    def step(k):
        for T, f, b in zip(trackers, frames, boxes):
            T.step(f[(k + 1) % 2], b)

    for k in range(warmup):
        step(k)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for k in range(warmup, warmup + steps):
        step(k)
    b.record()
    torch.cuda.synchronize()
    ok = 0
    for T, sp in zip(trackers, streams):
        n = int(T.offsets[len(sp.boxes)].item())
        ok += int(((T.status[:n].cpu().numpy() & 1) > 0).sum())
    del trackers
    return a.elapsed_time(b) / steps, ok


def measure_fp32_peak(local: int):
    """Measured FP32 multiply-add throughput of this GPU (TFLOP/s): the
    faster of scalar and packed chains (probe/fma_peak.cu), each launch about
    0.1 s, with the SM clock sampled meanwhile."""
    import ctypes
    import torch
    from paper_1910_06017_b300 import build as bld
    L = ctypes.CDLL(bld.build_probe())
    L.omt_probe_fma_tflops.restype = ctypes.c_double
    L.omt_probe_fma_tflops.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                       ctypes.POINTER(ctypes.c_float)]
    sink = torch.empty(SMS * 8 * 256 * 4, dtype=torch.float32, device=f"cuda:{local}")
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    res = {}
    for packed in (0, 1):
        ms = ctypes.c_float(0.0)
        best = 0.0
        for _ in range(3):
            t = L.omt_probe_fma_tflops(packed, 30000, ctypes.c_void_p(sink.data_ptr()),
                                       ctypes.byref(ms))
            best = max(best, t)
        res["packed" if packed else "scalar"] = {"tflops": best, "ms": float(ms.value)}
    clk = clocks.stop()
    peak = max(v["tflops"] for v in res.values())
    return peak, {"probe": "probe/fma_peak.cu: 8 independent FMA chains per thread, 8 CTAs of 256 "
                           "threads per SM, CUDA events, best of 3", **res, "clocks": clk}


def served(args, local):
    """Capacity of the serving loop (workload 5) for both paths: the highest
    common scale of the 25-60 fps arrival rates served completely with p99
    frame latency <= 40 ms (serve.capacity: doubling/halving, then three
    geometric bisections; 2 s of arrivals per probe)."""
    import torch
    from paper_1910_06017_b300 import omt, serve
    out = {"metric": "stream frames/s at p99 frame latency <= 40 ms",
           "workload": "64 streams {720x576,1920x1080,3840x2160}, Poisson 25-60 fps x scale, "
                       "20-300 boxes refreshed every 5-15 frames, <= 50 corners/box, 4 levels, "
                       "21x21, 40 GB admission budget; latency = arrival -> boxes ready, "
                       "frames copied from page-locked host memory inside it"}
    budget = 40 << 30
    for label, plain in (("batched_f16", False), ("plain_f32", True)):
        storage = omt.F32 if plain else omt.F16
        params = omt.default_params(levels=4, win=21, max_corners=50, storage=storage)
        specs, frames, det = serve.build_workload(2, 0.5)
        serve.serve(specs, frames, det, params, budget, plain=plain, deadline=0.5)   # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        best, probes = serve.capacity(64, params, plain, budget, p99_ms=40.0, duration=args.serve_s,
                                      bisect=3)
        out[label] = {"stream_frames_per_s": best["stream_frames_per_s"] if best else 0.0,
                      "latency_ms_p50": best["latency_ms_p50"] if best else None,
                      "latency_ms_p99": best["latency_ms_p99"] if best else None,
                      "rate_scale": best["fps_scale"] if best else None,
                      "probes": probes, "search_s": round(time.perf_counter() - t0, 1)}
        torch.cuda.empty_cache()
    b, p = out["batched_f16"]["stream_frames_per_s"], out["plain_f32"]["stream_frames_per_s"]
    out["ratio_batched_over_plain"] = b / p if p else None
    return out


def run_omt(args, ws, rank, local):
    import torch
    from paper_1910_06017_b300 import omt

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    storage = omt.F16 if args.storage == "f16" else omt.F32
    streams = make_streams(args.streams, rank)

    plain_ms, plain_ok = measure_plain(omt, torch, streams, dev, max(3, args.steps // 4), 3)
    torch.cuda.empty_cache()

    caps = [cap_of(sp) for sp in streams]
    prm = params_for(omt, storage, max(caps))
    if args.fb is not None:
        prm = prm.replace(fb_max=args.fb)  # forward-backward check in every step
    B = omt.BatchTracker([sp.size for sp in streams], prm, max_boxes=[len(sp.boxes) for sp in streams],
                         max_corners=caps, device=dev)
    fr_h = []
    for s, sp in enumerate(streams):
        B.prime(s, torch.from_numpy(sp.frame0).to(dev))
        B.frame[s][0].copy_(torch.from_numpy(sp.frame1))   # parity 0 reads frame 1
        B.frame[s][1].copy_(torch.from_numpy(sp.frame0))   # parity 1 reads frame 0
        B.set_boxes(s, torch.from_numpy(sp.boxes))
        fr_h.append((torch.from_numpy(sp.frame1).pin_memory(), torch.from_numpy(sp.frame0).pin_memory()))
    B.pack()
    for _ in range(args.warmup):
        B.step()
    torch.cuda.synchronize()
    # launch shape of the LK kernel, timed on this batch (results do not depend on it)
    tune_ms = B.autotune() if args.tune else {}
    torch.cuda.synchronize()
    if args.graph:
        B.capture()
        for _ in range(2):
            B.step()
        torch.cuda.synchronize()

    # ---- timed region: inputs resident, one step = all streams
    stream = torch.cuda.current_stream()
    clocks = Clocks(local)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev[0].record(stream)
    for k in range(args.steps):
        B.step()
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    step_ms = np.array([ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)])
    ms_total = ev[0].elapsed_time(ev[-1])

    ok_pts = n_pts = fb_lost = 0
    flops = 0.0
    for s in range(len(streams)):
        n = B.count(s)
        st = B.status[s][:n].cpu().numpy()
        fb_lost += int((st == omt.PT_LOST_FB).sum())
        it = B.iters[s][:n].cpu().numpy()
        ok_pts += int(((st & 1) > 0).sum())
        n_pts += n
        flops += lk_flops(it, st, LEVELS, WIN)

    # ---- per-phase kernel time: events around the LK and pyramid phases,
    # eager, same steps and stream
    ph_ev = []
    for k in range(args.steps):
        e = {p: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
             for p in (omt.PHASE_PYRAMID, omt.PHASE_LK, omt.PHASE_FB)}
        B.step_phases(events=e)
        ph_ev.append(e)
    torch.cuda.synchronize()
    lk_ms = float(np.mean([e[omt.PHASE_LK][0].elapsed_time(e[omt.PHASE_LK][1]) for e in ph_ev]))
    pyr_ms = float(np.mean([e[omt.PHASE_PYRAMID][0].elapsed_time(e[omt.PHASE_PYRAMID][1]) for e in ph_ev]))
    fb_ms = (float(np.mean([e[omt.PHASE_FB][0].elapsed_time(e[omt.PHASE_FB][1]) for e in ph_ev]))
             if B.fb else None)
    px0 = sum(sp.size[0] * sp.size[1] for sp in streams)
    pyr_bytes = px0 * pyramid_bytes_per_px(args.storage, LEVELS)

    # ---- end to end: every step's frames copied from page-locked host memory
    # and its boxes read back, through BatchTracker.run_pipelined (copies on a
    # second stream overlap the previous step's compute)
    torch.cuda.synchronize()
    par0 = B.cur
    t0 = time.perf_counter()
    h2d, d2h = B.run_pipelined(lambda k: [fr_h[s][(par0 + k) & 1] for s in range(len(streams))],
                               args.steps)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / args.steps

    ms_step = ms_total / args.steps
    ok_total, plain_ok_total = float(ok_pts), float(plain_ok)
    if ws > 1:
        (ms_step, e2e_s, plain_ms), (ok_total, plain_ok_total) = combine_ranks(
            [ms_step, e2e_s, plain_ms], [ok_pts, plain_ok], dev)
    value = ok_total / (ms_step * 1e-3)
    plain_value = plain_ok_total / (plain_ms * 1e-3)
    pk, pk_src = peaks()
    fp32_peak, fp32_probe = measure_fp32_peak(local)
    achieved = flops / (lk_ms * 1e-3) / 1e12
    serve_res = served(args, local) if args.serve and rank == 0 else None
    lk_tr = dram_traffic("lk_batch_kernel")
    pyr_tr = dram_traffic("pyramid_batch_kernel")
    level0_px = sum(w * h for w, h in (sp.size for sp in streams))
    return {
        "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {
            "workload": WORKLOAD,
            "path": "batched: one omt_batch_step per step" + (", CUDA graph" if args.graph else ""),
            "storage": args.storage, "streams_per_gpu": args.streams,
            "points_per_step": n_pts, "ok_points_per_step": ok_pts,
            **({"fb_max": args.fb, "fb_lost_points_per_step": fb_lost,
                "fb_ms_per_step": fb_ms} if args.fb is not None else {}),
            "stream_frames_per_s": args.streams * ws / (ms_step * 1e-3),
            "latency_ms_p50": float(np.percentile(step_ms, 50)),
            "latency_ms_p99": float(np.percentile(step_ms, 99)),
            "plain_f32_points_per_s": plain_value, "plain_f32_ms_per_step": plain_ms,
            "speedup_vs_plain_f32": value / plain_value,
            "l2": "working set > L2 (126 MB): no flush", "parallelism": f"replicas x{ws}",
            "lk_launch": {"warps_per_cta": B.caps.lk_warps or 4, "queue_chunk": B.caps.lk_chunk or 1,
                          "autotuned": bool(tune_ms),
                          "candidates_ms": {f"{w}x{c}": round(t, 4)
                                            for (w, c), t in tune_ms.get("lk", {}).items()}},
            "pyramid_launch": {"ctas_per_sm": B.caps.pyr_ctas_per_sm,
                               "candidates_ms": {str(c): round(t, 4)
                                                 for c, t in tune_ms.get("pyramid", {}).items()}},
            "corner_launch": {"list_ctas_per_sm": B.caps.corner_ctas_per_sm,
                              "select_ctas_per_sm": B.caps.select_ctas_per_sm,
                              "candidates_ms": {f"{c}x{s}": round(t, 4)
                                                for (c, s), t in tune_ms.get("corners", {}).items()}}},
        "e2e": {"value": ok_total / e2e_s, "unit": "points/s",
                "h2d_bytes_per_step": h2d // args.steps, "d2h_bytes_per_step": d2h // args.steps},
        "roofline": {"kernel": "lk_batch_kernel", "bound": "alu", "achieved": achieved,
                     "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                     # DRAM bytes of one launch on this workload (ncu capture of the
                     # same kernel source; see profiles/traffic.json)
                     "traffic": lk_tr["bytes_per_launch"] if lk_tr else None,
                     "peak_source": "measured in this run (FP32 multiply-add probe, of measured)",
                     "peak_probe": fp32_probe,
                     "nominal_tflops": SMS * FP32_LANES * 2 * pk.get("sm_max_mhz", 2032.0) / 1e6,
                     "lk_ms_per_step": lk_ms, "lk_share": lk_ms / ms_step},
        "roofline_pyramid": {"kernel": "pyramid_batch_kernel (all levels)", "bound": "hbm",
                             "achieved": pyr_bytes / (pyr_ms * 1e-3) / 1e9,
                             "peak": pk.get("hbm_gbs", 6400.0), "unit": "GB/s",
                             "frac": pyr_bytes / (pyr_ms * 1e-3) / 1e9 / pk.get("hbm_gbs", 6400.0),
                             # captured on a larger case, scaled per level-0 pixel
                             "traffic": (pyr_tr["bytes_per_level0_px"] * level0_px
                                         if pyr_tr and args.storage == "f16" else None),
                             "bytes_per_level0_px": pyramid_bytes_per_px(args.storage, LEVELS),
                             "ms_per_step": pyr_ms},
        "clocks": clk,
        "gpu_launches": (LEVELS + 5) * args.steps,
        **({"served": serve_res} if serve_res else {}),
    }


def run_reference(args, ws, rank):
    """The FP64 oracle on the host cores, on a bounded sample of the same
    workload: per step, one stream's pyramid pair, corners, LK and update."""
    from oracle import oracle as O
    sp = make_streams(1, rank)[0]
    O.lib()
    cores = O.max_threads()
    times, okc = [], 0
    for k in range(args.warmup + args.steps):
        t = time.perf_counter()
        P0 = O.Pyramid(sp.frame0, LEVELS)
        P1 = O.Pyramid(sp.frame1, LEVELS)
        pts, cnt = O.select_corners(sp.frame0, sp.boxes, cap_of(sp), min_dist=MIN_DIST)
        allp = np.concatenate([pts[i, :cnt[i]] for i in range(len(cnt))])
        out, st = O.lk_track(P0, P1, allp, win=WIN, max_iter=MAX_ITER, eps=EPS)
        off = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int32)
        O.update_boxes(sp.boxes, off, allp, out.astype(np.float32), st)
        dt = time.perf_counter() - t
        if k >= args.warmup:
            times.append(dt)
            okc = int(((st & 1) > 0).sum())
    sec = float(np.mean(times))
    value = okc / sec
    sample = f"stream 0 of the 32 per step ({sp.size[0]}x{sp.size[1]}, {okc} OK points)"
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "path": "FP64 CPU oracle"},
        "cpu_baseline": {"value": value, "unit": "points/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


# ------------------------------------------------------------ dense flow
FLOW_SIZE, FLOW_LEVELS, FLOW_BOXES = (1920, 1080), 4, 16
FLOW_METRIC = "dense flow frames/s (1920x1080)"
FLOW_WORKLOAD = ("1920x1080 frame pairs, texture shifted by (2.25, -1.5) px; per frame: "
                 "structure-texture, 4-level F32 pyramid, Huber-TV-L1 (3 warps x 30 iterations "
                 "per level), mean flow in 16 boxes")


def flow_frames(seed: int = 0):
    from paper_1910_06017_b300 import synth
    w, h = FLOW_SIZE
    rng = np.random.default_rng(synth.seed_for(6) + seed)
    tex = synth.Texture.draw(rng, w, h)
    f0 = synth.render_shift(tex, w, h, 0.0, 0.0)
    f1 = synth.render_shift(tex, w, h, 2.25, -1.5)
    boxes = synth.uniform_boxes(rng, w, h, FLOW_BOXES)
    return f0, f1, boxes


def flow_bytes_per_l0px(omt, fp) -> float:
    """Algorithmic DRAM bytes of the TV-L1 iteration launches per level-0
    pixel: a launch (one iteration, or two when fp.block is 2) reads the
    state once -- the extrapolated flow (8 B), the duals (16 B), the flow
    (8 B), the warped gradient (8 B), rho0 (4 B) -- and writes the duals,
    the flow and its extrapolation (32 B): 76 B per pixel and launch; each
    level adds a quarter of the one below."""
    area = sum(4.0 ** -L for L in range(FLOW_LEVELS))
    per = 2 if fp.block == 2 else 1
    launches = fp.iters // per + fp.iters % per
    return 76.0 * fp.warps * launches * area


def flow_launches_per_step(fp):
    """Kernels one flow step launches: the projection steps (two per launch
    when fp.block is 2) and the texture; one pyramid kernel per level; per
    level the upsampling and, per warp, the warp kernel and the primal-dual
    launches (pairs, then a single one for an odd count); the box means."""
    per = 2 if fp.block == 2 else 1
    st = fp.st_iters // per + fp.st_iters % per
    pd = fp.iters // per + fp.iters % per
    return st + 1 + FLOW_LEVELS + FLOW_LEVELS * (1 + fp.warps * (1 + pd)) + 1


def run_flow(args):
    """One step = one new frame: its texture, its F32 pyramid, the flow from
    the previous frame's pyramid, the mean flow in every box."""
    import torch
    from paper_1910_06017_b300 import omt
    dev = torch.device("cuda", 0)
    w, h = FLOW_SIZE
    f0, f1, boxes = flow_frames()
    fp = omt.default_flow_params()
    prm = omt.default_params(levels=FLOW_LEVELS)
    frames = [torch.from_numpy(f).to(dev) for f in (f0, f1)]
    host = [torch.from_numpy(f).pin_memory() for f in (f0, f1)]
    tex = [torch.zeros((h, w), dtype=torch.uint8, device=dev) for _ in range(2)]
    pyr = [omt.Pyramid(w, h, FLOW_LEVELS, omt.F32, dev) for _ in range(2)]
    st_scr = torch.empty(omt.lib().omt_structure_texture_scratch_bytes(w, h), dtype=torch.uint8, device=dev)
    tv_scr = torch.empty(omt.lib().omt_tvl1_scratch_bytes(w, h), dtype=torch.uint8, device=dev)
    flow = torch.zeros((h, w, 2), device=dev)
    bx = torch.from_numpy(np.ascontiguousarray(boxes, np.float32)).to(dev)
    bo = torch.zeros_like(bx)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > L2 (126 MB)

    def prime(k):
        omt.structure_texture(frames[k & 1], fp, tex[k & 1], st_scr)
        omt.build_pyramid(tex[k & 1], pyr[k & 1], prm)

    def step(k, ev=None):
        # frame k+1 arrives: its texture and pyramid, then the flow k -> k+1
        cur, nxt = k & 1, (k + 1) & 1
        omt.structure_texture(frames[nxt], fp, tex[nxt], st_scr)
        omt.build_pyramid(tex[nxt], pyr[nxt], prm)
        if ev:
            ev[0].record()
        omt.tvl1_flow(pyr[cur], pyr[nxt], fp, flow, tv_scr)
        if ev:
            ev[1].record()
        omt.box_mean_flow(flow, bx, bo)

    prime(0)
    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()
    clocks = Clocks(0)
    clocks.start()
    ms, tv = [], []
    for k in range(args.steps):
        flush.fill_(k & 255)    # L2 flushed between timed steps, outside the timed region
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        e[0].record()
        step(args.warmup + k, (e[1], e[2]))
        e[3].record()
        torch.cuda.synchronize()
        ms.append(e[0].elapsed_time(e[3]))
        tv.append(e[1].elapsed_time(e[2]))
    clk = clocks.stop()
    step_ms, tv_ms = float(np.mean(ms)), float(np.mean(tv))
    # end to end: the new frame copied from page-locked host memory, the boxes read back
    bo_h = torch.empty(bo.shape, dtype=torch.float32).pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for k in range(args.steps):
        frames[(k + 1) & 1].copy_(host[(k + 1) & 1], non_blocking=True)
        step(k)
        bo_h.copy_(bo, non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / args.steps
    byts = flow_bytes_per_l0px(omt, fp) * w * h
    pk, pk_src = peaks()
    hbm = pk.get("hbm_gbs", 6400.0)
    moved = (bo.cpu().numpy() - boxes)[:, :2]
    return {
        "metric": FLOW_METRIC, "value": 1e3 / step_ms, "unit": "frames/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": FLOW_WORKLOAD, "path": "omt_structure_texture + omt_build_pyramid + "
                   "omt_tvl1_flow + omt_box_mean_flow", "l2": "flushed between timed steps",
                   "tvl1_ms": tv_ms,
                   # steps alternate the pair's direction: +-(2.25, -1.5) px
                   "median_box_motion_last_step": np.median(moved, 0).tolist()},
        "e2e": {"value": 1e3 / e2e_ms, "unit": "frames/s", "h2d_bytes_per_step": w * h,
                "d2h_bytes_per_step": int(bo.numel() * 4)},
        "roofline": {"kernel": "pd2_kernel, the TV-L1 iterations (all levels)", "bound": "hbm",
                     "achieved": byts / (tv_ms * 1e-3) / 1e9, "peak": hbm,
                     "unit": "GB/s", "frac": byts / (tv_ms * 1e-3) / 1e9 / hbm,
                     "peak_source": pk_src, "traffic": None,
                     "bytes_per_level0_px": flow_bytes_per_l0px(omt, fp)},
        "clocks": clk,
        "gpu_launches": flow_launches_per_step(fp) * args.steps,
    }


def run_flow_reference(args):
    """The FP64 oracle's flow engine on the host cores, on a bounded sample:
    a 480x270 crop of the workload's frame pair per step (1/16 of the area),
    scaled to frames/s of the full frame by area."""
    from oracle import oracle as O
    f0, f1, boxes = flow_frames()
    c0, c1 = f0[:270, :480], f1[:270, :480]
    O.lib()
    P0 = O.Pyramid(O.structure_texture(c0), FLOW_LEVELS)   # the previous frame's, as on the GPU
    times = []
    for k in range(args.warmup + args.steps):
        t = time.perf_counter()
        T1 = O.structure_texture(c1)
        fl = O.tvl1(P0, O.Pyramid(T1, FLOW_LEVELS))
        O.box_mean_flow(fl, boxes / 4.0)
        if k >= args.warmup:
            times.append(time.perf_counter() - t)
    sec = float(np.mean(times)) * 16.0   # area of the full frame
    return {"value": 1.0 / sec, "unit": "frames/s", "cores": 1, "kind": "oracle",
            "sample": "480x270 crop of the 1920x1080 pair (the new frame's texture and "
                      "pyramid, 4-level flow, box means), time x16 by area"}


# ------------------------------------------------- beyond the hot path
def run_match(args):
    """The matching phase (Section V-A) at serving sizes: for n predicted
    boxes of a 1920x1080 frame against n detections (the predictions
    jittered, 10 % replaced), the device IoU matrix (CUDA events), its copy
    to page-locked host memory, the host assignment and the update (wall
    clock).  One JSON line per size."""
    import torch
    from paper_1910_06017_b300 import omt
    rng = np.random.default_rng(20191006)
    for n in (50, 300, 1000):
        x0, y0 = rng.uniform(0, 1800, n), rng.uniform(0, 960, n)
        w, h = rng.uniform(40, 150, n), rng.uniform(40, 150, n)
        pred = np.stack([x0, y0, x0 + w, y0 + h], 1).astype(np.float32)
        dets = pred + rng.normal(0, 4, pred.shape).astype(np.float32)
        drop = rng.uniform(0, 1, n) < 0.1
        dets[drop] = np.stack([x0[drop][::-1], y0[drop], x0[drop][::-1] + 60, y0[drop] + 60], 1)
        active = np.ones(n, np.uint8)
        pd, dd = torch.from_numpy(pred).cuda(), torch.from_numpy(dets).cuda()
        iou = torch.empty((n, n), dtype=torch.float64, device="cuda")
        for _ in range(3):
            omt.iou_matrix(pd, dd, iou)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 20
        e0.record()
        for _ in range(reps):
            omt.iou_matrix(pd, dd, iou)
        e1.record()
        torch.cuda.synchronize()
        iou_ms = e0.elapsed_time(e1) / reps
        host = torch.empty((n, n), dtype=torch.float64).pin_memory()
        t0 = time.perf_counter()
        host.copy_(iou)
        m = host.numpy()
        t1 = time.perf_counter()
        ma, mb = omt.assign(m, active)
        t2 = time.perf_counter()
        omt.update_tracks(pred, active, dets, ma, mb)
        t3 = time.perf_counter()
        print(json.dumps({"tracks": n, "detections": n, "iou_matrix_ms": round(iou_ms, 4),
                          "copy_ms": round(1e3 * (t1 - t0), 3), "assign_ms": round(1e3 * (t2 - t1), 3),
                          "update_ms": round(1e3 * (t3 - t2), 3), "matched": int((ma >= 0).sum())}))


def run_overlap(args):
    """Detection and tracking on one GPU at once (Section V-B runs the motion
    field and the detector concurrently).  The detector is a stub (YoloV3 and
    its weights are out of scope): per step, for every stream's frame, a
    chain of bf16 GEMMs of 4096 x 1024 x 1024 through torch (cuBLAS) on a
    CUDA stream of its own, 110 GFLOP per frame (about the two detector
    models).  The tracker is the batched step of the 32-stream workload (CUDA
    graph).  Median over the steps of CUDA events around tracking alone,
    detection alone and both issued every step on their two streams, also
    with the LK launch held to 2 CTAs per SM.  One JSON line."""
    import torch
    from paper_1910_06017_b300 import omt, synth
    dev = torch.device("cuda", 0)
    n_streams, gflop = args.streams, 110.0
    streams = [synth.stream_pair(s) for s in range(n_streams)]
    caps = [cap_of(sp) for sp in streams]
    prm = params_for(omt, omt.F16, max(caps))
    B = omt.BatchTracker([sp.size for sp in streams], prm, max_boxes=[len(sp.boxes) for sp in streams],
                         max_corners=caps, device=dev)
    for s, sp in enumerate(streams):
        B.prime(s, torch.from_numpy(sp.frame0).to(dev))
        B.frame[s][0].copy_(torch.from_numpy(sp.frame1))
        B.frame[s][1].copy_(torch.from_numpy(sp.frame0))
        B.set_boxes(s, torch.from_numpy(sp.boxes))
    B.pack()
    m, k, n = 4096, 1024, 1024
    n_gemm = max(1, int(round(gflop * n_streams / (2.0 * m * k * n / 1e9))))
    a = torch.randn(m, k, dtype=torch.bfloat16, device=dev)
    w = [torch.randn(k, n, dtype=torch.bfloat16, device=dev) for _ in range(4)]
    out = torch.empty(m, n, dtype=torch.bfloat16, device=dev)
    det = torch.cuda.Stream(device=dev)
    trk = torch.cuda.current_stream(dev)

    def detect():
        with torch.cuda.stream(det):
            for i in range(n_gemm):
                torch.matmul(a, w[i % 4], out=out)

    def timed(fn, steps):
        ms = []
        for _ in range(steps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(trk)
            det.wait_stream(trk)
            fn()
            trk.wait_stream(det)
            e1.record(trk)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return float(np.median(ms))

    res = {}
    for label, ctas in (("default", 0), ("lk_2_ctas_per_sm", 2)):
        B.caps.lk_ctas_per_sm = ctas
        B.capture()
        for _ in range(3):
            B.step()
            detect()
        track_ms = timed(B.step, args.steps)
        det_ms = timed(detect, args.steps)
        both_ms = timed(lambda: (detect(), B.step()), args.steps)
        res[label] = {"track_ms": track_ms, "detect_ms": det_ms, "both_ms": both_ms,
                      "saved_ms": track_ms + det_ms - both_ms,
                      "saved_frac_of_serial": (track_ms + det_ms - both_ms) / (track_ms + det_ms)}
    print(json.dumps({"workload": f"{n_streams} streams (bench workload) + stub detector "
                                  f"{gflop} GFLOP/frame ({n_gemm} bf16 GEMMs {m}x{k}x{n} per step)",
                      **res}))


def _median_ms(fn, steps, stream):
    """Median CUDA-event time (ms) of fn() on `stream` over `steps` runs,
    after three untimed runs."""
    import torch
    for _ in range(3):
        fn()
    ms = []
    for _ in range(steps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return float(np.median(ms))


def run_phases(args):
    """Where the batched step's time goes, on the bench workload: each phase
    of the step alone (pyramid, corners, LK, boxes), the pyramid and corner
    phases on their two streams as the step runs them, the eager step and
    the graph step.  Median CUDA-event times over the steps, launch shapes
    from the tuner.  One JSON line."""
    import torch
    from paper_1910_06017_b300 import omt
    dev = torch.device("cuda", 0)
    storage = omt.F16 if args.storage == "f16" else omt.F32
    streams = make_streams(args.streams, 0)
    caps = [cap_of(sp) for sp in streams]
    B = omt.BatchTracker([sp.size for sp in streams], params_for(omt, storage, max(caps)),
                         max_boxes=[len(sp.boxes) for sp in streams], max_corners=caps, device=dev)
    for s, sp in enumerate(streams):
        B.prime(s, torch.from_numpy(sp.frame0).to(dev))
        B.frame[s][0].copy_(torch.from_numpy(sp.frame1))
        B.frame[s][1].copy_(torch.from_numpy(sp.frame0))
        B.set_boxes(s, torch.from_numpy(sp.boxes))
    B.pack()
    for _ in range(args.warmup):
        B.step()
    if args.tune:
        B.autotune()
    torch.cuda.synchronize()
    main = torch.cuda.current_stream(dev)
    # the phases of the step that was just run (its table, frames and corners)
    dt = B.dev_tables[1 - B.cur]

    def phase(p):
        return lambda: omt.batch_phase(dt, B.caps, B.params, p, main)

    def side_by_side():
        B.side.wait_stream(main)
        omt.batch_phase(dt, B.caps, B.params, omt.PHASE_PYRAMID, main)
        omt.batch_phase(dt, B.caps, B.params, omt.PHASE_CORNERS, B.side)
        main.wait_stream(B.side)

    res = {name: _median_ms(fn, args.steps, main) for name, fn in (
        ("pyramid_ms", phase(omt.PHASE_PYRAMID)), ("corners_ms", phase(omt.PHASE_CORNERS)),
        ("pyramid_beside_corners_ms", side_by_side), ("lk_ms", phase(omt.PHASE_LK)),
        ("boxes_ms", phase(omt.PHASE_BOXES)))}
    res["eager_step_ms"] = _median_ms(B.step, args.steps, main)
    B.capture()
    res["graph_step_ms"] = _median_ms(B.step, args.steps, main)
    print(json.dumps({"workload": f"{args.streams} streams (bench workload), {args.storage} storage",
                      "caps": {"pyramid_ctas_per_sm": B.caps.pyr_ctas_per_sm,
                               "list_ctas_per_sm": B.caps.corner_ctas_per_sm,
                               "select_ctas_per_sm": B.caps.select_ctas_per_sm,
                               "lk_warps": B.caps.lk_warps, "lk_chunk": B.caps.lk_chunk},
                      **res}))


def run_lk_4k(args):
    """The batched LK phase at 31x31 and 5 levels on four streams of the
    3840x2160 large-motion pair (workload 4's frames, boxes and corner
    cap), F16 and F32 storage, for each of the tuner's LK launch shapes:
    median CUDA-event time over the steps.  One JSON line."""
    import torch
    from paper_1910_06017_b300 import omt, synth
    dev = torch.device("cuda", 0)
    pr = synth.rigid_pair()
    H, W = pr.frame0.shape
    ns = 4
    boxes = torch.from_numpy(np.ascontiguousarray(pr.boxes, np.float32))
    out = {"workload": f"{ns} streams of the 3840x2160 pair, {len(pr.boxes)} boxes, <= 250 corners "
                       "per box, 5 levels, 31x31"}
    for storage, name in ((omt.F16, "f16"), (omt.F32, "f32")):
        prm = omt.default_params(levels=5, win=31, max_corners=250, storage=storage)
        B = omt.BatchTracker([(W, H)] * ns, prm, max_boxes=len(pr.boxes), max_corners=[250] * ns,
                             device=dev)
        for s in range(ns):
            B.prime(s, torch.from_numpy(pr.frame0).to(dev))
            B.frame[s][0].copy_(torch.from_numpy(pr.frame1))
            B.frame[s][1].copy_(torch.from_numpy(pr.frame0))
            B.set_boxes(s, boxes)
        B.pack()
        B.step()
        torch.cuda.synchronize()
        main = torch.cuda.current_stream(dev)
        dt = B.dev_tables[1 - B.cur]
        ms = {}
        for w, c in B.TUNE_CANDIDATES:
            B.caps.lk_warps, B.caps.lk_chunk = w, c
            ms[f"{w}x{c}"] = _median_ms(
                lambda: omt.batch_phase(dt, B.caps, B.params, omt.PHASE_LK, main), args.steps, main)
        out[name] = {"points": sum(B.count(s) for s in range(ns)), "lk_ms_by_shape": ms,
                     "lk_ms": min(ms.values())}
        del B
        torch.cuda.empty_cache()
    print(json.dumps(out))


def run_working_level(args):
    """Tracking on the working level (Section V-A preprocessing: a pyramid
    level chosen by resolution is processed).  For the 3840x2160 pair with
    200 rigid regions and a 1920x1080 stream: the plain path's step time on
    level 0 and on the working level (CUDA events, mean of 20 steps, frames
    alternating) and, for the 4K pair, the median distance between each
    box's move and its region's true translation.  One JSON line."""
    import torch
    from paper_1910_06017_b300 import omt, synth
    dev = torch.device("cuda", 0)
    res = {}
    pr = synth.rigid_pair()
    sp = synth.stream_pair(0, workload=13)
    cases = [("3840x2160 rigid, 200 boxes", pr.frame0, pr.frame1, pr.boxes, pr.motions[:, :2], 250),
             ("1920x1080 stream, 64 boxes", sp.frame0, sp.frame1, sp.boxes, None, 100)]
    for name, f0, f1, boxes, truth, maxc in cases:
        h, w = f0.shape
        frames = [torch.from_numpy(f).to(dev) for f in (f0, f1)]
        b = torch.from_numpy(np.ascontiguousarray(boxes, np.float32)).to(dev)
        entry = {}
        for label, level in (("level0", 0), ("working", None)):
            params = omt.default_params(levels=4, win=21, max_corners=maxc, min_dist=3.0)
            T = omt.WorkingLevelTracker(w, h, params, len(boxes), level=level, device=dev)
            T.prime(frames[0])
            moved = (T.step(frames[1], b).cpu().numpy() - boxes)[:, :2]
            for k in range(3):
                T.step(frames[k & 1], b)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            steps = 20
            for k in range(steps):
                T.step(frames[k & 1], b)
            e1.record()
            torch.cuda.synchronize()
            entry[label] = {"level": T.level, "ms_per_step": e0.elapsed_time(e1) / steps}
            if truth is not None:
                entry[label]["median_box_error_px"] = float(np.median(np.hypot(*(moved - truth).T)))
        res[name] = entry
    print(json.dumps(res))


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or "unknown"


def oracle_legs():
    """The FP64 oracle, as it stands, on workloads 1, 2 and 4, with its LK
    on one thread and on every core it may use (OpenMP over points; the
    pyramids, corners and box update run on one thread in both): per leg the
    seconds of the whole per-frame path over the sample and the OK points
    per second of its LK step."""
    from oracle import oracle as O
    from paper_1910_06017_b300 import synth
    O.lib()
    cases = []
    p = synth.sd_pair()
    cases.append(("workload 1: 720x576 pair, 10 boxes, <= 50 corners, 3 levels, 21x21",
                  p.frame0, p.frame1, p.boxes, 50, 3, 21, None))
    clip = synth.affine_clip(n_frames=2)
    cases.append(("workload 2: 1920x1080 clip frames 0 -> 1, 16 boxes, <= 100 corners, 4 levels, "
                  "21x21", clip.frames[0], clip.frames[1], clip.gt_boxes[0], 100, 4, 21, None))
    pr = synth.rigid_pair()
    cases.append(("workload 4: 3840x2160 pair, 200 boxes, <= 250 corners, 5 levels, 31x31; LK on "
                  "a seeded 2,000-corner sample", pr.frame0, pr.frame1, pr.boxes, 250, 5, 31, 2000))
    legs = []
    for name, f0, f1, boxes, cap, levels, win, sample in cases:
        for threads in (1, 0):
            t0 = time.perf_counter()
            P0, P1 = O.Pyramid(f0, levels), O.Pyramid(f1, levels)
            pts, cnt = O.select_corners(f0, boxes, cap)
            allp = np.concatenate([pts[i, :cnt[i]] for i in range(len(cnt))])
            off = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int32)
            ub = boxes
            if sample:
                rng = np.random.default_rng(20191006 + 4)
                allp = allp[np.sort(rng.choice(len(allp), min(sample, len(allp)), replace=False))]
                off = np.array([0, len(allp)], np.int32)
                ub = np.array([[0, 0, f0.shape[1], f0.shape[0]]], np.float32)
            t1 = time.perf_counter()
            out, st = O.lk_track(P0, P1, allp, win=win, nthreads=threads)
            t2 = time.perf_counter()
            O.update_boxes(ub, off, allp, out.astype(np.float32), st)
            t3 = time.perf_counter()
            ok = int(((st & 1) > 0).sum())
            legs.append({"workload": name, "threads": threads or O.max_threads(),
                         "path_s": round(t3 - t0, 3), "lk_s": round(t2 - t1, 3), "ok_points": ok,
                         "lk_points_per_s": ok / (t2 - t1)})
    return legs


def cpu_baseline_sample():
    class A:
        steps, warmup = 1, 0
    cb = run_reference(A, 1, 0)["cpu_baseline"]
    cb["cpu_model"] = cpu_model()
    cb["affinity_cores"] = len(os.sched_getaffinity(0))
    cb["legs"] = oracle_legs()
    return cb


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="omt", choices=["omt", "reference"])
    ap.add_argument("--storage", default="f16", choices=["f32", "f16"])
    ap.add_argument("--streams", type=int, default=32)
    ap.add_argument("--no-graph", dest="graph", action="store_false")
    ap.add_argument("--no-tune", dest="tune", action="store_false",
                    help="keep the default LK launch shape instead of autotuning it")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serve", dest="serve", action="store_false",
                    help="skip the serving-loop capacity search (served)")
    ap.add_argument("--serve-s", type=float, default=2.0,
                    help="seconds of arrivals per probe of the capacity search")
    ap.add_argument("--match", action="store_true", help="time the matching phase (IoU + assignment)")
    ap.add_argument("--overlap", action="store_true",
                    help="tracking and a stub detector on two CUDA streams (Section V-B)")
    ap.add_argument("--working-level", action="store_true",
                    help="tracking on the working level chosen by resolution")
    ap.add_argument("--flow", action="store_true",
                    help="the dense flow engine (TV-L1) on 1920x1080 frames instead of the tracker")
    ap.add_argument("--fb", type=float, default=None, metavar="MAX",
                    help="forward-backward check in every step, threshold MAX px (default off)")
    ap.add_argument("--phases", action="store_true",
                    help="each phase of the batched step alone and side by side")
    ap.add_argument("--lk-4k", action="store_true",
                    help="the batched LK at 31x31 on four streams of the 4K pair")
    args = ap.parse_args()
    ws, rank, local = dist_env()
    if args.impl == "omt":
        args.warmup = max(args.warmup, 3)
    for flag, fn in (("match", run_match), ("overlap", run_overlap),
                     ("working_level", run_working_level), ("phases", run_phases),
                     ("lk_4k", run_lk_4k)):
        if getattr(args, flag):
            if rank == 0:
                fn(args)
            return
    if args.flow:
        if rank != 0:
            return
        if args.impl == "reference":
            a = argparse.Namespace(steps=max(1, args.steps // 10), warmup=0)
            cb = run_flow_reference(a)
            print(json.dumps({"impl": "reference", "metric": FLOW_METRIC, "value": cb["value"],
                              "unit": "frames/s", "n_gpus": ws, "steps": a.steps, "warmup": 0,
                              "ms_per_step": 1e3 / cb["value"], "higher_is_better": True,
                              "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                              "data": "synthetic", "config": {"workload": FLOW_WORKLOAD,
                                                              "path": "FP64 CPU oracle"},
                              "cpu_baseline": cb, "e2e": {"value": cb["value"], "unit": "frames/s",
                                                          "h2d_bytes_per_step": 0,
                                                          "d2h_bytes_per_step": 0}}))
            return
        res = run_flow(args)
        if not args.no_cpu_baseline:
            res["cpu_baseline"] = run_flow_reference(argparse.Namespace(steps=1, warmup=0))
        print(json.dumps(res))
        return
    if args.impl == "reference":
        # the oracle runs on rank 0 only; other ranks have no work
        if rank == 0:
            print(json.dumps(run_reference(args, ws, rank)))
        return
    if ws > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    res = run_omt(args, ws, rank, local)
    if rank == 0:
        if not args.no_cpu_baseline:
            res["cpu_baseline"] = cpu_baseline_sample()
        print(json.dumps(res))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
