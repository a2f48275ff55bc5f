"""Benchmark of the box-tracking hot path on the batched multi-stream workload.

Workload (one step): 32 independent video streams, resolutions drawn from
{720x576, 1280x720, 1920x1080}, each with a target of 2,000-20,000 points
(log-uniform) as Shi-Tomasi corners over an 8x8 grid of boxes, and a smooth
displacement field of at most 12 px between its two frames.  A step runs the
whole hot path for every stream: the pyramid of the new frame, the corners of
frame t inside the boxes, pyramidal LK (4 levels, 21x21 window, 30
iterations, eps 0.01) and the per-box median update.  Frames alternate
between each stream's two renders, so every step tracks a real pair.

Metric: LK tracked points/s (OK points only) over the whole job.  `value` is
measured with every input resident on the device; `e2e` moves each step's
frames host -> device from pinned memory and reads the boxes back.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl omt|reference]
                    [--storage f32|f16] [--streams S]
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

WORKLOAD = "32 streams {720x576,1280x720,1920x1080}, 2k-20k points/stream, |d|<=12 px, 4 levels, 21x21"
METRIC = "LK tracked points/s"
LEVELS, WIN, MAX_ITER, EPS = 4, 21, 30, 0.01
GRID = (8, 8)
FALLBACK_PEAKS = {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}
SMS, FP32_LANES = 148, 128


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return dict(FALLBACK_PEAKS), "fallback"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_bench_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
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
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


def make_streams(n_streams: int, rank: int):
    from paper_1910_06017_b300 import synth
    out = []
    for s in range(n_streams):
        sp = synth.stream_pair(rank * n_streams + s)
        out.append(sp)
    return out


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
    n_iter = it.sum()
    reached = np.zeros(len(it), np.int64)
    nz = it > 0
    # levels are stored [L0..Lm]; the walk goes from Lm down
    for i in range(levels):
        L = levels - 1 - i
        reached += np.where(np.any(nz[:, :L + 1], axis=1), 1, 0)
    lost_eig = (status & 2) > 0
    reached += lost_eig.astype(np.int64)
    return float(27 * N * reached.sum() + 12 * N * n_iter)


def run_omt(args, ws, rank, local):
    import torch
    from paper_1910_06017_b300 import omt

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    storage = omt.F16 if args.storage == "f16" else omt.F32
    streams = make_streams(args.streams, rank)
    trackers, frames_d, boxes_d, frames_h = [], [], [], []
    for sp in streams:
        w, h = sp.size
        cap = int(math.ceil(sp.n_target / (GRID[0] * GRID[1])))
        prm = omt.default_params(levels=LEVELS, win=WIN, max_iter=MAX_ITER, eps=EPS,
                                 max_corners=min(cap, omt.MAX_CORNERS), storage=storage,
                                 min_dist=3.0)
        T = omt.StreamTracker(w, h, prm, max_boxes=len(sp.boxes), device=dev)
        f0 = torch.from_numpy(sp.frame0).to(dev)
        f1 = torch.from_numpy(sp.frame1).to(dev)
        T.prime(f0)
        trackers.append(T)
        frames_d.append((f0, f1))
        boxes_d.append(torch.from_numpy(sp.boxes).to(dev))
        frames_h.append((torch.from_numpy(sp.frame0).pin_memory(), torch.from_numpy(sp.frame1).pin_memory()))
    stream = torch.cuda.current_stream()

    def step(k, lk_events=None):
        for s, T in enumerate(trackers):
            fn = frames_d[s][(k + 1) % 2]
            T.step(fn, boxes_d[s])

    # warm-up (also primes each tracker so step k tracks frame k%2 -> (k+1)%2)
    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()

    # the LK share of the step: events around each LK launch, measured in a
    # separate pass over the same steps (same launches, same stream)
    def timed_steps(k0, K, lk_time=False):
        ev = []
        for k in range(k0, k0 + K):
            for s, T in enumerate(trackers):
                fn = frames_d[s][(k + 1) % 2]
                if not lk_time:
                    T.step(fn, boxes_d[s])
                else:
                    _step_with_lk_events(omt, T, fn, boxes_d[s], ev)
        return ev

    clocks = Clocks(local)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    timed_steps(args.warmup, args.steps)
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    clk = clocks.stop()
    # points tracked in the last step, per stream (identical every step pair)
    ok_pts, n_pts, flops = 0, 0, 0.0
    for T, sp in zip(trackers, streams):
        nb = len(sp.boxes)
        n = int(T.offsets[nb].item())
        st = T.status[:n].cpu().numpy()
        it = T.iters[:n].cpu().numpy()
        ok_pts += int(((st & 1) > 0).sum())
        n_pts += n
        flops += lk_flops(it, st, LEVELS, WIN)
    # LK kernel timing pass
    ev = timed_steps(args.warmup + args.steps, args.steps, lk_time=True)
    torch.cuda.synchronize()
    lk_ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps

    # end to end: pinned host frames -> device each step, boxes back each step
    torch.cuda.synchronize()
    te = time.perf_counter()
    h2d = d2h = 0
    outs_h = [torch.empty((len(sp.boxes), 4), dtype=torch.float32).pin_memory() for sp in streams]
    for k in range(args.steps):
        for s, T in enumerate(trackers):
            fh = frames_h[s][(k + 1) % 2]
            fd = frames_d[s][(k + 1) % 2]
            fd.copy_(fh, non_blocking=True)
            h2d += fh.numel()
            bo = T.step(fd, boxes_d[s])
            outs_h[s].copy_(bo, non_blocking=True)
            d2h += bo.numel() * 4
        torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - te) / args.steps

    ms_step = ms / args.steps
    if ws > 1:
        import torch.distributed as dist
        t = torch.tensor([ms_step, e2e_s], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_step, e2e_s = float(t[0]), float(t[1])
        c = torch.tensor([ok_pts], dtype=torch.float64, device=dev)
        dist.all_reduce(c)
        ok_total = float(c[0])
    else:
        ok_total = float(ok_pts)
    value = ok_total / (ms_step * 1e-3)
    pk, pk_src = peaks()
    sm_mhz = pk.get("sm_max_mhz", 2032.0)
    fp32_peak = SMS * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12
    achieved = flops / (lk_ms * 1e-3) / 1e12
    launches_per_stream = LEVELS + 3 + 1 + 1
    res = {
        "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "path": "plain per-stream", "storage": args.storage,
                   "streams_per_gpu": args.streams, "points_per_step": n_pts,
                   "ok_points_per_step": ok_pts, "l2": "working set > L2 (126 MB): no flush",
                   "parallelism": f"replicas x{ws}"},
        "e2e": {"value": ok_total / e2e_s, "unit": "points/s", "h2d_bytes_per_step": h2d // args.steps,
                "d2h_bytes_per_step": d2h // args.steps},
        "roofline": {"kernel": "lk_kernel", "bound": "alu", "achieved": achieved,
                     "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                     "traffic": None,
                     "peak_source": f"148 SMs x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz ({pk_src} clock)",
                     "lk_ms_per_step": lk_ms, "lk_share": lk_ms / ms_step},
        "clocks": clk,
        "gpu_launches": launches_per_stream * args.streams * args.steps,
    }
    return res


def _step_with_lk_events(omt, T, frame_next, boxes, ev):
    import torch
    nb = boxes.shape[0]
    prev, nxt = T.pyr[T.cur], T.pyr[1 - T.cur]
    omt.build_pyramid(frame_next, nxt, T.params)
    omt.select_corners(prev, boxes, T.params, T.scratch, T.pts, T.offsets)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    omt.lk_track(prev, nxt, T.pts, T.params, T.pts_out, T.status, T.iters,
                 n_max=nb * T.params.max_corners, n_dev=T.offsets[nb:nb + 1])
    b.record()
    ev.append((a, b))
    omt.update_boxes(boxes, T.offsets, T.pts, T.pts_out, T.status, T.params, T.boxes_out[:nb],
                     T.nvalid[:nb])
    T.cur = 1 - T.cur


def run_reference(args, ws, rank):
    """The FP64 oracle on the host cores, on a bounded sample of the same
    workload: per step, one stream's pyramid pair, corners and LK."""
    from oracle import oracle as O
    streams = make_streams(1, rank)
    sp = streams[0]
    cap = int(math.ceil(sp.n_target / (GRID[0] * GRID[1])))
    O.lib()
    cores = O.max_threads()
    times, okc = [], 0
    for k in range(args.warmup + args.steps):
        t = time.perf_counter()
        P0 = O.Pyramid(sp.frame0, LEVELS)
        P1 = O.Pyramid(sp.frame1, LEVELS)
        pts, cnt = O.select_corners(sp.frame0, sp.boxes, cap, min_dist=3.0)
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
    sample = f"1 of 32 streams per step ({sp.size[0]}x{sp.size[1]}, {okc} OK points)"
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "path": "FP64 CPU oracle"},
        "cpu_baseline": {"value": value, "unit": "points/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def cpu_baseline_sample():
    """The oracle timed on this host on a bounded sample (one 720x576-1080p
    stream pair of the workload), for the cpu_baseline field."""
    class A:
        steps, warmup = 1, 0
    r = run_reference(A, 1, 0)
    return r["cpu_baseline"]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="omt", choices=["omt", "reference"])
    ap.add_argument("--storage", default="f32", choices=["f32", "f16"])
    ap.add_argument("--streams", type=int, default=32)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    ws, rank, local = dist_env()
    if args.warmup < 3 and args.impl == "omt":
        args.warmup = 3
    if ws > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, ws, rank)))
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
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
