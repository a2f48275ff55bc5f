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

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl omt|reference]
                    [--storage f16|f32] [--streams S] [--no-graph] [--no-tune]
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
        self.dev = device_index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_bench_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
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
    sm_mhz = pk.get("sm_max_mhz", 2032.0)
    fp32_peak = SMS * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12
    achieved = flops / (lk_ms * 1e-3) / 1e12
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
                          "candidates_ms": {f"{w}x{c}": round(t, 4) for (w, c), t in tune_ms.items()}}},
        "e2e": {"value": ok_total / e2e_s, "unit": "points/s",
                "h2d_bytes_per_step": h2d // args.steps, "d2h_bytes_per_step": d2h // args.steps},
        "roofline": {"kernel": "lk_batch_kernel", "bound": "alu", "achieved": achieved,
                     "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                     # DRAM bytes of one launch on this workload (ncu capture of the
                     # same kernel source; see profiles/traffic.json)
                     "traffic": lk_tr["bytes_per_launch"] if lk_tr else None,
                     "peak_source": f"148 SMs x 128 FP32 lanes x 2 flop x {sm_mhz:.0f} MHz ({pk_src} max clock)",
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


def cpu_baseline_sample():
    class A:
        steps, warmup = 1, 0
    return run_reference(A, 1, 0)["cpu_baseline"]


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
    ap.add_argument("--flow", action="store_true",
                    help="the dense flow engine (TV-L1) on 1920x1080 frames instead of the tracker")
    ap.add_argument("--fb", type=float, default=None, metavar="MAX",
                    help="forward-backward check in every step, threshold MAX px (default off)")
    args = ap.parse_args()
    ws, rank, local = dist_env()
    if args.impl == "omt":
        args.warmup = max(args.warmup, 3)
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
