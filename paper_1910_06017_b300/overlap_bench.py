"""Detection and tracking on one GPU at the same time (Section V-B: the
motion field and the detector run concurrently, about 20 % there).

    python -m paper_1910_06017_b300.overlap_bench [--streams 32] [--gflop-per-frame 110]

The detector is a stub (the paper's YoloV3 models and weights are out of
scope): per step, for every stream's frame, a chain of bf16 GEMMs of
4096 x 1024 x 1024 (8.6 GFLOP each) on a stream of its own, through torch
(cuBLAS), about the cost of the two detector models per frame by default.
The tracker is the batched step of the 32-stream bench workload (CUDA
graph).  Three timings, each the median over the steps of CUDA events on a
host-side clock that waits for both streams: tracking alone, detection
alone, and both issued every step on their two streams; the last also with
the LK launch held to 2 CTAs per SM, which leaves room on every SM for the
GEMMs.  One JSON line."""
import argparse
import json
import math

import numpy as np


def main():
    import torch
    from . import omt, synth

    ap = argparse.ArgumentParser()
    ap.add_argument("--streams", type=int, default=32)
    ap.add_argument("--gflop-per-frame", type=float, default=110.0)
    ap.add_argument("--steps", type=int, default=20)
    args = ap.parse_args()
    dev = torch.device("cuda", 0)
    streams = [synth.stream_pair(s) for s in range(args.streams)]
    caps = [int(math.ceil(sp.n_target / 64)) for sp in streams]   # 8 x 8 box grid
    prm = omt.default_params(levels=4, win=21, max_iter=30, eps=0.01, max_corners=max(caps),
                             storage=omt.F16, min_dist=3.0)
    B = omt.BatchTracker([sp.size for sp in streams], prm, max_boxes=[len(sp.boxes) for sp in streams],
                         max_corners=caps, device=dev)
    for s, sp in enumerate(streams):
        B.prime(s, torch.from_numpy(sp.frame0).to(dev))
        B.frame[s][0].copy_(torch.from_numpy(sp.frame1))
        B.frame[s][1].copy_(torch.from_numpy(sp.frame0))
        B.set_boxes(s, torch.from_numpy(sp.boxes))
    B.pack()

    m, k, n = 4096, 1024, 1024
    per_gemm = 2.0 * m * k * n / 1e9
    n_gemm = max(1, int(round(args.gflop_per_frame * args.streams / per_gemm)))
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
    print(json.dumps({"workload": f"{args.streams} streams (bench workload) + stub detector "
                                  f"{args.gflop_per_frame} GFLOP/frame ({n_gemm} bf16 GEMMs "
                                  f"{m}x{k}x{n} per step)", **res}))


if __name__ == "__main__":
    main()
