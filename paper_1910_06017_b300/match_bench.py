"""Timing of the matching phase (Section V-A) at serving sizes.

    python -m paper_1910_06017_b300.match_bench

For n predicted boxes against n detections (boxes of a 1920x1080 frame,
detections the predictions jittered, 10 % dropped and replaced): the device
IoU matrix (CUDA events), its copy to page-locked host memory, the host assignment and the update
(wall clock), one JSON line per size."""
import json
import time

import numpy as np


def main():
    import torch
    from . import omt
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


if __name__ == "__main__":
    main()
