"""Tracking on the working level (Section V-A preprocessing: the frame is
downscaled and a pyramid level chosen by its resolution is processed).

    python -m paper_1910_06017_b300.working_level_bench

For the 3840x2160 pair with rigid regions (200 boxes, up to 40 px and 3
degrees of motion) and a 1920x1080 stream of the bench workload: the step
time of the plain path on level 0 and on the working level (CUDA events,
mean of 20 steps, frames alternating), and the median distance between
each box's move and its region's true translation (the 4K pair; regions
that later regions overlap are included).  One JSON line."""
import json

import numpy as np


def main():
    import torch
    from . import omt, synth
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


if __name__ == "__main__":
    main()
