"""Writes the golden fixtures of this folder from the oracle alone.

Run from the repository root:  python tests/golden/make_golden.py
Every value stored here comes from oracle/ on inputs drawn by the seeded
generator; nothing comes from the CUDA path.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O  # noqa: E402
from paper_1910_06017_b300 import synth  # noqa: E402


def sd_crop_case():
    """A 64x48 crop of the 720x576 shifted pair (shift 1.37, -0.62)."""
    p = synth.sd_pair()
    f0 = np.ascontiguousarray(p.frame0[300:348, 200:264])
    f1 = np.ascontiguousarray(p.frame1[300:348, 200:264])
    boxes = np.array([[4.0, 3.0, 40.5, 30.0], [20.25, 10.0, 60.0, 45.0]], np.float32)
    levels, win, iters, eps, tau = 2, 9, 30, 0.01, 1e-3
    P0, P1 = O.Pyramid(f0, levels), O.Pyramid(f1, levels)
    pts, cnt = O.select_corners(f0, boxes, 12, quality=(1, 100), min_dist=5.0)
    allp = np.concatenate([pts[i, :cnt[i]] for i in range(len(boxes))])
    out, st, it, me = O.lk_track(P0, P1, allp, win=win, max_iter=iters, eps=eps, min_eig=tau,
                                 diagnostics=True)
    off = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int32)
    bo, nv = O.update_boxes(boxes, off, allp, out.astype(np.float32), st)
    return {
        "cite": ("Section V-A: Gaussian pyramid (binomial 5-tap, reflect-101), "
                 "Shi-Tomasi corners (exact integer response, per-box max, 1/100 "
                 "quality, 3x3 NMS, (R desc, raster asc), min distance 5), "
                 "Bouguet pyramidal Lucas-Kanade, per-box median update"),
        "source": "oracle/omt_oracle.c via tests/golden/make_golden.py",
        "w": 64, "h": 48,
        "frame0": f0.flatten().tolist(), "frame1": f1.flatten().tolist(),
        "boxes": boxes.tolist(),
        "params": {"levels": levels, "win": win, "max_iter": iters, "eps": eps,
                   "min_eig": tau, "max_corners": 12, "quality": [1, 100], "min_dist": 5.0},
        "level1_sum_x65536": int(round(P0.img[1].sum() * 256)),
        "counts": cnt.tolist(),
        "points": allp.tolist(),
        "pts_out": [[float(repr_x) for repr_x in r] for r in out.tolist()],
        "status": st.tolist(),
        "iters": it.tolist(),
        "boxes_out": bo.tolist(),
        "nvalid": nv.tolist(),
    }


def main():
    case = sd_crop_case()
    with open(os.path.join(HERE, "sd_crop_64x48.json"), "w") as f:
        json.dump(case, f, indent=None, separators=(",", ":"))
        f.write("\n")


if __name__ == "__main__":
    main()
