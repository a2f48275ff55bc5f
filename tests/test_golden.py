"""The oracle reproduces its committed golden fixture bit for bit.

The fixture (tests/golden/sd_crop_64x48.json) was written by
tests/golden/make_golden.py from the oracle alone; this guards the oracle
against accidental change.  The GPU parity tests reuse the same fixture.
"""
import json
import os

import numpy as np

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "sd_crop_64x48.json")


def load_golden():
    with open(GOLD) as f:
        g = json.load(f)
    w, h = g["w"], g["h"]
    g["frame0"] = np.array(g["frame0"], np.uint8).reshape(h, w)
    g["frame1"] = np.array(g["frame1"], np.uint8).reshape(h, w)
    g["boxes"] = np.array(g["boxes"], np.float32)
    g["points"] = np.array(g["points"], np.float32)
    g["pts_out"] = np.array(g["pts_out"], np.float64)
    g["status"] = np.array(g["status"], np.uint8)
    g["iters"] = np.array(g["iters"], np.uint8)
    g["boxes_out"] = np.array(g["boxes_out"], np.float64)
    return g


def test_oracle_matches_golden(oracle):
    g = load_golden()
    p = g["params"]
    P0 = oracle.Pyramid(g["frame0"], p["levels"])
    P1 = oracle.Pyramid(g["frame1"], p["levels"])
    assert int(round(P0.img[1].sum() * 256)) == g["level1_sum_x65536"]
    pts, cnt = oracle.select_corners(g["frame0"], g["boxes"], p["max_corners"],
                                     quality=tuple(p["quality"]), min_dist=p["min_dist"])
    assert cnt.tolist() == g["counts"]
    allp = np.concatenate([pts[i, :cnt[i]] for i in range(len(cnt))])
    np.testing.assert_array_equal(allp, g["points"])
    out, st, it, me = oracle.lk_track(P0, P1, allp, win=p["win"], max_iter=p["max_iter"],
                                      eps=p["eps"], min_eig=p["min_eig"], diagnostics=True)
    np.testing.assert_array_equal(out, g["pts_out"])
    np.testing.assert_array_equal(st, g["status"])
    np.testing.assert_array_equal(it, g["iters"])
    off = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int32)
    bo, nv = oracle.update_boxes(g["boxes"], off, allp, out.astype(np.float32), st)
    np.testing.assert_array_equal(bo, g["boxes_out"])
    assert nv.tolist() == g["nvalid"]
