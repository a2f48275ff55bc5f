"""Pins of the oracle's box update (Section V-A prediction).

Median (default) and mean aggregation of OK-point displacements, checked on
hand vectors, against numpy.median / numpy.mean, and end to end on a global
translation.
"""
import numpy as np
import pytest

from paper_1910_06017_b300 import synth

OK, LOST_EIG, LOST_OOB, NONCONV = 1, 2, 4, 8


def _run(oracle, dxs, sts, agg=0, box=(10.0, 20.0, 50.0, 70.0)):
    n = len(dxs)
    pts = np.zeros((n, 2), np.float32) + 100.0
    out = pts + np.asarray(dxs, np.float32).reshape(n, 2)
    bo, nv = oracle.update_boxes(np.array([box], np.float32), np.array([0, n], np.int32), pts, out,
                                 np.asarray(sts, np.uint8), aggregator=agg)
    return bo[0] - np.array(box), nv[0]


def test_median_odd(oracle):
    d, n = _run(oracle, [(3, 5), (-1, 0), (2, -7)], [OK, OK, OK])
    assert n == 3 and np.allclose(d, [2, 0, 2, 0])


def test_median_even_is_mean_of_middle(oracle):
    d, n = _run(oracle, [(1, 0), (4, 1), (2, 2), (10, 3)], [OK] * 4)
    assert n == 4 and np.allclose(d, [3, 1.5, 3, 1.5])


def test_lost_points_are_ignored(oracle):
    d, n = _run(oracle, [(1, 1), (100, 100), (3, 3), (-50, 7)],
                [OK, LOST_EIG, OK | NONCONV, LOST_OOB])
    assert n == 2 and np.allclose(d, [2, 2, 2, 2])


def test_all_lost_leaves_box(oracle):
    d, n = _run(oracle, [(1, 1), (2, 2)], [LOST_EIG, LOST_OOB])
    assert n == 0 and np.all(d == 0)
    bo, nv = oracle.update_boxes(np.array([[1, 2, 3, 4]], np.float32), np.array([0, 0], np.int32),
                                 np.zeros((0, 2), np.float32), np.zeros((0, 2), np.float32),
                                 np.zeros(0, np.uint8))
    assert nv[0] == 0 and np.all(bo[0] == [1, 2, 3, 4])


@pytest.mark.parametrize("agg", [0, 1])
def test_against_numpy(oracle, agg):
    rng = np.random.default_rng(5)
    nb = 40
    counts = rng.integers(0, 30, nb)
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    n = int(off[-1])
    pts = rng.uniform(0, 700, (n, 2)).astype(np.float32)
    out = (pts + rng.normal(0, 3, (n, 2))).astype(np.float32)
    st = rng.choice([OK, OK | NONCONV, LOST_EIG, LOST_OOB], n, p=[0.6, 0.1, 0.15, 0.15]).astype(np.uint8)
    boxes = rng.uniform(0, 500, (nb, 4)).astype(np.float32)
    bo, nv = oracle.update_boxes(boxes, off, pts, out, st, aggregator=agg)
    for b in range(nb):
        sel = slice(off[b], off[b + 1])
        ok = (st[sel] & OK) > 0
        d = out[sel][ok].astype(np.float64) - pts[sel][ok].astype(np.float64)
        assert nv[b] == ok.sum()
        if ok.sum() == 0:
            m = np.zeros(2)
        else:
            m = np.median(d, 0) if agg == 0 else np.mean(d, 0)
        np.testing.assert_allclose(bo[b], boxes[b].astype(np.float64) + np.concatenate([m, m]),
                                   rtol=0, atol=1e-9)


def test_global_translation_moves_every_box(oracle):
    p = synth.sd_pair()
    P0, P1 = oracle.Pyramid(p.frame0, 3), oracle.Pyramid(p.frame1, 3)
    pts, cnt = oracle.select_corners(p.frame0, p.boxes, 50)
    allp = np.concatenate([pts[i, :cnt[i]] for i in range(len(cnt))])
    out, st = oracle.lk_track(P0, P1, allp)
    off = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int32)
    bo, nv = oracle.update_boxes(p.boxes, off, allp, out.astype(np.float32), st)
    d = bo - p.boxes.astype(np.float64)
    assert np.all(nv == cnt)
    assert np.abs(d - [1.37, -0.62, 1.37, -0.62]).max() <= 0.02
