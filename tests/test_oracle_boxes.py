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


# ------------------------------------------------ median-flow scale (agg 2)

def _scale_box(oracle, pts, out, sts, box):
    n = len(pts)
    bo, nv = oracle.update_boxes(np.array([box], np.float32), np.array([0, n], np.int32),
                                 np.asarray(pts, np.float32), np.asarray(out, np.float32),
                                 np.asarray(sts, np.uint8), aggregator=2)
    return bo[0], nv[0]


def test_scale_hand_vectors(oracle):
    # pair distances |u|: 1, 2, sqrt(5); |v|: 2, 2, sqrt(8) -> ratios 2, 1,
    # sqrt(8/5); median sqrt(1.6).  Displacements (0,0), (1,0), (0,0): median 0.
    u = [(10, 10), (11, 10), (10, 12)]
    v = [(10, 10), (12, 10), (10, 12)]
    box = (0.0, 0.0, 20.0, 10.0)
    bo, n = _scale_box(oracle, u, v, [OK] * 3, box)
    s = np.sqrt(1.6)
    assert n == 3
    np.testing.assert_allclose(bo, [10 - 10 * s, 5 - 5 * s, 10 + 10 * s, 5 + 5 * s], rtol=0,
                               atol=1e-12)


def test_scale_of_a_pure_zoom(oracle):
    # points symmetric about the box centre, zoomed by s about it and moved by
    # t: every pair ratio is s and the median displacement is t
    rng = np.random.default_rng(11)
    c = np.array([64.0, 48.0])
    half = rng.uniform(-20, 20, (20, 2))
    u = np.concatenate([c + half, c - half])
    for s, t in ((1.25, (3.0, -2.0)), (0.8, (0.0, 0.5))):
        v = c + s * (u - c) + np.array(t)
        uf, vf = u.astype(np.float32), v.astype(np.float32)
        bo, n = _scale_box(oracle, uf, vf, [OK] * len(u), (44.0, 28.0, 84.0, 68.0))
        want = [64 + t[0] - 20 * s, 48 + t[1] - 20 * s, 64 + t[0] + 20 * s, 48 + t[1] + 20 * s]
        # float32 point storage limits the ratios to about 1e-6
        np.testing.assert_allclose(bo, want, atol=2e-4)


def test_scale_uses_the_first_64_ok_points_only(oracle):
    rng = np.random.default_rng(12)
    n = 150
    u = rng.uniform(0, 100, (n, 2))
    st = np.full(n, OK, np.uint8)
    st[rng.choice(n, 30, replace=False)] = LOST_EIG
    ok_idx = np.nonzero(st == OK)[0]
    first = ok_idx[:64]
    v = u * 3.0                      # later OK points zoom by 3, lost ones anyhow
    v[first] = u[first] * 1.5        # the first 64 OK points zoom by 1.5
    v[st != OK] = rng.uniform(-1e3, 1e3, ((st != OK).sum(), 2))
    bo, m = _scale_box(oracle, u.astype(np.float32), v.astype(np.float32), st, (0, 0, 10, 10))
    assert m == (st == OK).sum()
    w = bo[2] - bo[0]
    np.testing.assert_allclose(w, 15.0, atol=1e-4)


def test_scale_needs_two_points(oracle):
    box = (10.0, 20.0, 50.0, 70.0)
    for pts, out, sts in (([(5, 5)], [(7, 6)], [OK]), ([(5, 5), (9, 9)], [(7, 6), (0, 0)], [OK, LOST_OOB]),
                          ([(5, 5), (5, 5)], [(7, 6), (9, 6)], [OK, OK])):
        bo, _ = _scale_box(oracle, pts, out, sts, box)
        b0, _ = oracle.update_boxes(np.array([box], np.float32), np.array([0, len(pts)], np.int32),
                                    np.asarray(pts, np.float32), np.asarray(out, np.float32),
                                    np.asarray(sts, np.uint8), aggregator=0)
        np.testing.assert_allclose(bo, b0[0], atol=1e-12)   # scale 1: the plain median move
