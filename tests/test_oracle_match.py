"""Pins of the oracle's matching and update phases (Section V-A): IoU by
hand-computed cases, the assignment against brute force over all
assignments of tiny matrices, and the update by hand."""
import itertools

import numpy as np
import pytest


def test_iou_hand_cases(oracle):
    a = np.array([[0, 0, 10, 10], [0, 0, 10, 10], [0, 0, 10, 10], [2, 2, 4, 4], [0, 0, 0, 5]], np.float32)
    b = np.array([[0, 0, 10, 10], [5, 0, 15, 10], [20, 20, 30, 30], [0, 0, 10, 10], [0, 0, 10, 10]],
                 np.float32)
    m = oracle.iou_matrix(a, b)
    assert m[0, 0] == 1.0                       # identical
    assert m[1, 1] == 50.0 / 150.0              # half overlap: 50 / (100 + 100 - 50)
    assert m[2, 2] == 0.0                       # disjoint
    assert m[3, 3] == 4.0 / 100.0               # contained: area ratio
    assert m[4, 4] == 0.0                       # zero-area box
    # symmetric
    np.testing.assert_array_equal(oracle.iou_matrix(b, a), m.T)


def _brute(iou, active=None, iou_min=0.0):
    na, nb = iou.shape
    best = -1.0
    rows = [i for i in range(na) if active is None or active[i]]
    # every injective map of a subset of active rows to columns: pad with "none"
    cols = list(range(nb)) + [None] * len(rows)
    for perm in itertools.permutations(cols, len(rows)):
        tot = sum(iou[r, c] for r, c in zip(rows, perm) if c is not None and iou[r, c] > iou_min)
        best = max(best, tot)
    return best


@pytest.mark.parametrize("na,nb", [(1, 1), (3, 3), (4, 2), (2, 5), (5, 5), (6, 4)])
def test_assignment_is_optimal_against_brute_force(oracle, na, nb):
    rng = np.random.default_rng(20191006 + 31 * na + nb)
    for trial in range(12):
        iou = rng.uniform(0, 1, (na, nb)) * (rng.uniform(0, 1, (na, nb)) < 0.7)
        active = (rng.uniform(0, 1, na) < 0.8).astype(np.uint8) if trial % 2 else None
        ma, mb = oracle.assign(iou, active)
        # valid: a partial injection consistent in both directions, inactive rows unmatched
        for i, j in enumerate(ma):
            if j >= 0:
                assert mb[j] == i and iou[i, j] > 0.0
                assert active is None or active[i]
        for j, i in enumerate(mb):
            if i >= 0:
                assert ma[i] == j
        tot = sum(iou[i, j] for i, j in enumerate(ma) if j >= 0)
        assert abs(tot - _brute(iou, active)) <= 1e-12


def test_assignment_threshold_and_identity(oracle):
    iou = np.diag([0.9, 0.5, 0.2])
    ma, mb = oracle.assign(iou, iou_min=0.3)
    assert ma.tolist() == [0, 1, -1] and mb.tolist() == [0, 1, -1]
    # a global optimum can beat the greedy choice: greedy takes 0.9 and then 0.1
    iou = np.array([[0.9, 0.8], [0.8, 0.1]])
    ma, _ = oracle.assign(iou)
    assert ma.tolist() == [1, 0]


def test_update_by_hand(oracle):
    S = np.array([[0, 0, 10, 10], [20, 20, 30, 30], [50, 50, 60, 60]], np.float32)
    active = np.array([1, 1, 0], np.uint8)        # the third was lost earlier
    D = np.array([[21, 21, 31, 31], [100, 100, 110, 110]], np.float32)
    ma = np.array([-1, 0, -1], np.int32)
    md = np.array([1, -1], np.int32)
    boxes, act = oracle.update_tracks(S, active, D, ma, md)
    np.testing.assert_array_equal(boxes, [[0, 0, 10, 10], [21, 21, 31, 31], [50, 50, 60, 60],
                                          [100, 100, 110, 110]])
    assert act.tolist() == [0, 1, 0, 1]
