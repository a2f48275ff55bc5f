"""The library's assignment and update (host code of libomt) against the
oracle: the same maximal total IoU (the assignment itself may differ only
among equally good ones), valid partial injections, inactive rows left
out, the same update; and host-side argument checks."""
import ctypes

import numpy as np
import pytest

from paper_1910_06017_b300 import omt


def _valid(iou, ma, mb, active, iou_min):
    for i, j in enumerate(ma):
        if j >= 0:
            assert mb[j] == i and iou[i, j] > iou_min
            assert active is None or active[i]
    for j, i in enumerate(mb):
        if i >= 0:
            assert ma[i] == j


@pytest.mark.parametrize("na,nb", [(0, 0), (0, 5), (4, 0), (1, 1), (7, 7), (30, 12), (12, 30),
                                   (150, 150), (300, 220)])
def test_assignment_matches_oracle_total(oracle, na, nb):
    rng = np.random.default_rng(20191006 + 7 * na + nb)
    for trial in range(4):
        # box-like IoU structure: sparse, with ties and exact zeros
        iou = rng.uniform(0, 1, (na, nb)) * (rng.uniform(0, 1, (na, nb)) < 0.15)
        if trial == 1:
            iou = np.round(iou, 1)                      # many ties
        active = (rng.uniform(0, 1, na) < 0.9).astype(np.uint8) if trial >= 2 else None
        iou_min = 0.3 if trial == 3 else 0.0
        ma, mb = omt.assign(iou, active, iou_min)
        oa, ob = oracle.assign(iou, active, iou_min)
        _valid(iou, ma, mb, active, iou_min)
        if iou_min == 0.0:
            tot = sum(iou[i, j] for i, j in enumerate(ma) if j >= 0)
            otot = sum(iou[i, j] for i, j in enumerate(oa) if j >= 0)
            assert abs(tot - otot) <= 1e-9 * max(1.0, otot)
        if trial == 0:
            # no ties: the optimum is unique
            np.testing.assert_array_equal(ma, oa)
            np.testing.assert_array_equal(mb, ob)


def test_update_matches_oracle(oracle):
    rng = np.random.default_rng(7)
    S = rng.uniform(0, 500, (40, 4)).astype(np.float32)
    D = rng.uniform(0, 500, (25, 4)).astype(np.float32)
    active = (rng.uniform(0, 1, 40) < 0.8).astype(np.uint8)
    iou = oracle.iou_matrix(S, D)
    ms, md = oracle.assign(iou, active)
    b1, a1 = omt.update_tracks(S, active, D, ms, md)
    b2, a2 = oracle.update_tracks(S, active, D, ms, md)
    np.testing.assert_array_equal(b1, b2)
    np.testing.assert_array_equal(a1, a2)


def test_assign_argument_checks():
    lib = omt.lib()
    iou = np.zeros((3, 3))
    ma, mb = np.zeros(3, np.int32), np.zeros(3, np.int32)
    need = lib.omt_assign_workspace_bytes(3, 3)
    ws = np.zeros(need, np.uint8)
    p = lambda a: ctypes.c_void_p(a.ctypes.data)
    assert lib.omt_assign(p(iou), 3, 3, None, 0.0, p(ws), need - 1, p(ma), p(mb)) == omt.ENOMEM
    assert lib.omt_assign(p(iou), -1, 3, None, 0.0, p(ws), need, p(ma), p(mb)) == omt.EINVAL
    assert lib.omt_assign(p(iou), 3, 3, None, float("nan"), p(ws), need, p(ma), p(mb)) == omt.EINVAL
    assert lib.omt_assign(p(iou), 3, 3, None, 0.0, p(ws), need, p(ma), p(mb)) == omt.OK
    assert lib.omt_iou_matrix(None, 2, None, 2, None, None) == omt.EINVAL
    assert lib.omt_iou_matrix(None, 0, None, 0, None, None) == omt.OK
    # misaligned device box pointer (never dereferenced: rejected first)
    assert lib.omt_iou_matrix(ctypes.c_void_p(1 << 20 | 4), 2, ctypes.c_void_p(1 << 20), 2,
                              ctypes.c_void_p(1 << 21), None) == omt.EINVAL
