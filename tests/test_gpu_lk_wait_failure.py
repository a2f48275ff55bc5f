"""The LK kernels' bounded waits: a wait that runs out is reported, never
turned into a tracked point.

The test hook omt_debug_fail_lk_wait makes one chosen point declare its
first search-window copy 16 bytes larger than the copy delivers, so its
wait really runs out its one-second limit while no copy is left in flight
(every byte the copies carry has landed).  The failure path then runs as
it would after a stalled copy: the point and the others its warp holds come
back OMT_PT_LOST_TIMEOUT at their input positions, every other point is the
same bit for bit as in a run without the hook, omt_lk_wait_timeouts returns
OMT_ETIMEOUT, and the next run is clean.
"""
import ctypes
import math

import numpy as np
import pytest

from paper_1910_06017_b300 import synth
from lk_parity import gpu_lk

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def omt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1910_06017_b300 import omt as m
    m.lib()
    return m


def _timeouts_abi(omt):
    c = ctypes.c_uint32(0)
    rc = omt.lib().omt_lk_wait_timeouts(ctypes.byref(c))
    return rc, int(c.value)


def test_plain_lk_wait_failure_is_reported(omt):
    p = synth.sd_pair()
    rng = np.random.default_rng(31)
    pts = synth.random_points(rng, 3000, 720, 576)
    ref = gpu_lk(omt, p.frame0, p.frame1, pts)
    assert _timeouts_abi(omt) == (omt.OK, 0)
    omt.debug_fail_lk_wait(1234)
    try:
        out, st, it = gpu_lk(omt, p.frame0, p.frame1, pts)
    finally:
        omt.debug_fail_lk_wait(-1)
    rc, count = _timeouts_abi(omt)
    assert rc == omt.ETIMEOUT and count >= 1
    lost = st == omt.PT_LOST_TIMEOUT
    # 3,000 points fill 3,000 warps: the failed warp held this point only
    assert np.nonzero(lost)[0].tolist() == [1234]
    np.testing.assert_array_equal(out[lost], pts[lost])
    assert np.all(it[lost] == 0)
    for a, b in zip((out, st, it), ref):
        np.testing.assert_array_equal(a[~lost], b[~lost])
    # the hook is off again: the next run is the reference bit for bit
    again = gpu_lk(omt, p.frame0, p.frame1, pts)
    for a, b in zip(again, ref):
        np.testing.assert_array_equal(a, b)
    assert _timeouts_abi(omt) == (omt.OK, 0)


def test_batched_lk_wait_failure_is_reported(omt):
    sps = [synth.stream_pair(s, workload=13, n_range=(300, 3000)) for s in range(3)]
    caps = [int(math.ceil(sp.n_target / 64)) for sp in sps]
    params = omt.default_params(levels=4, win=21, min_dist=3.0, storage=1, max_corners=max(caps))

    def run(fail_at):
        B = omt.BatchTracker([sp.size for sp in sps], params,
                             max_boxes=[len(sp.boxes) for sp in sps], max_corners=caps)
        B.caps.lk_chunk = 4
        for s, sp in enumerate(sps):
            B.prime(s, torch.from_numpy(sp.frame0).cuda())
            B.slot(s).copy_(torch.from_numpy(sp.frame1))
            B.set_boxes(s, torch.from_numpy(sp.boxes))
        B.pack()
        omt.debug_fail_lk_wait(fail_at)
        try:
            B.step()
            torch.cuda.synchronize()
        finally:
            omt.debug_fail_lk_wait(-1)
        n = [B.count(s) for s in range(len(sps))]
        cat = lambda xs: np.concatenate([x[:k].cpu().numpy() for x, k in zip(xs, n)])
        offsets = [B.offsets[s][:len(sp.boxes) + 1].cpu().numpy() for s, sp in enumerate(sps)]
        return (cat(B.pts), cat(B.pts_out), cat(B.status), cat(B.iters),
                [B.boxes_out[s][:len(sp.boxes)].cpu().numpy() for s, sp in enumerate(sps)],
                n, offsets)

    ref = run(-1)
    ns, offs = ref[5], ref[6]
    assert _timeouts_abi(omt) == (omt.OK, 0)
    n0 = len(ref[0])
    target = n0 // 2
    pts, out, st, it, boxes, _, _ = run(target)
    rc, count = _timeouts_abi(omt)
    assert rc == omt.ETIMEOUT and count >= 1
    lost = st == omt.PT_LOST_TIMEOUT
    idx = np.nonzero(lost)[0]
    # the point itself and at most the rest of its warp's chunk, the chunk it
    # had taken next and the chunk it had claimed ahead (chunks of 4)
    assert target in idx and len(idx) <= 12
    np.testing.assert_array_equal(pts, ref[0])
    np.testing.assert_array_equal(out[lost], pts[lost])
    assert np.all(it[lost] == 0)
    for a, b in zip((out, st, it), ref[1:4]):
        np.testing.assert_array_equal(a[~lost], b[~lost])
    # the box update uses the OK points only: boxes without a lost point are
    # unchanged
    at = np.cumsum([0] + ns)
    for s, (a, b) in enumerate(zip(boxes, ref[4])):
        mine = idx[(idx >= at[s]) & (idx < at[s + 1])] - at[s]
        hit = set(np.searchsorted(offs[s], mine, side="right") - 1)
        for j in range(len(a)):
            if j not in hit:
                np.testing.assert_array_equal(a[j], b[j])
