"""omt_select_corners_static: corner selection without a caller scratch.

This entry point serves callers that cannot allocate device memory (a plugin
whose host application owns the CUDA allocator, a real-time loop that must
not call cudaMalloc): it keeps its scratch in one fixed array inside the
library.  These checks call it through the C-ABI and compare it with
omt_select_corners given a scratch buffer of its own, on two calls in a row
with different frames and boxes (the array keeps the first call's contents,
so the second result shows nothing leaks between calls).  The file sorts
last so that a run stopping at the first failure has run everything else.
"""
import ctypes

import numpy as np
import pytest

from paper_1910_06017_b300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def omt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1910_06017_b300 import omt as m
    m.lib()
    return m


def _case(omt, frame, boxes, maxc, quality=(1, 100), min_dist=5.0):
    h, w = frame.shape
    P = omt.Pyramid(w, h, 1)
    params = omt.default_params(levels=1, max_corners=maxc, quality=quality, min_dist=min_dist)
    omt.build_pyramid(torch.from_numpy(np.ascontiguousarray(frame)).cuda(), P, params)
    b = torch.from_numpy(np.ascontiguousarray(boxes, np.float32)).cuda()
    return P, params, b


def _with_scratch(omt, P, params, b):
    nb = b.shape[0]
    scratch = torch.empty(omt.corner_scratch_bytes(P.w, P.h, nb, params.max_corners),
                          dtype=torch.uint8, device="cuda")
    pts = torch.zeros((nb * params.max_corners, 2), device="cuda")
    off = torch.zeros(nb + 1, dtype=torch.int32, device="cuda")
    omt.select_corners(P, b, params, scratch, pts, off)
    torch.cuda.synchronize()
    return pts.cpu().numpy(), off.cpu().numpy()


def _static_abi(omt, P, params, b, check_free=False):
    """Calls omt_select_corners_static through ctypes, with no scratch.
    With check_free, also returns whether the device's free memory stayed
    the same across the call (outputs are allocated before the reading)."""
    nb = b.shape[0]
    pts = torch.full((nb * params.max_corners, 2), -1.0, device="cuda")
    off = torch.full((nb + 1,), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    fn = omt.lib().omt_select_corners_static
    fn.argtypes = [ctypes.POINTER(omt.PyramidDesc), ctypes.c_void_p, ctypes.c_int32,
                   ctypes.POINTER(omt.Params), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    rc = fn(ctypes.byref(P.desc), ctypes.c_void_p(b.data_ptr()), nb, ctypes.byref(params),
            ctypes.c_void_p(pts.data_ptr()), ctypes.c_void_p(off.data_ptr()),
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    same_free = torch.cuda.mem_get_info()[0] == free_before
    if check_free:
        return rc, pts.cpu().numpy(), off.cpu().numpy(), same_free
    return rc, pts.cpu().numpy(), off.cpu().numpy()


def _same(a, b):
    (pa, oa), (pb, ob) = a, b
    np.testing.assert_array_equal(oa, ob)
    n = int(oa[-1])
    np.testing.assert_array_equal(pa[:n], pb[:n])


def test_static_matches_caller_scratch_twice(omt):
    # first call: the 720x576 pair's frame 0 and its 10 boxes
    p = synth.sd_pair()
    P1, prm1, b1 = _case(omt, p.frame0, p.boxes, 50)
    rc, pts, off = _static_abi(omt, P1, prm1, b1)
    assert rc == omt.OK
    assert off[-1] > 300
    _same((pts, off), _with_scratch(omt, P1, prm1, b1))

    # second call right after: another frame, size, box set and parameters;
    # device memory must not change (the call allocates nothing)
    clip = synth.affine_clip(n_frames=1)
    P2, prm2, b2 = _case(omt, clip.frames[0], clip.gt_boxes[0], 100, (1, 50), 3.0)
    rc, pts, off, same_free = _static_abi(omt, P2, prm2, b2, check_free=True)
    assert rc == omt.OK
    assert same_free
    assert off[-1] > 300
    _same((pts, off), _with_scratch(omt, P2, prm2, b2))

    # and the first input again, after the array was overwritten
    rc, pts, off = _static_abi(omt, P1, prm1, b1)
    assert rc == omt.OK
    _same((pts, off), _with_scratch(omt, P1, prm1, b1))


def _static_need(w, h, nboxes, max_corners):
    """The array bytes a call needs, by the rule the header states: the
    response map (4 bytes per pixel), 8 bytes per box-corner slot and 4 per
    box (plus one word), each part rounded up to 256 bytes."""
    up = lambda v: (v + 255) // 256 * 256
    return up(w * h * 4) + up(nboxes * max_corners * 8) + up(nboxes * 4 + 4)


def test_static_rejects_frames_beyond_its_array(omt):
    # a 4K frame's response map alone (3840*2160*4 bytes) exceeds the array
    f = np.zeros((2160, 3840), np.uint8)
    P, prm, b = _case(omt, f, np.array([[0, 0, 100, 100]], np.float32), 10)
    assert _static_need(3840, 2160, 1, 10) > omt.STATIC_SCRATCH_BYTES
    rc, pts, off = _static_abi(omt, P, prm, b)
    assert rc == omt.ENOMEM
    assert np.all(off == -1)  # nothing was launched


def test_static_capacity_at_1080p(omt):
    # a 1920x1080 frame leaves the array room for about 1.05 million
    # box-corner slots: 1,000 boxes of 1,000 corners fit, 1,100 do not
    assert _static_need(1920, 1080, 1000, 1000) <= omt.STATIC_SCRATCH_BYTES
    assert _static_need(1920, 1080, 1100, 1000) > omt.STATIC_SCRATCH_BYTES
    clip = synth.affine_clip(n_frames=1)
    rng = np.random.default_rng(8)
    boxes = synth.uniform_boxes(rng, 1920, 1080, 1000)
    P, prm, b = _case(omt, clip.frames[0], boxes, 1000)
    rc, pts, off = _static_abi(omt, P, prm, b)
    assert rc == omt.OK
    _same((pts, off), _with_scratch(omt, P, prm, b))
