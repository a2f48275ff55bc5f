"""GPU parity of the working level (Section V-A preprocessing: a pyramid
level chosen by resolution) through the C-ABI.

The working frame (pyramid level L of an F32 pyramid rounded to u8) equals
the oracle's bit for bit for L = 0..2: those levels hold exact dyadic
values.  The working-level tracker then runs the ordinary kernels on the
working frames, so it must equal a plain tracker fed the oracle's working
frames and boxes scaled by 2^-L, bit for bit, with its boxes scaled back by
2^L exactly.
"""
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


def _t(a, dt=None):
    return torch.from_numpy(np.ascontiguousarray(a if dt is None else a.astype(dt))).cuda()


@pytest.mark.parametrize("size", [(720, 576), (1921, 1083), (37, 23), (3840, 2160)])
def test_working_frame_matches_oracle(omt, oracle, size):
    w, h = size
    rng = np.random.default_rng(w)
    f = synth.render_shift(synth.Texture.draw(rng, w, h), w, h)
    levels = (0, 1, 2) if w < 3000 else (2,)
    P = omt.Pyramid(w, h, 3, omt.F32)
    omt.build_pyramid(_t(f, np.uint8), P, omt.default_params(levels=3))
    for L in levels:
        lw, lh = P.level_size(L)
        out = torch.zeros((lh, lw + 5), dtype=torch.uint8, device="cuda")  # padded rows
        omt.level_u8(P, L, out[:, :lw])
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out[:, :lw].cpu().numpy(), oracle.level_u8(f, L),
                                      err_msg=str(L))


def test_rule_and_box_scaling(omt, oracle):
    for w, h in ((720, 576), (1280, 720), (1920, 1080), (2560, 1280), (3840, 2160)):
        assert omt.working_level(w, h) == oracle.working_level(w, h)
    b = np.array([[0.5, 1.25, 100.75, 37.0], [-3.0, 7.5, 9.0, 8.0]], np.float32)
    out = torch.zeros((2, 4), device="cuda")
    omt.scale_boxes(_t(b), 0.25, out)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), b * 0.25)


@pytest.mark.parametrize("which", ["1080p", "4k"])
def test_working_level_tracker_equals_plain_on_working_frames(omt, oracle, which):
    if which == "1080p":
        sp = synth.stream_pair(0, workload=13, n_range=(2000, 3000))  # 1920x1080
        f0, f1, boxes = sp.frame0, sp.frame1, sp.boxes
        L = 1
    else:
        pr = synth.rigid_pair(n_regions=60)
        f0, f1, boxes = pr.frame0, pr.frame1, pr.boxes
        L = 2
    h, w = f0.shape
    assert omt.working_level(w, h) == L
    params = omt.default_params(levels=3, max_corners=60, min_dist=3.0)
    T = omt.WorkingLevelTracker(w, h, params, len(boxes))
    T.prime(_t(f0, np.uint8))
    bo = T.step(_t(f1, np.uint8), _t(boxes, np.float32)).cpu().numpy()
    # the same kernels on the oracle's working frames
    w0, w1 = oracle.level_u8(f0, L), oracle.level_u8(f1, L)
    S = omt.StreamTracker(w0.shape[1], w0.shape[0], params, len(boxes))
    S.prime(_t(w0))
    so = S.step(_t(w1), _t(boxes * 2.0 ** -L, np.float32)).cpu().numpy()
    torch.cuda.synchronize()
    nb = len(boxes)
    n = int(S.offsets[nb].item())
    assert n == int(T.inner.offsets[nb].item()) and n > 100
    np.testing.assert_array_equal(T.inner.pts[:n].cpu().numpy(), S.pts[:n].cpu().numpy())
    np.testing.assert_array_equal(T.inner.status[:n].cpu().numpy(), S.status[:n].cpu().numpy())
    np.testing.assert_array_equal(T.inner.pts_out[:n].cpu().numpy(), S.pts_out[:n].cpu().numpy())
    np.testing.assert_array_equal(bo, so * 2.0 ** L)
