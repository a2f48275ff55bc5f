"""GPU parity of K1 (pyramid + gradients) and K2 (corner response and
selection) against the FP64 oracle, through the C-ABI.

Bar, F32 storage: levels 0-2 and the gradients of levels 0-1 bit-exact
(their values are dyadic and exact in FP32); level 3 and the gradients of
level 2 are the correctly rounded values of the definition (the kernel sums
exactly and rounds once), and deeper levels inherit the rounding of the
stored level they are formed from: every level within 2 FP32 ulps of the
oracle (level 4: at most 1.5), every gradient within 2 ulps of its own value
plus, from level 3 on, 2 ulps at the intensity scale (255) of the stored
level it differentiates.  F16 storage: bit-exact against the oracle's
half-precision storage (every level and gradient the correctly rounded half
of the definition applied to the level above as stored).  Corner response,
maximum flags and corner lists bit-exact.
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


def _gpu_pyramid(omt, frame, levels, storage=0, pad=0):
    h, w = frame.shape
    if pad:
        buf = torch.zeros((h, w + pad), dtype=torch.uint8, device="cuda")
        buf[:, :w] = torch.from_numpy(frame).cuda()
        f = buf[:, :w]
    else:
        f = torch.from_numpy(np.ascontiguousarray(frame)).cuda()
    P = omt.Pyramid(w, h, levels, storage)
    omt.build_pyramid(f, P, omt.default_params(levels=levels, storage=storage))
    torch.cuda.synchronize()
    return P


def _textured(w, h, seed):
    rng = np.random.default_rng(seed)
    tex = synth.Texture.draw(rng, w, h, n_blobs=max(8, w * h // 6000))
    return synth.render_shift(tex, w, h)


def _ulp32(x):
    return np.spacing(np.abs(np.asarray(x, np.float64)).astype(np.float32)).astype(np.float64)


@pytest.mark.parametrize("w,h,levels,pad", [(720, 576, 3, 0), (37, 23, 5, 13), (1920, 1080, 4, 0),
                                            (2, 3, 2, 0), (1, 1, 1, 0), (5, 4, 4, 3),
                                            (129, 65, 5, 0), (3840, 2160, 5, 0)])
def test_pyramid_f32_matches_oracle(omt, oracle, w, h, levels, pad):
    f = _textured(w, h, w * 7 + h)
    P = _gpu_pyramid(omt, f, levels, 0, pad)
    O = oracle.Pyramid(f, levels)
    for L in range(levels):
        img = P.image(L).cpu().numpy().astype(np.float64)
        grd = P.grad(L).cpu().numpy().astype(np.float64)
        if L <= 2:
            np.testing.assert_array_equal(img, O.img[L], err_msg=f"level {L}")
        else:
            # level 3 is the definition rounded once; level 4 adds the
            # rounding level 3 carries (< 1 ulp after averaging)
            ulps = np.abs(img - O.img[L]) / _ulp32(O.img[L])
            assert ulps.max() <= (0.5 if L == 3 else 2.0), (L, ulps.max())
        if L <= 1:
            np.testing.assert_array_equal(grd, O.grad[L], err_msg=f"grad {L}")
        else:
            bar = 2 * _ulp32(O.grad[L]) + (2 * _ulp32(255.0) if L >= 3 else 0.0)
            if L == 2:
                bar = 0.5 * _ulp32(O.grad[L])   # exact inputs, one rounding
            err = np.abs(grd - O.grad[L])
            assert np.all(err <= bar), (L, (err / _ulp32(O.grad[L])).max(), err.max())


@pytest.mark.parametrize("w,h,levels", [(720, 576, 3), (37, 23, 5), (1920, 1080, 4),
                                        (129, 65, 5), (3840, 2160, 5)])
def test_pyramid_f16_storage_bit_exact(omt, oracle, w, h, levels):
    f = _textured(w, h, 3)
    P = _gpu_pyramid(omt, f, levels, 1)
    O = oracle.Pyramid(f, levels, storage="f16")
    np.testing.assert_array_equal(P.image(0).cpu().numpy(), f)
    for L in range(levels):
        if L > 0:
            img = P.image(L).float().cpu().numpy().astype(np.float64) + 128.0
            np.testing.assert_array_equal(img, O.img[L], err_msg=f"level {L}")
        grd = P.grad(L).float().cpu().numpy().astype(np.float64)
        np.testing.assert_array_equal(grd, O.grad[L], err_msg=f"grad {L}")


def _local_max(R):
    h, w = R.shape
    flag = np.zeros_like(R, dtype=bool)
    c = R[1:-1, 1:-1]
    m = np.ones_like(c, dtype=bool)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            m &= c >= R[1 + dy:h - 1 + dy, 1 + dx:w - 1 + dx]
    flag[1:-1, 1:-1] = m
    return flag


@pytest.mark.parametrize("w,h", [(720, 576), (37, 23), (1920, 1080), (3, 3), (2, 9), (4099, 17)])
def test_corner_response_bit_exact(omt, oracle, w, h):
    f = _textured(w, h, 11 + w)
    P = _gpu_pyramid(omt, f, 1)
    out = torch.empty(h * w, dtype=torch.int32, device="cuda")
    omt.corner_response(P, out)
    torch.cuda.synchronize()
    g = out.cpu().numpy().view(np.uint32).reshape(h, w)
    R = oracle.corner_response(f)
    np.testing.assert_array_equal((g & 0x3FFFFFFF).astype(np.int64), R)
    np.testing.assert_array_equal((g >> 30) & 1, _local_max(R).astype(np.uint32))
    assert np.all((g >> 31) == 0)


def test_corner_response_random_noise_extremes(omt, oracle):
    # white noise of full amplitude drives the structure tensor to its bounds
    rng = np.random.default_rng(2)
    f = (rng.integers(0, 2, (64, 96)) * 255).astype(np.uint8)
    P = _gpu_pyramid(omt, f, 1)
    out = torch.empty(f.size, dtype=torch.int32, device="cuda")
    omt.corner_response(P, out)
    torch.cuda.synchronize()
    g = out.cpu().numpy().view(np.uint32).reshape(f.shape)
    np.testing.assert_array_equal((g & 0x3FFFFFFF).astype(np.int64), oracle.corner_response(f))


def _gpu_select(omt, P, boxes, params):
    nb = len(boxes)
    b = torch.from_numpy(np.ascontiguousarray(boxes, np.float32)).cuda()
    scratch = torch.empty(omt.corner_scratch_bytes(P.w, P.h, nb, params.max_corners),
                          dtype=torch.uint8, device="cuda")
    scratch.fill_(0xAB)
    pts = torch.full((max(1, nb * params.max_corners), 2), -7.0, device="cuda")
    off = torch.full((nb + 1,), -1, dtype=torch.int32, device="cuda")
    omt.select_corners(P, b if nb else None, params, scratch, pts, off)
    torch.cuda.synchronize()
    off = off.cpu().numpy()
    pts = pts.cpu().numpy()
    return [pts[off[i]:off[i + 1]] for i in range(nb)], off


def _check_select(omt, oracle, f, boxes, maxc, quality=(1, 100), min_dist=5.0, P=None):
    if P is None:
        P = _gpu_pyramid(omt, f, 1)
    params = omt.default_params(levels=P.levels, max_corners=maxc, quality=quality, min_dist=min_dist)
    got, off = _gpu_select(omt, P, boxes, params)
    want_pts, want_cnt = oracle.select_corners(f, boxes, maxc, quality=quality, min_dist=min_dist)
    assert off[0] == 0 and np.all(np.diff(off) == want_cnt)
    for i in range(len(boxes)):
        np.testing.assert_array_equal(got[i], want_pts[i, :want_cnt[i]], err_msg=f"box {i}")
    return want_cnt


def test_select_sd_pair(omt, oracle):
    p = synth.sd_pair()
    cnt = _check_select(omt, oracle, p.frame0, p.boxes, 50)
    assert cnt.sum() > 300


def test_select_golden(omt, oracle):
    from tests.test_golden import load_golden
    g = load_golden()
    P = _gpu_pyramid(omt, g["frame0"], g["params"]["levels"])
    params = omt.default_params(levels=g["params"]["levels"], max_corners=g["params"]["max_corners"],
                                quality=tuple(g["params"]["quality"]), min_dist=g["params"]["min_dist"])
    got, off = _gpu_select(omt, P, g["boxes"], params)
    assert np.diff(off).tolist() == g["counts"]
    np.testing.assert_array_equal(np.concatenate(got), g["points"])


def test_select_ragged_boxes(omt, oracle):
    w, h = 203, 157
    f = _textured(w, h, 5)
    boxes = np.array([[0, 0, w, h], [3.5, 2.0, 30.0, 25.5], [10.0, 10.0, 10.0, 20.0],
                      [-50, -5, 20.25, 18.75], [190, 150, 400, 400], [w + 5, 0, w + 50, 10],
                      [1.0, 1.0, 2.0, 2.0], [0.5, 0.5, 1.5, 1.5], [np.nan, 0, 10, 10],
                      [40, 30, 20, 50], [5.999, 7.001, 60.0001, 61.9999]], np.float32)
    for maxc, q, md in [(50, (1, 100), 5.0), (7, (1, 4), 3.0), (1, (1, 100), 0.0),
                        (300, (0, 1), 2.5), (0, (1, 100), 5.0), (4096, (0, 1), 0.0)]:
        _check_select(omt, oracle, f, boxes, maxc, q, md)


def test_select_no_boxes(omt, oracle):
    f = _textured(64, 48, 1)
    P = _gpu_pyramid(omt, f, 1)
    got, off = _gpu_select(omt, P, np.zeros((0, 4), np.float32), omt.default_params(levels=1))
    assert off.tolist() == [0]


def test_select_constant_and_rank_one(omt, oracle):
    for f in [np.full((64, 80), 99, np.uint8),
              np.tile(synth.quantise(128 + 90 * np.sin(np.arange(80) / 2.0)), (64, 1))]:
        boxes = np.array([[3, 3, 77, 61], [0, 0, 80, 64]], np.float32)
        _check_select(omt, oracle, f, boxes, 50)


def test_select_many_candidates_uses_chunks(omt, oracle):
    # quality 0 and min distance 0 keep every positive local maximum of a
    # 1080p full-frame box: far more candidates than one shared-memory sort
    f = _textured(1920, 1080, 17)
    R = oracle.corner_response(f)
    assert _local_max(R)[1:-1, 1:-1].sum() > 3 * 8192
    boxes = np.array([[0, 0, 1920, 1080], [100, 100, 1500, 900]], np.float32)
    _check_select(omt, oracle, f, boxes, 4096, (0, 1), 0.0)
    _check_select(omt, oracle, f, boxes, 4096, (0, 1), 3.0)


def test_select_1080p_workload(omt, oracle):
    clip = synth.affine_clip(n_frames=1)
    _check_select(omt, oracle, clip.frames[0], clip.gt_boxes[0], 100)


def test_select_4k_workload(omt, oracle):
    pr = synth.rigid_pair(n_regions=200)
    cnt = _check_select(omt, oracle, pr.frame0, pr.boxes, 250)
    assert cnt.sum() > 20000


def test_select_weak_maxima_overflow_quality_fits(omt, oracle):
    # faint noise makes thousands of weak local maxima in the box; a few
    # strong squares set R_max so that the quality test keeps only their
    # corners: the box overflows the first gather but not the second
    rng = np.random.default_rng(23)
    w, h = 640, 480
    f = (128 + rng.integers(-2, 3, size=(h, w))).astype(np.uint8)
    for k in range(12):
        x0, y0 = 40 + 48 * (k % 6) * 2, 60 + 150 * (k // 6)
        f[y0:y0 + 30, x0:x0 + 30] = 250 if k % 2 else 5
    R = oracle.corner_response(f)
    lm = _local_max(R) & (R > 0)
    box = (slice(10, 470), slice(5, 635))
    assert lm[box].sum() > 4096
    assert (lm[box] & (R[box] * 100 > R[box].max())).sum() < 1024
    boxes = np.array([[5, 10, 635, 470], [0, 0, w, h]], np.float32)
    _check_select(omt, oracle, f, boxes, 200)
    _check_select(omt, oracle, f, boxes, 20, (1, 100), 12.0)
