"""GPU parity of the forward-backward consistency check (omt_fb_check and
the batched OMT_PHASE_FB) against the FP64 oracle, through the C-ABI.

The decision kernel is compared with the oracle bit for bit on hand
vectors.  The whole check (forward LK, backward LK from the forward results,
decision) is compared with the oracle's composition: FP32 and FP64 round
trips differ by the flow tolerance (or, where a stopping iteration differs,
by up to about eps), so decisions are compared outside a guard band of
0.03 px around fb_max.  The batched phase must equal the plain calls bit for
bit (same device code), and the box update must drop the LOST_FB points.
"""
import math

import numpy as np
import pytest

from paper_1910_06017_b300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

OK, LOST_EIG, LOST_OOB, NONCONV, LOST_FB = 1, 2, 4, 8, 16
BAND = 0.03


@pytest.fixture(scope="module")
def omt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1910_06017_b300 import omt as m
    m.lib()
    return m


def _t(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a, dt)).cuda()


def test_fb_check_kernel_matches_oracle_hand_vectors(omt, oracle):
    pts = np.array([[10, 10], [10, 10], [10, 10], [10, 10], [10, 10], [5, 5], [5, 5],
                    [7.5, 2.25]], np.float32)
    back = np.array([[10.375, 10.5], [10.375, 10.5 + 2.0 ** -20], [10.0, 10.0], [13.0, 14.0],
                     [10.0, 10.25], [50.0, 50.0], [5.0, 5.0], [7.5, 2.25]], np.float32)
    sb = np.array([OK, OK, LOST_EIG, OK, OK | NONCONV, OK, OK, OK], np.uint8)
    st = np.array([OK, OK, OK, OK, OK | NONCONV, LOST_EIG, LOST_OOB, OK | NONCONV], np.uint8)
    for fb_max in (0.625, 0.0, 3.0, float("inf")):
        want = oracle.fb_check(pts, back.astype(np.float64), sb, st, fb_max)
        g = _t(st, np.uint8)
        omt.fb_check(_t(pts, np.float32), _t(back, np.float32), _t(sb, np.uint8), fb_max, g)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(g.cpu().numpy(), want, err_msg=str(fb_max))


def test_fb_check_count_from_device_and_bad_arguments(omt):
    n = 1000
    rng = np.random.default_rng(3)
    pts = rng.uniform(0, 100, (n, 2)).astype(np.float32)
    back = pts + rng.normal(0, 1, (n, 2)).astype(np.float32)
    st = np.full(n, OK, np.uint8)
    sb = np.full(n, OK, np.uint8)
    g = _t(st, np.uint8)
    m = torch.tensor([600], dtype=torch.int32, device="cuda")
    omt.fb_check(_t(pts, np.float32), _t(back, np.float32), _t(sb, np.uint8), 1.0, g,
                 n_max=n, n_dev=m)
    torch.cuda.synchronize()
    got = g.cpu().numpy()
    e = np.hypot(*(back - pts).T)
    assert np.all(got[600:] == OK)                     # beyond the device count: untouched
    np.testing.assert_array_equal(got[:600] == OK, e[:600] <= 1.0)
    omt.fb_check(_t(pts, np.float32), _t(back, np.float32), _t(sb, np.uint8), 1.0, g, n_max=0)
    with pytest.raises(RuntimeError):
        omt.fb_check(_t(pts, np.float32), _t(back, np.float32), _t(sb, np.uint8), float("nan"), g)


def _pyr(omt, frame, levels, storage=0):
    h, w = frame.shape
    P = omt.Pyramid(w, h, levels, storage)
    omt.build_pyramid(torch.from_numpy(np.ascontiguousarray(frame)).cuda(), P,
                      omt.default_params(levels=levels, storage=storage))
    return P


def _gpu_fb(omt, f0, f1, pts, fb_max, **kw):
    params = omt.default_params(**kw)
    P0, P1 = _pyr(omt, f0, params.levels), _pyr(omt, f1, params.levels)
    n = len(pts)
    p = _t(pts, np.float32)
    out = torch.zeros((n, 2), device="cuda")
    back = torch.zeros((n, 2), device="cuda")
    st = torch.zeros(n, dtype=torch.uint8, device="cuda")
    sb = torch.zeros(n, dtype=torch.uint8, device="cuda")
    omt.lk_track_fb(P0, P1, p, params, fb_max, out, st, back, sb)
    torch.cuda.synchronize()
    return out.cpu().numpy(), st.cpu().numpy(), back.cpu().numpy(), sb.cpu().numpy()


def _occluded_scene():
    rng = np.random.default_rng(7)
    w, h = 320, 240
    tex = synth.Texture.draw(rng, w, h)
    other = synth.Texture.draw(np.random.default_rng(8), w, h)
    f0 = synth.render_shift(tex, w, h, 0.0, 0.0)
    f1 = synth.render_shift(tex, w, h, 2.0, 1.0)
    occ = (slice(80, 170), slice(100, 210))
    f1[occ] = synth.render_shift(other, w, h, 0.0, 0.0)[occ]
    return f0, f1


@pytest.mark.parametrize("scene", ["sd_pair", "occluded"])
def test_plain_fb_matches_oracle(omt, oracle, scene):
    if scene == "sd_pair":
        p = synth.sd_pair()
        f0, f1, boxes, kw, fb_max = p.frame0, p.frame1, p.boxes, dict(levels=3, win=21), 0.05
        maxc, md = 50, 5.0
    else:
        f0, f1 = _occluded_scene()
        boxes = np.array([[0, 0, f0.shape[1], f0.shape[0]]], np.float32)
        kw, fb_max, maxc, md = dict(levels=3, win=15), 0.5, 400, 4.0
    pts, cnt = oracle.select_corners(f0, boxes, maxc, min_dist=md)
    allp = np.concatenate([pts[i, :cnt[i]] for i in range(len(cnt))])
    o_out, o_st, o_back, o_sb = oracle.lk_track_fb(oracle.Pyramid(f0, kw["levels"]),
                                                   oracle.Pyramid(f1, kw["levels"]), allp, fb_max,
                                                   eps=0.01, max_iter=30, min_eig=1e-3,
                                                   win=kw["win"])
    g_out, g_st, g_back, g_sb = _gpu_fb(omt, f0, f1, allp, fb_max, eps=0.01, max_iter=30, **kw)
    # decisions away from the threshold agree; both forward runs OK there
    e = np.hypot(*(o_back - allp).T)
    fwd_o = ((o_st & OK) > 0) | (o_st == LOST_FB)
    fwd_g = ((g_st & OK) > 0) | (g_st == LOST_FB)
    clear = fwd_o & fwd_g & ((o_sb & OK) > 0) & ((g_sb & OK) > 0) & (np.abs(e - fb_max) > BAND)
    assert clear.mean() > 0.8, clear.mean()
    np.testing.assert_array_equal(g_st[clear] == LOST_FB, o_st[clear] == LOST_FB)
    assert ((o_st & OK) > 0).sum() > 0
    if scene == "occluded":  # the SD pair's round trips all close (median 1e-4 px)
        assert (o_st == LOST_FB).sum() > 20
    # a LOST_FB point keeps its forward position; the statuses are valid
    assert set(np.unique(g_st)) <= {OK, OK | NONCONV, LOST_EIG, LOST_OOB, LOST_FB}


def _streams(n, first=0):
    return [synth.stream_pair(s, workload=13, n_range=(300, 3000)) for s in range(first, first + n)]


def _cap(sp):
    return int(math.ceil(sp.n_target / 64))


@pytest.mark.parametrize("storage", [0, 1])
def test_batched_fb_equals_plain_calls(omt, oracle, storage):
    sps = _streams(4, first=60)
    fb_max = 0.05
    params = omt.default_params(levels=4, win=21, min_dist=3.0, storage=storage,
                                max_corners=max(_cap(sp) for sp in sps), fb_max=fb_max)
    sizes = [sp.size for sp in sps]
    B = omt.BatchTracker(sizes, params, max_boxes=[len(sp.boxes) for sp in sps],
                         max_corners=[_cap(sp) for sp in sps])
    for s, sp in enumerate(sps):
        B.prime(s, torch.from_numpy(sp.frame0).cuda())
        B.slot(s).copy_(torch.from_numpy(sp.frame1))
        B.set_boxes(s, torch.from_numpy(sp.boxes))
    B.pack()
    B.capture()
    B.step()
    torch.cuda.synchronize()
    n_fb = 0
    for s, sp in enumerate(sps):
        n = B.count(s)
        pts = B.pts[s][:n]
        prm = params.replace(max_corners=_cap(sp))
        P0 = _pyr(omt, sp.frame0, 4, storage)
        P1 = _pyr(omt, sp.frame1, 4, storage)
        out = torch.zeros((n, 2), device="cuda")
        back = torch.zeros((n, 2), device="cuda")
        st = torch.zeros(n, dtype=torch.uint8, device="cuda")
        sb = torch.zeros(n, dtype=torch.uint8, device="cuda")
        omt.lk_track_fb(P0, P1, pts, prm, fb_max, out, st, back, sb)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(B.pts_out[s][:n].cpu().numpy(), out.cpu().numpy())
        np.testing.assert_array_equal(B.pts_back[s][:n].cpu().numpy(), back.cpu().numpy())
        np.testing.assert_array_equal(B.status_back[s][:n].cpu().numpy(), sb.cpu().numpy())
        got_st = B.status[s][:n].cpu().numpy()
        np.testing.assert_array_equal(got_st, st.cpu().numpy())
        n_fb += int((got_st == LOST_FB).sum())
        # the box update moved each box by the median over its OK points only
        nb = B.nboxes[s]
        off = B.offsets[s][:nb + 1].cpu().numpy()
        want, nv = oracle.update_boxes(sp.boxes, off, pts.cpu().numpy(), out.cpu().numpy(),
                                       got_st)
        np.testing.assert_array_equal(B.nvalid[s][:nb].cpu().numpy(), nv)
        np.testing.assert_allclose(B.boxes_out[s][:nb].cpu().numpy(), want, atol=1e-3)
    assert n_fb > 0
    assert omt.lk_wait_timeouts() == 0
