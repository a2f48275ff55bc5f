"""GPU parity of K3 (pyramidal LK) and K4 (box update) against the FP64
oracle, through the C-ABI, and end-to-end steps of the whole path.

Bar for flow, both storages: within 1e-3 px of the oracle run on the
pyramid the GPU stores (F32: the FP64 definition; F16: the oracle's
half-precision storage, which the F16 kernels produce bit for bit) on every
point whose per-level iteration counts agree; a stopping iteration that
differs stays within eps and is counted; statuses identical outside the
guard band lambda_min/N in [0.9 tau, 1.1 tau] and the points the
conditioning probe marks (tests/lk_parity.py).  Half-precision storage
itself is stated per workload against the FP64 oracle on unquantised
pyramids: within 0.02 px on every converged point, p99 and mean within
0.02 px on all OK points, the NONCONV share counted and bounded.
"""
import numpy as np
import pytest

from paper_1910_06017_b300 import synth
from lk_parity import (FLOW_TOL, F16_TOL, LOST_EIG, LOST_OOB, NONCONV, OK, compare, error_vs_fp64,
                       gpu_lk, gpu_pyramid, oracle_lk)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def omt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1910_06017_b300 import omt as m
    m.lib()
    return m


def _pyr(omt, frame, levels, storage=0):
    return gpu_pyramid(omt, frame, levels, storage)


def test_lk_sd_pair_corners(omt, oracle):
    p = synth.sd_pair()
    pts, cnt = oracle.select_corners(p.frame0, p.boxes, 50)
    allp = np.concatenate([pts[i, :cnt[i]] for i in range(len(cnt))])
    compare(omt, oracle, p.frame0, p.frame1, allp, label="SD pair corners")


def test_lk_fixed_iterations_all_points(omt, oracle):
    p = synth.sd_pair()
    rng = np.random.default_rng(3)
    pts = np.stack([rng.uniform(0, 719, 2000), rng.uniform(0, 575, 2000)], 1).astype(np.float32)
    g_out, g_st, g_it = gpu_lk(omt, p.frame0, p.frame1, pts, levels=3, win=21, max_iter=10, eps=0.0)
    (o_out, o_st, o_it, o_me), unstable = oracle_lk(oracle, p.frame0, p.frame1, pts, max_iter=10,
                                                    eps=0.0, probe=True)
    band = np.any((o_me >= 0.9e-3) & (o_me <= 1.1e-3), axis=1)
    stable = ~unstable & ~band
    print(f"fixed 10 iterations, 2000 random points: excluded by the conditioning probe "
          f"{unstable.sum()}, in the tau guard band {band.sum()}")
    assert unstable.mean() <= 0.05
    assert np.all(g_st[stable] == o_st[stable])
    both = ((g_st & OK) > 0) & stable
    assert both.mean() > 0.8
    assert np.abs(g_out[both] - o_out[both]).max() <= FLOW_TOL


def test_lk_identical_frames_exact_zero(omt, oracle):
    p = synth.sd_pair()
    rng = np.random.default_rng(4)
    pts = np.stack([rng.uniform(0, 719, 500), rng.uniform(0, 575, 500)], 1).astype(np.float32)
    out, st, it = gpu_lk(omt, p.frame0, p.frame0, pts)
    ok = (st & OK) > 0
    assert ok.mean() > 0.9
    np.testing.assert_array_equal(out[ok], pts[ok])
    assert np.all(it[ok] == 1)


@pytest.mark.parametrize("win,levels", [(3, 1), (7, 2), (15, 4), (21, 5), (31, 5), (9, 8)])
def test_lk_window_and_level_sweep(omt, oracle, win, levels):
    rng = np.random.default_rng(win * 10 + levels)
    w, h = 331, 257
    tex = synth.Texture.draw(rng, w, h, n_blobs=24)
    f0 = synth.render_shift(tex, w, h)
    f1 = synth.render_shift(tex, w, h, 2.3, -1.7)
    pts = np.stack([rng.uniform(0, w - 1, 600), rng.uniform(0, h - 1, 600)], 1).astype(np.float32)
    compare(omt, oracle, f0, f1, pts, win=win, levels=levels, min_ok=0.5, max_unstable=0.12,
            label=f"random points, win {win}, {levels} levels")


def test_lk_borders_and_oob(omt, oracle):
    rng = np.random.default_rng(12)
    w, h = 96, 80
    tex = synth.Texture.low_frequency(rng, w + 40, h + 40)
    f0 = synth.render_shift(tex, w, h, 0, 0)
    f1 = synth.render_shift(tex, w, h, 6.0, -5.0)
    pts = np.concatenate([np.stack([rng.uniform(0, w - 1, 300), rng.uniform(0, h - 1, 300)], 1),
                          np.array([[w - 1, 3], [w - 2.5, h - 1], [0, 0], [95, 79]])]).astype(np.float32)
    compare(omt, oracle, f0, f1, pts, levels=2, win=11, min_ok=0.3, max_unstable=0.12,
            label="borders")


def test_lk_one_dimensional_texture_lost(omt):
    w, h = 96, 64
    x = np.arange(w, dtype=np.float64)
    f0 = synth.quantise(np.tile(128 + 80 * np.sin(2 * np.pi * x / 17.0), (h, 1)))
    f1 = synth.quantise(np.tile(128 + 80 * np.sin(2 * np.pi * (x - 1.3) / 17.0), (h, 1)))
    pts = np.stack([np.linspace(12, 80, 10), np.linspace(12, 50, 10)], 1).astype(np.float32)
    out, st, it = gpu_lk(omt, f0, f1, pts, levels=2, win=11)
    assert np.all(st == LOST_EIG)
    np.testing.assert_array_equal(out, pts)


def test_lk_empty_and_device_count(omt, oracle):
    p = synth.sd_pair()
    out, st, it = gpu_lk(omt, p.frame0, p.frame1, np.zeros((0, 2), np.float32))
    assert out.shape == (0, 2)
    # n_dev limits the work to the first points; the rest stay untouched
    params = omt.default_params()
    P0, P1 = _pyr(omt, p.frame0, 3), _pyr(omt, p.frame1, 3)
    pts = torch.tensor([[100.0, 100.0], [200.0, 300.0], [400.0, 50.0]], device="cuda")
    o = torch.full((3, 2), -1.0, device="cuda")
    s = torch.full((3,), 255, dtype=torch.uint8, device="cuda")
    n_dev = torch.tensor([2], dtype=torch.int32, device="cuda")
    omt.lk_track(P0, P1, pts, params, o, s, None, n_max=3, n_dev=n_dev)
    torch.cuda.synchronize()
    assert s[2].item() == 255 and o[2, 0].item() == -1.0
    assert (s[:2].cpu().numpy() & OK).all()


def test_lk_points_outside_the_input_domain(omt, oracle):
    # non-finite coordinates and coordinates beyond 2^24 px come back
    # LOST_OOB and unchanged, as in the oracle; the other points are unaffected
    p = synth.sd_pair()
    far = np.array([[np.nan, 10.0], [10.0, np.inf], [3.0e9, 5.0], [-3.0e9, -7.0e9], [1.0e20, 1.0],
                    [-16777300.0, 5.0]], np.float32)
    good = np.array([[100.0, 100.0], [200.0, 300.0]], np.float32)
    pts = np.concatenate([good[:1], far, good[1:]])
    out, st, it = gpu_lk(omt, p.frame0, p.frame1, pts)
    assert st[1:7].tolist() == [LOST_OOB] * 6
    assert np.all(it[1:7] == 0)
    np.testing.assert_array_equal(out[3:7], far[2:6])
    ref_out, ref_st, _ = gpu_lk(omt, p.frame0, p.frame1, good)
    np.testing.assert_array_equal(out[[0, 7]], ref_out)
    np.testing.assert_array_equal(st[[0, 7]], ref_st)
    o_out, o_st, _, _ = oracle_lk(oracle, p.frame0, p.frame1, far)
    assert o_st.tolist() == [LOST_OOB] * 6


def test_lk_batch_independence(omt):
    # a point's result does not depend on the launch shape or batch mates
    p = synth.sd_pair()
    rng = np.random.default_rng(9)
    pts = np.stack([rng.uniform(0, 719, 3000), rng.uniform(0, 575, 3000)], 1).astype(np.float32)
    full = gpu_lk(omt, p.frame0, p.frame1, pts)
    for sl in [slice(0, 1), slice(17, 400), slice(2999, 3000)]:
        part = gpu_lk(omt, p.frame0, p.frame1, pts[sl])
        for a, b in zip(full, part):
            np.testing.assert_array_equal(a[sl], b)


def test_lk_f16_storage_sd_pair(omt, oracle):
    # workload 1 (the SD pair, 3 levels, 21x21): the F16 path against the
    # oracle on half-precision storage at the FP32 bar, and the cost of the
    # storage against the FP64 oracle
    p = synth.sd_pair()
    pts, cnt = oracle.select_corners(p.frame0, p.boxes, 50)
    allp = np.concatenate([pts[i, :cnt[i]] for i in range(len(cnt))])
    g_out, g_st, _, _ = compare(omt, oracle, p.frame0, p.frame1, allp, storage=1,
                                label="SD pair corners")
    o_out, o_st = oracle_lk(oracle, p.frame0, p.frame1, allp)[:2]
    error_vs_fp64("SD pair, F16 storage", g_out, g_st, o_out, o_st, max_nonconv=0.05)


def test_lk_4k_large_motion_sample(omt, oracle):
    # workload 4 (3840x2160, 200 rigid regions moving up to 40 px and 3
    # degrees, 5 levels, 31x31): 3,000 sampled corners
    pr = synth.rigid_pair()
    pts, cnt = oracle.select_corners(pr.frame0, pr.boxes, 250)
    allp = np.concatenate([pts[i, :cnt[i]] for i in range(len(cnt))])
    rng = np.random.default_rng(1)
    sample = allp[rng.choice(len(allp), 3000, replace=False)]
    kw = dict(levels=5, win=31, max_iter=30, eps=0.01)
    o_out, o_st = oracle_lk(oracle, pr.frame0, pr.frame1, sample, **kw)[:2]
    stats = {}
    for storage in (0, 1):
        g_out, g_st, _, _ = compare(omt, oracle, pr.frame0, pr.frame1, sample, storage=storage,
                                    min_ok=0.5, label="4K sample", **kw)
        # against the FP64 oracle on unquantised pyramids; most NONCONV
        # points straddle two regions that move differently (their window's
        # translation model does not fit, the iteration oscillates)
        name = f"4K sample, {'F16' if storage else 'F32'} storage"
        stats[storage] = error_vs_fp64(name, g_out, g_st, o_out, o_st)
    # storing the pyramid in half precision costs accuracy
    assert stats[1]["mean"] >= stats[0]["mean"]


# ------------------------------------------------------------------ boxes

def _gpu_update(omt, boxes, off, pts, out, st, agg):
    params = omt.default_params(aggregator=agg)
    nb = len(boxes)
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dt)).cuda()
    bo = torch.empty((nb, 4), device="cuda")
    nv = torch.empty(nb, dtype=torch.int32, device="cuda")
    omt.update_boxes(t(boxes, np.float32), t(off, np.int32), t(pts.reshape(-1, 2), np.float32),
                     t(out.reshape(-1, 2), np.float32), t(st, np.uint8), params, bo, nv)
    torch.cuda.synchronize()
    return bo.cpu().numpy(), nv.cpu().numpy()


@pytest.mark.parametrize("agg", [0, 1, 2])
def test_update_boxes_matches_oracle(omt, oracle, agg):
    rng = np.random.default_rng(5 + agg)
    nb = 300
    counts = rng.integers(0, 400, nb)
    counts[:3] = [0, 1, 2]
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    n = int(off[-1])
    pts = rng.uniform(0, 3800, (n, 2)).astype(np.float32)
    out = (pts + rng.normal(0, 5, (n, 2))).astype(np.float32)
    st = rng.choice([OK, OK | NONCONV, LOST_EIG, LOST_OOB], n, p=[0.6, 0.1, 0.15, 0.15]).astype(np.uint8)
    boxes = rng.uniform(0, 3000, (nb, 4)).astype(np.float32)
    g, gn = _gpu_update(omt, boxes, off, pts, out, st, agg)
    o, on = oracle.update_boxes(boxes, off, pts, out, st, aggregator=agg)
    np.testing.assert_array_equal(gn, on)
    # agg 2: FP32 ratios against FP64 ones move the median scale by a few
    # ulps, times box half-sizes up to 1.5e3 px
    np.testing.assert_allclose(g, o, rtol=0, atol={0: 5e-4, 1: 1e-3, 2: 2e-3}[agg])
    if agg == 2:
        w = (g[:, 2] - g[:, 0]) / (boxes[:, 2] - boxes[:, 0])
        assert np.all(np.isclose(w[:2], 1.0)) and np.std(w[3:]) > 1e-4  # <2 points: scale 1


def test_update_boxes_scale_of_a_zoom(omt, oracle):
    # every box's points zoom by its own factor about the box centre
    rng = np.random.default_rng(21)
    nb, k = 40, 90
    boxes = np.zeros((nb, 4), np.float32)
    pts, out = [], []
    for b in range(nb):
        c = rng.uniform(200, 1800, 2)
        hw = rng.uniform(20, 120, 2)
        boxes[b] = [c[0] - hw[0], c[1] - hw[1], c[0] + hw[0], c[1] + hw[1]]
        u = c + rng.uniform(-1, 1, (k, 2)) * hw
        s = rng.uniform(0.7, 1.4)
        pts.append(u)
        out.append(c + s * (u - c) + rng.uniform(-5, 5, 2))
    pts = np.concatenate(pts).astype(np.float32)
    out = np.concatenate(out).astype(np.float32)
    off = (np.arange(nb + 1) * k).astype(np.int32)
    st = np.full(nb * k, OK, np.uint8)
    g, gn = _gpu_update(omt, boxes, off, pts, out, st, 2)
    o, on = oracle.update_boxes(boxes, off, pts, out, st, aggregator=2)
    np.testing.assert_array_equal(gn, on)
    np.testing.assert_allclose(g, o, rtol=0, atol=1e-3)


def test_update_boxes_hand_vectors(omt):
    boxes = np.array([[10, 20, 50, 70], [0, 0, 5, 5], [1, 1, 2, 2]], np.float32)
    pts = np.zeros((7, 2), np.float32) + 100
    d = np.array([[3, 5], [-1, 0], [2, -7], [1, 0], [4, 1], [2, 2], [10, 3]], np.float32)
    st = np.array([OK, OK, OK, OK, OK | NONCONV, LOST_EIG, OK], np.uint8)
    off = np.array([0, 3, 7, 7], np.int32)
    g, gn = _gpu_update(omt, boxes, off, pts, pts + d, st, 0)
    np.testing.assert_array_equal(gn, [3, 3, 0])
    np.testing.assert_array_equal(g[0], [12, 20, 52, 70])
    np.testing.assert_array_equal(g[1], [4, 1, 9, 6])
    np.testing.assert_array_equal(g[2], boxes[2])


# ------------------------------------------------------------ end to end

def test_stream_tracker_sd_step(omt, oracle):
    p = synth.sd_pair()
    params = omt.default_params()
    T = omt.StreamTracker(720, 576, params, max_boxes=16)
    T.prime(torch.from_numpy(p.frame0).cuda())
    boxes = torch.from_numpy(p.boxes).cuda()
    bo = T.step(torch.from_numpy(p.frame1).cuda(), boxes)
    torch.cuda.synchronize()
    # oracle pipeline on the same frames
    pts, cnt = oracle.select_corners(p.frame0, p.boxes, 50)
    allp = np.concatenate([pts[i, :cnt[i]] for i in range(len(cnt))])
    O0, O1 = oracle.Pyramid(p.frame0, 3), oracle.Pyramid(p.frame1, 3)
    o_out, o_st = oracle.lk_track(O0, O1, allp)
    off = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int32)
    o_b, o_nv = oracle.update_boxes(p.boxes, off, allp, o_out.astype(np.float32), o_st)
    np.testing.assert_array_equal(T.offsets[:len(p.boxes) + 1].cpu().numpy(), off)
    np.testing.assert_array_equal(T.pts[:off[-1]].cpu().numpy(), allp)
    np.testing.assert_array_equal(T.nvalid[:len(p.boxes)].cpu().numpy(), o_nv)
    np.testing.assert_allclose(bo.cpu().numpy(), o_b, rtol=0, atol=2e-3)
    assert np.abs(bo.cpu().numpy() - p.boxes - [1.37, -0.62, 1.37, -0.62]).max() <= 0.02


def test_1080p_clip_trajectory_matches_oracle(omt, oracle):
    # Section V-A loop on the whole 64-frame 1080p affine clip (workload 2):
    # detections every 5th frame, prediction in between; GPU and oracle box
    # trajectories must agree on every frame.
    n = 64
    clip = synth.affine_clip(n_frames=n)
    params = omt.default_params(levels=4, max_corners=100)
    T = omt.StreamTracker(1920, 1080, params, max_boxes=16)
    T.prime(torch.from_numpy(clip.frames[0]).cuda())
    gb = clip.gt_boxes[0].astype(np.float32)
    ob = gb.copy()
    worst = []
    for t in range(1, n):
        if (t - 1) % 5 == 0:
            gb = clip.gt_boxes[t - 1].astype(np.float32)
            ob = gb.copy()
        g = T.step(torch.from_numpy(clip.frames[t]).cuda(), torch.from_numpy(gb).cuda())
        torch.cuda.synchronize()
        gb = g.cpu().numpy().copy()
        pts, cnt = oracle.select_corners(clip.frames[t - 1], ob, 100)
        allp = np.concatenate([pts[i, :cnt[i]] for i in range(len(cnt))])
        O0, O1 = oracle.Pyramid(clip.frames[t - 1], 4), oracle.Pyramid(clip.frames[t], 4)
        o_out, o_st = oracle.lk_track(O0, O1, allp)
        off = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int32)
        ob, _ = oracle.update_boxes(ob, off, allp, o_out.astype(np.float32), o_st)
        ob = ob.astype(np.float32)
        worst.append(float(np.abs(gb - ob).max()))
        assert worst[-1] <= 0.05, (t, worst[-1])
    print(f"1080p clip, {n} frames: max box corner difference per frame: median "
          f"{np.median(worst):.2e} px, max {max(worst):.2e}")
