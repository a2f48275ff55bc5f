"""The batched path (omt_batch_step) against the plain per-stream calls.

Both run the same per-tile / per-box / per-point device code, so every
result must agree bit for bit: the new pyramids, the corner lists and
offsets, the tracked points, statuses and iteration counts, the boxes.
Also: a stream gives the same result alone as in a mix of streams, a CUDA
graph replay equals the eager step, and membership below the capacities
works.  The plain path is itself held to the oracle by the other tests.
"""
import math

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


def _streams(n, first=0):
    out = []
    for s in range(first, first + n):
        sp = synth.stream_pair(s, workload=13, n_range=(300, 3000))
        out.append(sp)
    # a stream with an empty box list and one with boxes off the frame
    return out


def _cap(sp):
    return int(math.ceil(sp.n_target / 64))


def _run_plain(omt, sps, params, boxes_list):
    res = []
    for sp, boxes in zip(sps, boxes_list):
        w, h = sp.size
        prm = params.replace(max_corners=_cap(sp))
        T = omt.StreamTracker(w, h, prm, max_boxes=max(1, len(boxes)))
        T.prime(torch.from_numpy(sp.frame0).cuda())
        b = torch.from_numpy(np.ascontiguousarray(boxes, np.float32)).cuda()
        nb = len(boxes)
        if nb:
            bo = T.step(torch.from_numpy(sp.frame1).cuda(), b)
        else:
            omt.build_pyramid(torch.from_numpy(sp.frame1).cuda(), T.pyr[1], prm)
            T.offsets.zero_()
            T.cur = 1
            bo = T.boxes_out[:0]
        torch.cuda.synchronize()
        n = int(T.offsets[nb].item()) if nb else 0
        res.append(dict(
            offsets=T.offsets[:nb + 1].cpu().numpy(), pts=T.pts[:n].cpu().numpy(),
            out=T.pts_out[:n].cpu().numpy(), st=T.status[:n].cpu().numpy(),
            it=T.iters[:n].cpu().numpy(), boxes=bo.cpu().numpy(),
            nvalid=T.nvalid[:nb].cpu().numpy(), pyr=T.pyr[1].buffer.cpu().numpy()))
    return res


def _make_batch(omt, sps, params, boxes_list, graph=False):
    sizes = [sp.size for sp in sps]
    B = omt.BatchTracker(sizes, params, max_boxes=[max(1, len(b)) for b in boxes_list],
                         max_corners=[_cap(sp) for sp in sps])
    for s, (sp, boxes) in enumerate(zip(sps, boxes_list)):
        B.prime(s, torch.from_numpy(sp.frame0).cuda())
        B.slot(s).copy_(torch.from_numpy(sp.frame1))
        B.set_boxes(s, torch.from_numpy(np.ascontiguousarray(boxes, np.float32)))
    B.pack()
    return B


def _batch_results(B, sps):
    res = []
    for s in range(len(sps)):
        nb = B.nboxes[s]
        n = B.count(s)
        res.append(dict(
            offsets=B.offsets[s][:nb + 1].cpu().numpy(), pts=B.pts[s][:n].cpu().numpy(),
            out=B.pts_out[s][:n].cpu().numpy(), st=B.status[s][:n].cpu().numpy(),
            it=B.iters[s][:n].cpu().numpy(), boxes=B.boxes_out[s][:nb].cpu().numpy(),
            nvalid=B.nvalid[s][:nb].cpu().numpy(),
            pyr=B.pyr[s][B.cur].buffer.cpu().numpy()))
    return res


def _assert_same(a, b, pyramids=True):
    for k in a:
        if k == "pyr" and not pyramids:
            continue
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


def _pyr_planes(omt, buf, w, h, levels, storage):
    """The payload of every plane of a pyramid buffer (pitch padding is
    never written, so only the planes are compared)."""
    import ctypes
    d = omt.PyramidDesc()
    n = omt.pyramid_bytes(w, h, levels, storage)
    assert omt.lib().omt_pyramid_init(ctypes.byref(d), w, h, levels, storage,
                                      ctypes.c_void_p(1 << 20), n) == 0  # layout only
    out = []
    for L in range(levels):
        lv = d.lv[L]
        esz = 1 if L == 0 else (4 if storage == 0 else 2)
        gsz = 8 if storage == 0 else 4
        out.append(buf[lv.img_off:lv.img_off + lv.img_pitch * lv.h].reshape(lv.h, lv.img_pitch)[:, :lv.w * esz])
        out.append(buf[lv.grad_off:lv.grad_off + lv.grad_pitch * lv.h].reshape(lv.h, lv.grad_pitch)[:, :lv.w * gsz])
    return out


@pytest.mark.parametrize("storage", [0, 1])
def test_batch_equals_plain_bitwise(omt, storage):
    sps = _streams(6)
    boxes_list = [sp.boxes for sp in sps]
    boxes_list[2] = np.zeros((0, 4), np.float32)  # a stream with no boxes
    boxes_list[3] = np.concatenate([sps[3].boxes, [[5000, 5000, 5100, 5100], [-40, -40, -10, -10]]]).astype(np.float32)
    params = omt.default_params(levels=4, win=21, min_dist=3.0, storage=storage,
                                max_corners=max(_cap(sp) for sp in sps))
    plain = _run_plain(omt, sps, params, boxes_list)
    B = _make_batch(omt, sps, params, boxes_list)
    B.step()
    torch.cuda.synchronize()
    got = _batch_results(B, sps)
    for s, (a, b) in enumerate(zip(plain, got)):
        w, h = sps[s].size
        _assert_same({k: v for k, v in a.items() if k != "pyr"}, {k: v for k, v in b.items() if k != "pyr"})
        for x, y in zip(_pyr_planes(omt, a["pyr"], w, h, 4, storage), _pyr_planes(omt, b["pyr"], w, h, 4, storage)):
            np.testing.assert_array_equal(x, y)
    assert sum(len(r["st"]) for r in got) > 1000


def test_alone_equals_in_the_mix(omt):
    sps = _streams(5, first=20)
    params = omt.default_params(levels=4, win=21, min_dist=3.0,
                                max_corners=max(_cap(sp) for sp in sps))
    boxes_list = [sp.boxes for sp in sps]
    B = _make_batch(omt, sps, params, boxes_list)
    B.step()
    torch.cuda.synchronize()
    mix = _batch_results(B, sps)
    for s in (0, 3):
        A = _make_batch(omt, [sps[s]], params, [boxes_list[s]])
        A.step()
        torch.cuda.synchronize()
        alone = _batch_results(A, [sps[s]])[0]
        _assert_same({k: v for k, v in alone.items() if k != "pyr"},
                     {k: v for k, v in mix[s].items() if k != "pyr"})


def test_graph_replay_equals_eager(omt):
    sps = _streams(4, first=40)
    params = omt.default_params(levels=4, win=21, min_dist=3.0, storage=1,
                                max_corners=max(_cap(sp) for sp in sps))
    boxes_list = [sp.boxes for sp in sps]
    E = _make_batch(omt, sps, params, boxes_list)
    G = _make_batch(omt, sps, params, boxes_list)
    G.step()             # one eager step before capture (library one-time setup)
    for s, sp in enumerate(sps):      # rewind G to frame 0 -> 1
        G.cur = 0
        G.prime(s, torch.from_numpy(sp.frame0).cuda())
    torch.cuda.synchronize()
    G.capture()
    for k in range(3):
        for s, sp in enumerate(sps):
            f = sp.frame1 if k % 2 == 0 else sp.frame0
            E.slot(s).copy_(torch.from_numpy(f))
            G.slot(s).copy_(torch.from_numpy(f))
        E.step()
        G.step()
        torch.cuda.synchronize()
        for a, b in zip(_batch_results(E, sps), _batch_results(G, sps)):
            _assert_same({k2: v for k2, v in a.items() if k2 != "pyr"},
                         {k2: v for k2, v in b.items() if k2 != "pyr"})


def test_membership_below_capacity(omt):
    sps = _streams(3, first=60)
    params = omt.default_params(levels=3, win=15, min_dist=3.0,
                                max_corners=max(_cap(sp) for sp in sps))
    boxes_list = [sp.boxes for sp in sps]
    plain = _run_plain(omt, sps, params, boxes_list)
    sizes = [sp.size for sp in sps] + [(1920, 1080)]
    B = omt.BatchTracker(sizes, params, max_boxes=[64, 64, 64, 64],
                         max_corners=[_cap(sp) for sp in sps] + [10])
    for s, sp in enumerate(sps):
        B.prime(s, torch.from_numpy(sp.frame0).cuda())
        B.slot(s).copy_(torch.from_numpy(sp.frame1))
        B.set_boxes(s, torch.from_numpy(sp.boxes))
    # the fourth stream exists in the capacities but has nothing to track
    B.set_boxes(3, torch.zeros((0, 4)))
    B.prime(3, B.slot(3))
    B.pack()
    B.step()
    torch.cuda.synchronize()
    got = _batch_results(B, sps)
    for a, b in zip(plain, got):
        _assert_same({k: v for k, v in a.items() if k != "pyr"}, {k: v for k, v in b.items() if k != "pyr"})


def test_run_pipelined_equals_stepwise(omt):
    """Frames uploaded on a copy stream while the previous step computes give
    the same boxes as copying each step's frames before it runs."""
    sps = _streams(3, first=80)
    params = omt.default_params(levels=4, win=21, min_dist=3.0, storage=1,
                                max_corners=max(_cap(sp) for sp in sps))
    boxes_list = [sp.boxes for sp in sps]
    A = _make_batch(omt, sps, params, boxes_list)
    P = _make_batch(omt, sps, params, boxes_list)
    fr = [(torch.from_numpy(sp.frame1).pin_memory(), torch.from_numpy(sp.frame0).pin_memory())
          for sp in sps]
    want = []
    for k in range(5):
        for s in range(len(sps)):
            A.slot(s).copy_(fr[s][k & 1])
        A.step()
        torch.cuda.synchronize()
        want.append([A.boxes_out[s][:len(sps[s].boxes)].cpu().numpy() for s in range(len(sps))])
    got = {}
    h2d, d2h = P.run_pipelined(lambda k: [fr[s][k & 1] for s in range(len(sps))], 5,
                               consume=lambda k, b: got.__setitem__(k, [x.numpy().copy() for x in b]))
    assert sorted(got) == list(range(5))
    for k in range(5):
        for s in range(len(sps)):
            np.testing.assert_array_equal(got[k][s], want[k][s])
    assert h2d == 5 * sum(sp.size[0] * sp.size[1] for sp in sps)


def test_lk_launch_shape_does_not_change_results(omt):
    """Every launch shape the tuner may pick (LK warps per CTA and
    work-queue chunk; CTAs per SM of the pyramid, corner-list and select
    kernels) gives the same pyramids, corners, points, statuses, iterations
    and boxes bit for bit, and autotune keeps one of its candidates."""
    sps = _streams(4, first=100)
    params = omt.default_params(levels=4, win=21, min_dist=3.0, storage=1,
                                max_corners=max(_cap(sp) for sp in sps))
    boxes_list = [sp.boxes for sp in sps]
    ref = None
    for warps, chunk, pyr, lst, sel in [(4, 1, 0, 0, 0), (2, 4, 1, 1, 1), (8, 2, 2, 8, 4),
                                        (1, 16, 4, 4, 2)]:
        B = _make_batch(omt, sps, params, boxes_list)
        B.caps.lk_warps, B.caps.lk_chunk = warps, chunk
        B.caps.pyr_ctas_per_sm, B.caps.corner_ctas_per_sm, B.caps.select_ctas_per_sm = pyr, lst, sel
        B.step()
        torch.cuda.synchronize()
        got = _batch_results(B, sps)
        if ref is None:
            ref = got
        else:
            for a, b, sp in zip(ref, got, sps):
                _assert_same(a, b, pyramids=False)
                w, h = sp.size
                for x, y in zip(_pyr_planes(omt, a["pyr"], w, h, 4, 1),
                                _pyr_planes(omt, b["pyr"], w, h, 4, 1)):
                    np.testing.assert_array_equal(x, y)
    B = _make_batch(omt, sps, params, boxes_list)
    times = B.autotune(reps=2)
    assert (B.caps.lk_warps, B.caps.lk_chunk) in times["lk"] and min(times["lk"].values()) > 0
    assert B.caps.pyr_ctas_per_sm in times["pyramid"] and min(times["pyramid"].values()) > 0
    assert (B.caps.corner_ctas_per_sm, B.caps.select_ctas_per_sm) in times["corners"]
    B.step()
    torch.cuda.synchronize()
    for a, b in zip(ref, _batch_results(B, sps)):
        _assert_same({k: v for k, v in a.items() if k != "pyr"}, {k: v for k, v in b.items() if k != "pyr"})


@pytest.mark.parametrize("storage", [0, 1])
def test_batch_equals_plain_win31_five_levels(omt, storage):
    """The largest window (31x31) and five levels, as for 3840x2160 frames,
    through the batched path (whose launch clamps the warps per CTA to the
    shared memory their staging areas need) equal the plain calls."""
    sps = _streams(3, first=120)
    boxes_list = [sp.boxes for sp in sps]
    params = omt.default_params(levels=5, win=31, min_dist=3.0, storage=storage,
                                max_corners=max(_cap(sp) for sp in sps))
    plain = _run_plain(omt, sps, params, boxes_list)
    for warps in (4, 8):
        B = _make_batch(omt, sps, params, boxes_list)
        B.caps.lk_warps, B.caps.lk_chunk = warps, 2
        B.step()
        torch.cuda.synchronize()
        for a, b in zip(plain, _batch_results(B, sps)):
            _assert_same({k: v for k, v in a.items() if k != "pyr"}, {k: v for k, v in b.items() if k != "pyr"})


@pytest.mark.slow
def test_bench_workload_f16_step_against_oracle(omt, oracle):
    """The benchmark's step itself (workload 3: 32 streams, 221 k corners,
    4 levels, 21x21, F16-stored pyramids, one CUDA-graph replay of
    omt_batch_step) against the oracle: every stream's corner list bit for
    bit, then a seeded 5 % sample of the points tracked -- against the
    oracle on half-precision storage at the FP32 bar, and against the FP64
    oracle on unquantised pyramids as the error of the storage."""
    from lk_parity import check, error_vs_fp64, oracle_lk
    sps = [synth.stream_pair(s) for s in range(32)]
    caps = [_cap(sp) for sp in sps]
    params = omt.default_params(levels=4, win=21, max_iter=30, eps=0.01, min_dist=3.0,
                                storage=1, max_corners=max(caps))
    B = omt.BatchTracker([sp.size for sp in sps], params, max_boxes=[len(sp.boxes) for sp in sps],
                         max_corners=caps)
    for s, sp in enumerate(sps):
        B.prime(s, torch.from_numpy(sp.frame0).cuda())
        B.slot(s).copy_(torch.from_numpy(sp.frame1))
        B.set_boxes(s, torch.from_numpy(sp.boxes))
    B.pack()
    B.capture()
    B.step()
    torch.cuda.synchronize()
    rng = np.random.default_rng(synth.seed_for(3))
    cols = {k: [] for k in ("g_out", "g_st", "g_it", "pts", "o_out", "o_st", "o_it", "o_me",
                            "unstable", "d_out", "d_st")}
    total = 0
    for s, sp in enumerate(sps):
        n = B.count(s)
        total += n
        g_pts = B.pts[s][:n].cpu().numpy()
        pts, cnt = oracle.select_corners(sp.frame0, sp.boxes, caps[s], min_dist=3.0)
        np.testing.assert_array_equal(B.offsets[s][:len(sp.boxes) + 1].cpu().numpy(),
                                      np.concatenate([[0], np.cumsum(cnt)]))
        allp = np.concatenate([pts[i, :cnt[i]] for i in range(len(cnt))])
        np.testing.assert_array_equal(g_pts, allp)
        pick = np.sort(rng.choice(n, int(round(0.05 * n)), replace=False))
        sample = allp[pick]
        kw = dict(levels=4, win=21, max_iter=30, eps=0.01)
        (o_out, o_st, o_it, o_me), unstable = oracle_lk(oracle, sp.frame0, sp.frame1, sample,
                                                        probe=True, storage=1, **kw)
        d_out, d_st = oracle_lk(oracle, sp.frame0, sp.frame1, sample, **kw)[:2]
        for k, v in (("g_out", B.pts_out[s][:n].cpu().numpy()[pick]),
                     ("g_st", B.status[s][:n].cpu().numpy()[pick]),
                     ("g_it", B.iters[s][:n].cpu().numpy()[pick]), ("pts", sample),
                     ("o_out", o_out), ("o_st", o_st), ("o_it", o_it), ("o_me", o_me),
                     ("unstable", unstable), ("d_out", d_out), ("d_st", d_st)):
            cols[k].append(v)
    c = {k: np.concatenate(v) for k, v in cols.items()}
    assert total == 221227, total
    # every stream's points lie in its own frame: validity per stream is
    # covered by check() with the largest frame's bounds
    check(f"32-stream batched F16 step, 5 % sample ({len(c['pts'])} of {total})", c["g_out"],
          c["g_st"], c["g_it"], c["pts"], (1080, 1920), c["o_out"], c["o_st"], c["o_it"],
          c["o_me"], c["unstable"], 1e-3, 0.01)
    error_vs_fp64("32-stream batched F16 step, 5 % sample", c["g_out"], c["g_st"], c["d_out"],
                  c["d_st"], max_nonconv=0.2)


def test_lk_staging_waits_never_time_out(omt):
    # every window copy of the LK kernels above landed within its wait limit
    torch.cuda.synchronize()
    assert omt.lk_wait_timeouts() == 0
    assert omt.lk_wait_timeouts() == 0  # the read restarts the count


def test_candidate_list_overflow_in_the_batch(omt, oracle):
    """A box with more than 1,024 candidate corners (noise of full amplitude,
    quality 0: every positive local maximum is a candidate) overflows its
    candidate list: the batched step then selects it through the response
    map of the strips that touch it, and still equals the plain calls bit
    for bit.  The next step, without that box, equals the plain calls too
    (the step-wide overflow word is reset)."""
    from paper_1910_06017_b300.synth import StreamPair
    rng = np.random.default_rng(77)
    base = synth.stream_pair(3, workload=13, n_range=(300, 3000))
    f0 = base.frame0.copy()
    f0[40:260, 60:360] = rng.integers(0, 256, size=(220, 300)).astype(np.uint8)
    box = [60, 40, 360, 260]
    R = oracle.corner_response(f0)
    Rc = R[1:-1, 1:-1]
    nb = np.stack([R[1 + dy:R.shape[0] - 1 + dy, 1 + dx:R.shape[1] - 1 + dx]
                   for dy in (-1, 0, 1) for dx in (-1, 0, 1)]).max(axis=0)
    lm = np.zeros_like(R, bool)
    lm[1:-1, 1:-1] = (Rc >= nb) & (Rc > 0)
    assert lm[40:260, 60:360].sum() > 1024   # more candidates than a list holds
    noisy = StreamPair(f0, base.frame1, np.concatenate([base.boxes[:20], [box]]).astype(np.float32),
                       base.n_target, base.size)
    sps = _streams(2, first=60) + [noisy]
    params = omt.default_params(levels=4, win=21, min_dist=0.0, storage=1, quality=(0, 1),
                                max_corners=max(_cap(sp) for sp in sps))
    boxes_list = [sp.boxes for sp in sps]
    plain = _run_plain(omt, sps, params, boxes_list)
    B = _make_batch(omt, sps, params, boxes_list)
    B.step()
    torch.cuda.synchronize()
    for a, b in zip(plain, _batch_results(B, sps)):
        _assert_same(a, b, pyramids=False)
    # second step (frame 1 -> frame 0 in the other slot): the noisy box is gone
    boxes2 = [sp.boxes for sp in sps[:2]] + [noisy.boxes[:20]]
    for s, (sp, b) in enumerate(zip(sps, boxes2)):
        B.slot(s).copy_(torch.from_numpy(sp.frame0))
        B.set_boxes(s, torch.from_numpy(np.ascontiguousarray(b, np.float32)))
    B.pack()
    B.step()
    torch.cuda.synchronize()
    back = [StreamPair(sp.frame1, sp.frame0, b, sp.n_target, sp.size) for sp, b in zip(sps, boxes2)]
    plain2 = _run_plain(omt, back, params, boxes2)
    for a, b in zip(plain2, _batch_results(B, back)):
        _assert_same(a, b, pyramids=False)
