"""Pins of the oracle's forward-backward consistency check.

The decision itself is pinned by hand vectors (status kept, status set to
LOST_FB, the threshold's closed end, lost forward runs untouched).  The
composition with the tracker is pinned by exact zero round trips on
identical frames, round trips that close to well under a tenth of a pixel
on a rendered sub-pixel shift, and an occluded region whose points cannot
come back while the rest of the frame does.
"""
import numpy as np

from paper_1910_06017_b300 import synth

OK, LOST_EIG, LOST_OOB, NONCONV, LOST_FB = 1, 2, 4, 8, 16


def test_fb_check_hand_vectors(oracle):
    pts = np.array([[10, 10], [10, 10], [10, 10], [10, 10], [10, 10], [5, 5], [5, 5],
                    [7.5, 2.25]], np.float32)
    back = np.array([[10.375, 10.5],  # |e| = 0.625 exactly: closes at fb_max 0.625
                     [10.375, 10.5 + 2.0 ** -20],  # just beyond
                     [10.0, 10.0],    # exact return, but the backward run was lost
                     [13.0, 14.0],    # far
                     [10.0, 10.25],   # NONCONV forward point that closes
                     [50.0, 50.0],    # forward lost: untouched
                     [5.0, 5.0],      # forward lost (OOB): untouched
                     [7.5, 2.25]], np.float64)
    sb = np.array([OK, OK, LOST_EIG, OK, OK | NONCONV, OK, OK, OK], np.uint8)
    st = np.array([OK, OK, OK, OK, OK | NONCONV, LOST_EIG, LOST_OOB, OK | NONCONV], np.uint8)
    got = oracle.fb_check(pts, back, sb, st, 0.625)
    assert got.tolist() == [OK, LOST_FB, LOST_FB, LOST_FB, OK | NONCONV, LOST_EIG, LOST_OOB,
                            OK | NONCONV]
    # fb_max = 0 keeps only exact returns
    got0 = oracle.fb_check(pts, back, sb, st, 0.0)
    assert got0.tolist() == [LOST_FB] * 5 + [LOST_EIG, LOST_OOB, OK | NONCONV]
    # the input statuses are not modified in place
    assert st.tolist()[0] == OK


def test_identical_frames_round_trip_is_exact(oracle):
    p = synth.sd_pair()
    P = oracle.Pyramid(p.frame0, 3)
    pts, cnt = oracle.select_corners(p.frame0, p.boxes, 50)
    allp = np.concatenate([pts[i, :cnt[i]] for i in range(len(cnt))])
    out, st, back, sb = oracle.lk_track_fb(P, P, allp, 0.0, win=21, max_iter=30, eps=0.01,
                                           min_eig=1e-3)
    ok = (st & OK) > 0
    assert ok.mean() > 0.95
    # zero flow both ways: the round trip closes exactly, even at fb_max 0
    np.testing.assert_array_equal(back[ok], allp[ok].astype(np.float64))
    assert not np.any(st == LOST_FB)


def test_subpixel_shift_round_trips_close(oracle):
    p = synth.sd_pair(low_frequency=True, quantised=False)
    P0, P1 = oracle.Pyramid(p.frame0, 3), oracle.Pyramid(p.frame1, 3)
    pts, cnt = oracle.select_corners(np.clip(np.floor(p.frame0 + 0.5), 0, 255).astype(np.uint8),
                                     p.boxes, 50)
    allp = np.concatenate([pts[i, :cnt[i]] for i in range(len(cnt))])
    out, st, back, sb = oracle.lk_track_fb(P0, P1, allp, 0.1, win=21, max_iter=30, eps=0.01,
                                           min_eig=1e-3)
    fwd_ok = (sb & OK) > 0
    e = np.hypot(*(back - allp).T)
    kept = (st & OK) > 0
    assert kept.mean() > 0.9
    # every kept point closes within the threshold; the shift is recovered
    assert np.all(e[kept] <= 0.1)
    assert np.median(e[kept]) < 0.01
    d = out[kept] - allp[kept]
    assert np.allclose(np.median(d, axis=0), p.shift, atol=0.01)
    assert fwd_ok.sum() >= kept.sum()


def test_occluded_region_fails_the_round_trip(oracle):
    # frame 1: the whole frame moves by (2, 1) px, except a square whose
    # content is replaced by an unrelated texture (an occluder)
    rng = np.random.default_rng(7)
    w, h = 320, 240
    tex = synth.Texture.draw(rng, w, h)
    other = synth.Texture.draw(np.random.default_rng(8), w, h)
    f0 = synth.render_shift(tex, w, h, 0.0, 0.0)
    f1 = synth.render_shift(tex, w, h, 2.0, 1.0)
    occ = (slice(80, 170), slice(100, 210))
    f1[occ] = synth.render_shift(other, w, h, 0.0, 0.0)[occ]
    P0, P1 = oracle.Pyramid(f0, 3), oracle.Pyramid(f1, 3)
    pts, cnt = oracle.select_corners(f0, np.array([[0, 0, w, h]], np.float32), 400, min_dist=4.0)
    allp = pts[0, :cnt[0]]
    out, st, back, sb = oracle.lk_track_fb(P0, P1, allp, 0.5, win=15, max_iter=30, eps=0.01,
                                           min_eig=1e-3)
    # points well inside the occluder, and well away from it (window reach)
    x, y = allp[:, 0], allp[:, 1]
    inside = (x > 115) & (x < 195) & (y > 95) & (y < 155)
    outside = (x < 80) | (x > 230) | (y < 60) | (y > 190)
    assert inside.sum() >= 20 and outside.sum() >= 100
    fb = st == LOST_FB
    assert fb[inside].mean() > 0.5
    assert fb[outside].mean() < 0.05
