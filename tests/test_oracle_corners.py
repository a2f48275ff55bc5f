"""Pins of the oracle's Shi-Tomasi response and corner selection.

The response is checked against math.isqrt, scipy's convolution of the same
Scharr kernel and numpy's symmetric eigensolver; the selection against a
naive repeated-extraction re-implementation on tiny boxes and against images
whose corners are known by construction.
"""
import math

import numpy as np
import pytest
import scipy.ndimage as ndi

from paper_1910_06017_b300 import synth

SCHARR_X = np.array([[-3, 0, 3], [-10, 0, 10], [-3, 0, 3]], dtype=np.int64)


def test_isqrt_against_math(oracle):
    rng = np.random.default_rng(3)
    vals = [0, 1, 2, 3, 4, 15, 16, 17, (1 << 57) - 1, 1 << 57, (1 << 62)]
    for s in [1, 2, 1000, 46340, 3 << 20, (1 << 31) - 1, 1 << 31, 3037000499]:
        vals += [s * s - 1, s * s, s * s + 1]
    vals += [int(v) for v in rng.integers(0, 1 << 62, 2000, dtype=np.int64)]
    for v in vals:
        assert oracle.isqrt(v) == math.isqrt(v), v


def _raw_scharr_lib(f):
    fi = f.astype(np.int64)
    return (ndi.correlate(fi, SCHARR_X, mode="mirror"),
            ndi.correlate(fi, SCHARR_X.T, mode="mirror"))


def _response_independent(f):
    gx, gy = _raw_scharr_lib(f)
    box = np.ones((3, 3), np.int64)
    a = ndi.correlate(gx * gx, box, mode="mirror")
    b = ndi.correlate(gx * gy, box, mode="mirror")
    c = ndi.correlate(gy * gy, box, mode="mirror")
    R = np.zeros(f.shape, np.int64)
    for idx in np.ndindex(f.shape):
        A, B, C = int(a[idx]), int(b[idx]), int(c[idx])
        R[idx] = (A + C) - math.isqrt((A - C) ** 2 + 4 * B * B)
    return R, a, b, c


def test_scharr_raw_matches_library(oracle):
    rng = np.random.default_rng(5)
    for shape in [(17, 23), (2, 9), (40, 3)]:
        f = rng.integers(0, 256, shape, dtype=np.uint8)
        gx, gy = oracle.scharr_raw(f)
        lx, ly = _raw_scharr_lib(f)
        np.testing.assert_array_equal(gx, lx)
        np.testing.assert_array_equal(gy, ly)


def test_response_is_twice_lambda_min(oracle):
    rng = np.random.default_rng(9)
    f = rng.integers(0, 256, (31, 37), dtype=np.uint8)
    R = oracle.corner_response(f)
    Ri, a, b, c = _response_independent(f)
    np.testing.assert_array_equal(R, Ri)
    M = np.stack([np.stack([a, b], -1), np.stack([b, c], -1)], -2).astype(np.float64)
    lam = np.linalg.eigvalsh(M)[..., 0]
    slack = 1e-6 * np.maximum(1.0, (a + c))
    assert np.all(R >= 2 * lam - slack)
    assert np.all(R < 2 * lam + 1 + slack)
    assert np.all(R >= 0)


@pytest.mark.parametrize("kind", ["grating_x", "diagonal_ramp"])
def test_rank_one_images_have_no_corners(oracle, kind):
    # A rank-1 gradient field (I = f(x), or I = x + y) has b^2 = a c, so the
    # response vanishes wherever the 5x5 support stays off the reflected border.
    h, w = 48, 64
    y, x = np.mgrid[0:h, 0:w]
    if kind == "grating_x":
        f = np.clip(np.floor(128 + 90 * np.sin(2 * np.pi * x / 13.0) + 0.5), 0, 255).astype(np.uint8)
    else:
        f = (x + y + 20).astype(np.uint8)
    R = oracle.corner_response(f)
    assert np.all(R[2:-2, 2:-2] == 0)
    boxes = np.array([[3, 3, w - 3, h - 3], [5.5, 3.25, 40, 30]], np.float32)
    pts, cnt = oracle.select_corners(f, boxes, 50)
    assert cnt.tolist() == [0, 0]


def test_square_corners(oracle):
    f = np.zeros((64, 64), np.uint8)
    f[20:44, 20:44] = 200
    pts, cnt = oracle.select_corners(f, np.array([[0, 0, 64, 64]], np.float32), 10, min_dist=5)
    assert cnt[0] == 4
    got = sorted(map(tuple, pts[0, :4].tolist()))
    want = [(19.5, 19.5), (19.5, 43.5), (43.5, 19.5), (43.5, 43.5)]
    for g, t in zip(got, want):
        assert abs(g[0] - t[0]) <= 1.0 and abs(g[1] - t[1]) <= 1.0, (got, want)


def test_checkerboard_crossings(oracle):
    n = 10
    y, x = np.mgrid[0:80, 0:80]
    f = np.where(((x // n) + (y // n)) % 2 == 0, 40, 210).astype(np.uint8)
    pts, cnt = oracle.select_corners(f, np.array([[5, 5, 75, 75]], np.float32), 100, min_dist=5)
    c = int(cnt[0])
    assert c == 49
    p = pts[0, :c]
    # every crossing lies between pixels k*n - 1 and k*n
    near = np.abs(p - (np.round((p + 0.5) / n) * n - 0.5))
    assert np.all(near <= 1.0)
    cells = {tuple(np.round((q + 0.5) / n).astype(int)) for q in p}
    assert len(cells) == 49


def _naive_select(R, w, h, box, cap, qnum, qden, min_dist):
    """Repeated extraction: take the best remaining candidate (R desc, raster
    index asc) that keeps min_dist to those taken, until cap or none left."""
    x0, y0, x1, y1 = [float(v) for v in box]
    elig = [(x, y) for y in range(1, h - 1) for x in range(1, w - 1)
            if x0 <= x < x1 and y0 <= y < y1]
    rmax = max([int(R[y, x]) for x, y in elig], default=0)
    cands = []
    for x, y in elig:
        r = int(R[y, x])
        if r <= 0 or qden * r <= qnum * rmax:
            continue
        if all(r >= int(R[y + dy, x + dx]) for dy in (-1, 0, 1) for dx in (-1, 0, 1)):
            cands.append((x, y, r))
    t = float(np.float32(min_dist) * np.float32(min_dist))
    taken = []
    remaining = list(cands)
    while remaining and len(taken) < cap:
        best = None
        for c in remaining:
            if best is None or c[2] > best[2] or (c[2] == best[2] and c[1] * w + c[0] < best[1] * w + best[0]):
                best = c
        remaining.remove(best)
        if all((best[0] - a) ** 2 + (best[1] - b) ** 2 >= t for a, b in taken):
            taken.append((best[0], best[1]))
    return taken


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_selection_matches_naive(oracle, seed):
    rng = np.random.default_rng(100 + seed)
    w, h = 48, 40
    tex = synth.Texture.draw(rng, w, h, n_blobs=12, sigma=(2.0, 6.0), period=(5.0, 12.0))
    X, Y = synth.pixel_grid(w, h)
    f = synth.quantise(tex.evaluate(X, Y))
    Rind, *_ = _response_independent(f)
    boxes = np.array([[0, 0, w, h], [3.5, 2.0, 30.0, 25.5], [10.0, 10.0, 10.0, 20.0],
                      [-5, -5, 20.25, 18.75], [30, 20, 60, 60]], np.float32)
    for cap, q, md in [(8, (1, 100), 5.0), (50, (1, 4), 3.0), (3, (1, 100), 0.0), (20, (0, 1), 2.5)]:
        pts, cnt = oracle.select_corners(f, boxes, cap, quality=q, min_dist=md)
        for b in range(len(boxes)):
            want = _naive_select(Rind, w, h, boxes[b], cap, q[0], q[1], md)
            got = [tuple(map(int, p)) for p in pts[b, :cnt[b]].tolist()]
            assert got == want, (b, cap, q, md)
    # an empty box selects nothing
    assert cnt[2] == 0
