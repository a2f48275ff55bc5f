"""Pins of the oracle's pyramid and gradients (Section V-A preprocessing).

Each check ties the oracle to something other than itself: closed forms of
the binomial reduce and the Scharr derivative on polynomials, dyadic
exactness, and library convolutions of the same definitions.
"""
import numpy as np
import pytest
import scipy.ndimage as ndi

K5 = np.array([1.0, 4.0, 6.0, 4.0, 1.0])
SCHARR_X = np.array([[-3.0, 0.0, 3.0], [-10.0, 0.0, 10.0], [-3.0, 0.0, 3.0]])


def test_level_sizes(oracle):
    got = [oracle.level_size(37, 23, L) for L in range(5)]
    assert got == [(37, 23), (19, 12), (10, 6), (5, 3), (3, 2)]
    assert oracle.level_size(1, 1, 4) == (1, 1)


@pytest.mark.parametrize("n", [2, 3, 4, 5, 7])
def test_reflect101_matches_numpy_reflect(oracle, n):
    # numpy's 'reflect' pad mirrors about the edge sample without repeating it
    pad = 3 * n
    ref = np.pad(np.arange(n), pad, mode="reflect")
    for i in range(-pad, n + pad):
        assert oracle.reflect101(i, n) == ref[i + pad]
    assert oracle.reflect101(-3, 1) == 0


def test_constant_image(oracle):
    f = np.full((23, 37), 77, np.uint8)
    P = oracle.Pyramid(f, 4)
    for L in range(4):
        assert np.all(P.img[L] == 77.0)
        assert np.all(P.grad[L] == 0.0)


def test_affine_ramp(oracle):
    h, w = 30, 40
    y, x = np.mgrid[0:h, 0:w]
    f = (3 * x + 2 * y + 5).astype(np.uint8)
    P = oracle.Pyramid(f, 3)
    # level 0 interior: Ix = alpha, Iy = beta exactly
    assert np.all(P.grad[0][1:-1, 1:-1, 0] == 3.0)
    assert np.all(P.grad[0][1:-1, 1:-1, 1] == 2.0)
    # level 1 interior (5-tap support inside the image): 2 alpha X + 2 beta Y + gamma
    l1 = P.img[1]
    Y, X = np.mgrid[0:l1.shape[0], 0:l1.shape[1]]
    inner = (2 * X - 2 >= 0) & (2 * X + 2 <= w - 1) & (2 * Y - 2 >= 0) & (2 * Y + 2 <= h - 1)
    assert np.all(l1[inner] == (6 * X + 4 * Y + 5)[inner])
    # level-1 gradient interior (stencil on interior level-1 values): 2 alpha, 2 beta
    g1 = P.grad[1]
    inner2 = inner & np.roll(inner, 1, 0) & np.roll(inner, -1, 0) & np.roll(inner, 1, 1) & np.roll(inner, -1, 1)
    inner2[0, :] = inner2[-1, :] = False
    inner2[:, 0] = inner2[:, -1] = False
    assert inner2.sum() > 10
    assert np.all(g1[inner2][:, 0] == 6.0) and np.all(g1[inner2][:, 1] == 4.0)


def test_quadratic_closed_forms(oracle):
    # I = x^2: the binomial reduce adds sum k_i i^2 / 16 = 1 per unit of the
    # quadratic coefficient, so level 1 = 4 X^2 + 1 and level 2 = 16 Y^2 + 5;
    # the Scharr derivative of x^2 is exactly 2x.
    h, w = 16, 64
    x = np.tile(np.arange(w, dtype=np.float64), (h, 1))
    P = oracle.Pyramid(x * x, 3)
    X1 = np.arange(P.img[1].shape[1])
    ok1 = (2 * X1 - 2 >= 0) & (2 * X1 + 2 <= w - 1)
    assert np.all(P.img[1][:, ok1] == (4.0 * X1 * X1 + 1.0)[ok1])
    X2 = np.arange(P.img[2].shape[1])
    w1 = P.img[1].shape[1]
    ok2 = (2 * X2 - 2 >= 1) & (2 * X2 + 2 <= w1 - 2) & (4 * X2 + 6 <= w - 1)
    assert ok2.sum() >= 3
    assert np.all(P.img[2][:, ok2] == (16.0 * X2 * X2 + 5.0)[ok2])
    assert np.all(P.grad[0][:, 1:-1, 0] == 2.0 * x[:, 1:-1])
    assert np.all(P.grad[0][:, :, 1] == 0.0)


def test_bilinear_product_gradient(oracle):
    # I = x y: Ix = y and Iy = x in the interior (smoothing keeps linear terms)
    h, w = 20, 24
    y, x = np.mgrid[0:h, 0:w].astype(np.float64)
    P = oracle.Pyramid(x * y, 1)
    assert np.all(P.grad[0][1:-1, 1:-1, 0] == y[1:-1, 1:-1])
    assert np.all(P.grad[0][1:-1, 1:-1, 1] == x[1:-1, 1:-1])


def test_dyadic_exactness(oracle):
    rng = np.random.default_rng(7)
    f = rng.integers(0, 256, (41, 53), dtype=np.uint8)
    P = oracle.Pyramid(f, 5)
    for L in range(5):
        v = P.img[L] * 2.0 ** (8 * L)
        assert np.all(v == np.round(v)), L
        assert P.img[L].min() >= 0.0 and P.img[L].max() <= 255.0


@pytest.mark.parametrize("shape", [(41, 53), (9, 6), (64, 64), (3, 5)])
def test_matches_library_convolution(oracle, shape):
    rng = np.random.default_rng(11)
    f = rng.integers(0, 256, shape, dtype=np.uint8)
    levels = 3
    P = oracle.Pyramid(f, levels)
    k2 = np.outer(K5, K5) / 256.0
    cur = f.astype(np.float64)
    for L in range(levels):
        np.testing.assert_array_equal(P.img[L], cur)
        gx = ndi.correlate(cur, SCHARR_X / 32.0, mode="mirror")
        gy = ndi.correlate(cur, SCHARR_X.T / 32.0, mode="mirror")
        if min(cur.shape) >= 2:
            np.testing.assert_allclose(P.grad[L][..., 0], gx, rtol=0, atol=1e-12)
            np.testing.assert_allclose(P.grad[L][..., 1], gy, rtol=0, atol=1e-12)
        if min(cur.shape) >= 3:
            nxt = ndi.correlate(cur, k2, mode="mirror")[::2, ::2]
        else:
            break
        cur = nxt


# --------------------------------------------------- half-precision storage
# A pyramid stored in half precision keeps level 0 as the u8 frame, every
# level L >= 1 as half(I - 128) computed from level L-1 as stored, and every
# gradient plane as the half of the gradient of its stored level.

def _half(v):
    return v.astype(np.float16).astype(np.float64)


@pytest.mark.parametrize("shape", [(41, 53), (64, 64), (9, 6)])
def test_f16_storage_matches_library_convolution(oracle, shape):
    rng = np.random.default_rng(12)
    f = rng.integers(0, 256, shape, dtype=np.uint8)
    levels = 4
    P = oracle.Pyramid(f, levels, storage="f16")
    k2 = np.outer(K5, K5) / 256.0
    cur = f.astype(np.float64)
    for L in range(levels):
        np.testing.assert_array_equal(P.img[L], cur)
        if min(cur.shape) >= 2:
            gx = ndi.correlate(cur, SCHARR_X / 32.0, mode="mirror")
            gy = ndi.correlate(cur, SCHARR_X.T / 32.0, mode="mirror")
            np.testing.assert_array_equal(P.grad[L][..., 0], _half(gx))
            np.testing.assert_array_equal(P.grad[L][..., 1], _half(gy))
        if min(cur.shape) < 3 or L + 1 == levels:
            break
        cur = _half(ndi.correlate(cur, k2, mode="mirror")[::2, ::2] - 128.0) + 128.0


def test_f16_storage_values_and_error_bound(oracle):
    rng = np.random.default_rng(13)
    f = rng.integers(0, 256, (57, 71), dtype=np.uint8)
    levels = 5
    H = oracle.Pyramid(f, levels, storage="f16")
    D = oracle.Pyramid(f, levels)
    np.testing.assert_array_equal(H.img[0], D.img[0])
    for L in range(levels):
        # every stored value is a half (levels >= 1 offset by 128)
        if L:
            assert np.all(_half(H.img[L] - 128.0) == H.img[L] - 128.0)
        assert np.all(_half(H.grad[L]) == H.grad[L])
        # the binomial reduction averages (non-negative weights summing to
        # one), so each level adds at most half a half-ulp of |I - 128| <=
        # 128 (2^-5) to the error of the one above; the gradient moves by at
        # most the level's error (|Scharr| sums to one per axis) plus its
        # own rounding (|I_x| <= 128)
        e_img = np.abs(H.img[L] - D.img[L]).max()
        assert e_img <= L * 2.0 ** -5, (L, e_img)
        e_grad = np.abs(H.grad[L] - D.grad[L]).max()
        assert e_grad <= L * 2.0 ** -5 + 2.0 ** -5, (L, e_grad)
    # frames whose level-1 values need no more than a half's precision
    # (|I - 128| < 8: the half grid there is 2^-8 or finer, and level-1
    # values are multiples of 2^-8) give level 1 exactly
    g = rng.integers(121, 136, (40, 48), dtype=np.uint8)
    np.testing.assert_array_equal(oracle.Pyramid(g, 2, storage="f16").img[1],
                                  oracle.Pyramid(g, 2).img[1])
