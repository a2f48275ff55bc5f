"""Pins of the oracle's working frame (Section V-A preprocessing: a pyramid
level chosen by the input resolution).

Level 0 is the frame itself; a constant frame stays constant at every
level; an affine ramp a x + b y + c becomes 2^L a X + 2^L b Y + c in the
interior of level L (the binomial kernel is symmetric and sums to one),
rounded; values stay in [0, 255]; the level rule follows the frame width.
"""
import numpy as np


def test_level_zero_is_the_frame(oracle):
    rng = np.random.default_rng(1)
    f = rng.integers(0, 256, (37, 53)).astype(np.uint8)
    np.testing.assert_array_equal(oracle.level_u8(f, 0), f)


def test_constant_frame(oracle):
    for v in (0, 99, 255):
        f = np.full((50, 70), v, np.uint8)
        for L in (1, 2):
            out = oracle.level_u8(f, L)
            assert out.shape == tuple(reversed(oracle.level_size(70, 50, L)))
            assert np.all(out == v)


def test_affine_ramp(oracle):
    # x + y + 10 (slopes 1, 1): level L holds 2^L X + 2^L Y + 10 in its interior
    h, w = 96, 128
    y, x = np.mgrid[0:h, 0:w]
    g = (x + y + 10).astype(np.uint8)
    for L in (1, 2):
        out = oracle.level_u8(g, L).astype(int)
        lh, lw = out.shape
        Y, X = np.mgrid[0:lh, 0:lw]
        m = 2 * (L + 1)
        inner = (slice(m, lh - m), slice(m, lw - m))
        want = (2 ** L) * X + (2 ** L) * Y + 10
        np.testing.assert_array_equal(out[inner], want[inner])


def test_rule_by_width(oracle):
    assert oracle.working_level(720, 576) == 0
    assert oracle.working_level(1280, 720) == 0
    assert oracle.working_level(1920, 1080) == 1
    assert oracle.working_level(2560, 1280) == 1
    assert oracle.working_level(3840, 2160) == 2
