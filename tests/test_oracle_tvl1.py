"""Pins of the oracle's dense flow engine (Section IV: structure-texture
decomposition, Huber-TV-L1 flow; Section V-A: mean-in-box prediction).

The structure-texture step is pinned by the constant image (closed form),
equivariance under a brightness offset, and the ROF energy it must lower;
the flow by exact zero flow on identical frames and the recovery of
rendered translations, sub-pixel and beyond a single level's reach; the box
prediction by hand vectors and the half-open pixel convention.
"""
import numpy as np

from paper_1910_06017_b300 import synth


def _tex(rng, w, h, low=False):
    t = synth.Texture.low_frequency(rng, w, h) if low else synth.Texture.draw(rng, w, h)
    return t


def test_structure_texture_constant_image(oracle):
    for v in (0, 37, 128, 255):
        f = np.full((24, 32), v, np.uint8)
        T = oracle.structure_texture(f)
        # S = I exactly (no gradient, the duals stay 0): T = k (1 - alpha) I
        want = np.clip(np.floor(oracle.ST_K * (1 - oracle.ST_ALPHA) * v + 128 + 0.5), 0, 255)
        assert np.all(T == want), (v, np.unique(T))


def _rof_energy(S, I, theta):
    gx = np.zeros_like(S); gy = np.zeros_like(S)
    gx[:, :-1] = S[:, 1:] - S[:, :-1]
    gy[:-1, :] = S[1:, :] - S[:-1, :]
    return np.sqrt(gx ** 2 + gy ** 2).sum() + ((S - I) ** 2).sum() / (2 * theta)


def test_structure_texture_offset_and_energy(oracle):
    rng = np.random.default_rng(4)
    w, h = 96, 72
    f = synth.render_shift(_tex(rng, w, h), w, h)
    f = np.clip(f, 20, 200).astype(np.uint8)
    T = oracle.structure_texture(f).astype(int)
    T10 = oracle.structure_texture(f + 10).astype(int)
    # ROF commutes with a brightness offset: the texture moves by k (1 - alpha) 10 = 1
    assert np.mean(T10 - T == 1) > 0.999
    # the structure lowers the ROF energy below the image's own, and more
    # iterations lower it further
    k, th = oracle.ST_K, oracle.ST_THETA
    _, S = oracle.structure_texture(f, with_structure=True)
    _, S5 = oracle.structure_texture(f, iters=5, with_structure=True)
    I = f.astype(float)
    e, e5, e0 = _rof_energy(S, I, th), _rof_energy(S5, I, th), _rof_energy(I, I, th)
    assert e < e5 < e0, (e, e5, e0)
    # the texture keeps the edges and drops the slow variation
    assert T.std() < 0.6 * k * f.std()


def test_identical_frames_give_zero_flow(oracle):
    rng = np.random.default_rng(5)
    w, h = 80, 64
    f = synth.render_shift(_tex(rng, w, h), w, h)
    P = oracle.Pyramid(f, 3)
    fl = oracle.tvl1(P, P)
    assert np.all(fl == 0.0)


def test_translation_is_recovered(oracle):
    rng = np.random.default_rng(3)
    w, h = 160, 120
    tex = _tex(rng, w, h)
    for shift, levels, tol in (((1.37, -0.62), 3, 0.02), ((5.5, 3.25), 4, 0.05)):
        f0 = synth.render_shift(tex, w, h, 0, 0)
        f1 = synth.render_shift(tex, w, h, *shift)
        T0, T1 = oracle.structure_texture(f0), oracle.structure_texture(f1)
        fl = oracle.tvl1(oracle.Pyramid(T0, levels), oracle.Pyramid(T1, levels))
        inner = fl[20:-20, 20:-20].reshape(-1, 2)
        err = np.abs(inner - np.array(shift))
        assert err.mean() < tol, (shift, err.mean(0))
        assert np.allclose(np.median(inner, 0), shift, atol=tol)


def test_box_mean_flow_hand_vectors(oracle):
    h, w = 6, 8
    fl = np.zeros((h, w, 2))
    fl[..., 0] = np.arange(w)[None, :]          # u1 = x
    fl[..., 1] = 2.0
    boxes = np.array([[0, 0, 2, 1],             # pixels (0,0), (1,0): mean u1 0.5
                      [1.5, 2, 4, 3],           # pixels x = 2, 3: mean 2.5
                      [20, 20, 30, 30],         # outside: stays
                      [-3, -3, 0.5, 0.5],       # only pixel (0, 0)
                      [7, 5, 9, 9]], np.float32)  # pixel (7, 5)
    out = oracle.box_mean_flow(fl, boxes)
    want = boxes.astype(float) + np.array([[0.5, 2, 0.5, 2], [2.5, 2, 2.5, 2], [0, 0, 0, 0],
                                            [0, 2, 0, 2], [7, 2, 7, 2]])
    np.testing.assert_allclose(out, want, atol=1e-12)
