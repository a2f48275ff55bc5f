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


# ------------------------------------------------- the iteration body
# Section IV's engine minimises, per warp, the sum over both flow components
# of the Huber-regularised total variation plus lambda times the L1 data
# term |rho(u)|, rho(u) = r0 + g . u, by a primal-dual projected gradient
# scheme.  The pins below hold each piece of the oracle's iteration to that
# definition by routes that share none of its expressions: the adjoint
# identity of its difference operators, brute-force minimisation of the two
# proximal problems, a matrix-form restatement of the generic Chambolle-Pock
# iteration, and the optimality conditions of the converged saddle point.

SIGMA = TAU = 1.0 / np.sqrt(8.0)


def _huber(z, eps):
    n = np.hypot(z[..., 0], z[..., 1])
    return np.where(n <= eps, n * n / (2 * eps), n - eps / 2)


def test_div_is_the_negative_adjoint_of_grad(oracle):
    rng = np.random.default_rng(11)
    for h, w in ((1, 1), (1, 7), (6, 1), (9, 13)):
        u = rng.normal(size=(h, w))
        p = rng.normal(size=(h, w, 2))
        g = oracle.grad_fwd(u)
        d = oracle.div_bwd(p)
        lhs, rhs = (g * p).sum(), -(u * d).sum()
        assert abs(lhs - rhs) <= 1e-12 * (1 + abs(lhs)), (h, w, lhs, rhs)
    # forward differences of a ramp, zero on the last column / row
    y, x = np.mgrid[0:5, 0:6].astype(float)
    g = oracle.grad_fwd(3 * x - 2 * y + 1)
    assert np.all(g[:, :-1, 0] == 3) and np.all(g[:, -1, 0] == 0)
    assert np.all(g[:-1, :, 1] == -2) and np.all(g[-1, :, 1] == 0)


def test_dual_step_is_the_resolvent_of_the_huber_conjugate(oracle):
    # The conjugate of the Huber norm h_eps is eps/2 |q|^2 on the unit disc
    # (+inf outside), so the dual step must be argmin over |q| <= 1 of
    # |q - (p + sigma g)|^2 / (2 sigma) + eps/2 |q|^2: found here on a grid.
    s = np.linspace(-1, 1, 1601)
    qx, qy = np.meshgrid(s, s)
    inside = qx ** 2 + qy ** 2 <= 1.0
    phi = np.linspace(0, 2 * np.pi, 40001)   # and the disc's edge, finely
    qx = np.concatenate([qx[inside], np.cos(phi)])
    qy = np.concatenate([qy[inside], np.sin(phi)])
    rng = np.random.default_rng(12)
    for eps in (0.05, 0.5, 2.0):
        for scale in (0.2, 0.8, 3.0):   # inside and outside the disc
            p = rng.uniform(-1, 1, 2) * 0.5
            g = rng.normal(size=2) * scale / SIGMA
            v = p + SIGMA * g
            obj = ((qx - v[0]) ** 2 + (qy - v[1]) ** 2) / (2 * SIGMA) + eps / 2 * (qx ** 2 + qy ** 2)
            k = np.argmin(obj)
            got = np.array(oracle.tvl1_dual(p, g, SIGMA, eps))
            assert np.hypot(*got) <= 1.0 + 1e-15
            # within the grid's reach of the best grid point, and no grid
            # point beats it
            assert np.abs(got - [qx[k], qy[k]]).max() <= 2.5e-3, (eps, scale, got)
            here = (np.sum((got - v) ** 2) / (2 * SIGMA) + eps / 2 * np.sum(got ** 2))
            assert here <= obj[k] + 1e-12


def test_prox_is_the_argmin_of_the_data_term(oracle):
    # u <- argmin_v |v - t|^2 / (2 tau) + lambda |r0 + g . v|, checked on a
    # grid around t, for the three branches (rho(t) below, inside and above
    # the band +-tau lambda |g|^2) and g = 0.
    lam = 10.0
    g = np.array([0.3, -0.2])
    t = np.array([0.4, 1.1])
    band = TAU * lam * (g @ g)
    rho_t = lambda r0: r0 + g @ t
    cases = [(-g @ t - 3 * band, g), (-g @ t + 0.4 * band, g), (-g @ t + 3 * band, g),
             (0.7, np.zeros(2))]
    seen = set()
    for r0, gg in cases:
        reach = TAU * lam * np.hypot(*gg) + 0.05
        s = np.linspace(-reach, reach, 2001)
        vx, vy = np.meshgrid(t[0] + s, t[1] + s)
        obj = ((vx - t[0]) ** 2 + (vy - t[1]) ** 2) / (2 * TAU) + lam * np.abs(r0 + gg[0] * vx + gg[1] * vy)
        k = np.argmin(obj)
        got = np.array(oracle.tvl1_prox(t, r0, gg, TAU, lam))
        step = s[1] - s[0]
        assert np.abs(got - [vx.flat[k], vy.flat[k]]).max() <= 2 * step, (r0, got)
        here = np.sum((got - t) ** 2) / (2 * TAU) + lam * abs(r0 + gg @ got)
        assert here <= obj.flat[k] + 1e-12, (r0, here, obj.flat[k])
        r = rho_t(r0) if gg.any() else 0.0
        seen.add(int(np.sign(r)) if abs(r) > band else 0)
    assert seen == {-1, 0, 1}


def _grad_matrix(h, w):
    """Forward differences (zero at the last column/row) as a sparse (2n, n)
    matrix acting on row-major fields: rows 0..n-1 give gx, n..2n-1 gy."""
    import scipy.sparse as sp

    def d1(m):
        D = sp.diags([-np.ones(m), np.ones(m - 1)], [0, 1], shape=(m, m)).tolil()
        D[m - 1, m - 1] = 0.0
        return D.tocsr()
    return sp.vstack([sp.kron(sp.identity(h), d1(w)), sp.kron(d1(h), sp.identity(w))]).tocsr()


def _chambolle_pock(gw, r0, u, p, iters, lam, eps):
    """The generic primal-dual iteration of Chambolle and Pock (2011, with
    theta = 1) for min_u sum_d H_eps(K u_d) + lam sum |r0 + g . u|, written
    with the operator K as a matrix, the dual resolvent as scaling and
    projection, and the primal resolvent by a scalar minimisation along g."""
    from scipy.optimize import minimize_scalar
    h, w = r0.shape
    n = h * w
    K = _grad_matrix(h, w)
    U = u.reshape(n, 2).copy()
    Y = [p.reshape(n, 4)[:, 0:2].copy(), p.reshape(n, 4)[:, 2:4].copy()]
    G = gw.reshape(n, 2)
    R = r0.reshape(n)
    Ub = U.copy()
    for _ in range(iters):
        for d in range(2):
            Ku = K @ Ub[:, d]
            y = (Y[d] + SIGMA * np.stack([Ku[:n], Ku[n:]], 1)) / (1 + SIGMA * eps)
            nrm = np.maximum(1.0, np.hypot(y[:, 0], y[:, 1]))
            Y[d] = y / nrm[:, None]
        T = np.stack([U[:, d] - TAU * (K.T @ np.concatenate([Y[d][:, 0], Y[d][:, 1]]))
                      for d in range(2)], 1)
        Un = T.copy()
        for i in range(n):
            g = G[i]
            gg = g @ g
            if gg == 0:
                continue
            # the minimiser lies on t + s g
            f = lambda s: (s * s * gg) / (2 * TAU) + lam * abs(R[i] + g @ T[i] + s * gg)
            reach = TAU * lam + abs(R[i] + g @ T[i]) / gg + 1.0
            s = minimize_scalar(f, bounds=(-reach, reach), method="bounded",
                                options={"xatol": 1e-14, "maxiter": 2000}).x
            kink = -(R[i] + g @ T[i]) / gg   # where rho vanishes: taken if it is lower
            if f(kink) < f(s):
                s = kink
            Un[i] = T[i] + s * g
        Ub = 2 * Un - U
        U = Un
    P = np.concatenate([Y[0], Y[1]], 1)
    return U.reshape(h, w, 2), P.reshape(h, w, 4)


def test_iterations_match_a_matrix_form_chambolle_pock(oracle):
    rng = np.random.default_rng(13)
    h, w = 8, 8
    gw = rng.normal(0, 0.3, (h, w, 2))
    gw[3, 4] = 0.0
    r0 = rng.normal(0, 0.2, (h, w))
    u = rng.normal(0, 0.5, (h, w, 2))
    p = np.zeros((h, w, 4))
    for lam, eps in ((10.0, 0.05), (1.0, 0.7)):
        for iters in (1, 2, 5):
            ou, op = oracle.tvl1_iterations(gw, r0, u, p, iters, lam=lam, eps=eps)
            mu, mp = _chambolle_pock(gw, r0, u, p, iters, lam, eps)
            # the scalar minimiser locates a smooth minimum to about the square
            # root of the FP64 epsilon; a wrong step would move values by 1e-2+
            np.testing.assert_allclose(op, mp, rtol=0, atol=1e-6)
            np.testing.assert_allclose(ou, mu, rtol=0, atol=1e-6)


def test_iterations_converge_to_the_optimality_conditions(oracle):
    # At the saddle point the duals are the Huber gradient of each flow
    # component, p_d = grad u_d / max(eps, |grad u_d|), and div p lies in
    # lam g d|rho|(u): parallel to g, lam g sign(rho) where rho != 0 and at
    # most lam in size where rho = 0; the energy falls to its minimum.
    rng = np.random.default_rng(14)
    h, w = 10, 12
    gw = rng.normal(0, 0.3, (h, w, 2))
    gw[2, 3] = 0.0
    r0 = rng.normal(0, 0.2, (h, w))
    u0 = rng.normal(0, 0.5, (h, w, 2))
    lam, eps = 2.0, 0.05

    def energy(u):
        tv = sum(_huber(oracle.grad_fwd(u[..., d]), eps).sum() for d in range(2))
        return tv + lam * np.abs(r0 + (gw * u).sum(-1)).sum()

    e = [energy(oracle.tvl1_iterations(gw, r0, u0, np.zeros((h, w, 4)), k, lam=lam, eps=eps)[0])
         for k in (0, 10, 100, 5000)]
    assert e[0] > e[1] > e[2] > e[3] and e[2] - e[3] < 1e-2 * (e[0] - e[3]), e
    u, p = oracle.tvl1_iterations(gw, r0, u0, np.zeros((h, w, 4)), 5000, lam=lam, eps=eps)
    for d in range(2):
        g = oracle.grad_fwd(u[..., d])
        want = g / np.maximum(eps, np.hypot(g[..., 0], g[..., 1]))[..., None]
        np.testing.assert_allclose(p[..., 2 * d:2 * d + 2], want, rtol=0, atol=1e-10)
    dv = np.stack([oracle.div_bwd(p[..., 0:2]), oracle.div_bwd(p[..., 2:4])], -1)
    gn2 = (gw * gw).sum(-1)
    has = gn2 > 0
    cross = dv[..., 0] * gw[..., 1] - dv[..., 1] * gw[..., 0]
    assert np.abs(cross[has]).max() <= 1e-10
    assert np.abs(dv[~has]).max() <= 1e-10
    mu = (dv * gw).sum(-1)[has] / gn2[has]
    rho = (r0 + (gw * u).sum(-1))[has]
    assert np.all(np.abs(mu) <= lam * (1 + 1e-12))
    off = np.abs(rho) > 1e-9
    assert off.sum() > 20
    np.testing.assert_allclose(mu[off], lam * np.sign(rho[off]), rtol=1e-10)


def test_warp_linearisation(oracle):
    # rho(u0) = I1(x + u0) - I0(x): on a ramp I1 = a x + b y + c (exact under
    # bilinear sampling away from the clamped border) and u0 constant,
    # gw = (a, b)/255 and r0 + gw . u0 = (I1(x + u0) - I0) / 255
    h, w = 12, 14
    y, x = np.mgrid[0:h, 0:w].astype(float)
    a, b, c = 3.0, -2.0, 100.0
    I1 = a * x + b * y + c
    G1 = np.stack([np.full((h, w), a), np.full((h, w), b)], -1)
    I0 = np.full((h, w), 50.0)
    u = np.zeros((h, w, 2)) + [0.3, 0.7]
    gw, r0 = oracle.tvl1_warp(I0, I1, G1, u)
    inner = (slice(0, h - 2), slice(0, w - 2))
    np.testing.assert_allclose(gw[inner], np.broadcast_to([a / 255, b / 255], gw[inner].shape), atol=1e-15)
    warped = a * (x + 0.3) + b * (y + 0.7) + c
    np.testing.assert_allclose((r0 + (gw * u).sum(-1))[inner], ((warped - I0) / 255)[inner], atol=1e-12)
