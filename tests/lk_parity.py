"""Shared LK parity helpers of the GPU tests (K3 against the FP64 oracle).

gpu_lk runs omt_lk_track through the C-ABI.  oracle_lk runs the oracle on
the pyramid the GPU path stores: FP64 levels for F32 storage, the oracle's
half-precision storage for F16 (every level and gradient the correctly
rounded half of the definition applied to the level above as stored, which
the F16 kernels produce bit for bit), so the same FP32 bar applies to both
storages.  error_vs_fp64 states the error of a run against the oracle on
unquantised FP64 pyramids: the cost of half-precision storage itself.

Conditioning probe: the oracle is run twice more with every pyramid value
multiplied by (1 + 2^-20 z), z ~ N(0, 1): perturbations of about 16 FP32
ulps, the size of the rounding FP32 arithmetic carries.  A point whose
oracle status, iteration counts or position (by more than 1e-4 px) changes
under that noise sits on a decision no FP32 computation can reproduce
(oscillating or divergent iterations, stops right at eps, centres at the
window bound); such points are counted, must stay a small minority, and are
only checked for validity.
"""
import numpy as np

OK, LOST_EIG, LOST_OOB, NONCONV = 1, 2, 4, 8
FLOW_TOL = 1e-3
F16_TOL = 0.02


def _torch():
    import torch
    return torch


def gpu_pyramid(omt, frame, levels, storage=0):
    torch = _torch()
    h, w = frame.shape
    P = omt.Pyramid(w, h, levels, storage)
    omt.build_pyramid(torch.from_numpy(np.ascontiguousarray(frame)).cuda(), P,
                      omt.default_params(levels=levels, storage=storage))
    return P


def gpu_lk(omt, f0, f1, pts, storage=0, **kw):
    torch = _torch()
    params = omt.default_params(storage=storage, **kw)
    P0, P1 = gpu_pyramid(omt, f0, params.levels, storage), gpu_pyramid(omt, f1, params.levels, storage)
    n = len(pts)
    p = torch.from_numpy(np.ascontiguousarray(pts, np.float32).reshape(-1, 2)).cuda()
    out = torch.full((max(n, 1), 2), np.nan, device="cuda")
    st = torch.full((max(n, 1),), 255, dtype=torch.uint8, device="cuda")
    it = torch.full((max(n, 1), params.levels), 255, dtype=torch.uint8, device="cuda")
    omt.lk_track(P0, P1, p, params, out, st, it, n_max=n)
    torch.cuda.synchronize()
    return out.cpu().numpy()[:n], st.cpu().numpy()[:n], it.cpu().numpy()[:n]


def oracle_lk(oracle, f0, f1, pts, levels=3, win=21, max_iter=30, eps=0.01, min_eig=1e-3,
              probe=False, storage=0):
    kind = "f16" if storage else "f64"
    O0, O1 = oracle.Pyramid(f0, levels, kind), oracle.Pyramid(f1, levels, kind)
    kw = dict(win=win, max_iter=max_iter, eps=eps, min_eig=min_eig, diagnostics=True)
    res = oracle.lk_track(O0, O1, pts, **kw)
    if not probe:
        return res
    unstable = np.zeros(len(res[1]), bool)
    base = [(P.img_flat.copy(), P.grad_flat.copy()) for P in (O0, O1)]
    for seed in (12345, 54321):
        rng = np.random.default_rng(seed)
        for P, (img, grad) in zip((O0, O1), base):
            P.img_flat[:] = img * (1.0 + 2.0 ** -20 * rng.standard_normal(img.shape))
            P.grad_flat[:] = grad * (1.0 + 2.0 ** -20 * rng.standard_normal(grad.shape))
        res2 = oracle.lk_track(O0, O1, pts, **kw)
        unstable |= ((res[1] != res2[1]) | np.any(res[2] != res2[2], axis=1) |
                     (np.abs(res[0] - res2[0]).max(axis=1) > 1e-4))
    return res, unstable


def check(label, g_out, g_st, g_it, pts, shape, o_out, o_st, o_it, o_me, unstable, tau, eps,
          tol=FLOW_TOL, min_ok=0.9, max_unstable=0.05):
    """The parity rules of a GPU run against the oracle on the same stored
    pyramid; prints what was excluded and why."""
    n = len(o_st)
    band = np.any((o_me >= 0.9 * tau) & (o_me <= 1.1 * tau), axis=1)
    stable = ~unstable & ~band
    same_status = g_st == o_st
    ok = (g_st & OK) > 0
    agree = np.all(g_it == o_it, axis=1) & same_status & stable
    both = agree & ok
    differ = stable & ~agree & ok & ((o_st & OK) > 0)
    err = np.abs(g_out[both] - o_out[both]).max(initial=0.0)
    derr = np.abs(g_out[differ] - o_out[differ]).max(initial=0.0)
    print(f"{label}: {n} points; excluded by the conditioning probe {unstable.sum()} "
          f"({unstable.mean():.2%}), in the tau guard band {band.sum()}; compared at "
          f"{tol:g} px: {both.sum()} (max {err:.2e}); stopping iteration differs: "
          f"{differ.sum()} (max {derr:.2e} px, bar eps = {eps:g})")
    assert unstable.mean() <= max_unstable, unstable.mean()
    bad = np.nonzero(stable & ~same_status)[0]
    assert len(bad) == 0, (bad[:10], g_st[bad[:10]], o_st[bad[:10]])
    assert ok.mean() >= min_ok, ok.mean()
    assert err <= tol, err
    # a stopping iteration that differs at the finest level leaves the two
    # results one sub-eps step apart; differing coarser levels re-converge
    if differ.any():
        assert derr <= eps, derr
    assert differ.mean() <= 0.05
    # validity everywhere: lost points report their input, OK points stay inside
    lost = ~ok
    np.testing.assert_array_equal(g_out[lost], np.asarray(pts, np.float32)[lost])
    h, w = shape
    assert np.all(g_out[ok] >= 0) and np.all(g_out[ok, 0] <= w - 1) and np.all(g_out[ok, 1] <= h - 1)
    assert set(np.unique(g_st)) <= {OK, OK | NONCONV, LOST_EIG, LOST_OOB}


def compare(omt, oracle, f0, f1, pts, storage=0, tol=FLOW_TOL, min_ok=0.9, max_unstable=0.05,
            label="LK", **kw):
    params = dict(levels=3, win=21, max_iter=30, eps=0.01, min_eig=1e-3)
    params.update(kw)
    g_out, g_st, g_it = gpu_lk(omt, f0, f1, pts, storage, **params)
    (o_out, o_st, o_it, o_me), unstable = oracle_lk(oracle, f0, f1, pts, probe=True,
                                                    storage=storage, **params)
    check(f"{label} ({'F16' if storage else 'F32'} storage)", g_out, g_st, g_it, pts, f0.shape,
          o_out, o_st, o_it, o_me, unstable, params["min_eig"], params["eps"], tol, min_ok,
          max_unstable)
    return g_out, g_st, o_out, o_st


def error_vs_fp64(label, g_out, g_st, o_out, o_st, tol=F16_TOL, max_status_differs=0.01,
                  max_nonconv=0.5):
    """Error of a run against the FP64 oracle on unquantised pyramids, over
    every point OK in both with the same status: max, p99 and mean gated at
    tol on the points the oracle converges (max) and on all of them (p99,
    mean); points the oracle leaves NONCONV (still oscillating at max_iter,
    so any perturbation moves them) and status differences are counted and
    bounded."""
    n = len(o_st)
    same = g_st == o_st
    both = ((g_st & OK) > 0) & same
    conv = both & (o_st == OK)
    nonc = both & ((o_st & NONCONV) > 0)
    e = np.hypot(*(g_out - o_out).T)
    stats = dict(n=n, ok=int(both.sum()), max=float(e[both].max(initial=0.0)),
                 p99=float(np.percentile(e[both], 99)) if both.any() else 0.0,
                 mean=float(e[both].mean()) if both.any() else 0.0,
                 conv=int(conv.sum()), conv_max=float(e[conv].max(initial=0.0)),
                 nonconv=int(nonc.sum()), nonconv_max=float(e[nonc].max(initial=0.0)),
                 status_differs=int((~same).sum()))
    print(f"{label}: |GPU - FP64 oracle| over {stats['ok']} of {n} points OK with the oracle's "
          f"status: max {stats['max']:.2e} px, p99 {stats['p99']:.2e}, mean {stats['mean']:.2e}; "
          f"converged {stats['conv']}: max {stats['conv_max']:.2e}; NONCONV {stats['nonconv']}: "
          f"max {stats['nonconv_max']:.2e}; status differs on {stats['status_differs']}")
    assert stats["conv_max"] <= tol, stats
    assert stats["p99"] <= tol and stats["mean"] <= tol, stats
    assert stats["status_differs"] <= max_status_differs * n, stats
    assert stats["nonconv"] <= max_nonconv * max(stats["ok"], 1), stats
    return stats
