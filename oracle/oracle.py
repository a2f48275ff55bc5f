"""ctypes wrapper of the FP64 CPU oracle (omt_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
benchmark's CPU baseline, never by the product path.  It builds
``liboracle.so`` next to this file with gcc on first use.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from ctypes import POINTER, c_double, c_float, c_int, c_int32, c_int64, c_long, c_size_t, c_uint8, c_uint64

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "omt_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

OK, LOST_EIG, LOST_OOB, NONCONV = 1, 2, 4, 8


def build(force: bool = False) -> str:
    """Compile liboracle.so (plain C, -O2, OpenMP) if missing or stale."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11",
                               "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        L.orc_reflect101.argtypes = [c_int, c_int]
        L.orc_reflect101.restype = c_int
        L.orc_level_size.argtypes = [c_int, c_int, c_int, POINTER(c_int), POINTER(c_int)]
        L.orc_pyramid_elems.argtypes = [c_int, c_int, c_int]
        L.orc_pyramid_elems.restype = c_size_t
        L.orc_pyramid.argtypes = [POINTER(c_uint8), c_int, c_int, c_long, c_int,
                                  POINTER(c_double), POINTER(c_double)]
        L.orc_pyramid_f64.argtypes = [POINTER(c_double), c_int, c_int, c_int,
                                      POINTER(c_double), POINTER(c_double)]
        L.orc_isqrt.argtypes = [c_uint64]
        L.orc_isqrt.restype = c_uint64
        L.orc_scharr_raw.argtypes = [POINTER(c_uint8), c_int, c_int, c_long,
                                     POINTER(c_int32), POINTER(c_int32)]
        L.orc_corner_response.argtypes = [POINTER(c_uint8), c_int, c_int, c_long, POINTER(c_int64)]
        L.orc_select_corners.argtypes = [POINTER(c_uint8), c_int, c_int, c_long, POINTER(c_float), c_int,
                                         c_int, c_int, c_int, c_float, POINTER(c_float), POINTER(c_int32)]
        L.orc_select_corners.restype = c_int
        L.orc_lk_track.argtypes = [POINTER(c_double)] * 4 + [
            c_int, c_int, c_int, POINTER(c_float), c_int, c_int, c_int, c_double, c_double,
            POINTER(c_double), POINTER(c_uint8), POINTER(c_uint8), POINTER(c_double), c_int]
        L.orc_update_boxes.argtypes = [POINTER(c_float), POINTER(c_int32), POINTER(c_float),
                                       POINTER(c_float), POINTER(c_uint8), c_int, c_int,
                                       POINTER(c_double), POINTER(c_int32)]
        L.orc_fb_check.argtypes = [POINTER(c_float), POINTER(c_double), POINTER(c_uint8), c_int,
                                   c_double, POINTER(c_uint8)]
        L.orc_structure_texture.argtypes = [POINTER(c_uint8), c_int, c_int, c_long, c_double,
                                            c_double, c_double, c_int, POINTER(c_uint8), c_long,
                                            POINTER(c_double)]
        L.orc_tvl1.argtypes = [POINTER(c_double), POINTER(c_double), POINTER(c_double), c_int, c_int,
                               c_int, c_double, c_double, c_int, c_int, POINTER(c_double)]
        L.orc_grad_fwd.argtypes = [POINTER(c_double), c_int, c_int, POINTER(c_double)]
        L.orc_div_bwd.argtypes = [POINTER(c_double), c_int, c_int, POINTER(c_double)]
        L.orc_tvl1_dual.argtypes = [c_double] * 6 + [POINTER(c_double)] * 2
        L.orc_tvl1_prox.argtypes = [c_double] * 7 + [POINTER(c_double)] * 2
        L.orc_tvl1_iterations.argtypes = [POINTER(c_double), POINTER(c_double), c_int, c_int,
                                          c_double, c_double, c_int, POINTER(c_double),
                                          POINTER(c_double)]
        L.orc_tvl1_warp.argtypes = [POINTER(c_double)] * 3 + [c_int, c_int] + [POINTER(c_double)] * 3
        L.orc_box_mean_flow.argtypes = [POINTER(c_double), c_int, c_int, POINTER(c_float), c_int,
                                        POINTER(c_double)]
        L.orc_working_level.argtypes = [c_int, c_int]
        L.orc_working_level.restype = c_int
        L.orc_level_u8.argtypes = [POINTER(c_uint8), c_int, c_int, c_long, c_int, POINTER(c_uint8)]
        L.orc_max_threads.restype = c_int
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(POINTER(t)) if a is not None else None


def level_size(w: int, h: int, level: int):
    a, b = c_int(), c_int()
    lib().orc_level_size(w, h, level, ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


class Pyramid:
    """Oracle pyramid of one frame: img[L] (h_L, w_L) and grad[L] (h_L, w_L, 2).

    storage "f64" (default): every level and gradient plane in FP64, from
    the definitions (Section V-A preprocessing; binomial reduction, Scharr).
    storage "f16": the values a pyramid stored in half precision holds --
    level 0 is the u8 frame; each level L >= 1 is the binomial reduction of
    level L-1 *as stored*, rounded to half(I - 128) (the value kept is that
    half plus 128); each gradient plane is the Scharr gradient of its level
    as stored, rounded to half.  The reduction and the gradient are the FP64
    ones of the "f64" pyramid, applied level by level to the stored values."""

    def __init__(self, frame: np.ndarray, levels: int, storage: str = "f64"):
        """frame: uint8 (a video frame) or float64 (an unquantised render)."""
        h, w = frame.shape
        self.w, self.h, self.levels, self.storage = w, h, levels, storage
        n = lib().orc_pyramid_elems(w, h, levels)
        self.img_flat = np.zeros(n, np.float64)
        self.grad_flat = np.zeros(2 * n, np.float64)
        if storage == "f16":
            self._build_f16(frame, levels)
        elif frame.dtype == np.uint8:
            f = np.ascontiguousarray(frame)
            lib().orc_pyramid(_p(f, c_uint8), w, h, w, levels, _p(self.img_flat, c_double),
                              _p(self.grad_flat, c_double))
        else:
            f = np.ascontiguousarray(frame, dtype=np.float64)
            lib().orc_pyramid_f64(_p(f, c_double), w, h, levels, _p(self.img_flat, c_double),
                                  _p(self.grad_flat, c_double))
        self.img, self.grad = [], []
        off = 0
        for L in range(levels):
            lw, lh = level_size(w, h, L)
            self.img.append(self.img_flat[off:off + lw * lh].reshape(lh, lw))
            self.grad.append(self.grad_flat[2 * off:2 * (off + lw * lh)].reshape(lh, lw, 2))
            off += lw * lh

    def _build_f16(self, frame, levels):
        assert frame.dtype == np.uint8, "half storage starts from a u8 frame"
        h, w = frame.shape
        cur = np.ascontiguousarray(frame, dtype=np.float64)   # level L as stored
        off = 0
        for L in range(levels):
            lw, lh = level_size(w, h, L)
            # the FP64 gradient of the stored level and the FP64 reduction of it
            two = min(2, levels - L)
            n2 = lib().orc_pyramid_elems(lw, lh, two)
            img2 = np.zeros(n2, np.float64)
            grad2 = np.zeros(2 * n2, np.float64)
            lib().orc_pyramid_f64(_p(cur, c_double), lw, lh, two, _p(img2, c_double),
                                  _p(grad2, c_double))
            self.img_flat[off:off + lw * lh] = cur.reshape(-1)
            self.grad_flat[2 * off:2 * (off + lw * lh)] = \
                grad2[:2 * lw * lh].astype(np.float16).astype(np.float64)
            off += lw * lh
            if two == 2:
                nw, nh = level_size(w, h, L + 1)
                nxt = img2[lw * lh:lw * lh + nw * nh].reshape(nh, nw)
                cur = np.ascontiguousarray((nxt - 128.0).astype(np.float16).astype(np.float64) + 128.0)


def isqrt(d: int) -> int:
    return int(lib().orc_isqrt(d))


def reflect101(i: int, n: int) -> int:
    return lib().orc_reflect101(i, n)


def scharr_raw(frame: np.ndarray):
    f = np.ascontiguousarray(frame, dtype=np.uint8)
    h, w = f.shape
    gx = np.zeros((h, w), np.int32)
    gy = np.zeros((h, w), np.int32)
    lib().orc_scharr_raw(_p(f, c_uint8), w, h, w, _p(gx, c_int32), _p(gy, c_int32))
    return gx, gy


def corner_response(frame: np.ndarray) -> np.ndarray:
    f = np.ascontiguousarray(frame, dtype=np.uint8)
    h, w = f.shape
    R = np.zeros((h, w), np.int64)
    lib().orc_corner_response(_p(f, c_uint8), w, h, w, _p(R, c_int64))
    return R


def select_corners(frame: np.ndarray, boxes: np.ndarray, max_corners: int,
                   quality=(1, 100), min_dist: float = 5.0):
    """Returns (pts (nboxes, max_corners, 2) float32, counts (nboxes,) int32)."""
    f = np.ascontiguousarray(frame, dtype=np.uint8)
    h, w = f.shape
    b = np.ascontiguousarray(boxes, dtype=np.float32).reshape(-1, 4)
    nb = b.shape[0]
    pts = np.zeros((nb, max(max_corners, 0), 2), np.float32)
    counts = np.zeros(nb, np.int32)
    lib().orc_select_corners(_p(f, c_uint8), w, h, w, _p(b, c_float), nb, max_corners,
                             int(quality[0]), int(quality[1]), float(min_dist),
                             _p(pts, c_float), _p(counts, c_int32))
    return pts, counts


def lk_track(prev: Pyramid, nxt: Pyramid, pts: np.ndarray, win: int = 21, max_iter: int = 30,
             eps: float = 0.01, min_eig: float = 1e-3, nthreads: int = 0, diagnostics: bool = False):
    """Returns (pts_out (n, 2) float64, status (n,) uint8[, iters (n, L), mineig (n, L)])."""
    assert prev.w == nxt.w and prev.h == nxt.h and prev.levels == nxt.levels
    p = np.ascontiguousarray(pts, dtype=np.float32).reshape(-1, 2)
    n = p.shape[0]
    out = np.zeros((n, 2), np.float64)
    st = np.zeros(n, np.uint8)
    it = np.zeros((n, prev.levels), np.uint8) if diagnostics else None
    me = np.zeros((n, prev.levels), np.float64) if diagnostics else None
    lib().orc_lk_track(_p(prev.img_flat, c_double), _p(prev.grad_flat, c_double),
                       _p(nxt.img_flat, c_double), _p(nxt.grad_flat, c_double),
                       prev.w, prev.h, prev.levels, _p(p, c_float), n, win, max_iter,
                       float(eps), float(min_eig), _p(out, c_double), _p(st, c_uint8),
                       _p(it, c_uint8), _p(me, c_double), int(nthreads))
    if diagnostics:
        return out, st, it, me
    return out, st


def update_boxes(boxes, offsets, pts, pts_out, status, aggregator: int = 0):
    """Returns (boxes_out (nboxes, 4) float64, nvalid (nboxes,) int32)."""
    b = np.ascontiguousarray(boxes, dtype=np.float32).reshape(-1, 4)
    o = np.ascontiguousarray(offsets, dtype=np.int32)
    p = np.ascontiguousarray(pts, dtype=np.float32).reshape(-1, 2)
    q = np.ascontiguousarray(pts_out, dtype=np.float32).reshape(-1, 2)
    s = np.ascontiguousarray(status, dtype=np.uint8)
    nb = b.shape[0]
    out = np.zeros((nb, 4), np.float64)
    nv = np.zeros(nb, np.int32)
    lib().orc_update_boxes(_p(b, c_float), _p(o, c_int32), _p(p, c_float), _p(q, c_float),
                           _p(s, c_uint8), nb, int(aggregator), _p(out, c_double), _p(nv, c_int32))
    return out, nv


def fb_check(pts, pts_back, status_back, status, fb_max: float):
    """Forward-backward check: the forward statuses with the points whose
    round trip u -> v -> u' does not close within fb_max (or whose backward
    run was lost) set to LOST_FB."""
    p = np.ascontiguousarray(pts, dtype=np.float32).reshape(-1, 2)
    q = np.ascontiguousarray(pts_back, dtype=np.float64).reshape(-1, 2)
    sb = np.ascontiguousarray(status_back, dtype=np.uint8)
    st = np.array(status, dtype=np.uint8, copy=True)
    lib().orc_fb_check(_p(p, c_float), _p(q, c_double), _p(sb, c_uint8), p.shape[0],
                       float(fb_max), _p(st, c_uint8))
    return st


def lk_track_fb(prev: Pyramid, nxt: Pyramid, pts, fb_max: float, **kw):
    """Forward LK from prev to nxt, backward LK from the results, and the
    forward-backward check: (pts_out, status, pts_back, status_back).  The
    backward run starts from the forward results as float32, the precision
    points are stored in."""
    out, st = lk_track(prev, nxt, pts, **kw)
    back, sb = lk_track(nxt, prev, out.astype(np.float32), **kw)
    return out, fb_check(pts, back, sb, st, fb_max), back, sb


def working_level(w: int, h: int) -> int:
    """Pyramid level processed for a w x h frame (Section V-A preprocessing)."""
    return int(lib().orc_working_level(w, h))


def level_u8(frame, level: int):
    """Level `level` of the frame's pyramid rounded to u8: the working frame."""
    f = np.ascontiguousarray(frame, dtype=np.uint8)
    h, w = f.shape
    lw, lh = level_size(w, h, level)
    out = np.zeros((lh, lw), np.uint8)
    lib().orc_level_u8(_p(f, c_uint8), w, h, w, int(level), _p(out, c_uint8))
    return out


# Section IV readings of the dense flow engine (see omt_oracle.c)
ST_THETA, ST_ALPHA, ST_K, ST_ITERS = 0.125, 0.95, 2.0, 100
TVL1_LAMBDA, TVL1_EPS, TVL1_WARPS, TVL1_ITERS = 10.0, 0.05, 3, 30


def structure_texture(frame, theta=ST_THETA, alpha=ST_ALPHA, k=ST_K, iters=ST_ITERS,
                      with_structure: bool = False):
    """u8 texture image of a u8 frame (ROF structure removed)[, structure]."""
    f = np.ascontiguousarray(frame, dtype=np.uint8)
    h, w = f.shape
    out = np.zeros((h, w), np.uint8)
    S = np.zeros((h, w), np.float64) if with_structure else None
    lib().orc_structure_texture(_p(f, c_uint8), w, h, w, float(theta), float(alpha), float(k),
                                int(iters), _p(out, c_uint8), w, _p(S, c_double))
    return (out, S) if with_structure else out


def tvl1(prev: Pyramid, nxt: Pyramid, lam=TVL1_LAMBDA, eps=TVL1_EPS, warps=TVL1_WARPS,
         iters=TVL1_ITERS):
    """Dense flow (h, w, 2) float64 from prev to nxt, level-0 pixels."""
    assert prev.w == nxt.w and prev.h == nxt.h and prev.levels == nxt.levels
    out = np.zeros((prev.h, prev.w, 2), np.float64)
    lib().orc_tvl1(_p(prev.img_flat, c_double), _p(nxt.img_flat, c_double),
                   _p(nxt.grad_flat, c_double), prev.w, prev.h, prev.levels, float(lam),
                   float(eps), int(warps), int(iters), _p(out, c_double))
    return out


def grad_fwd(u):
    """Forward differences of a (h, w) field, zero at the last row/column: (h, w, 2)."""
    f = np.ascontiguousarray(u, dtype=np.float64)
    h, w = f.shape
    g = np.zeros((h, w, 2), np.float64)
    lib().orc_grad_fwd(_p(f, c_double), w, h, _p(g, c_double))
    return g


def div_bwd(p):
    """Divergence of a (h, w, 2) dual field, the negative adjoint of grad_fwd: (h, w)."""
    q = np.ascontiguousarray(p, dtype=np.float64)
    h, w = q.shape[:2]
    d = np.zeros((h, w), np.float64)
    lib().orc_div_bwd(_p(q, c_double), w, h, _p(d, c_double))
    return d


def tvl1_dual(p, g, sigma, eps):
    """One pixel's Huber-TV dual step of one flow component: (qx, qy)."""
    qx, qy = c_double(), c_double()
    lib().orc_tvl1_dual(float(p[0]), float(p[1]), float(g[0]), float(g[1]), float(sigma),
                        float(eps), ctypes.byref(qx), ctypes.byref(qy))
    return qx.value, qy.value


def tvl1_prox(t, r0, g, tau, lam):
    """One pixel's prox of tau lam |r0 + g . v| at v = t: (v1, v2)."""
    v1, v2 = c_double(), c_double()
    lib().orc_tvl1_prox(float(t[0]), float(t[1]), float(r0), float(g[0]), float(g[1]),
                        float(tau), float(lam), ctypes.byref(v1), ctypes.byref(v2))
    return v1.value, v2.value


def tvl1_iterations(gw, r0, u, p, iters, lam=TVL1_LAMBDA, eps=TVL1_EPS):
    """iters primal-dual iterations of one warp on one level: (u, p) after
    them; gw (h, w, 2), r0 (h, w), u (h, w, 2), p (h, w, 4)."""
    G = np.ascontiguousarray(gw, dtype=np.float64)
    R = np.ascontiguousarray(r0, dtype=np.float64)
    h, w = R.shape
    U = np.array(u, dtype=np.float64, copy=True, order="C")
    P = np.array(p, dtype=np.float64, copy=True, order="C")
    lib().orc_tvl1_iterations(_p(G, c_double), _p(R, c_double), w, h, float(lam), float(eps),
                              int(iters), _p(U, c_double), _p(P, c_double))
    return U, P


def tvl1_warp(I0, I1, G1, u):
    """Linearisation of one warp: (gw (h, w, 2), r0 (h, w))."""
    a = np.ascontiguousarray(I0, dtype=np.float64)
    b = np.ascontiguousarray(I1, dtype=np.float64)
    g = np.ascontiguousarray(G1, dtype=np.float64)
    U = np.ascontiguousarray(u, dtype=np.float64)
    h, w = a.shape
    gw = np.zeros((h, w, 2), np.float64)
    r0 = np.zeros((h, w), np.float64)
    lib().orc_tvl1_warp(_p(a, c_double), _p(b, c_double), _p(g, c_double), w, h, _p(U, c_double),
                        _p(gw, c_double), _p(r0, c_double))
    return gw, r0


def box_mean_flow(flow, boxes):
    """Boxes moved by the mean flow over their pixels: (nboxes, 4) float64."""
    fl = np.ascontiguousarray(flow, dtype=np.float64)
    h, w = fl.shape[:2]
    b = np.ascontiguousarray(boxes, dtype=np.float32).reshape(-1, 4)
    out = np.zeros((b.shape[0], 4), np.float64)
    lib().orc_box_mean_flow(_p(fl, c_double), w, h, _p(b, c_float), b.shape[0], _p(out, c_double))
    return out


def iou_matrix(a, b):
    """IoU of every pair (na, nb) float64, Section V-A matching score."""
    A = np.ascontiguousarray(a, dtype=np.float32).reshape(-1, 4)
    B = np.ascontiguousarray(b, dtype=np.float32).reshape(-1, 4)
    out = np.zeros((A.shape[0], B.shape[0]), np.float64)
    lib().orc_iou_matrix(_p(A, c_float), A.shape[0], _p(B, c_float), B.shape[0], _p(out, c_double))
    return out


def assign(iou, active=None, iou_min: float = 0.0):
    """Maximum-total-IoU assignment (Hungarian method): (match_a, match_b)."""
    m = np.ascontiguousarray(iou, dtype=np.float64)
    na, nb = m.shape
    act = None if active is None else np.ascontiguousarray(active, dtype=np.uint8)
    ma = np.zeros(na, np.int32)
    mb = np.zeros(nb, np.int32)
    lib().orc_assign(_p(m, c_double), na, nb, None if act is None else _p(act, c_uint8),
                     ctypes.c_double(iou_min), _p(ma, c_int32), _p(mb, c_int32))
    return ma, mb


def update_tracks(boxes_s, active_s, boxes_d, match_s, match_d):
    """Update phase: (boxes (n, 4) float32, active (n,) uint8)."""
    S = np.ascontiguousarray(boxes_s, dtype=np.float32).reshape(-1, 4)
    D = np.ascontiguousarray(boxes_d, dtype=np.float32).reshape(-1, 4)
    a = np.ascontiguousarray(active_s, dtype=np.uint8)
    ms = np.ascontiguousarray(match_s, dtype=np.int32)
    md = np.ascontiguousarray(match_d, dtype=np.int32)
    out = np.zeros((S.shape[0] + D.shape[0], 4), np.float32)
    act = np.zeros(S.shape[0] + D.shape[0], np.uint8)
    n = np.zeros(1, np.int32)
    lib().orc_update_tracks(_p(S, c_float), _p(a, c_uint8), S.shape[0], _p(D, c_float), D.shape[0],
                            _p(ms, c_int32), _p(md, c_int32), _p(out, c_float), _p(act, c_uint8),
                            _p(n, c_int32))
    return out[:n[0]], act[:n[0]]


def max_threads() -> int:
    return lib().orc_max_threads()
