"""Thin ctypes binding of libomt (include/omt.h).

Argument marshalling only: every step of the tracking path runs in the CUDA
kernels behind the C-ABI.  Torch provides device memory and streams.  There
is no CPU fallback: if libomt.so is missing or fails to load, every call
raises.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, Structure, c_float, c_int32, c_int64, c_size_t, c_uint8, c_uint32, c_void_p

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libomt.so")
ABI_VERSION = 400   # the library version whose structure layouts this binding mirrors

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ECHECK = 0, -1, -2, -3, -4, -5
F32, F16 = 0, 1
PT_OK, PT_LOST_EIG, PT_LOST_OOB, PT_NONCONV = 1, 2, 4, 8
MAX_LEVELS = 8
MAX_CORNERS = 4096

EXPORTED = [
    "omt_default_params", "omt_validate_params", "omt_pyramid_bytes", "omt_pyramid_init",
    "omt_build_pyramid", "omt_corner_response", "omt_corner_scratch_bytes",
    "omt_select_corners", "omt_lk_track", "omt_update_boxes", "omt_error_string",
    "omt_version", "omt_select_corners_static", "omt_batch_table_bytes", "omt_batch_pack",
    "omt_batch_step", "omt_batch_upload", "omt_batch_phase", "omt_iou_matrix",
    "omt_assign_workspace_bytes", "omt_assign", "omt_update_tracks", "omt_lk_wait_timeouts",
    "omt_fb_check", "omt_default_flow_params", "omt_structure_texture_scratch_bytes",
    "omt_tvl1_scratch_bytes", "omt_structure_texture", "omt_tvl1_flow", "omt_box_mean_flow",
    "omt_working_level", "omt_level_u8", "omt_scale_boxes", "omt_debug_fail_lk_wait",
]
PHASE_PYRAMID, PHASE_CORNERS, PHASE_LK, PHASE_BOXES, PHASE_FB = 0, 1, 2, 3, 4
PT_OK, PT_LOST_EIG, PT_LOST_OOB, PT_NONCONV, PT_LOST_FB, PT_LOST_TIMEOUT = 1, 2, 4, 8, 16, 32
BATCH_MAX_STREAMS = 256
STATIC_SCRATCH_BYTES = 16 << 20


class OmtError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {error_string(code)} ({code})")
        self.code = code


class Params(Structure):
    _fields_ = [("levels", c_int32), ("win", c_int32), ("max_iter", c_int32), ("eps", c_float),
                ("min_eig", c_float), ("quality_num", c_int32), ("quality_den", c_int32),
                ("min_dist", c_float), ("max_corners", c_int32), ("storage", c_int32),
                ("aggregator", c_int32), ("fb_max", c_float)]

    def replace(self, **kw) -> "Params":
        p = Params()
        ctypes.pointer(p)[0] = self
        for k, v in kw.items():
            setattr(p, k, v)
        return p

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class Level(Structure):
    _fields_ = [("w", c_int32), ("h", c_int32), ("img_off", c_int64), ("img_pitch", c_int64),
                ("grad_off", c_int64), ("grad_pitch", c_int64)]


class PyramidDesc(Structure):
    _fields_ = [("w", c_int32), ("h", c_int32), ("levels", c_int32), ("storage", c_int32),
                ("base", c_void_p), ("bytes", c_size_t), ("lv", Level * MAX_LEVELS)]


class BatchStream(Structure):
    _fields_ = [("frame", c_void_p), ("frame_pitch", c_size_t), ("prev", PyramidDesc),
                ("next", PyramidDesc), ("boxes", c_void_p), ("nboxes", c_int32),
                ("max_corners", c_int32), ("scratch", c_void_p), ("scratch_bytes", c_size_t),
                ("pts", c_void_p), ("pts_out", c_void_p), ("status", c_void_p),
                ("iters", c_void_p), ("offsets", c_void_p), ("boxes_out", c_void_p),
                ("nvalid", c_void_p), ("pts_back", c_void_p), ("status_back", c_void_p)]


class FlowParams(Structure):
    _fields_ = [("st_theta", c_float), ("st_alpha", c_float), ("st_k", c_float),
                ("st_iters", c_int32), ("lambda_", c_float), ("eps", c_float), ("warps", c_int32),
                ("iters", c_int32), ("block", c_int32)]


class BatchCaps(Structure):
    _fields_ = [("max_streams", c_int32), ("max_boxes", c_int32), ("max_w", c_int32),
                ("max_h", c_int32), ("max_corners", c_int32),
                ("lk_warps", c_int32), ("lk_ctas_per_sm", c_int32), ("lk_chunk", c_int32),
                ("pyr_ctas_per_sm", c_int32), ("corner_ctas_per_sm", c_int32),
                ("select_ctas_per_sm", c_int32), ("reserved", c_int32)]


_lib = None


def lib():
    """The loaded libomt.so (raises if it is missing; never falls back)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError(f"libomt.so not built at {LIB_PATH}; run python -m paper_1910_06017_b300.build")
        L = ctypes.CDLL(LIB_PATH)
        P = POINTER(PyramidDesc)
        L.omt_default_params.argtypes = [POINTER(Params)]
        L.omt_default_params.restype = None
        L.omt_validate_params.argtypes = [POINTER(Params)]
        L.omt_pyramid_bytes.argtypes = [c_int32, c_int32, c_int32, c_int32]
        L.omt_pyramid_bytes.restype = c_size_t
        L.omt_pyramid_init.argtypes = [P, c_int32, c_int32, c_int32, c_int32, c_void_p, c_size_t]
        L.omt_build_pyramid.argtypes = [c_void_p, c_int32, c_int32, c_size_t, POINTER(Params), P, c_void_p]
        L.omt_corner_response.argtypes = [P, c_void_p, c_void_p]
        L.omt_corner_scratch_bytes.argtypes = [c_int32, c_int32, c_int32, c_int32]
        L.omt_corner_scratch_bytes.restype = c_size_t
        L.omt_select_corners.argtypes = [P, c_void_p, c_int32, POINTER(Params), c_void_p, c_size_t,
                                         c_void_p, c_void_p, c_void_p]
        L.omt_lk_track.argtypes = [P, P, c_void_p, c_int32, c_void_p, POINTER(Params), c_void_p,
                                   c_void_p, c_void_p, c_void_p]
        L.omt_update_boxes.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int32,
                                       POINTER(Params), c_void_p, c_void_p, c_void_p]
        L.omt_error_string.argtypes = [c_int32]
        L.omt_error_string.restype = ctypes.c_char_p
        L.omt_version.restype = c_int32
        if L.omt_version() != ABI_VERSION:
            raise OSError(f"{LIB_PATH} is version {L.omt_version()}, the binding's structures are "
                          f"those of version {ABI_VERSION}; rebuild the library")
        L.omt_iou_matrix.argtypes = [c_void_p, c_int32, c_void_p, c_int32, c_void_p, c_void_p]
        L.omt_assign_workspace_bytes.argtypes = [c_int32, c_int32]
        L.omt_assign_workspace_bytes.restype = c_size_t
        L.omt_assign.argtypes = [c_void_p, c_int32, c_int32, c_void_p, ctypes.c_double, c_void_p,
                                 c_size_t, c_void_p, c_void_p]
        L.omt_update_tracks.argtypes = [c_void_p, c_void_p, c_int32, c_void_p, c_int32, c_void_p,
                                        c_void_p, c_void_p, c_void_p, c_void_p]
        L.omt_lk_wait_timeouts.argtypes = [c_void_p]
        L.omt_debug_fail_lk_wait.argtypes = [c_int64]
        L.omt_default_flow_params.argtypes = [POINTER(FlowParams)]
        L.omt_working_level.argtypes = [c_int32, c_int32]
        L.omt_working_level.restype = c_int32
        L.omt_level_u8.argtypes = [POINTER(PyramidDesc), c_int32, c_void_p, c_size_t, c_void_p]
        L.omt_scale_boxes.argtypes = [c_void_p, c_int32, c_float, c_void_p, c_void_p]
        L.omt_structure_texture_scratch_bytes.argtypes = [c_int32, c_int32]
        L.omt_structure_texture_scratch_bytes.restype = c_size_t
        L.omt_tvl1_scratch_bytes.argtypes = [c_int32, c_int32]
        L.omt_tvl1_scratch_bytes.restype = c_size_t
        L.omt_structure_texture.argtypes = [c_void_p, c_int32, c_int32, c_size_t,
                                            POINTER(FlowParams), c_void_p, c_size_t, c_void_p,
                                            c_size_t, c_void_p]
        L.omt_tvl1_flow.argtypes = [POINTER(PyramidDesc), POINTER(PyramidDesc), POINTER(FlowParams),
                                    c_void_p, c_void_p, c_size_t, c_void_p]
        L.omt_box_mean_flow.argtypes = [c_void_p, c_int32, c_int32, c_void_p, c_int32, c_void_p,
                                        c_void_p]
        L.omt_fb_check.argtypes = [c_void_p, c_void_p, c_void_p, c_int32, c_void_p, c_float,
                                   c_void_p, c_void_p]
        L.omt_batch_table_bytes.argtypes = [POINTER(BatchCaps)]
        L.omt_batch_table_bytes.restype = c_size_t
        L.omt_batch_pack.argtypes = [POINTER(BatchStream), c_int32, POINTER(Params),
                                     POINTER(BatchCaps), c_void_p, c_size_t]
        L.omt_batch_step.argtypes = [c_void_p, POINTER(BatchCaps), POINTER(Params), c_void_p,
                                     c_size_t, c_void_p]
        L.omt_batch_upload.argtypes = [c_void_p, POINTER(BatchCaps), c_void_p, c_size_t, c_void_p]
        L.omt_batch_phase.argtypes = [c_void_p, POINTER(BatchCaps), POINTER(Params), c_int32,
                                      c_void_p]
        _lib = L
    return _lib


def error_string(code: int) -> str:
    return lib().omt_error_string(code).decode()


def _check(code: int, what: str):
    if code != OK:
        raise OmtError(code, what)


def _ptr(t):
    """Device address of a torch tensor, or None."""
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def default_params(**kw) -> Params:
    p = Params()
    lib().omt_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if k == "quality" and isinstance(v, (tuple, list)):
            p.quality_num, p.quality_den = int(v[0]), int(v[1])
        else:
            setattr(p, k, v)
    return p


def validate_params(p: Params) -> int:
    return lib().omt_validate_params(ctypes.byref(p))


def pyramid_bytes(w: int, h: int, levels: int, storage: int = F32) -> int:
    return int(lib().omt_pyramid_bytes(w, h, levels, storage))


class Pyramid:
    """A frame's pyramid in a torch-allocated device buffer."""

    def __init__(self, w: int, h: int, levels: int, storage: int = F32, device="cuda", buffer=None):
        import torch
        n = pyramid_bytes(w, h, levels, storage)
        if n == 0:
            raise OmtError(EINVAL, "pyramid shape")
        self.buffer = torch.empty(n, dtype=torch.uint8, device=device) if buffer is None else buffer
        self.desc = PyramidDesc()
        _check(lib().omt_pyramid_init(ctypes.byref(self.desc), w, h, levels, storage,
                                      _ptr(self.buffer), self.buffer.numel()), "omt_pyramid_init")
        self.w, self.h, self.levels, self.storage = w, h, levels, storage

    def level_size(self, L: int):
        return self.desc.lv[L].w, self.desc.lv[L].h

    def image(self, L: int):
        """Level L as a torch tensor (uint8 for L = 0, float32/float16 otherwise)."""
        import torch
        lv = self.desc.lv[L]
        raw = self.buffer[lv.img_off: lv.img_off + lv.img_pitch * lv.h].view(lv.h, lv.img_pitch)
        if L == 0:
            return raw[:, :lv.w]
        dt = torch.float32 if self.storage == F32 else torch.float16
        return raw.view(dt)[:, :lv.w]

    def grad(self, L: int):
        """Level L gradients (h, w, 2) as float32 or float16."""
        import torch
        lv = self.desc.lv[L]
        raw = self.buffer[lv.grad_off: lv.grad_off + lv.grad_pitch * lv.h].view(lv.h, lv.grad_pitch)
        dt = torch.float32 if self.storage == F32 else torch.float16
        return raw.view(dt)[:, :2 * lv.w].reshape(lv.h, lv.w, 2)


def build_pyramid(frame, pyr: Pyramid, params: Params, stream=None):
    """frame: 2-D uint8 CUDA tensor (rows may be padded: stride(0) is the pitch)."""
    assert frame.dtype.itemsize == 1 and frame.dim() == 2 and frame.stride(1) == 1
    h, w = frame.shape
    _check(lib().omt_build_pyramid(_ptr(frame), w, h, frame.stride(0), ctypes.byref(params),
                                   ctypes.byref(pyr.desc), _stream(stream)), "omt_build_pyramid")


def corner_response(pyr: Pyramid, out, stream=None):
    """out: int32/uint32-sized CUDA tensor of h*w elements."""
    _check(lib().omt_corner_response(ctypes.byref(pyr.desc), _ptr(out), _stream(stream)),
           "omt_corner_response")


def corner_scratch_bytes(w: int, h: int, nboxes: int, max_corners: int) -> int:
    return int(lib().omt_corner_scratch_bytes(w, h, nboxes, max_corners))


def select_corners(pyr: Pyramid, boxes, params: Params, scratch, pts, offsets, stream=None):
    """boxes float32 (nb, 4); pts float32 (nb*max_corners, 2); offsets int32 (nb+1)."""
    nb = boxes.shape[0] if boxes is not None else 0
    _check(lib().omt_select_corners(ctypes.byref(pyr.desc), _ptr(boxes), nb, ctypes.byref(params),
                                    _ptr(scratch), scratch.numel() * scratch.element_size(),
                                    _ptr(pts), _ptr(offsets), _stream(stream)), "omt_select_corners")


def select_corners_static(pyr: Pyramid, boxes, params: Params, pts, offsets, stream=None):
    """select_corners without a scratch argument: the library's own fixed
    device array is used instead (for callers that cannot allocate).  Calls
    share that array, so they must not overlap on the GPU."""
    L = lib()
    fn = L.omt_select_corners_static
    fn.argtypes = [POINTER(PyramidDesc), c_void_p, c_int32, POINTER(Params), c_void_p, c_void_p,
                   c_void_p]
    nb = boxes.shape[0] if boxes is not None else 0
    _check(fn(ctypes.byref(pyr.desc), _ptr(boxes), nb, ctypes.byref(params), _ptr(pts),
              _ptr(offsets), _stream(stream)), "omt_select_corners_static")


def lk_track(prev: Pyramid, nxt: Pyramid, pts, params: Params, pts_out, status, iters=None,
             n_max=None, n_dev=None, stream=None):
    n = pts.shape[0] if n_max is None else n_max
    _check(lib().omt_lk_track(ctypes.byref(prev.desc), ctypes.byref(nxt.desc), _ptr(pts), n,
                              _ptr(n_dev), ctypes.byref(params), _ptr(pts_out), _ptr(status),
                              _ptr(iters), _stream(stream)), "omt_lk_track")


def fb_check(pts, pts_back, status_back, fb_max: float, status, n_max=None, n_dev=None,
             stream=None):
    """Forward-backward check (device tensors): status[i] with OK becomes
    LOST_FB unless status_back[i] has OK and |pts_back[i] - pts[i]| <= fb_max."""
    n = pts.shape[0] if n_max is None else n_max
    _check(lib().omt_fb_check(_ptr(pts), _ptr(pts_back), _ptr(status_back), n, _ptr(n_dev),
                              float(fb_max), _ptr(status), _stream(stream)), "omt_fb_check")


def lk_track_fb(prev: Pyramid, nxt: Pyramid, pts, params: Params, fb_max: float, pts_out, status,
                pts_back, status_back, iters=None, n_max=None, n_dev=None, stream=None):
    """Forward LK (prev -> nxt), backward LK from its results (nxt -> prev)
    and the forward-backward check, as three calls on one stream."""
    lk_track(prev, nxt, pts, params, pts_out, status, iters, n_max, n_dev, stream)
    lk_track(nxt, prev, pts_out, params, pts_back, status_back, None, n_max, n_dev, stream)
    fb_check(pts, pts_back, status_back, fb_max, status, n_max, n_dev, stream)


def working_level(w: int, h: int) -> int:
    """Pyramid level processed for a w x h frame: 0 SD/HD, 1 2K, 2 4K."""
    return int(lib().omt_working_level(w, h))


def level_u8(pyr: "Pyramid", level: int, out, stream=None):
    """Level `level` of an F32 pyramid rounded to u8 into out (device (h_L, w_L))."""
    _check(lib().omt_level_u8(ctypes.byref(pyr.desc), int(level), _ptr(out), out.stride(0),
                              _stream(stream)), "omt_level_u8")


def scale_boxes(boxes, scale: float, out, stream=None):
    """out = boxes * scale (device (n, 4) float32)."""
    _check(lib().omt_scale_boxes(_ptr(boxes), boxes.shape[0], float(scale), _ptr(out),
                                 _stream(stream)), "omt_scale_boxes")


def default_flow_params(**kw) -> FlowParams:
    """Dense-flow parameters (the library's readings), with overrides;
    `lambda_` is the data weight."""
    p = FlowParams()
    lib().omt_default_flow_params(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def structure_texture(frame, params: FlowParams, texture, scratch=None, stream=None):
    """u8 texture image of a u8 device frame (h, w) into texture (h, w)."""
    import torch
    h, w = frame.shape
    n = lib().omt_structure_texture_scratch_bytes(w, h)
    if scratch is None:
        scratch = torch.empty(n, dtype=torch.uint8, device=frame.device)
    _check(lib().omt_structure_texture(_ptr(frame), w, h, frame.stride(0), ctypes.byref(params),
                                       _ptr(texture), texture.stride(0), _ptr(scratch),
                                       scratch.numel(), _stream(stream)), "omt_structure_texture")


def tvl1_flow(prev: "Pyramid", nxt: "Pyramid", params: FlowParams, flow, scratch=None,
              stream=None):
    """Dense flow (device (h, w, 2) float32) from prev to nxt (F32 pyramids)."""
    import torch
    n = lib().omt_tvl1_scratch_bytes(prev.w, prev.h)
    if scratch is None:
        scratch = torch.empty(n, dtype=torch.uint8, device=flow.device)
    _check(lib().omt_tvl1_flow(ctypes.byref(prev.desc), ctypes.byref(nxt.desc),
                               ctypes.byref(params), _ptr(flow), _ptr(scratch), scratch.numel(),
                               _stream(stream)), "omt_tvl1_flow")


def box_mean_flow(flow, boxes, boxes_out, stream=None):
    """Boxes moved by the mean flow inside them (device tensors)."""
    h, w = flow.shape[:2]
    _check(lib().omt_box_mean_flow(_ptr(flow), w, h, _ptr(boxes), boxes.shape[0], _ptr(boxes_out),
                                   _stream(stream)), "omt_box_mean_flow")


def update_boxes(boxes, offsets, pts, pts_out, status, params: Params, boxes_out, nvalid=None,
                 stream=None):
    nb = boxes.shape[0]
    _check(lib().omt_update_boxes(_ptr(boxes), _ptr(offsets), _ptr(pts), _ptr(pts_out),
                                  _ptr(status), nb, ctypes.byref(params), _ptr(boxes_out),
                                  _ptr(nvalid), _stream(stream)), "omt_update_boxes")


def iou_matrix(a, b, out, stream=None):
    """IoU of every pair of boxes (device tensors (na, 4), (nb, 4) float32)
    into out (device (na, nb) float64), Section V-A matching score."""
    _check(lib().omt_iou_matrix(_ptr(a), a.shape[0], _ptr(b), b.shape[0], _ptr(out), _stream(stream)),
           "omt_iou_matrix")


def _np_ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None and a.size else None


def assign(iou, active=None, iou_min: float = 0.0):
    """Maximum-total-IoU assignment (host numpy (na, nb) float64): returns
    (match_a, match_b) int32, -1 where unmatched."""
    import numpy as np
    m = np.ascontiguousarray(iou, dtype=np.float64)
    na, nb = m.shape
    act = None if active is None else np.ascontiguousarray(active, dtype=np.uint8)
    ws = np.empty(max(1, lib().omt_assign_workspace_bytes(na, nb)), np.uint8)
    ma, mb = np.empty(na, np.int32), np.empty(nb, np.int32)
    _check(lib().omt_assign(_np_ptr(m), na, nb, _np_ptr(act), float(iou_min), _np_ptr(ws), ws.size,
                            _np_ptr(ma), _np_ptr(mb)), "omt_assign")
    return ma, mb


def update_tracks(boxes_s, active_s, boxes_d, match_s, match_d):
    """Update phase on host arrays: returns (boxes (n, 4) float32, active (n,) uint8)."""
    import numpy as np
    S = np.ascontiguousarray(boxes_s, dtype=np.float32).reshape(-1, 4)
    D = np.ascontiguousarray(boxes_d, dtype=np.float32).reshape(-1, 4)
    a = np.ascontiguousarray(active_s, dtype=np.uint8)
    ms, md = np.ascontiguousarray(match_s, dtype=np.int32), np.ascontiguousarray(match_d, dtype=np.int32)
    out = np.zeros((S.shape[0] + D.shape[0], 4), np.float32)
    act = np.zeros(S.shape[0] + D.shape[0], np.uint8)
    n = np.zeros(1, np.int32)
    _check(lib().omt_update_tracks(_np_ptr(S), _np_ptr(a), S.shape[0], _np_ptr(D), D.shape[0],
                                   _np_ptr(ms), _np_ptr(md), _np_ptr(out), _np_ptr(act),
                                   ctypes.c_void_p(n.ctypes.data)), "omt_update_tracks")
    return out[:n[0]], act[:n[0]]


def lk_wait_timeouts() -> int:
    """LK window-copy waits that reached their time limit since the previous
    call (0 unless the copy engine stalled; the points concerned came back
    PT_LOST_TIMEOUT).  The C call returns OMT_ETIMEOUT when the count is not
    0; here the count is the answer."""
    c = ctypes.c_uint32(0)
    rc = lib().omt_lk_wait_timeouts(ctypes.byref(c))
    if rc != ETIMEOUT:
        _check(rc, "omt_lk_wait_timeouts")
    return int(c.value)


def debug_fail_lk_wait(point: int) -> None:
    """Test hook: make the wait for the first search window of LK point
    `point` run out (omt_debug_fail_lk_wait); -1 turns it off."""
    _check(lib().omt_debug_fail_lk_wait(int(point)), "omt_debug_fail_lk_wait")


def match_and_update(pred, active, dets, iou_min: float = 0.0, stream=None):
    """Matching and update phases for one stream: pred (device (ns, 4)
    float32, the predicted scene objects), active (host (ns,) uint8), dets
    (device (nd, 4) float32).  The IoU matrix is computed on the device and
    read back; the assignment and update run on the host.  Returns
    (boxes (n, 4) float32, active (n,) uint8, match_s, match_d) on the host."""
    import numpy as np
    import torch
    ns, nd = pred.shape[0], dets.shape[0]
    iou = torch.empty((ns, nd), dtype=torch.float64, device=pred.device)
    iou_matrix(pred, dets, iou, stream)
    host = torch.empty((ns, nd), dtype=torch.float64).pin_memory()
    host.copy_(iou)
    m = host.numpy()
    ms, md = assign(m, active, iou_min)
    boxes, act = update_tracks(pred.cpu().numpy(), active, dets.cpu().numpy(), ms, md)
    return boxes, act, ms, md


class StreamTracker:
    """Per-stream state for the plain path: two pyramids (t, t+1) that swap
    roles, and the buffers one step needs.  step() runs the whole hot path
    (pyramid of the new frame, corners of frame t inside the boxes, LK, box
    update) as five asynchronous C-ABI calls with no host synchronisation."""

    def __init__(self, w: int, h: int, params: Params, max_boxes: int, device="cuda"):
        import torch
        self.w, self.h, self.params = w, h, params
        self.pyr = [Pyramid(w, h, params.levels, params.storage, device),
                    Pyramid(w, h, params.levels, params.storage, device)]
        self.cur = 0
        self.max_boxes = max_boxes
        cap = max(1, max_boxes * params.max_corners)
        self.scratch = torch.empty(corner_scratch_bytes(w, h, max_boxes, params.max_corners),
                                   dtype=torch.uint8, device=device)
        self.pts = torch.empty((cap, 2), dtype=torch.float32, device=device)
        self.pts_out = torch.empty((cap, 2), dtype=torch.float32, device=device)
        self.status = torch.empty(cap, dtype=torch.uint8, device=device)
        self.iters = torch.empty((cap, params.levels), dtype=torch.uint8, device=device)
        self.offsets = torch.empty(max_boxes + 1, dtype=torch.int32, device=device)
        self.boxes_out = torch.empty((max(1, max_boxes), 4), dtype=torch.float32, device=device)
        self.nvalid = torch.empty(max(1, max_boxes), dtype=torch.int32, device=device)

    def prime(self, frame, stream=None):
        build_pyramid(frame, self.pyr[self.cur], self.params, stream)

    def step(self, frame_next, boxes, stream=None, with_iters: bool = True):
        """Track boxes (nb, 4) of frame t into frame t+1; returns boxes_out[:nb]."""
        nb = boxes.shape[0]
        assert nb <= self.max_boxes
        prev, nxt = self.pyr[self.cur], self.pyr[1 - self.cur]
        build_pyramid(frame_next, nxt, self.params, stream)
        select_corners(prev, boxes, self.params, self.scratch, self.pts, self.offsets, stream)
        cap = nb * self.params.max_corners
        lk_track(prev, nxt, self.pts, self.params, self.pts_out, self.status,
                 self.iters if with_iters else None, n_max=cap, n_dev=self.offsets[nb:nb + 1],
                 stream=stream)
        update_boxes(boxes, self.offsets, self.pts, self.pts_out, self.status, self.params,
                     self.boxes_out[:nb], self.nvalid[:nb], stream)
        self.cur = 1 - self.cur
        return self.boxes_out[:nb]


class WorkingLevelTracker:
    """The plain path on a frame's working level (Section V-A preprocessing:
    a pyramid level chosen by resolution).  Each incoming frame is reduced
    to its working frame (an F32 pyramid of level+1 levels, its last level
    rounded to u8), and a StreamTracker of the working size tracks the boxes
    scaled into level-L pixels; boxes come back in level-0 pixels.  Every
    step is C-ABI calls on one stream."""

    def __init__(self, w: int, h: int, params: Params, max_boxes: int, level=None,
                 device="cuda"):
        import torch
        self.level = working_level(w, h) if level is None else int(level)
        self.reduce = default_params(levels=self.level + 1, storage=F32)
        self.full = Pyramid(w, h, self.level + 1, F32, device)
        self.lw, self.lh = self.full.level_size(self.level)
        self.work = torch.empty((self.lh, self.lw), dtype=torch.uint8, device=device)
        self.inner = StreamTracker(self.lw, self.lh, params, max_boxes, device)
        self.boxes_work = torch.empty((max(1, max_boxes), 4), dtype=torch.float32, device=device)
        self.boxes_out = torch.empty((max(1, max_boxes), 4), dtype=torch.float32, device=device)

    def _working_frame(self, frame, stream=None):
        build_pyramid(frame, self.full, self.reduce, stream)
        level_u8(self.full, self.level, self.work, stream)

    def prime(self, frame, stream=None):
        self._working_frame(frame, stream)
        self.inner.prime(self.work, stream)

    def step(self, frame_next, boxes, stream=None):
        """Track boxes (nb, 4, level-0 px) of frame t into frame t+1."""
        nb = boxes.shape[0]
        self._working_frame(frame_next, stream)
        scale_boxes(boxes, 2.0 ** -self.level, self.boxes_work[:nb], stream)
        out = self.inner.step(self.work, self.boxes_work[:nb], stream)
        scale_boxes(out, 2.0 ** self.level, self.boxes_out[:nb], stream)
        return self.boxes_out[:nb]


# ------------------------------------------------------------------ batched

def batch_table_bytes(caps: BatchCaps) -> int:
    return int(lib().omt_batch_table_bytes(ctypes.byref(caps)))


def batch_pack(streams, params: Params, caps: BatchCaps, table):
    """streams: sequence of BatchStream; table: host uint8 tensor (pinned for graphs)."""
    arr = (BatchStream * max(1, len(streams)))(*streams)
    _check(lib().omt_batch_pack(arr, len(streams), ctypes.byref(params), ctypes.byref(caps),
                                ctypes.c_void_p(table.data_ptr()), table.numel()), "omt_batch_pack")


def batch_step(table, caps: BatchCaps, params: Params, dev_table, stream=None):
    _check(lib().omt_batch_step(ctypes.c_void_p(table.data_ptr()), ctypes.byref(caps),
                                ctypes.byref(params), _ptr(dev_table), dev_table.numel(),
                                _stream(stream)), "omt_batch_step")


def batch_upload(table, caps: BatchCaps, dev_table, stream=None):
    _check(lib().omt_batch_upload(ctypes.c_void_p(table.data_ptr()), ctypes.byref(caps),
                                  _ptr(dev_table), dev_table.numel(), _stream(stream)),
           "omt_batch_upload")


def batch_phase(dev_table, caps: BatchCaps, params: Params, phase: int, stream=None):
    _check(lib().omt_batch_phase(_ptr(dev_table), ctypes.byref(caps), ctypes.byref(params),
                                 phase, _stream(stream)), "omt_batch_phase")


class BatchTracker:
    """Many independent streams advanced by one omt_batch_step per step.

    Every stream keeps, resident on the device, two pyramids that swap roles
    (frame t, frame t+1), two frame slots (the step with parity p reads
    frame t+1 from slot p), its input and output boxes, point buffers and
    corner scratch.  Two tables (one per
    pyramid parity) are packed into page-locked host memory and copied to two
    device tables by pack(); a step runs 4 + levels launches for all streams
    over the table of its parity.  capture() records each parity's step in a
    CUDA graph, which step() then replays.
    """

    def __init__(self, sizes, params: Params, max_boxes, max_corners=None, device="cuda",
                 with_iters: bool = True, overlap: bool = True):
        import torch
        self.params = params
        # run the corner phase (frame t) on a second stream beside the
        # pyramid phase (frame t+1): they touch disjoint buffers
        self.overlap = overlap
        self.device = torch.device(device)
        n = len(sizes)
        if isinstance(max_boxes, int):
            max_boxes = [max_boxes] * n
        if max_corners is None:
            max_corners = [params.max_corners] * n
        elif isinstance(max_corners, int):
            max_corners = [max_corners] * n
        self.sizes, self.max_boxes, self.max_corners = list(sizes), list(max_boxes), list(max_corners)
        self.caps = BatchCaps(n, int(sum(max_boxes)), max(w for w, _ in sizes),
                              max(h for _, h in sizes), max(max(max_corners), params.max_corners))
        dev = self.device
        self.pyr, self.frame, self.boxes, self.boxes_out = [], [], [], []
        self.pts, self.pts_out, self.status, self.iters, self.offsets, self.nvalid = [], [], [], [], [], []
        # the backward run of the forward-backward check (params.fb_max >= 0)
        self.fb = params.fb_max >= 0
        self.pts_back, self.status_back = [], []
        self.scratch, self.nboxes = [], [0] * n
        # every stream's output boxes in one buffer, so one copy reads them all
        nbs = [max(1, nb) for nb in max_boxes]
        self.boxes_out_all = torch.zeros((sum(nbs), 4), dtype=torch.float32, device=dev)
        self.boxes_out_at = [sum(nbs[:i]) for i in range(n)]
        for (w, h), nb, mc in zip(sizes, max_boxes, max_corners):
            self.pyr.append([Pyramid(w, h, params.levels, params.storage, dev),
                             Pyramid(w, h, params.levels, params.storage, dev)])
            self.frame.append([torch.zeros((h, w), dtype=torch.uint8, device=dev) for _ in range(2)])
            cap = max(1, nb * mc)
            self.boxes.append(torch.zeros((max(1, nb), 4), dtype=torch.float32, device=dev))
            at = self.boxes_out_at[len(self.boxes_out)]
            self.boxes_out.append(self.boxes_out_all[at:at + max(1, nb)])
            self.pts.append(torch.zeros((cap, 2), dtype=torch.float32, device=dev))
            self.pts_out.append(torch.zeros((cap, 2), dtype=torch.float32, device=dev))
            self.status.append(torch.zeros(cap, dtype=torch.uint8, device=dev))
            self.pts_back.append(torch.zeros((cap, 2), dtype=torch.float32, device=dev)
                                 if self.fb else None)
            self.status_back.append(torch.zeros(cap, dtype=torch.uint8, device=dev)
                                    if self.fb else None)
            self.iters.append(torch.zeros((cap, params.levels), dtype=torch.uint8, device=dev)
                              if with_iters else None)
            self.offsets.append(torch.zeros(nb + 1, dtype=torch.int32, device=dev))
            self.nvalid.append(torch.zeros(max(1, nb), dtype=torch.int32, device=dev))
            self.scratch.append(torch.empty(corner_scratch_bytes(w, h, nb, mc), dtype=torch.uint8,
                                            device=dev))
        nbytes = batch_table_bytes(self.caps)
        self.tables = [torch.empty(nbytes, dtype=torch.uint8).pin_memory() for _ in range(2)]
        self.dev_tables = [torch.empty(nbytes, dtype=torch.uint8, device=dev) for _ in range(2)]
        self.cur = 0
        self.graphs = [None, None]
        self.side = torch.cuda.Stream(device=dev)

    def _desc(self, s: int, parity: int) -> BatchStream:
        d = BatchStream()
        f = self.frame[s][parity]
        d.frame, d.frame_pitch = f.data_ptr(), f.stride(0)
        d.prev = self.pyr[s][parity].desc
        d.next = self.pyr[s][1 - parity].desc
        d.boxes = self.boxes[s].data_ptr()
        d.nboxes = self.nboxes[s]
        d.max_corners = self.max_corners[s]
        d.scratch, d.scratch_bytes = self.scratch[s].data_ptr(), self.scratch[s].numel()
        d.pts, d.pts_out = self.pts[s].data_ptr(), self.pts_out[s].data_ptr()
        d.status = self.status[s].data_ptr()
        d.iters = self.iters[s].data_ptr() if self.iters[s] is not None else None
        d.offsets = self.offsets[s].data_ptr()
        d.boxes_out, d.nvalid = self.boxes_out[s].data_ptr(), self.nvalid[s].data_ptr()
        if self.fb:
            d.pts_back, d.status_back = self.pts_back[s].data_ptr(), self.status_back[s].data_ptr()
        return d

    def slot(self, s: int):
        """Device frame slot the next step reads frame t+1 of stream s from."""
        return self.frame[s][self.cur]

    def set_boxes(self, s: int, boxes):
        """Boxes of stream s on frame t (device or host tensor (nb, 4))."""
        nb = boxes.shape[0]
        assert nb <= self.max_boxes[s]
        if nb:
            self.boxes[s][:nb].copy_(boxes, non_blocking=True)
        self.nboxes[s] = nb
        self.graphs = [None, None]

    def pack(self, stream=None):
        """Pack both parities' tables and copy them to the device (on
        `stream`, ordered after the steps already queued there)."""
        for parity in range(2):
            batch_pack([self._desc(s, parity) for s in range(len(self.sizes))], self.params,
                       self.caps, self.tables[parity])
            batch_upload(self.tables[parity], self.caps, self.dev_tables[parity], stream)

    def _phases(self, parity, events=None, stream=None):
        if self.overlap and not events:
            import torch
            main = stream if stream is not None else torch.cuda.current_stream(self.device)
            dt = self.dev_tables[parity]
            self.side.wait_stream(main)
            batch_phase(dt, self.caps, self.params, PHASE_PYRAMID, main)
            batch_phase(dt, self.caps, self.params, PHASE_CORNERS, self.side)
            main.wait_stream(self.side)
            batch_phase(dt, self.caps, self.params, PHASE_LK, main)
            if self.fb:
                batch_phase(dt, self.caps, self.params, PHASE_FB, main)
            batch_phase(dt, self.caps, self.params, PHASE_BOXES, main)
            return
        events = events or {}
        phases = (PHASE_PYRAMID, PHASE_CORNERS, PHASE_LK) + ((PHASE_FB,) if self.fb else ()) + \
            (PHASE_BOXES,)
        for phase in phases:
            ev = events.get(phase)
            if ev:
                ev[0].record()
            batch_phase(self.dev_tables[parity], self.caps, self.params, phase, stream)
            if ev:
                ev[1].record()

    def prime(self, s: int, frame, stream=None):
        """Build stream s's frame-t pyramid from a u8 device frame."""
        build_pyramid(frame, self.pyr[s][self.cur], self.params, stream)

    def capture(self):
        """Capture each parity's step in a CUDA graph (after one eager step)."""
        import torch
        self.pack()
        self.graphs = [None, None]
        torch.cuda.synchronize()
        for parity in range(2):
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, capture_error_mode="relaxed"):
                self._phases(parity)
            self.graphs[parity] = g

    def step(self, stream=None):
        """Advance every stream: frame slots hold frame t+1, boxes frame t's."""
        if self.graphs[self.cur] is not None:
            self.graphs[self.cur].replay()
        else:
            self._phases(self.cur, stream=stream)
        self.cur = 1 - self.cur

    def step_phases(self, events=None, stream=None):
        """The step as its four phases, eagerly.  events: optional dict phase ->
        (start, end) CUDA events recorded around that phase."""
        self._phases(self.cur, events, stream)
        self.cur = 1 - self.cur

    # Launch shapes the autotuner tries: (warps per CTA, points per work-queue take).
    TUNE_CANDIDATES = tuple((w, c) for w in (2, 4, 8) for c in (1, 2, 4))
    # CTAs per SM of the pyramid kernels, and (list kernel, select kernel) of
    # the corner phase; 0 = as many as fit
    TUNE_PYRAMID = (0, 1, 2, 4)
    TUNE_CORNERS = tuple((c, s) for c in (0, 4, 8) for s in (0, 2, 4))

    def _time_phase(self, phase, reps, stream, setup=()):
        """Median CUDA-event time (ms) of `phase` over `reps` runs after one
        untimed run; the phases in `setup` run before each (not timed)."""
        import torch
        par = self.cur
        ms = []
        for k in range(reps + 1):
            for p in setup:
                batch_phase(self.dev_tables[par], self.caps, self.params, p, stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            batch_phase(self.dev_tables[par], self.caps, self.params, phase, stream)
            e1.record()
            e1.synchronize()
            if k:
                ms.append(e0.elapsed_time(e1))
        return sorted(ms)[len(ms) // 2]

    def autotune(self, candidates=None, reps: int = 3, stream=None) -> dict:
        """Pick the batched launch shapes that are fastest on this batch.

        Each phase's shape is timed alone with CUDA events on the caller's
        own batch (the median of `reps` runs after one untimed run) and the
        fastest is kept in self.caps: CTAs per SM of the pyramid kernels
        (TUNE_PYRAMID), CTAs per SM of the corner-list and select kernels
        (TUNE_CORNERS, with the counters reset by the phase itself), then,
        with the corners of frame t selected, warps per CTA and work-queue
        chunk of the LK kernel (`candidates`, default TUNE_CANDIDATES).  No
        result depends on any shape.  The state afterwards is as before the
        call except for the rebuilt frame t+1 pyramids; captured graphs are
        dropped (capture again).  Returns {"lk": {(warps, chunk): ms},
        "pyramid": {ctas: ms}, "corners": {(list_ctas, select_ctas): ms}}."""
        out = {"pyramid": {}, "corners": {}, "lk": {}}
        for c in self.TUNE_PYRAMID:
            self.caps.pyr_ctas_per_sm = int(c)
            out["pyramid"][int(c)] = self._time_phase(PHASE_PYRAMID, reps, stream)
        self.caps.pyr_ctas_per_sm = min(out["pyramid"], key=out["pyramid"].get)
        for c, s in self.TUNE_CORNERS:
            self.caps.corner_ctas_per_sm, self.caps.select_ctas_per_sm = int(c), int(s)
            out["corners"][(int(c), int(s))] = self._time_phase(PHASE_CORNERS, reps, stream)
        self.caps.corner_ctas_per_sm, self.caps.select_ctas_per_sm = min(
            out["corners"], key=out["corners"].get)
        batch_phase(self.dev_tables[self.cur], self.caps, self.params, PHASE_PYRAMID, stream)
        batch_phase(self.dev_tables[self.cur], self.caps, self.params, PHASE_CORNERS, stream)
        for w, c in list(candidates or self.TUNE_CANDIDATES):
            self.caps.lk_warps, self.caps.lk_chunk = int(w), int(c)
            out["lk"][(int(w), int(c))] = self._time_phase(PHASE_LK, reps, stream)
        self.caps.lk_warps, self.caps.lk_chunk = min(out["lk"], key=out["lk"].get)
        self.graphs = [None, None]
        return out

    def count(self, s: int) -> int:
        return int(self.offsets[s][self.nboxes[s]].item())

    def run_pipelined(self, frames_for, steps: int, consume=None, copy_stream=None):
        """Run `steps` steps with host frames in and boxes out, overlapping
        the copies with compute.

        frames_for(k) returns step k's frames (page-locked host u8 tensors,
        one per stream, frame t+1 of every stream).  They are copied on a
        copy stream while step k-1 computes; the compute stream waits for
        them.  Step k reads the frame slots of its parity, which step k-2
        read last, so the copy for step k waits for step k-2.  After each
        step its output boxes are copied to page-locked host memory (two
        alternating buffers) and consume(k, boxes) runs on the host once
        they have arrived, while step k+1 computes.  Returns the bytes
        copied host to device and device to host."""
        import torch
        comp = torch.cuda.current_stream(self.device)
        up = copy_stream or torch.cuda.Stream(device=self.device)
        n = len(self.sizes)
        outs_all = [torch.empty(self.boxes_out_all.shape, dtype=torch.float32).pin_memory()
                    for _ in range(2)]
        at = self.boxes_out_at
        outs = [[o[at[s]:at[s] + max(1, self.nboxes[s])] for s in range(n)] for o in outs_all]
        h2d = d2h = 0
        done_step = [None] * steps
        done_d2h = [None] * steps

        def upload(k, parity):
            nonlocal h2d
            with torch.cuda.stream(up):
                if k >= 2:
                    up.wait_event(done_step[k - 2])
                for s, f in enumerate(frames_for(k)):
                    self.frame[s][parity].copy_(f, non_blocking=True)
                    h2d += f.numel() * f.element_size()
                e = torch.cuda.Event()
                e.record(up)
            return e

        ready = upload(0, self.cur)
        for k in range(steps):
            comp.wait_event(ready)
            self.step()
            done_step[k] = torch.cuda.Event()
            done_step[k].record(comp)
            outs_all[k & 1].copy_(self.boxes_out_all, non_blocking=True)
            d2h += self.boxes_out_all.numel() * 4
            done_d2h[k] = torch.cuda.Event()
            done_d2h[k].record(comp)
            if k + 1 < steps:
                ready = upload(k + 1, self.cur)
            if k >= 1:
                done_d2h[k - 1].synchronize()
                if consume:
                    consume(k - 1, [outs[(k - 1) & 1][s][:self.nboxes[s]] for s in range(n)])
        if steps:
            done_d2h[steps - 1].synchronize()
            if consume:
                consume(steps - 1, [outs[(steps - 1) & 1][s][:self.nboxes[s]] for s in range(n)])
        return h2d, d2h
