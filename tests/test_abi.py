"""The C-ABI library loads on a machine without a GPU, exports every entry
point include/omt.h declares, and rejects bad arguments on the host before
any launch (these calls never reach the device)."""
import ctypes
import os
import re

import pytest

from paper_1910_06017_b300 import omt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(omt_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported():
    lib = omt.lib()
    declared = _declared()
    assert len(declared) >= 12
    for name in declared:
        assert hasattr(lib, name), name
    assert set(omt.EXPORTED) <= set(declared)


def test_nm_lists_symbols():
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", omt.LIB_PATH], capture_output=True,
                         text=True).stdout
    for name in _declared():
        assert re.search(rf"\bT {name}\b", out), name


def test_default_params_are_valid():
    p = omt.default_params()
    assert omt.validate_params(p) == omt.OK
    assert (p.levels, p.win, p.max_iter, p.max_corners) == (3, 21, 30, 50)
    assert (p.quality_num, p.quality_den) == (1, 100)


@pytest.mark.parametrize("field,value", [("levels", 0), ("levels", 9), ("win", 4), ("win", 33),
                                         ("win", 1), ("max_iter", 0), ("max_iter", 256),
                                         ("eps", -1.0), ("eps", float("nan")),
                                         ("min_eig", -0.1), ("quality_den", 0),
                                         ("quality_num", -1), ("min_dist", -1.0),
                                         ("max_corners", -1), ("max_corners", 4097),
                                         ("storage", 2), ("aggregator", 2)])
def test_invalid_params_rejected(field, value):
    p = omt.default_params().replace(**{field: value})
    assert omt.validate_params(p) == omt.EINVAL


def test_pyramid_layout_alignment():
    for (w, h, L, st) in [(720, 576, 3, 0), (37, 23, 5, 1), (1, 1, 8, 0), (3840, 2160, 5, 1)]:
        n = omt.pyramid_bytes(w, h, L, st)
        assert n > 0
        d = omt.PyramidDesc()
        fake = 1 << 20  # never dereferenced: init is host-only
        assert omt.lib().omt_pyramid_init(ctypes.byref(d), w, h, L, st, ctypes.c_void_p(fake), n) == 0
        lw, lh = w, h
        for i in range(L):
            lv = d.lv[i]
            assert (lv.w, lv.h) == (lw, lh)
            assert lv.img_off % 256 == 0 and lv.grad_off % 256 == 0
            assert lv.img_pitch % 128 == 0 and lv.grad_pitch % 128 == 0
            esz = 1 if i == 0 else (4 if st == 0 else 2)
            assert lv.img_pitch >= lw * esz and lv.grad_pitch >= lw * 2 * (4 if st == 0 else 2)
            assert lv.grad_off >= lv.img_off + lv.img_pitch * lh
            lw, lh = (lw + 1) >> 1, (lh + 1) >> 1
        assert omt.lib().omt_pyramid_init(ctypes.byref(d), w, h, L, st, ctypes.c_void_p(fake), n - 1) == omt.ENOMEM
        assert omt.lib().omt_pyramid_init(ctypes.byref(d), w, h, L, st, ctypes.c_void_p(fake + 64), n) == omt.EINVAL
    assert omt.pyramid_bytes(0, 5, 3, 0) == 0
    assert omt.pyramid_bytes(5, 5, 9, 0) == 0


def test_invalid_calls_rejected_before_launch():
    lib = omt.lib()
    p = omt.default_params()
    d = omt.PyramidDesc()
    n = omt.pyramid_bytes(64, 48, 3, 0)
    assert lib.omt_pyramid_init(ctypes.byref(d), 64, 48, 3, 0, ctypes.c_void_p(1 << 20), n) == 0
    fake = ctypes.c_void_p(1 << 24)
    # frame size differs from the pyramid's
    assert lib.omt_build_pyramid(fake, 65, 48, 65, ctypes.byref(p), ctypes.byref(d), None) == omt.EINVAL
    # pitch below width
    assert lib.omt_build_pyramid(fake, 64, 48, 63, ctypes.byref(p), ctypes.byref(d), None) == omt.EINVAL
    # params storage differs from the pyramid's
    p16 = p.replace(storage=1)
    assert lib.omt_build_pyramid(fake, 64, 48, 64, ctypes.byref(p16), ctypes.byref(d), None) == omt.EINVAL
    # scratch too small
    need = lib.omt_corner_scratch_bytes(64, 48, 4, 50)
    assert lib.omt_select_corners(ctypes.byref(d), fake, 4, ctypes.byref(p), ctypes.c_void_p(1 << 26),
                                  need - 1, fake, fake, None) == omt.ENOMEM
    # misaligned scratch
    assert lib.omt_select_corners(ctypes.byref(d), fake, 4, ctypes.byref(p), ctypes.c_void_p((1 << 26) + 8),
                                  need, fake, fake, None) == omt.EINVAL
    # pyramids of different shape
    d2 = omt.PyramidDesc()
    n2 = omt.pyramid_bytes(64, 40, 3, 0)
    assert lib.omt_pyramid_init(ctypes.byref(d2), 64, 40, 3, 0, ctypes.c_void_p(1 << 22), n2) == 0
    assert lib.omt_lk_track(ctypes.byref(d), ctypes.byref(d2), fake, 10, None, ctypes.byref(p),
                            fake, fake, None, None) == omt.EINVAL
    # a corrupted descriptor is rejected
    d.lv[1].img_off += 256
    assert lib.omt_corner_response(ctypes.byref(d), fake, None) == omt.EINVAL
    # in-place box update is rejected
    assert lib.omt_update_boxes(fake, fake, fake, fake, fake, 3, ctypes.byref(p), fake, None,
                                None) == omt.EINVAL
    # zero boxes is a no-op
    assert lib.omt_update_boxes(None, None, None, None, None, 0, ctypes.byref(p), None, None,
                                None) == omt.OK


def test_error_strings():
    assert omt.error_string(omt.OK) == "success"
    assert "invalid" in omt.error_string(omt.EINVAL)
    assert omt.error_string(12345) == "unknown error"
