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
                                         ("storage", 2), ("aggregator", 3), ("aggregator", -1),
                                         ("fb_max", float("nan"))])
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


def test_struct_layouts_match_header(tmp_path):
    """The ctypes mirrors have the C structs' sizes and field offsets."""
    import subprocess
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "omt.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(omt_params), sizeof(omt_pyramid),
         sizeof(omt_batch_stream), sizeof(omt_batch_caps), sizeof(omt_level));
  printf("%zu %zu %zu %zu\n", offsetof(omt_batch_stream, prev), offsetof(omt_batch_stream, boxes),
         offsetof(omt_batch_stream, scratch), offsetof(omt_batch_stream, nvalid));
  printf("%zu %zu\n", offsetof(omt_pyramid, base), offsetof(omt_pyramid, lv));
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()
    got = list(map(int, out))
    want = [ctypes.sizeof(omt.Params), ctypes.sizeof(omt.PyramidDesc), ctypes.sizeof(omt.BatchStream),
            ctypes.sizeof(omt.BatchCaps), ctypes.sizeof(omt.Level),
            omt.BatchStream.prev.offset, omt.BatchStream.boxes.offset, omt.BatchStream.scratch.offset,
            omt.BatchStream.nvalid.offset, omt.PyramidDesc.base.offset, omt.PyramidDesc.lv.offset]
    assert got == want


def _fake_stream(w, h, nb, mc, base, levels=3, storage=0):
    """A batch stream description over made-up, well-aligned addresses (the
    pack step only reads the description, never the memory)."""
    d = omt.BatchStream()
    n = omt.pyramid_bytes(w, h, levels, storage)
    lib = omt.lib()
    assert lib.omt_pyramid_init(ctypes.byref(d.prev), w, h, levels, storage, ctypes.c_void_p(base), n) == 0
    assert lib.omt_pyramid_init(ctypes.byref(d.next), w, h, levels, storage,
                                ctypes.c_void_p(base + (1 << 28)), n) == 0
    p = base + (1 << 29)
    d.frame, d.frame_pitch = p, w
    d.boxes, d.nboxes, d.max_corners = p + (1 << 24), nb, mc
    d.scratch = p + (2 << 24)
    d.scratch_bytes = omt.corner_scratch_bytes(w, h, nb, mc)
    d.pts, d.pts_out, d.status = p + (3 << 24), p + (4 << 24), p + (5 << 24)
    d.iters, d.offsets = None, p + (6 << 24)
    d.boxes_out, d.nvalid = p + (7 << 24), None
    return d


def test_batch_pack_validation():
    import numpy as np
    prm = omt.default_params(levels=3, max_corners=50)
    caps = omt.BatchCaps(4, 100, 1920, 1080, 64)
    n = omt.batch_table_bytes(caps)
    assert n > 0
    table = np.zeros(n, np.uint8)
    tp = ctypes.c_void_p(table.ctypes.data)
    lib = omt.lib()
    ok = [_fake_stream(720, 576, 10, 50, 1 << 32), _fake_stream(1920, 1080, 64, 64, 2 << 32)]
    arr = (omt.BatchStream * 2)(*ok)
    assert lib.omt_batch_pack(arr, 2, ctypes.byref(prm), ctypes.byref(caps), tp, n) == omt.OK
    # header: two streams, 74 boxes
    hdr = np.frombuffer(table[:12].tobytes(), np.int32)
    assert hdr.tolist() == [2, 4, 74]
    bad = []
    s = _fake_stream(720, 576, 101, 50, 1 << 32); bad.append(("boxes over caps", s, omt.EINVAL))
    s = _fake_stream(3840, 2160, 1, 50, 1 << 32); bad.append(("frame over caps", s, omt.EINVAL))
    s = _fake_stream(720, 576, 10, 65, 1 << 32); bad.append(("corners over caps", s, omt.EINVAL))
    s = _fake_stream(720, 576, 10, 50, 1 << 32); s.scratch_bytes -= 1; bad.append(("short scratch", s, omt.ENOMEM))
    s = _fake_stream(720, 576, 10, 50, 1 << 32); s.boxes_out = s.boxes; bad.append(("aliased boxes", s, omt.EINVAL))
    s = _fake_stream(720, 576, 10, 50, 1 << 32, levels=4); bad.append(("levels differ", s, omt.EINVAL))
    s = _fake_stream(720, 576, 10, 50, 1 << 32); s.frame_pitch = 700; bad.append(("pitch", s, omt.EINVAL))
    for what, s, code in bad:
        arr = (omt.BatchStream * 1)(s)
        assert lib.omt_batch_pack(arr, 1, ctypes.byref(prm), ctypes.byref(caps), tp, n) == code, what
    arr = (omt.BatchStream * 5)(*([ok[0]] * 5))
    assert lib.omt_batch_pack(arr, 5, ctypes.byref(prm), ctypes.byref(caps), tp, n) == omt.EINVAL
    # launch-shape fields out of range are rejected
    for field, value in [("lk_warps", 9), ("lk_warps", -1), ("lk_ctas_per_sm", 33), ("lk_chunk", 17),
                         ("pyr_ctas_per_sm", 33), ("pyr_ctas_per_sm", -1),
                         ("corner_ctas_per_sm", 33), ("select_ctas_per_sm", -1), ("reserved", 1)]:
        bad_caps = omt.BatchCaps(4, 100, 1920, 1080, 64)
        setattr(bad_caps, field, value)
        assert omt.batch_table_bytes(bad_caps) == 0, field
    good = omt.BatchCaps(4, 100, 1920, 1080, 64, 8, 2, 16)
    assert omt.batch_table_bytes(good) == n
    good = omt.BatchCaps(4, 100, 1920, 1080, 64, 8, 2, 16, 32, 32, 32)
    assert omt.batch_table_bytes(good) == n
    assert lib.omt_batch_pack(arr, 1, ctypes.byref(prm), ctypes.byref(caps), tp, n - 1) == omt.ENOMEM


def test_batch_pack_forward_backward_arrays():
    import numpy as np
    caps = omt.BatchCaps(2, 100, 1920, 1080, 64)
    n = omt.batch_table_bytes(caps)
    table = np.zeros(n, np.uint8)
    tp = ctypes.c_void_p(table.ctypes.data)
    lib = omt.lib()
    prm = omt.default_params(levels=3, max_corners=50, fb_max=0.5)
    s = _fake_stream(720, 576, 10, 50, 1 << 32)
    arr = (omt.BatchStream * 1)(s)
    # the check needs its backward arrays
    assert lib.omt_batch_pack(arr, 1, ctypes.byref(prm), ctypes.byref(caps), tp, n) == omt.EINVAL
    s.pts_back, s.status_back = (1 << 29) + (1 << 32) + (8 << 24), (1 << 29) + (1 << 32) + (9 << 24)
    arr = (omt.BatchStream * 1)(s)
    assert lib.omt_batch_pack(arr, 1, ctypes.byref(prm), ctypes.byref(caps), tp, n) == omt.OK
    s.pts_back += 4  # float2 array misaligned
    arr = (omt.BatchStream * 1)(s)
    assert lib.omt_batch_pack(arr, 1, ctypes.byref(prm), ctypes.byref(caps), tp, n) == omt.EINVAL
    # without the check they are not needed; a step must use the packed threshold
    off = omt.default_params(levels=3, max_corners=50)
    s = _fake_stream(720, 576, 10, 50, 1 << 32)
    arr = (omt.BatchStream * 1)(s)
    assert lib.omt_batch_pack(arr, 1, ctypes.byref(off), ctypes.byref(caps), tp, n) == omt.OK
    assert lib.omt_batch_step(tp, ctypes.byref(caps), ctypes.byref(prm), ctypes.c_void_p(1 << 40),
                              n, None) == omt.EINVAL
    # omt_fb_check argument checks (host only)
    fake = ctypes.c_void_p(1 << 30)
    assert lib.omt_fb_check(fake, fake, fake, 10, None, ctypes.c_float(float("nan")), fake,
                            None) == omt.EINVAL
    assert lib.omt_fb_check(fake, fake, fake, -1, None, ctypes.c_float(1.0), fake, None) == omt.EINVAL
    assert lib.omt_fb_check(None, None, None, 0, None, ctypes.c_float(1.0), None, None) == omt.OK
    assert lib.omt_fb_check(None, fake, fake, 10, None, ctypes.c_float(1.0), fake, None) == omt.EINVAL


def test_flow_engine_arguments_rejected_before_launch():
    lib = omt.lib()
    fp = omt.default_flow_params()
    assert omt.validate_params(omt.default_params()) == omt.OK
    fake = ctypes.c_void_p(1 << 24)
    n = lib.omt_structure_texture_scratch_bytes(64, 48)
    assert n > 0 and lib.omt_structure_texture_scratch_bytes(0, 48) == 0
    # pitch below width, short scratch, bad parameters
    assert lib.omt_structure_texture(fake, 64, 48, 63, ctypes.byref(fp), fake, 64, fake, n,
                                     None) == omt.EINVAL
    assert lib.omt_structure_texture(fake, 64, 48, 64, ctypes.byref(fp), fake, 64, fake, n - 1,
                                     None) == omt.ENOMEM
    assert fp.block == 2
    for bad in (omt.default_flow_params(iters=0), omt.default_flow_params(block=0),
                omt.default_flow_params(block=3)):
        assert lib.omt_structure_texture(fake, 64, 48, 64, ctypes.byref(bad), fake, 64, fake, n,
                                         None) == omt.EINVAL
    # the flow needs F32 pyramids of one shape
    d0, d1, d16 = omt.PyramidDesc(), omt.PyramidDesc(), omt.PyramidDesc()
    m = omt.pyramid_bytes(64, 48, 3, 0)
    assert lib.omt_pyramid_init(ctypes.byref(d0), 64, 48, 3, 0, ctypes.c_void_p(1 << 20), m) == 0
    assert lib.omt_pyramid_init(ctypes.byref(d1), 64, 48, 3, 0, ctypes.c_void_p(1 << 22), m) == 0
    m16 = omt.pyramid_bytes(64, 48, 3, 1)
    assert lib.omt_pyramid_init(ctypes.byref(d16), 64, 48, 3, 1, ctypes.c_void_p(1 << 23), m16) == 0
    t = lib.omt_tvl1_scratch_bytes(64, 48)
    assert lib.omt_tvl1_flow(ctypes.byref(d0), ctypes.byref(d16), ctypes.byref(fp), fake, fake, t,
                             None) == omt.EINVAL
    assert lib.omt_tvl1_flow(ctypes.byref(d0), ctypes.byref(d0), ctypes.byref(fp), fake, fake, t,
                             None) == omt.EINVAL
    assert lib.omt_tvl1_flow(ctypes.byref(d0), ctypes.byref(d1), ctypes.byref(fp), fake, fake, t - 1,
                             None) == omt.ENOMEM
    bad = omt.default_flow_params(block=3)
    assert lib.omt_tvl1_flow(ctypes.byref(d0), ctypes.byref(d1), ctypes.byref(bad), fake, fake, t,
                             None) == omt.EINVAL
    # box means: in place and misaligned boxes are rejected; zero boxes is a no-op
    assert lib.omt_box_mean_flow(fake, 64, 48, fake, 3, fake, None) == omt.EINVAL
    assert lib.omt_box_mean_flow(fake, 64, 48, ctypes.c_void_p((1 << 24) + 8), 3,
                                 ctypes.c_void_p(1 << 25), None) == omt.EINVAL
    assert lib.omt_box_mean_flow(None, 64, 48, None, 0, None, None) == omt.OK


def test_working_level_arguments_rejected_before_launch():
    lib = omt.lib()
    assert [lib.omt_working_level(w, h) for w, h in ((720, 576), (1920, 1080), (3840, 2160))] == [0, 1, 2]
    d32, d16 = omt.PyramidDesc(), omt.PyramidDesc()
    assert lib.omt_pyramid_init(ctypes.byref(d32), 64, 48, 3, 0, ctypes.c_void_p(1 << 20),
                                omt.pyramid_bytes(64, 48, 3, 0)) == 0
    assert lib.omt_pyramid_init(ctypes.byref(d16), 64, 48, 3, 1, ctypes.c_void_p(1 << 22),
                                omt.pyramid_bytes(64, 48, 3, 1)) == 0
    fake = ctypes.c_void_p(1 << 24)
    assert lib.omt_level_u8(ctypes.byref(d16), 1, fake, 64, None) == omt.EINVAL   # F16 storage
    assert lib.omt_level_u8(ctypes.byref(d32), 3, fake, 64, None) == omt.EINVAL   # no such level
    assert lib.omt_level_u8(ctypes.byref(d32), 1, fake, 31, None) == omt.EINVAL   # pitch < 32
    assert lib.omt_scale_boxes(None, 0, ctypes.c_float(0.5), None, None) == omt.OK
    assert lib.omt_scale_boxes(ctypes.c_void_p((1 << 24) + 4), 2, ctypes.c_float(0.5), fake,
                               None) == omt.EINVAL


def test_library_version_matches_the_binding():
    # the binding's ctypes structures mirror one library version's layouts;
    # loading another version raises instead of misreading a structure
    assert omt.lib().omt_version() == omt.ABI_VERSION == 400
