"""CPU-only checks of the C ABI: the library loads, exports every function
that ``include/morph.h`` declares, and rejects bad arguments on the host
before any device work (no GPU call is made by these tests)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def M():
    from paper_0712_0121_gb300 import build
    build.build_morph()
    from paper_0712_0121_gb300 import morph
    return morph


def declared_functions():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            text = "\n".join(l for l in text.splitlines() if not l.lstrip().startswith("#"))
            names += re.findall(r"MORPH_API\s+[\w\s\*]*?\b(\w+)\s*\(", text)
    return names


def test_header_declares_the_api():
    names = declared_functions()
    for n in ("morph_erode_rect", "morph_dilate_rect", "morph_open_rect", "morph_close_rect",
              "rle_from_bitmap", "rle_to_bitmap"):
        assert n in names


def test_library_exports_every_declared_symbol(M):
    lib = ctypes.CDLL(M.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert M.abi_version() == 1


def _img(M, fmt=1, W=100, H=10, words=0x10000, stride=2):
    d = M.morph_image()
    d.fmt, d.width, d.height, d.reserved = fmt, W, H, 0
    d.words = words
    d.stride_words = stride
    return d


def _call(M, op, dst, src, sw=3, sh=3, ox=1, oy=1, ws=None, nws=0):
    return M.lib().morph_rect(op, ctypes.byref(dst) if dst is not None else None,
                              ctypes.byref(src) if src is not None else None, sw, sh, ox, oy, ws,
                              nws, None)


def test_host_argument_checks(M):
    src = _img(M, words=0x10000)
    dst = _img(M, words=0x90000)
    E = M.MORPH_EINVAL
    assert _call(M, 0, None, src) == E
    assert _call(M, 0, dst, None) == E
    assert _call(M, 7, dst, src) == E                      # op
    assert _call(M, 0, dst, src, sw=0) == E                # SE size
    assert _call(M, 0, dst, src, sw=3, ox=3) == E          # origin outside
    assert _call(M, 0, dst, src, sh=2, oy=-1) == E
    bad = _img(M, words=0x90000, W=99)
    assert _call(M, 0, bad, src) == E                      # size mismatch
    alias = _img(M, words=0x10008)
    assert _call(M, 0, alias, src) == E                    # overlap
    short = _img(M, words=0x90000, stride=1)
    assert _call(M, 0, short, src) == E                    # stride < ceil(W/64)
    mis = _img(M, words=0x90004)
    assert _call(M, 0, mis, src) == E                      # 64-bit words not aligned
    res = _img(M, words=0x90000)
    res.reserved = 1
    assert _call(M, 0, res, src) == E
    assert b"reserved" in M.lib().morph_last_error()


def test_batch_host_launch_rejects_null_buffers(M):
    """``morph_batch_launch_host`` checks its host and device buffers before
    any CUDA call: a NULL buffer with a nonzero size is MORPH_EINVAL."""
    L, E = M.lib(), M.MORPH_EINVAL
    buf = ctypes.create_string_buffer(64)
    p = ctypes.addressof(buf)
    assert L.morph_batch_launch_host(None, None, None, 0, None, p, 16, None, None, 0, None) == E
    assert b"NULL buffer" in L.morph_last_error()
    assert L.morph_batch_launch_host(None, None, None, 0, p, None, 16, None, None, 0, None) == E
    assert L.morph_batch_launch_host(None, None, None, 0, None, None, 0, None, p, 16, None) == E
    assert L.morph_batch_launch_host(None, None, None, 0, None, None, 0, p, None, 16, None) == E


def test_rle_checks_and_workspace(M):
    def rle(W=100, H=10, rp=0x1000, runs=0x2000, cap=100):
        d = M.morph_image()
        d.fmt, d.width, d.height = 2, W, H
        d.row_ptr, d.runs, d.capacity_runs = rp, runs, cap
        return d
    src, dst = rle(), rle(rp=0x5000, runs=0x6000)
    assert _call(M, 0, dst, src) == M.MORPH_ENOMEM               # no workspace
    need = M.lib().morph_workspace_size(2, ctypes.byref(dst), ctypes.byref(src), 3, 3, 1, 1)
    assert need >= 10 * 4
    assert _call(M, 2, dst, src, ws=0x900000, nws=need - 1) == M.MORPH_ENOMEM
    wide = rle(W=70000)
    assert _call(M, 0, rle(W=70000, rp=0x5000, runs=0x6000), wide) == M.MORPH_EINVAL
    assert _call(M, 0, rle(rp=0x1004, runs=0x6000), src) == M.MORPH_EINVAL  # row_ptr overlap
    mixed = _img(M, words=0x90000)
    assert _call(M, 0, mixed, src) == M.MORPH_EINVAL              # packed dst, RLE src
    odd = rle(rp=0x5000, runs=0x6002)
    assert _call(M, 0, odd, src, ws=0x900000, nws=need) == M.MORPH_EINVAL  # runs not 4-byte aligned
    assert b"aligned" in M.lib().morph_last_error()


def test_packed_workspace_only_for_wide_rectangles(M):
    src = _img(M, W=5000, stride=79)
    dst = _img(M, W=5000, stride=79, words=0x9000000)
    f = M.lib().morph_workspace_size
    assert f(0, ctypes.byref(dst), ctypes.byref(src), 257, 3, 128, 1) == 0
    assert f(0, ctypes.byref(dst), ctypes.byref(src), 259, 3, 129, 1) > 0
    assert f(2, ctypes.byref(dst), ctypes.byref(src), 600, 1, 0, 0) > 0
    small = _img(M, W=100)
    assert f(0, ctypes.byref(_img(M, W=100, words=0x9000000)), ctypes.byref(small), 600, 1, 0, 0) == 0


def test_components_and_histogram_checks(M):
    """Host checks of the connected-component and run-length-statistics
    entry points; every case fails before any device work."""
    L = M.lib()

    def rle(W=100, H=10, rp=0x1000, runs=0x2000, cap=100):
        d = M.morph_image()
        d.fmt, d.width, d.height = 2, W, H
        d.row_ptr, d.runs, d.capacity_runs = rp, runs, cap
        return d
    src = rle()
    need = L.morph_components_workspace_size(ctypes.byref(src))
    assert need >= 4 * (10 + 11 + 100)
    assert need % 256 == 0
    lab, st, nc, ws = 0x10000, 0x20000, 0x30000, 0x40000

    def cc(labels=lab, stats=st, max_c=50, n=nc, s=src, conn=4, w=ws, nw=need):
        return L.morph_rle_components(labels, stats, max_c, n, ctypes.byref(s) if s else None, conn,
                                      w, nw, None)
    assert cc(conn=6) == M.MORPH_EINVAL
    assert cc(labels=None) == M.MORPH_EINVAL
    assert cc(n=None) == M.MORPH_EINVAL
    assert cc(s=None) == M.MORPH_EINVAL
    assert cc(s=_img(M, words=0x90000)) == M.MORPH_EINVAL       # packed src
    assert cc(max_c=-1) == M.MORPH_EINVAL
    assert cc(labels=0x1002) == M.MORPH_EINVAL                  # misaligned
    assert cc(labels=0x2000 + 8) == M.MORPH_EINVAL              # labels overlap the runs
    assert cc(stats=0x10000 + 64) == M.MORPH_EINVAL             # stats overlap the labels
    assert cc(w=None) == M.MORPH_ENOMEM
    assert cc(nw=need - 1) == M.MORPH_ENOMEM
    assert cc(w=ws + 16) == M.MORPH_EINVAL                      # workspace not 256-aligned
    packed = _img(M, words=0x90000)
    assert L.morph_components_workspace_size(ctypes.byref(packed)) == 0
    hb, hw = 0x50000, 0x60000
    assert L.morph_run_length_hist(hb, hw, ctypes.byref(packed), None) == M.MORPH_EINVAL
    assert L.morph_run_length_hist(hb, hb + 8, ctypes.byref(src), None) == M.MORPH_EINVAL  # overlap
    assert L.morph_run_length_hist(hb + 4, hw, ctypes.byref(src), None) == M.MORPH_EINVAL  # misaligned
    assert L.morph_run_length_hist(None, None, ctypes.byref(src), None) == M.MORPH_OK      # nothing to do


def test_transpose_checks(M):
    L = M.lib()
    src = _img(M, W=100, H=10, words=0x10000, stride=2)
    good = _img(M, W=10, H=100, words=0x90000, stride=1)
    bad = _img(M, W=100, H=10, words=0x90000, stride=2)
    assert L.morph_transpose(ctypes.byref(bad), ctypes.byref(src), None) == M.MORPH_EINVAL  # not transposed sizes
    assert b"transpose" in L.morph_last_error()
    over = _img(M, W=10, H=100, words=0x10000 + 8, stride=1)
    assert L.morph_transpose(ctypes.byref(over), ctypes.byref(src), None) == M.MORPH_EINVAL  # overlap

    def rle(W, H, rp, runs, cap=100):
        d = M.morph_image()
        d.fmt, d.width, d.height = 2, W, H
        d.row_ptr, d.runs, d.capacity_runs = rp, runs, cap
        return d
    rs = rle(100, 10, 0x1000, 0x2000)
    rd = rle(10, 100, 0x5000, 0x6000)
    need = L.morph_rle_transpose_workspace_size(ctypes.byref(rs))
    assert need >= 10 * 4 * 4 + 100 * 4 + 100 * 4
    assert L.morph_transpose(ctypes.byref(rd), ctypes.byref(rs), None) == M.MORPH_EINVAL  # RLE to packed entry
    assert L.morph_rle_transpose(ctypes.byref(rd), ctypes.byref(rs), None, 0, None) == M.MORPH_ENOMEM
    assert L.morph_rle_transpose(ctypes.byref(rd), ctypes.byref(rs), 0x900010, need, None) == M.MORPH_EINVAL
    assert L.morph_rle_transpose(ctypes.byref(rs), ctypes.byref(rs), 0x900000, need, None) == M.MORPH_EINVAL
    assert L.morph_rle_transpose(ctypes.byref(good), ctypes.byref(rs), 0x900000, need, None) == M.MORPH_EINVAL


def test_sheared_line_checks(M):
    L = M.lib()
    i32 = ctypes.c_int32 * 10
    shift = i32(*range(10))
    src = _img(M, W=100, H=10, words=0x10000, stride=2)
    dst = _img(M, W=100, H=10, words=0x90000, stride=2)
    need = L.morph_sheared_line_workspace_size(0, ctypes.byref(src), shift, 10, 5, 0)
    assert need > 0 and need % 256 == 0
    assert L.morph_sheared_line_workspace_size(0, ctypes.byref(src), shift, 9, 5, 0) == 0   # wrong count

    def call(op=0, n=10, length=5, origin=2, horizontal=0, ws=0x900000, nws=need, s=src):
        return L.morph_sheared_line(op, ctypes.byref(dst), ctypes.byref(s), shift, n, length, origin,
                                    horizontal, ws, nws, None)
    assert call(op=7) == M.MORPH_EINVAL
    assert call(n=9) == M.MORPH_EINVAL
    assert call(horizontal=1) == M.MORPH_EINVAL          # needs one shift per column (100)
    assert call(length=0) == M.MORPH_EINVAL
    assert call(origin=5) == M.MORPH_EINVAL
    assert call(ws=None) == M.MORPH_ENOMEM
    assert call(nws=need - 1) == M.MORPH_ENOMEM
    assert call(ws=0x900010) == M.MORPH_EINVAL           # not 256-byte aligned
    assert call(s=_img(M, W=100, H=10, words=0x90000 + 8, stride=2)) == M.MORPH_EINVAL  # overlap


def test_layout_checks(M):
    L = M.lib()
    page = _img(M, W=100, H=10, words=0x10000, stride=2)
    need = L.morph_layout_workspace_size(ctypes.byref(page))
    assert need > 0 and need % 256 == 0
    wide = _img(M, W=70000, H=10, words=0x10000, stride=1100)
    assert L.morph_layout_workspace_size(ctypes.byref(wide)) == 0
    gaps = (ctypes.c_int32 * 2)()

    def call(pg=page, boxes=0x50000, max_b=10, n=0x60000, pct=90, ws=0x900000, nws=need):
        return L.morph_layout_boxes(boxes, max_b, n, gaps, ctypes.byref(pg) if pg else None, pct, ws, nws,
                                    None)
    assert call(pg=None) == M.MORPH_EINVAL
    assert call(pg=wide) == M.MORPH_EINVAL
    assert call(boxes=None) == M.MORPH_EINVAL
    assert call(n=None) == M.MORPH_EINVAL
    assert call(max_b=-1) == M.MORPH_EINVAL
    assert call(pct=0) == M.MORPH_EINVAL
    assert call(pct=101) == M.MORPH_EINVAL
    assert call(ws=None) == M.MORPH_ENOMEM
    assert call(nws=need - 1) == M.MORPH_ENOMEM
    assert call(ws=0x900010) == M.MORPH_EINVAL


def test_line_element_through_the_abi_equals_the_oracle_table(M):
    """morph_line_element (host arithmetic of the library, no GPU) against
    the oracle's independently written table, whose own pins are exact
    tables worked out by hand."""
    import numpy as np

    import oracle
    angles = [0.0, 45.0, 90.0, 135.0, -20.0, 170.0, 60.0, -75.0, -45.0, 44.999, 45.001, 89.5, -89.5,
              12.34, 1000.0, -3600.0 + 7.5]
    for angle in angles:
        for r, W, H in [(0, 1, 1), (12, 61, 40), (25, 300, 257), (7, 5, 900)]:
            buf = (ctypes.c_int32 * max(W, H))()
            n, L, o, hz = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
            st = M.lib().morph_line_element(angle, r, W, H, buf, max(W, H), ctypes.byref(n), ctypes.byref(L),
                                            ctypes.byref(o), ctypes.byref(hz))
            assert st == M.MORPH_OK
            shift, length, origin, horizontal = oracle.line_table(angle, r, W, H)
            assert (L.value, o.value, bool(hz.value)) == (length, origin, horizontal), (angle, r)
            assert n.value == shift.shape[0]
            assert np.array_equal(np.frombuffer(buf, np.int32)[:n.value], shift), (angle, r, W, H)
            # the binding returns the same table
            s2, L2, o2, h2 = M.line_element(angle, r, W, H)
            assert np.array_equal(s2, shift) and (L2, o2, h2) == (length, origin, horizontal)


def test_line_element_rejects_bad_arguments(M):
    buf = (ctypes.c_int32 * 8)()
    out = [ctypes.c_int() for _ in range(4)]
    refs = [ctypes.byref(v) for v in out]
    lib = M.lib()
    assert lib.morph_line_element(10.0, 3, 8, 8, buf, 8, *refs) == M.MORPH_OK
    assert lib.morph_line_element(10.0, 3, 9, 8, buf, 8, *refs) == M.MORPH_EINVAL  # capacity
    assert b"capacity" in lib.morph_last_error()
    assert lib.morph_line_element(float("nan"), 3, 8, 8, buf, 8, *refs) == M.MORPH_EINVAL
    assert lib.morph_line_element(10.0, -1, 8, 8, buf, 8, *refs) == M.MORPH_EINVAL
    assert lib.morph_line_element(10.0, 3, 0, 8, buf, 8, *refs) == M.MORPH_EINVAL
    assert lib.morph_line_element(10.0, 3, 8, 8, None, 8, *refs) == M.MORPH_EINVAL
