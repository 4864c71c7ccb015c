"""Plain CPU oracle for rectangular binary morphology, run-length coding,
connected components of RLE images, run-length statistics, transposition,
sheared line structuring elements and their skew tables, and the layout
analysis built from them.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product library never calls it, and the two share no code.

The arithmetic lives in ``morph_oracle.c`` (plain loops on unpacked bytes, see
its header for the definitions and the boundary reading).  This module only
compiles it with gcc, loads it with ctypes and marshals numpy arrays.

Conventions (all arrays are numpy):
  * a bitmap is ``uint8[H, W]`` with values 0/1, row 0 first;
  * an RLE image is ``(row_ptr int32[H+1], runs uint16[N, 2])`` with runs
    ``[start, end)`` per row, ascending and separated by gaps (the paper's
    section "Run Length Image Coding", half-open reading).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "morph_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``morph_oracle.c`` into ``liboracle.so`` (gcc, OpenMP)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fvisibility=hidden",
           "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            u8p = ctypes.POINTER(ctypes.c_uint8)
            i32p = ctypes.POINTER(ctypes.c_int32)
            u16p = ctypes.POINTER(ctypes.c_uint16)
            ci = ctypes.c_int
            for name in ("oracle_erode_rect", "oracle_dilate_rect"):
                f = getattr(lib, name)
                f.argtypes = [u8p, u8p, ci, ci, ci, ci, ci, ci, ci]
                f.restype = None
            for name in ("oracle_erode_rect_sep", "oracle_dilate_rect_sep"):
                f = getattr(lib, name)
                f.argtypes = [u8p, u8p, ci, ci, ci, ci, ci, ci, ci]
                f.restype = ci
            for name in ("oracle_erode_mask", "oracle_dilate_mask"):
                f = getattr(lib, name)
                f.argtypes = [u8p, u8p, ci, ci, u8p, ci, ci, ci, ci, ci]
                f.restype = None
            lib.oracle_rect_batch.argtypes = [u8p, u8p, ctypes.c_int64, ci, ci, ci, ci, ci, ci, ci]
            lib.oracle_rect_batch.restype = ci
            lib.oracle_rle_count.argtypes = [i32p, u8p, ci, ci]
            lib.oracle_rle_count.restype = ctypes.c_int64
            lib.oracle_rle_encode.argtypes = [i32p, u16p, u8p, ci, ci]
            lib.oracle_rle_encode.restype = None
            lib.oracle_rle_decode.argtypes = [u8p, i32p, u16p, ci, ci]
            lib.oracle_rle_decode.restype = ci
            i64p = ctypes.POINTER(ctypes.c_int64)
            lib.oracle_rle_components.argtypes = [i32p, i32p, u16p, ci, ci]
            lib.oracle_rle_components.restype = ctypes.c_int64
            lib.oracle_rle_component_stats.argtypes = [i64p, i32p, i32p, u16p, ci, ctypes.c_int64]
            lib.oracle_rle_component_stats.restype = None
            lib.oracle_run_length_hist.argtypes = [i64p, i64p, i32p, u16p, ci, ci]
            lib.oracle_run_length_hist.restype = None
            lib.oracle_transpose.argtypes = [u8p, u8p, ci, ci]
            lib.oracle_transpose.restype = None
            lib.oracle_rle_transpose_sweep.argtypes = [i32p, u16p, ctypes.c_int64, i32p, u16p, ci, ci]
            lib.oracle_rle_transpose_sweep.restype = ctypes.c_int64
            lib.oracle_sheared_line.argtypes = [u8p, u8p, ci, ci, i32p, ci, ci, ci]
            lib.oracle_sheared_line.restype = None
            lib.oracle_layout_gap.argtypes = [i64p, ci, ci]
            lib.oracle_layout_gap.restype = ci
            _lib = lib
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _as_img(img) -> np.ndarray:
    a = np.ascontiguousarray(img, dtype=np.uint8)
    if a.ndim != 2:
        raise ValueError("bitmap must be 2D uint8")
    if a.size and a.max() > 1:
        raise ValueError("bitmap values must be 0/1")
    return a


def _check_se(sw, sh, ox, oy):
    if sw < 1 or sh < 1 or not (0 <= ox < sw) or not (0 <= oy < sh):
        raise ValueError("bad structuring element %dx%d origin (%d,%d)" % (sw, sh, ox, oy))


def centre(sw: int, sh: int):
    """Default origin of a sw x sh rectangle: (floor(sw/2), floor(sh/2))."""
    return sw // 2, sh // 2


# ------------------------------------------------------------ rectangle ops

def erode(img, sw, sh, ox=None, oy=None, mode="brute", threads=1) -> np.ndarray:
    """Clipped-window erosion by a sw x sh rectangle with origin (ox, oy)."""
    return _rect(img, sw, sh, ox, oy, mode, threads, dilate=False)


def dilate(img, sw, sh, ox=None, oy=None, mode="brute", threads=1) -> np.ndarray:
    """Clipped-window dilation (reflected rectangle) with origin (ox, oy)."""
    return _rect(img, sw, sh, ox, oy, mode, threads, dilate=True)


def opening(img, sw, sh, ox=None, oy=None, mode="brute", threads=1) -> np.ndarray:
    """Opening = dilation of the erosion, same rectangle and origin."""
    e = erode(img, sw, sh, ox, oy, mode, threads)
    return dilate(e, sw, sh, ox, oy, mode, threads)


def closing(img, sw, sh, ox=None, oy=None, mode="brute", threads=1) -> np.ndarray:
    """Closing = erosion of the dilation, same rectangle and origin."""
    d = dilate(img, sw, sh, ox, oy, mode, threads)
    return erode(d, sw, sh, ox, oy, mode, threads)


OPS = {"erode": erode, "dilate": dilate, "open": opening, "close": closing}


def apply(op: str, img, sw, sh, ox=None, oy=None, mode="brute", threads=1) -> np.ndarray:
    return OPS[op](img, sw, sh, ox, oy, mode, threads)


def _rect(img, sw, sh, ox, oy, mode, threads, dilate):
    if ox is None or oy is None:
        cx, cy = centre(sw, sh)
        ox = cx if ox is None else ox
        oy = cy if oy is None else oy
    _check_se(sw, sh, ox, oy)
    a = _as_img(img)
    H, W = a.shape
    out = np.empty_like(a)
    if a.size == 0:
        return out
    lib = _load()
    if mode == "brute":
        f = lib.oracle_dilate_rect if dilate else lib.oracle_erode_rect
        f(_ptr(out, ctypes.c_uint8), _ptr(a, ctypes.c_uint8), W, H, sw, sh, ox, oy, threads)
    elif mode == "separable":
        f = lib.oracle_dilate_rect_sep if dilate else lib.oracle_erode_rect_sep
        if f(_ptr(out, ctypes.c_uint8), _ptr(a, ctypes.c_uint8), W, H, sw, sh, ox, oy, threads):
            raise MemoryError("oracle separable mode: allocation failed")
    else:
        raise ValueError("mode must be 'brute' or 'separable'")
    return out


def rect_batch(imgs: np.ndarray, sw, sh, ox, oy, op: str) -> np.ndarray:
    """Apply one op to n images ``uint8[n, H, W]`` (brute force)."""
    _check_se(sw, sh, ox, oy)
    a = np.ascontiguousarray(imgs, dtype=np.uint8)
    n, H, W = a.shape
    out = np.empty_like(a)
    code = {"erode": 0, "dilate": 1, "open": 2, "close": 3}[op]
    if _load().oracle_rect_batch(_ptr(out, ctypes.c_uint8), _ptr(a, ctypes.c_uint8), n, W, H,
                                 sw, sh, ox, oy, code):
        raise MemoryError("oracle batch: allocation failed")
    return out


# ----------------------------------------------------------------- masks
# Section "Morphology with Arbitrary Masks": the structuring element is a
# bitmap ``uint8[mh, mw]`` (1 = in the element) with origin (ox, oy); the
# definitions are the rectangle ones over the element's pixels (see
# ``oracle_erode_mask`` in morph_oracle.c).  Two evaluation modes:
#   brute — the pixel-at-a-time definition (C);
#   runs  — the paper's run-at-a-time loop: for every horizontal run of the
#           element, the image's clipped row minimum over the run's pixels,
#           shifted to the run's place, ANDed into the result (numpy; the
#           image is embedded in an all-ones canvas so that the clipped
#           window is a plain window).

def _as_mask(mask) -> np.ndarray:
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    if m.ndim != 2 or m.size == 0:
        raise ValueError("mask must be a non-empty 2D array")
    m = (m != 0).astype(np.uint8)
    if not m.any():
        raise ValueError("mask has no pixel")
    return m


def mask_runs(mask):
    """Horizontal runs of the element: list of (j, x0, w), row by row, left
    to right (the runs the paper's loop iterates over)."""
    m = _as_mask(mask)
    out = []
    for j in range(m.shape[0]):
        d = np.diff(np.concatenate(([0], m[j].astype(np.int8), [0])))
        starts, ends = np.flatnonzero(d == 1), np.flatnonzero(d == -1)
        out += [(j, int(a), int(b - a)) for a, b in zip(starts, ends)]
    return out


def reflect_mask(mask, ox, oy):
    """The reflected element (i, j) -> (mw-1-i, mh-1-j) and its origin."""
    m = _as_mask(mask)
    return m[::-1, ::-1].copy(), m.shape[1] - 1 - ox, m.shape[0] - 1 - oy


def _mask_call(img, mask, ox, oy, threads, dilate):
    m = _as_mask(mask)
    mh, mw = m.shape
    if not (0 <= ox < mw and 0 <= oy < mh):
        raise ValueError("origin outside the mask")
    a = _as_img(img)
    H, W = a.shape
    out = np.empty_like(a)
    if a.size:
        f = _load().oracle_dilate_mask if dilate else _load().oracle_erode_mask
        f(_ptr(out, ctypes.c_uint8), _ptr(a, ctypes.c_uint8), W, H, _ptr(m, ctypes.c_uint8), mw, mh,
          ox, oy, threads)
    return out


def _erode_mask_runs(img, mask, ox, oy):
    m = _as_mask(mask)
    mh, mw = m.shape
    a = _as_img(img)
    H, W = a.shape
    P = max(mw, mh)
    canvas = np.ones((H + 2 * P, W + 2 * P), np.uint8)
    canvas[P:P + H, P:P + W] = a
    Wc = canvas.shape[1]
    out = np.ones((H, W), np.uint8)
    for j, x0, w in mask_runs(m):
        # S[:, x] = min of canvas[:, x .. x+w-1]: the run's pixels, left end at x
        S = canvas[:, 0:Wc - w + 1].copy()
        for i in range(1, w):
            np.minimum(S, canvas[:, i:Wc - w + 1 + i], out=S)
        dy, dx = j - oy, x0 - ox
        out &= S[P + dy:P + dy + H, P + dx:P + dx + W]
    return out


def erode_mask(img, mask, ox, oy, mode="brute", threads=1) -> np.ndarray:
    """Clipped-window erosion by an arbitrary element with origin (ox, oy)."""
    if mode == "brute":
        return _mask_call(img, mask, ox, oy, threads, dilate=False)
    if mode == "runs":
        m = _as_mask(mask)
        if not (0 <= ox < m.shape[1] and 0 <= oy < m.shape[0]):
            raise ValueError("origin outside the mask")
        return _erode_mask_runs(img, m, ox, oy)
    raise ValueError("mode must be 'brute' or 'runs'")


def dilate_mask(img, mask, ox, oy, mode="brute", threads=1) -> np.ndarray:
    """Clipped-window dilation by an arbitrary element (reflected window)."""
    if mode == "brute":
        return _mask_call(img, mask, ox, oy, threads, dilate=True)
    if mode == "runs":
        # the max over the reflected window is 1 - the min of the complement
        r, rx, ry = reflect_mask(mask, ox, oy)
        return 1 - _erode_mask_runs(1 - _as_img(img), r, rx, ry)
    raise ValueError("mode must be 'brute' or 'runs'")


def apply_mask(op: str, img, mask, ox, oy, mode="brute", threads=1) -> np.ndarray:
    """erode / dilate / open (= dilate of erode) / close (= erode of dilate)."""
    if op == "erode":
        return erode_mask(img, mask, ox, oy, mode, threads)
    if op == "dilate":
        return dilate_mask(img, mask, ox, oy, mode, threads)
    if op == "open":
        return dilate_mask(erode_mask(img, mask, ox, oy, mode, threads), mask, ox, oy, mode, threads)
    if op == "close":
        return erode_mask(dilate_mask(img, mask, ox, oy, mode, threads), mask, ox, oy, mode, threads)
    raise ValueError("op must be erode, dilate, open or close")


def disc_mask(r: int) -> np.ndarray:
    """Digital disc of radius r: (i-r)^2 + (j-r)^2 <= r^2, size (2r+1)^2."""
    j, i = np.mgrid[0:2 * r + 1, 0:2 * r + 1]
    return (((i - r) ** 2 + (j - r) ** 2) <= r * r).astype(np.uint8)


# ----------------------------------------------------------------- RLE

def rle_encode(img):
    """Canonical runs of each row -> (row_ptr int32[H+1], runs uint16[N, 2])."""
    a = _as_img(img)
    H, W = a.shape
    if W > 65535:
        raise ValueError("RLE rows are limited to 65535 pixels (16-bit run ends)")
    lib = _load()
    n = int(lib.oracle_rle_count(None, _ptr(a, ctypes.c_uint8), W, H)) if a.size else 0
    row_ptr = np.zeros(H + 1, dtype=np.int32)
    runs = np.zeros((n, 2), dtype=np.uint16)
    if a.size:
        lib.oracle_rle_encode(_ptr(row_ptr, ctypes.c_int32), _ptr(runs, ctypes.c_uint16),
                              _ptr(a, ctypes.c_uint8), W, H)
    return row_ptr, runs


def rle_decode(row_ptr, runs, W: int, H: int) -> np.ndarray:
    """Paint the runs of each row into a 0/1 bitmap.  Raises on a run list
    that is not canonical (empty, out of range, touching or unsorted)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    rn = np.ascontiguousarray(runs, dtype=np.uint16).reshape(-1, 2)
    if rp.shape != (H + 1,) or rp[0] != 0 or rp[-1] != rn.shape[0] or np.any(np.diff(rp) < 0):
        raise ValueError("row_ptr is not a valid prefix array")
    out = np.empty((H, W), dtype=np.uint8)
    if out.size == 0:
        return out
    if rn.shape[0] == 0:
        rn = np.zeros((1, 2), dtype=np.uint16)
    if _load().oracle_rle_decode(_ptr(out, ctypes.c_uint8), _ptr(rp, ctypes.c_int32),
                                 _ptr(rn, ctypes.c_uint16), W, H):
        raise ValueError("run list is not canonical")
    return out


def rle_apply(op: str, row_ptr, runs, W, H, sw, sh, ox=None, oy=None, mode="brute", threads=1):
    """Morphology on an RLE image, by its plain definition: decode, apply the
    byte-image op, encode the result."""
    img = rle_decode(row_ptr, runs, W, H)
    return rle_encode(apply(op, img, sw, sh, ox, oy, mode, threads))


# ------------------------------------------------- connected components ---

def _rle_arrays(row_ptr, runs):
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ru = np.ascontiguousarray(runs, dtype=np.uint16).reshape(-1, 2)
    if ru.shape[0] == 0:
        ru = np.zeros((1, 2), np.uint16)  # a valid pointer; no run is read
    return rp, ru


def rle_components(row_ptr, runs, H: int, connectivity: int = 4):
    """Label the runs of an RLE image by connected component (union-find over
    runs that touch in adjacent lines, section "Connected Component Extraction
    and Statistics").  Returns ``(labels int32[N], n_components)``; components
    are numbered in raster order of their first run.  connectivity 4: runs
    sharing a column; 8: also diagonal neighbours."""
    if connectivity not in (4, 8):
        raise ValueError("connectivity must be 4 or 8")
    rp, ru = _rle_arrays(row_ptr, runs)
    n = int(rp[H])
    labels = np.zeros(max(n, 1), np.int32)
    count = _load().oracle_rle_components(_ptr(labels, ctypes.c_int32), _ptr(rp, ctypes.c_int32),
                                          _ptr(ru, ctypes.c_uint16), int(H), int(connectivity))
    return labels[:n], int(count)


def rle_component_stats(labels, n_components: int, row_ptr, runs, H: int) -> np.ndarray:
    """Per component: ``int64[n, 7]`` = x0, y0, x1, y1 (half-open bounding
    box), area, sum of x, sum of y over its pixels (pixel-by-pixel loop)."""
    rp, ru = _rle_arrays(row_ptr, runs)
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    if lab.size == 0:
        lab = np.zeros(1, np.int32)
    out = np.zeros((max(n_components, 1), 7), np.int64)
    _load().oracle_rle_component_stats(_ptr(out, ctypes.c_int64), _ptr(lab, ctypes.c_int32),
                                       _ptr(rp, ctypes.c_int32), _ptr(ru, ctypes.c_uint16), int(H),
                                       int(n_components))
    return out[:n_components]


def run_length_hist(row_ptr, runs, W: int, H: int):
    """Histograms ``(black int64[W+1], white int64[W+1])`` of the lengths of
    the black runs and of the white runs (gaps, those at the row ends
    included; an empty row is one white run of length W)."""
    rp, ru = _rle_arrays(row_ptr, runs)
    black = np.zeros(W + 1, np.int64)
    white = np.zeros(W + 1, np.int64)
    _load().oracle_run_length_hist(_ptr(black, ctypes.c_int64), _ptr(white, ctypes.c_int64),
                                   _ptr(rp, ctypes.c_int32), _ptr(ru, ctypes.c_uint16), int(W), int(H))
    return black, white


# ------------------------------------------------------------ transpose ---

def transpose(img) -> np.ndarray:
    """The transposed bitmap ``out[x, y] = img[y, x]`` (plain loop in C)."""
    a = _as_img(img)
    H, W = a.shape
    out = np.zeros((W, H), np.uint8)
    _load().oracle_transpose(_ptr(out, ctypes.c_uint8), _ptr(a, ctypes.c_uint8), W, H)
    return out


def rle_transpose(row_ptr, runs, W: int, H: int):
    """Transpose of an RLE image (section "Efficient Transpose"):
    decode, transpose, encode; the result has width H and height W."""
    return rle_encode(transpose(rle_decode(row_ptr, runs, W, H)))


def rle_transpose_sweep(row_ptr, runs, W: int, H: int):
    """Transpose of an RLE image by the sweep of section "Efficient
    Transpose" (a list of open column intervals with their start lines,
    merged with each input line; see ``oracle_rle_transpose_sweep``), never
    decoding a pixel: (row_ptr int32[W+1], runs uint16[N, 2]) of the H x W
    result (width H, height W)."""
    if H > 65535:
        raise ValueError("the transpose's rows are H wide: H must be <= 65535 (16-bit run ends)")
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    rn = np.ascontiguousarray(runs, dtype=np.uint16).reshape(-1, 2)
    if rp.shape != (H + 1,) or rp[0] != 0 or rp[-1] != rn.shape[0] or np.any(np.diff(rp) < 0):
        raise ValueError("row_ptr is not a valid prefix array")
    if rn.shape[0] == 0:
        rn = np.zeros((1, 2), dtype=np.uint16)
    out_rp = np.zeros(W + 1, dtype=np.int32)
    # a column holds at most ceil(H / 2) separated runs
    cap = W * ((H + 1) // 2)
    out = np.zeros((max(cap, 1), 2), dtype=np.uint16)
    n = int(_load().oracle_rle_transpose_sweep(_ptr(out_rp, ctypes.c_int32), _ptr(out, ctypes.c_uint16),
                                               cap, _ptr(rp, ctypes.c_int32), _ptr(rn, ctypes.c_uint16),
                                               W, H))
    if n == -1:
        raise ValueError("run list is not canonical")
    if n < 0:
        raise MemoryError("transpose sweep failed (%d)" % n)
    return out_rp, out[:n].copy()


# --------------------------------------------------- sheared line SEs ---

def sheared_line(op: str, img, shift, length: int, origin: int, horizontal: bool = False) -> np.ndarray:
    """Erode / dilate / open / close by a line sheared by ``shift`` (section
    "Morphology with Lines at Arbitrary Orientations"): skew, axis-parallel
    line of ``length`` pixels with origin ``origin``, skew back, written out
    pixel by pixel (see ``oracle_sheared_line``).  ``horizontal``: the line
    runs along the rows and ``shift[x]`` moves column x down (the transposed
    case)."""
    a = _as_img(img)
    if horizontal:
        return transpose(sheared_line(op, transpose(a), shift, length, origin, False))
    H, W = a.shape
    sh = np.ascontiguousarray(shift, dtype=np.int32)
    if sh.shape != (H,):
        raise ValueError("one shift per line")
    if not (1 <= length and 0 <= origin < length):
        raise ValueError("bad line")

    def one(x, dil):
        out = np.zeros_like(x)
        _load().oracle_sheared_line(_ptr(out, ctypes.c_uint8), _ptr(x, ctypes.c_uint8), W, H,
                                    _ptr(sh, ctypes.c_int32), int(length), int(origin), int(dil))
        return out
    if op == "erode":
        return one(a, 0)
    if op == "dilate":
        return one(a, 1)
    if op == "open":
        return one(one(a, 0), 1)
    if op == "close":
        return one(one(a, 1), 0)
    raise ValueError(op)



def line_table(angle_deg: float, half_length: int, width: int, height: int):
    """Skew table and line of a line element at an angle (section "Morphology
    with Lines at Arbitrary Orientations": skew perpendicular to the line by
    the tangent of its angle from the nearer axis, then an axis-parallel line
    of about 2 r cos(angle) pixels; the paper fixes neither the rounding nor
    the axis at exactly 45 degrees).

    Reading: the angle is in degrees counterclockwise from the x axis with
    image rows growing downwards, reduced to [-90, 90).  A line within 45
    degrees of the x axis (45 included) runs along the rows: the table has
    one entry per column, the nearest integer (ties upwards) to x tan(a),
    and moves column x down.  Any other line runs along the columns: one
    entry per row, the nearest integer to y tan(90 - a), moving row y right.
    The line has 2 c + 1 pixels with c = half_length |cos| of that same
    angle rounded to the nearest integer (ties away from zero), origin c.
    Double precision, as the C library computes tan and cos.

    Returns ``(shift int32 array, length, origin, horizontal)`` — the
    arguments of ``sheared_line``."""
    if half_length < 0 or width < 1 or height < 1 or not math.isfinite(angle_deg):
        raise ValueError("bad line element")
    a = math.fmod(float(angle_deg) + 90.0, 180.0)
    if a < 0.0:
        a += 180.0
    a -= 90.0
    along_rows = -45.0 <= a <= 45.0
    off = a if along_rows else 90.0 - a
    rad = off * (math.pi / 180.0)
    t = math.tan(rad)
    n = width if along_rows else height
    shift = np.empty(n, np.int32)
    for i in range(n):
        shift[i] = math.floor(i * t + 0.5)
    v = half_length * abs(math.cos(rad))
    c = int(math.floor(v + 0.5))  # v >= 0: ties away from zero
    return shift, 2 * c + 1, c, along_rows


# ------------------------------------------------------- layout analysis --

def layout_gap(white, lmax: int, pct: int) -> int:
    """Gap estimate from a white-run histogram (section "Document Analysis
    Performance"; the rule is the reading stated in ``oracle_layout_gap``):
    the smallest L in 1..lmax whose white runs of length <= L are at least
    pct percent of those of length 1..lmax, 0 if there are none."""
    if lmax < 1 or not (1 <= pct <= 100):
        raise ValueError("lmax >= 1 and pct in 1..100")
    w = np.zeros(lmax + 1, np.int64)
    src = np.asarray(white, dtype=np.int64)
    k = min(lmax + 1, src.shape[0])
    w[:k] = src[:k]
    return int(_load().oracle_layout_gap(_ptr(w, ctypes.c_int64), int(lmax), int(pct)))


def layout_boxes(page, pct: int = 90):
    """The paper's morphological layout analysis (section "Document Analysis
    Performance"), composed from the oracle's own steps: white-run histograms
    along the lines and, through the transpose, along the columns; a gap
    estimate from each (``layout_gap`` with lmax = 1/16 of the line, at
    least 1); dilation by a (gap_h + 1) x (gap_v + 1) rectangle with its
    origin at the centre; the 8-connected components of the result and their
    records (``rle_component_stats``), numbered in raster order.

    Returns ``((gap_h, gap_v), records int64[n, 7])``."""
    a = _as_img(page)
    H, W = a.shape
    rp, runs = rle_encode(a)
    _, white_h = run_length_hist(rp, runs, W, H)
    rpt, runst = rle_encode(transpose(a))
    _, white_v = run_length_hist(rpt, runst, H, W)
    gh = layout_gap(white_h, max(W // 16, 1), pct)
    gv = layout_gap(white_v, max(H // 16, 1), pct)
    sw, sh = gh + 1, gv + 1
    d = dilate(a, sw, sh, sw // 2, sh // 2, mode="separable")
    rpd, runsd = rle_encode(d)
    labels, n = rle_components(rpd, runsd, H, 8)
    return (gh, gv), rle_component_stats(labels, n, rpd, runsd, H)
