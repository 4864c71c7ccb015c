"""Python binding of ``libmorph.so`` (the C ABI in ``include/morph.h``).

Argument marshalling only: every pixel of every operation is computed by the
CUDA kernels behind the ABI.  PyTorch supplies device memory (tensors) and
streams.  Importing this module loads the library and raises if it has not
been built — there is no fallback path.

Images:
  * :class:`Packed` — a torch tensor of shape ``[H, stride_words]`` with dtype
    ``torch.int32`` (``MORPH_PACKED32``) or ``torch.int64``
    (``MORPH_PACKED64``) holding little-endian bit rows;
  * :class:`Rle` — ``row_ptr`` (int32 ``[H+1]``), ``runs`` (int16 ``[cap, 2]``
    holding uint16 start/end pairs), ``n_runs`` (int64 ``[1]``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmorph.so")

MORPH_OK, MORPH_EINVAL, MORPH_ECAPACITY, MORPH_ENOMEM, MORPH_ECUDA, MORPH_ETIMEOUT = range(6)
PACKED32, PACKED64, RLE = 0, 1, 2
ERODE, DILATE, OPEN, CLOSE, TO_RLE = 0, 1, 2, 3, 4
OPS = {"erode": ERODE, "dilate": DILATE, "open": OPEN, "close": CLOSE}
PATH_PACKED, PATH_RLE = 0, 1


class MorphError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s: %s" % (_status_name(status), message))
        self.status = status


class morph_image(ctypes.Structure):
    _fields_ = [
        ("fmt", ctypes.c_int32),
        ("width", ctypes.c_int32),
        ("height", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("words", ctypes.c_void_p),
        ("stride_words", ctypes.c_int64),
        ("row_ptr", ctypes.c_void_p),
        ("runs", ctypes.c_void_p),
        ("capacity_runs", ctypes.c_int64),
        ("n_runs", ctypes.c_void_p),
    ]


class morph_job(ctypes.Structure):
    _fields_ = [
        ("op", ctypes.c_int32),
        ("path", ctypes.c_int32),
        ("se_w", ctypes.c_int32),
        ("se_h", ctypes.c_int32),
        ("origin_x", ctypes.c_int32),
        ("origin_y", ctypes.c_int32),
        ("depends_on", ctypes.c_int32),
        ("tile_rows", ctypes.c_int32),
        ("words_per_thread", ctypes.c_int32),
        ("src", morph_image),
        ("dst", morph_image),
    ]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libmorph.so is not built (run __graft_entry__.build() or "
                          "python -m paper_0712_0121_gb300.build); there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    img_p = ctypes.POINTER(morph_image)
    vp, sz, ci = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int
    for name in ("morph_erode_rect", "morph_dilate_rect", "morph_open_rect", "morph_close_rect"):
        f = getattr(lib, name)
        f.argtypes = [img_p, img_p, ci, ci, ci, ci, vp, sz, vp]
        f.restype = ci
    lib.morph_rect.argtypes = [ci, img_p, img_p, ci, ci, ci, ci, vp, sz, vp]
    lib.morph_rect.restype = ci
    lib.morph_workspace_size.argtypes = [ci, img_p, img_p, ci, ci, ci, ci]
    lib.morph_workspace_size.restype = sz
    u8p = ctypes.POINTER(ctypes.c_uint8)
    lib.morph_mask_workspace_size.argtypes = [ci, img_p, img_p, u8p, ci, ci, ci, ci]
    lib.morph_mask_workspace_size.restype = sz
    lib.morph_mask.argtypes = [ci, img_p, img_p, u8p, ci, ci, ci, ci, vp, sz, vp]
    lib.morph_mask.restype = ci
    lib.morph_convert_workspace_size.argtypes = [ci]
    lib.morph_convert_workspace_size.restype = sz
    lib.rle_from_bitmap.argtypes = [img_p, img_p, vp, sz, vp]
    lib.rle_from_bitmap.restype = ci
    lib.rle_to_bitmap.argtypes = [img_p, img_p, vp]
    lib.rle_to_bitmap.restype = ci
    i32p = ctypes.POINTER(ctypes.c_int32)
    lib.morph_sheared_line_workspace_size.argtypes = [ci, img_p, i32p, ci, ci, ci]
    lib.morph_sheared_line_workspace_size.restype = sz
    lib.morph_sheared_line.argtypes = [ci, img_p, img_p, i32p, ci, ci, ci, ci, vp, sz, vp]
    lib.morph_sheared_line.restype = ci
    lib.morph_line_element.argtypes = [ctypes.c_double, ci, ci, ci, i32p, ci, ctypes.POINTER(ci),
                                       ctypes.POINTER(ci), ctypes.POINTER(ci), ctypes.POINTER(ci)]
    lib.morph_line_element.restype = ci
    lib.morph_transpose.argtypes = [img_p, img_p, vp]
    lib.morph_transpose.restype = ci
    lib.morph_rle_transpose_workspace_size.argtypes = [img_p]
    lib.morph_rle_transpose_workspace_size.restype = sz
    lib.morph_rle_transpose.argtypes = [img_p, img_p, vp, sz, vp]
    lib.morph_rle_transpose.restype = ci
    lib.morph_layout_workspace_size.argtypes = [img_p]
    lib.morph_layout_workspace_size.restype = sz
    lib.morph_layout_boxes.argtypes = [vp, ctypes.c_int64, vp, i32p, img_p, ci, vp, sz, vp]
    lib.morph_layout_boxes.restype = ci
    lib.morph_components_workspace_size.argtypes = [img_p]
    lib.morph_components_workspace_size.restype = sz
    lib.morph_rle_components.argtypes = [vp, vp, ctypes.c_int64, vp, img_p, ci, vp, sz, vp]
    lib.morph_rle_components.restype = ci
    lib.morph_run_length_hist.argtypes = [vp, vp, img_p, vp]
    lib.morph_run_length_hist.restype = ci
    lib.morph_sync_status.argtypes = [vp]
    lib.morph_sync_status.restype = ci
    lib.morph_last_error.argtypes = []
    lib.morph_last_error.restype = ctypes.c_char_p
    lib.morph_status_string.argtypes = [ci]
    lib.morph_status_string.restype = ctypes.c_char_p
    lib.morph_abi_version.argtypes = []
    lib.morph_abi_version.restype = ci
    job_p = ctypes.POINTER(morph_job)
    lib.morph_batch_plan_bytes.argtypes = [job_p, ci, ci, ci]
    lib.morph_batch_plan_bytes.restype = sz
    lib.morph_batch_plan_build.argtypes = [vp, sz, job_p, ci, ci, ci]
    lib.morph_batch_plan_build.restype = ci
    lib.morph_batch_workspace_size.argtypes = [vp]
    lib.morph_batch_workspace_size.restype = sz
    lib.morph_batch_kernels.argtypes = [vp]
    lib.morph_batch_kernels.restype = ci
    lib.morph_batch_items.argtypes = [vp]
    lib.morph_batch_items.restype = ci
    lib.morph_batch_plan_debug.argtypes = [vp, ci, ctypes.c_longlong]
    lib.morph_batch_plan_debug.restype = ci
    lib.morph_batch_launch.argtypes = [vp, vp, vp, sz, ci, vp]
    lib.morph_batch_launch.restype = ci
    lib.morph_batch_launch_host.argtypes = [vp, vp, vp, sz, vp, vp, sz, vp, vp, sz, vp]
    lib.morph_batch_launch_host.restype = ci
    lib.morph_rle_rect_noalloc.argtypes = [ci, img_p, img_p, ci, ci, ci, ci, vp]
    lib.morph_rle_rect_noalloc.restype = ci
    return lib


_lib = _load()


def lib() -> ctypes.CDLL:
    return _lib


def _status_name(st: int) -> str:
    return _lib.morph_status_string(st).decode()


def _check(st: int) -> None:  # noqa: D103
    if st != MORPH_OK:
        raise MorphError(st, _lib.morph_last_error().decode())


def _stream_handle(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


# --------------------------------------------------------------- images

class Packed:
    """A packed bitmap on the device: ``words`` is ``[H, stride]`` int32/int64."""

    def __init__(self, words: torch.Tensor, width: int):
        if words.dtype not in (torch.int32, torch.int64) or words.dim() != 2:
            raise ValueError("words must be a 2D int32 or int64 tensor")
        self.words = words
        self.width = int(width)
        self.height = int(words.shape[0])
        self.fmt = PACKED32 if words.dtype == torch.int32 else PACKED64

    @property
    def word_bits(self) -> int:
        return 32 if self.fmt == PACKED32 else 64

    @staticmethod
    def empty(width: int, height: int, word_bits: int = 64, device="cuda", stride=None) -> "Packed":
        dt = torch.int32 if word_bits == 32 else torch.int64
        nw = (width + word_bits - 1) // word_bits
        stride = nw if stride is None else stride
        return Packed(torch.empty((height, stride), dtype=dt, device=device), width)

    def desc(self) -> morph_image:
        d = morph_image()
        d.fmt, d.width, d.height, d.reserved = self.fmt, self.width, self.height, 0
        d.words = self.words.data_ptr()
        d.stride_words = self.words.stride(0)
        return d


class Rle:
    """A run-length image on the device (CSR of uint16 (start, end) runs)."""

    def __init__(self, row_ptr: torch.Tensor, runs: torch.Tensor, width: int,
                 n_runs: torch.Tensor | None = None):
        self.row_ptr = row_ptr
        self.runs = runs
        self.width = int(width)
        self.height = int(row_ptr.shape[0]) - 1
        self.n_runs = n_runs if n_runs is not None else torch.zeros(1, dtype=torch.int64,
                                                                    device=row_ptr.device)
        self.fmt = RLE

    @property
    def capacity(self) -> int:
        return int(self.runs.shape[0])

    @staticmethod
    def empty(width: int, height: int, capacity: int, device="cuda") -> "Rle":
        return Rle(torch.zeros(height + 1, dtype=torch.int32, device=device),
                   torch.empty((max(capacity, 1), 2), dtype=torch.int16, device=device), width)

    def desc(self) -> morph_image:
        d = morph_image()
        d.fmt, d.width, d.height, d.reserved = RLE, self.width, self.height, 0
        d.row_ptr = self.row_ptr.data_ptr()
        d.runs = self.runs.data_ptr()
        d.capacity_runs = self.capacity
        d.n_runs = self.n_runs.data_ptr()
        return d

    def to_numpy(self):
        """(row_ptr int32[H+1], runs uint16[N, 2]) on the host (synchronises)."""
        rp = self.row_ptr.cpu().numpy()
        n = int(rp[-1])
        runs = self.runs[:n].cpu().numpy().view(np.uint16).reshape(-1, 2)
        return rp, runs

    @staticmethod
    def from_numpy(row_ptr, runs, width, device="cuda", capacity=None) -> "Rle":
        rp = torch.as_tensor(np.ascontiguousarray(row_ptr, dtype=np.int32), device=device)
        r = np.ascontiguousarray(runs, dtype=np.uint16).reshape(-1, 2)
        cap = max(capacity or r.shape[0], 1)
        buf = np.zeros((cap, 2), dtype=np.uint16)
        buf[: r.shape[0]] = r
        rt = torch.as_tensor(buf.view(np.int16), device=device)
        n = torch.tensor([r.shape[0]], dtype=torch.int64, device=device)
        return Rle(rp, rt, width, n)


# ---------------------------------------------------------------- layout

def pack(img, word_bits: int = 64, device="cuda", stride=None) -> Packed:
    """0/1 ``uint8[H, W]`` array -> :class:`Packed` (LSB-first rows)."""
    a = np.ascontiguousarray(img, dtype=np.uint8)
    H, W = a.shape
    nw = (W + word_bits - 1) // word_bits
    stride = nw if stride is None else stride
    b = np.packbits(a, axis=1, bitorder="little")
    rowbytes = stride * word_bits // 8
    out = np.zeros((H, rowbytes), dtype=np.uint8)
    out[:, : b.shape[1]] = b
    dt = np.int32 if word_bits == 32 else np.int64
    t = torch.from_numpy(out.view(dt).reshape(H, stride).copy())
    return Packed(t.to(device), W)


def unpack(p: Packed) -> np.ndarray:
    """:class:`Packed` -> 0/1 ``uint8[H, W]`` on the host (synchronises)."""
    raw = p.words.cpu().numpy().view(np.uint8).reshape(p.height, -1)
    return np.unpackbits(raw, axis=1, bitorder="little")[:, : p.width].copy()


# ------------------------------------------------------------ operations

def workspace_size(op, dst, src, se_w: int, se_h: int, origin_x=None, origin_y=None) -> int:
    ox = se_w // 2 if origin_x is None else origin_x
    oy = se_h // 2 if origin_y is None else origin_y
    return int(_lib.morph_workspace_size(OPS.get(op, op), ctypes.byref(dst.desc()),
                                         ctypes.byref(src.desc()), se_w, se_h, ox, oy))


def _ws_args(workspace):
    if workspace is None:
        return None, 0
    return workspace.data_ptr(), workspace.numel() * workspace.element_size()


def morph_rect(op, dst, src, se_w: int, se_h: int, origin_x=None, origin_y=None,
               workspace: torch.Tensor | None = None, stream=None) -> None:
    """Erode / dilate / open / close ``src`` into ``dst`` (same family of
    format).  Origin defaults to the centre (se_w // 2, se_h // 2).  When the
    operation needs a workspace and none is given, one is allocated here."""
    ox = se_w // 2 if origin_x is None else origin_x
    oy = se_h // 2 if origin_y is None else origin_y
    opc = OPS.get(op, op)
    if workspace is None:
        n = workspace_size(opc, dst, src, se_w, se_h, ox, oy)
        if n:
            dev = src.row_ptr.device if src.fmt == RLE else src.words.device
            workspace = torch.empty(n, dtype=torch.uint8, device=dev)
    wp, wn = _ws_args(workspace)
    _check(_lib.morph_rect(opc, ctypes.byref(dst.desc()), ctypes.byref(src.desc()), se_w, se_h,
                           ox, oy, wp, wn, _stream_handle(stream)))


def morph_erode_rect(dst, src, se_w, se_h, origin_x=None, origin_y=None, workspace=None, stream=None):
    morph_rect(ERODE, dst, src, se_w, se_h, origin_x, origin_y, workspace, stream)


def morph_dilate_rect(dst, src, se_w, se_h, origin_x=None, origin_y=None, workspace=None, stream=None):
    morph_rect(DILATE, dst, src, se_w, se_h, origin_x, origin_y, workspace, stream)


def morph_open_rect(dst, src, se_w, se_h, origin_x=None, origin_y=None, workspace=None, stream=None):
    morph_rect(OPEN, dst, src, se_w, se_h, origin_x, origin_y, workspace, stream)


def morph_close_rect(dst, src, se_w, se_h, origin_x=None, origin_y=None, workspace=None, stream=None):
    morph_rect(CLOSE, dst, src, se_w, se_h, origin_x, origin_y, workspace, stream)


def mask_workspace_size(op, dst, src, mask: np.ndarray, origin_x: int, origin_y: int) -> int:
    m = _mask_bytes(mask)
    return int(_lib.morph_mask_workspace_size(OPS.get(op, op), ctypes.byref(dst.desc()),
                                              ctypes.byref(src.desc()),
                                              m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                              m.shape[1], m.shape[0], origin_x, origin_y))


def _mask_bytes(mask) -> np.ndarray:
    m = np.ascontiguousarray(mask)
    if m.ndim != 2:
        raise ValueError("mask must be 2D")
    return np.ascontiguousarray(m != 0, dtype=np.uint8)


def morph_mask(op, dst, src, mask, origin_x=None, origin_y=None,
               workspace: torch.Tensor | None = None, stream=None) -> None:
    """Erode / dilate / open / close ``src`` into ``dst`` (both
    :class:`Packed` or both :class:`Rle`) by an arbitrary structuring element
    ``mask`` (2D array, nonzero = in the element).  Origin defaults to the
    centre (mask_w // 2, mask_h // 2).  A workspace is allocated here when
    none is given."""
    m = _mask_bytes(mask)
    mh, mw = m.shape
    ox = mw // 2 if origin_x is None else origin_x
    oy = mh // 2 if origin_y is None else origin_y
    opc = OPS.get(op, op)
    if workspace is None:
        n = mask_workspace_size(opc, dst, src, m, ox, oy)
        if n:
            dev = src.row_ptr.device if src.fmt == RLE else src.words.device
            workspace = torch.empty(n, dtype=torch.uint8, device=dev)
    wp, wn = _ws_args(workspace)
    _check(_lib.morph_mask(opc, ctypes.byref(dst.desc()), ctypes.byref(src.desc()),
                           m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), mw, mh, ox, oy, wp, wn,
                           _stream_handle(stream)))


def rle_rect_noalloc(op, dst: "Rle", src: "Rle", se_w: int, se_h: int, origin_x=None,
                     origin_y=None, stream=None) -> None:
    """RLE erode or dilate without any workspace or allocation (for callers
    that may not allocate device memory); images up to 65536 rows.  Calls that
    overlap on the GPU share the library's fixed scratch and must not run
    concurrently."""
    ox = se_w // 2 if origin_x is None else origin_x
    oy = se_h // 2 if origin_y is None else origin_y
    _check(_lib.morph_rle_rect_noalloc(OPS.get(op, op), ctypes.byref(dst.desc()),
                                       ctypes.byref(src.desc()), se_w, se_h, ox, oy,
                                       _stream_handle(stream)))


def convert_workspace_size(height: int) -> int:
    return int(_lib.morph_convert_workspace_size(height))


def rle_from_bitmap(dst: Rle, src: Packed, workspace: torch.Tensor | None = None, stream=None) -> None:
    if workspace is None:
        workspace = torch.empty(max(convert_workspace_size(src.height), 1), dtype=torch.uint8,
                                device=src.words.device)
    wp, wn = _ws_args(workspace)
    _check(_lib.rle_from_bitmap(ctypes.byref(dst.desc()), ctypes.byref(src.desc()), wp, wn,
                                _stream_handle(stream)))


def rle_to_bitmap(dst: Packed, src: Rle, stream=None) -> None:
    _check(_lib.rle_to_bitmap(ctypes.byref(dst.desc()), ctypes.byref(src.desc()),
                              _stream_handle(stream)))


# -------------------------------------------------------- sheared lines

def line_element(angle_deg: float, half_length: int, width: int, height: int):
    """Skew table and line of a line element of half length r at an angle
    (degrees, counterclockwise from the x axis), computed by the library's
    ``morph_line_element``.  Returns (shift int32 array, length, origin,
    horizontal), the arguments of ``sheared_line``."""
    cap = max(int(width), int(height), 1)
    shift = np.zeros(cap, np.int32)
    n, L, o, hz = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(_lib.morph_line_element(float(angle_deg), int(half_length), int(width), int(height),
                                   shift.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), cap,
                                   ctypes.byref(n), ctypes.byref(L), ctypes.byref(o), ctypes.byref(hz)))
    return shift[:n.value].copy(), L.value, o.value, bool(hz.value)


def sheared_line_workspace_size(op, src: Packed, shift, length: int, horizontal: bool = False) -> int:
    sh = np.ascontiguousarray(shift, dtype=np.int32)
    return int(_lib.morph_sheared_line_workspace_size(
        OPS.get(op, op), ctypes.byref(src.desc()), sh.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
        int(sh.shape[0]), int(length), int(bool(horizontal))))


def sheared_line(op, dst: Packed, src: Packed, shift, length: int, origin=None, horizontal: bool = False,
                 workspace: torch.Tensor | None = None, stream=None) -> None:
    """Erode / dilate / open / close by a line sheared by the table ``shift``
    (one entry per line, or per column when ``horizontal``): skew, axis-parallel
    line of ``length`` pixels, skew back.  See ``line_element`` for a table from
    an angle."""
    sh = np.ascontiguousarray(shift, dtype=np.int32)
    o = length // 2 if origin is None else origin
    opc = OPS.get(op, op)
    if workspace is None:
        n = sheared_line_workspace_size(opc, src, sh, length, horizontal)
        workspace = torch.empty(max(n, 1), dtype=torch.uint8, device=src.words.device)
    wp, wn = _ws_args(workspace)
    _check(_lib.morph_sheared_line(opc, ctypes.byref(dst.desc()), ctypes.byref(src.desc()),
                                   sh.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), int(sh.shape[0]),
                                   int(length), int(o), int(bool(horizontal)), wp, wn,
                                   _stream_handle(stream)))


# ------------------------------------------------------------ transpose

def transpose(dst: Packed, src: Packed, stream=None) -> None:
    """dst (H x W) = transpose of packed src (W x H)."""
    _check(_lib.morph_transpose(ctypes.byref(dst.desc()), ctypes.byref(src.desc()),
                                _stream_handle(stream)))


def rle_transpose_workspace_size(src: Rle) -> int:
    return int(_lib.morph_rle_transpose_workspace_size(ctypes.byref(src.desc())))


def rle_transpose(dst: Rle, src: Rle, workspace: torch.Tensor | None = None, stream=None) -> None:
    """dst (H x W, RLE) = transpose of RLE src (W x H): the columns of src as rows."""
    if workspace is None:
        workspace = torch.empty(max(rle_transpose_workspace_size(src), 1), dtype=torch.uint8,
                                device=src.row_ptr.device)
    wp, wn = _ws_args(workspace)
    _check(_lib.morph_rle_transpose(ctypes.byref(dst.desc()), ctypes.byref(src.desc()), wp, wn,
                                    _stream_handle(stream)))


# ------------------------------------------------- connected components

COMPONENT_FIELDS = ("x0", "y0", "x1", "y1", "area", "sum_x", "sum_y")


def components_workspace_size(src: Rle) -> int:
    return int(_lib.morph_components_workspace_size(ctypes.byref(src.desc())))


def rle_components(src: Rle, connectivity: int = 4, labels: torch.Tensor | None = None,
                   stats: torch.Tensor | bool | None = True, n_components: torch.Tensor | None = None,
                   workspace: torch.Tensor | None = None, stream=None):
    """Connected components of an RLE image (union-find over runs that touch
    in adjacent lines).  Returns ``(labels, stats, n_components)`` as device
    tensors: ``labels`` int32[capacity] (one per run, components numbered in
    raster order of their first run), ``stats`` int64[max_components, 7]
    with the columns of ``COMPONENT_FIELDS`` (or None), ``n_components``
    int64[1].  ``stats=True`` sizes the statistics for every possible
    component (one per run); pass a tensor to bound them."""
    dev = src.row_ptr.device
    if labels is None:
        labels = torch.empty(max(src.capacity, 1), dtype=torch.int32, device=dev)
    if stats is True:
        stats = torch.empty((max(src.capacity, 1), 7), dtype=torch.int64, device=dev)
    elif stats is False:
        stats = None
    if n_components is None:
        n_components = torch.zeros(1, dtype=torch.int64, device=dev)
    if workspace is None:
        workspace = torch.empty(max(components_workspace_size(src), 1), dtype=torch.uint8, device=dev)
    wp, wn = _ws_args(workspace)
    max_c = int(stats.shape[0]) if stats is not None else 0
    _check(_lib.morph_rle_components(labels.data_ptr(), stats.data_ptr() if stats is not None else None,
                                     max_c, n_components.data_ptr(), ctypes.byref(src.desc()),
                                     int(connectivity), wp, wn, _stream_handle(stream)))
    return labels, stats, n_components


def layout_workspace_size(page: Packed) -> int:
    return int(_lib.morph_layout_workspace_size(ctypes.byref(page.desc())))


def layout_boxes(page: Packed, coverage_pct: int = 90, max_boxes: int = 65536,
                 boxes: torch.Tensor | None = None, n_boxes: torch.Tensor | None = None,
                 workspace: torch.Tensor | None = None, stream=None):
    """Layout blocks of a packed page: gap estimates from white run lengths,
    dilation by the estimated rectangle, bounding boxes of the 8-connected
    components.  Returns ``(boxes int64[max_boxes, 7], n_boxes int64[1],
    (gap_h, gap_v))``; columns of ``boxes`` as ``COMPONENT_FIELDS``."""
    dev = page.words.device
    if boxes is None:
        boxes = torch.empty((max(max_boxes, 1), 7), dtype=torch.int64, device=dev)
    if n_boxes is None:
        n_boxes = torch.zeros(1, dtype=torch.int64, device=dev)
    if workspace is None:
        workspace = torch.empty(max(layout_workspace_size(page), 1), dtype=torch.uint8, device=dev)
    wp, wn = _ws_args(workspace)
    gaps = (ctypes.c_int32 * 2)()
    _check(_lib.morph_layout_boxes(boxes.data_ptr(), int(boxes.shape[0]), n_boxes.data_ptr(), gaps,
                                   ctypes.byref(page.desc()), int(coverage_pct), wp, wn,
                                   _stream_handle(stream)))
    return boxes, n_boxes, (int(gaps[0]), int(gaps[1]))


def run_length_hist(src: Rle, black: torch.Tensor | None = None, white: torch.Tensor | None = None,
                    stream=None):
    """Histograms int64[width + 1] of black and white run lengths of an RLE
    image (white runs: the gaps of each row, those at its ends included)."""
    dev = src.row_ptr.device
    if black is None:
        black = torch.empty(src.width + 1, dtype=torch.int64, device=dev)
    if white is None:
        white = torch.empty(src.width + 1, dtype=torch.int64, device=dev)
    _check(_lib.morph_run_length_hist(black.data_ptr(), white.data_ptr(), ctypes.byref(src.desc()),
                                      _stream_handle(stream)))
    return black, white


def sync_status(stream=None) -> int:
    """Wait for the stream; return the latched device status (and clear it)."""
    return int(_lib.morph_sync_status(_stream_handle(stream)))


def abi_version() -> int:
    return int(_lib.morph_abi_version())


# ----------------------------------------------------------------- batch

class Batch:
    """One batch launch over many packed pages (``morph_batch_*``).

    ``jobs``: list of dicts with keys ``op`` ("erode"/"dilate"/"open"/"close"
    or code, or "to_rle"), ``se`` ((se_w, se_h); not for "to_rle"), optional
    ``origin`` ((ox, oy), default centre), ``path`` ("packed" or "rle"),
    ``src`` (:class:`Packed`), ``dst`` (:class:`Packed`, or :class:`Rle` for
    "to_rle"), optional ``depends_on`` (index of an earlier job) and
    ``tile_rows`` (row-band height of packed tiles) and ``words_per_thread``
    (2 or 4: the packed tile's word tile; 0 = the planner's choice).
    The plan is built on the host, copied to the device once, and every
    :meth:`launch` is one call of ``morph_batch_launch`` (:attr:`kernels`
    kernel launches: grouped tile launches and the persistent kernel;
    graph-capturable)."""

    def __init__(self, jobs, tile_rows: int = 0, rle_runs_per_row: int = 0, device="cuda",
                 debug=None):
        n = len(jobs)
        if n < 1:
            raise ValueError("empty batch")
        arr = (morph_job * n)()
        self._keep = []
        for k, j in enumerate(jobs):
            sw, sh = j.get("se", (1, 1))
            ox, oy = j.get("origin") or (sw // 2, sh // 2)
            path = j.get("path", "packed")
            arr[k].op = TO_RLE if j["op"] == "to_rle" else OPS.get(j["op"], j["op"])
            arr[k].depends_on = j.get("depends_on", -1)
            arr[k].tile_rows = j.get("tile_rows", 0)
            arr[k].words_per_thread = j.get("words_per_thread", 0)
            arr[k].path = PATH_RLE if path in ("rle", PATH_RLE) else PATH_PACKED
            arr[k].se_w, arr[k].se_h, arr[k].origin_x, arr[k].origin_y = sw, sh, ox, oy
            arr[k].src = j["src"].desc()
            arr[k].dst = j["dst"].desc()
            self._keep.append((j["src"], j["dst"]))
        nbytes = int(_lib.morph_batch_plan_bytes(arr, n, tile_rows, rle_runs_per_row))
        if nbytes == 0:
            # rebuild into a 1-byte buffer to get the reason
            _check(_lib.morph_batch_plan_build(None, 0, arr, n, tile_rows, rle_runs_per_row))
            raise MorphError(MORPH_EINVAL, "batch plan rejected")
        self.host_plan = np.zeros(nbytes, dtype=np.uint8)
        hp = self.host_plan.ctypes.data
        _check(_lib.morph_batch_plan_build(hp, nbytes, arr, n, tile_rows, rle_runs_per_row))
        for what, value in (debug or []):
            _check(_lib.morph_batch_plan_debug(hp, what, value))
        self.dev_plan = torch.from_numpy(self.host_plan).to(device)
        self.ws_bytes = int(_lib.morph_batch_workspace_size(hp))
        self.workspace = torch.empty(max(self.ws_bytes, 1), dtype=torch.uint8, device=device)
        self.n_items = int(_lib.morph_batch_items(hp))
        self.n_jobs = n

    def debug(self, what: int, value: int) -> None:
        """``morph_batch_plan_debug`` on the host plan (test and timing hooks)."""
        _check(_lib.morph_batch_plan_debug(self.host_plan.ctypes.data, what, value))

    @property
    def kernels(self) -> int:
        """Kernel launches one :meth:`launch` makes."""
        return int(_lib.morph_batch_kernels(self.host_plan.ctypes.data))

    def launch(self, stream=None, n_ctas: int = 0) -> None:
        _check(_lib.morph_batch_launch(self.dev_plan.data_ptr(), self.host_plan.ctypes.data,
                                       self.workspace.data_ptr(), self.ws_bytes, n_ctas,
                                       _stream_handle(stream)))

    def launch_host(self, h_in: torch.Tensor, d_in: torch.Tensor, h_out: torch.Tensor, d_out: torch.Tensor,
                    stream=None) -> None:
        """``morph_batch_launch_host``: copy ``h_in`` (host, pinned) into
        ``d_in``, launch, copy ``d_out`` into ``h_out`` (host, pinned), all on
        ``stream``; the plan's pages live in ``d_in`` / ``d_out``."""
        nin, nout = h_in.numel() * h_in.element_size(), h_out.numel() * h_out.element_size()
        if d_in.numel() * d_in.element_size() < nin or d_out.numel() * d_out.element_size() < nout:
            raise ValueError("device buffers smaller than the host buffers")
        _check(_lib.morph_batch_launch_host(self.dev_plan.data_ptr(), self.host_plan.ctypes.data,
                                            self.workspace.data_ptr(), self.ws_bytes, h_in.data_ptr(),
                                            d_in.data_ptr(), nin, h_out.data_ptr(), d_out.data_ptr(), nout,
                                            _stream_handle(stream)))

    def capture(self, n_ctas: int = 0) -> "torch.cuda.CUDAGraph":
        """Capture one launch in a CUDA graph (replay with ``g.replay()``)."""
        self.launch(n_ctas=n_ctas)  # warm-up outside the capture (sets kernel attributes)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.launch(n_ctas=n_ctas)
        return g
