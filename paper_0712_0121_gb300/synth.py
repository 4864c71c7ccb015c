"""Seeded synthetic document pages (stand-ins for scanned journal pages and
a binarised map, neither of which is available here).

This module holds no morphology: it paints glyph-like rectangles, blurs noise
and draws Bernoulli pixels (``csrc/synth.c``).  It serves both the oracle tests
and the GPU path, so both see identical bytes.  Pages are ``uint8[H, W]`` 0/1
arrays, row 0 first.

Seed convention for the workloads: ``0x5EED0000 + 1000 * config + page``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None


def _load():
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build_synth()
            lib = ctypes.CDLL(path)
            u8p = ctypes.POINTER(ctypes.c_uint8)
            ci, cd, u64 = ctypes.c_int, ctypes.c_double, ctypes.c_uint64
            lib.synth_text.argtypes = [u8p, ci, ci, u64, cd, ci, ci, ci, ci, ci, ci, ci, ci, ci, cd]
            lib.synth_text.restype = cd
            lib.synth_halftone.argtypes = [u8p, ci, ci, u64, cd, cd]
            lib.synth_halftone.restype = cd
            lib.synth_noise.argtypes = [u8p, ci, ci, u64, cd]
            lib.synth_noise.restype = cd
            lib.synth_bernoulli.argtypes = [u8p, ctypes.c_int64, u64, cd]
            lib.synth_bernoulli.restype = None
            lib.synth_ints.argtypes = [ctypes.POINTER(ctypes.c_int32), ctypes.c_int64, u64, ci, ci]
            lib.synth_ints.restype = None
            lib.synth_unif.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.c_int64, u64]
            lib.synth_unif.restype = None
            _lib = lib
    return _lib


def _u8(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def seed_for(config: int, page: int) -> int:
    return 0x5EED0000 + 1000 * config + page


def text_page(W, H, seed, density, glyph=(6, 10, 10, 12), gap=(4, 6), ncols=1, n_ruled=0,
              n_filled=0, tol=0.005):
    """Lines of glyph boxes (w in glyph[0..1], h in glyph[2..3]) with random
    interior strokes; returns (page, ink fraction)."""
    out = np.empty((H, W), dtype=np.uint8)
    d = _load().synth_text(_u8(out), W, H, seed, density, glyph[0], glyph[1], glyph[2], glyph[3],
                           gap[0], gap[1], ncols, n_ruled, n_filled, tol)
    return out, float(d)


def halftone_page(W, H, seed, density=0.45, sigma=2.0):
    """Gaussian-blurred iid noise thresholded at the (1 - density) quantile."""
    out = np.empty((H, W), dtype=np.uint8)
    d = _load().synth_halftone(_u8(out), W, H, seed, density, sigma)
    if d < 0:
        raise MemoryError("halftone generator: allocation failed")
    return out, float(d)


def noise_page(W, H, seed, p=0.05):
    """Salt-and-pepper: iid Bernoulli(p) pixels."""
    out = np.empty((H, W), dtype=np.uint8)
    d = _load().synth_noise(_u8(out), W, H, seed, p)
    return out, float(d)


def random_bits(shape, seed, p=0.5) -> np.ndarray:
    out = np.empty(shape, dtype=np.uint8)
    _load().synth_bernoulli(_u8(out), out.size, seed, p)
    return out


def randint(n, seed, lo, hi) -> np.ndarray:
    out = np.empty(n, dtype=np.int32)
    _load().synth_ints(out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), n, seed, lo, hi)
    return out


def uniform(n, seed) -> np.ndarray:
    out = np.empty(n, dtype=np.float64)
    _load().synth_unif(out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n, seed)
    return out


# ------------------------------------------------------------ workloads

def glyph_scale(W: int) -> float:
    """Glyph size relative to a 300 dpi letter page (2550 px wide)."""
    return W / 2550.0


def document_page(W, H, seed, density, ncols=None):
    """Generic text document of any size: 20-30 px glyphs at 300 dpi scaled
    with the page width, 2-3 columns, ruled lines and filled boxes."""
    s = glyph_scale(W)
    g = (max(2, round(20 * s)), max(3, round(30 * s)), max(2, round(20 * s)), max(3, round(30 * s)))
    gap = (max(1, round(4 * s)), max(2, round(8 * s)))
    if ncols is None:
        ncols = 2 + int(randint(1, seed ^ 0xC015, 0, 1)[0])
    return text_page(W, H, seed, density, glyph=g, gap=gap, ncols=ncols, n_ruled=4, n_filled=3)


def config1_page(page: int = 0):
    """512 x 512, glyph boxes about 8 x 12 px, 4-6 px gaps, about 10 % ink."""
    return text_page(512, 512, seed_for(1, page), 0.10, glyph=(6, 10, 10, 12), gap=(4, 6))


def config2_page(page: int = 0):
    """2550 x 3300 (letter at 300 dpi), 20-30 px glyphs, 2-3 columns, ruled
    lines and filled rectangles, about 8 % ink."""
    return document_page(2550, 3300, seed_for(2, page), 0.08)


CONFIG3_KINDS = ("blank", "text", "halftone", "noise")


def config3_page(kind: str, page: int = 0, W: int = 5100, H: int = 6600):
    """5100 x 6600 (600 dpi) density sweep: near-blank 0.5 %, text 8 %,
    clustered halftone 45 % (sigma 2 px), salt-and-pepper 5 %."""
    seed = seed_for(3, 10 * page + CONFIG3_KINDS.index(kind))
    if kind == "blank":
        return document_page(W, H, seed, 0.005)
    if kind == "text":
        return document_page(W, H, seed, 0.08)
    if kind == "halftone":
        return halftone_page(W, H, seed, 0.45, 2.0)
    if kind == "noise":
        return noise_page(W, H, seed, 0.05)
    raise ValueError(kind)


CONFIG4_SIZES = ((1700, 2200), (2550, 3300), (3300, 5100), (5100, 6600))
CONFIG4_SES = ((3, 3), (5, 5), (9, 9), (15, 15), (31, 31), (1, 41), (41, 1), (101, 1))
CONFIG4_OPS = ("erode", "dilate", "open", "close")


def config4_jobs(n: int = 256, seed: int = seed_for(4, 0)):
    """Per-page (size, ink density, SE, op) of the uneven batch: sizes uniform
    over four page formats, density uniform in 1-30 %, SE uniform over
    {3, 5, 9, 15, 31} squares and the bars 1x41, 41x1, 101x1, op uniform."""
    sizes = randint(n, seed + 1, 0, len(CONFIG4_SIZES) - 1)
    ses = randint(n, seed + 2, 0, len(CONFIG4_SES) - 1)
    ops = randint(n, seed + 3, 0, len(CONFIG4_OPS) - 1)
    dens = 0.01 + 0.29 * uniform(n, seed + 4)
    jobs = []
    for i in range(n):
        W, H = CONFIG4_SIZES[sizes[i]]
        sw, sh = CONFIG4_SES[ses[i]]
        jobs.append(dict(W=W, H=H, density=float(dens[i]), se=(sw, sh),
                         op=CONFIG4_OPS[ops[i]], seed=seed_for(4, 1 + i)))
    return jobs


def config4_page(job):
    return document_page(job["W"], job["H"], job["seed"], job["density"])


def line_shifts(n: int, slope: float) -> np.ndarray:
    """Skew table of a line with the given slope (pixels across per pixel
    along): shift[i] = floor(i * slope + 1/2), the nearest integer."""
    return np.floor(np.arange(n) * float(slope) + 0.5).astype(np.int32)
