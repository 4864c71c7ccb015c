"""morph_rle_rect_noalloc — the entry point for callers that may not allocate
device memory (its scratch is a fixed array inside the library).

Checked through the C ABI against the regular RLE entry point (which uses a
caller workspace), bit for bit, on two calls in a row.  This file is
collected last so that a run stopping at the first failure has already run
every other test; it also passes alone in a fresh process, where its first
call is the one that sets up the scratch address on the device."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_0712_0121_gb300 import synth

pytestmark = pytest.mark.gpu

M = pytest.importorskip("paper_0712_0121_gb300.morph")


def rle_of(img):
    rp, runs = oracle.rle_encode(img)
    return M.Rle.from_numpy(rp, runs, img.shape[1])


def noalloc(op, dst, src, sw, sh, ox, oy):
    st = M.lib().morph_rle_rect_noalloc(M.OPS[op], ctypes.byref(dst.desc()), ctypes.byref(src.desc()),
                                        sw, sh, ox, oy, torch.cuda.current_stream().cuda_stream)
    assert st == M.MORPH_OK, M.lib().morph_last_error()


def test_noalloc_matches_workspace_entry_point_twice():
    cases = [
        (synth.text_page(640, 480, 501, 0.15, glyph=(4, 9, 6, 12), gap=(2, 5))[0], "erode", 5, 3, 2, 1),
        (synth.random_bits((300, 777), 502, 0.6), "dilate", 3, 7, 0, 6),
    ]
    for img, op, sw, sh, ox, oy in cases:  # two calls in a row, different inputs and ops
        H, W = img.shape
        src = rle_of(img)
        got = M.Rle.empty(W, H, H * ((W + 1) // 2))
        ref = M.Rle.empty(W, H, H * ((W + 1) // 2))
        noalloc(op, got, src, sw, sh, ox, oy)
        M.morph_rect(op, ref, src, sw, sh, ox, oy)
        assert M.sync_status() == M.MORPH_OK
        g_rp, g_runs = got.to_numpy()
        r_rp, r_runs = ref.to_numpy()
        assert np.array_equal(g_rp, r_rp)
        assert np.array_equal(g_runs, r_runs)
        assert int(got.n_runs.item()) == int(ref.n_runs.item())


def test_noalloc_rejects_images_taller_than_its_scratch():
    d = M.morph_image()
    d.fmt, d.width, d.height = M.RLE, 10, 65537
    d.row_ptr, d.runs, d.capacity_runs = 0x1000, 0x2000, 10
    s = M.morph_image()
    s.fmt, s.width, s.height = M.RLE, 10, 65537
    s.row_ptr, s.runs, s.capacity_runs = 0x900000, 0xA00000, 10
    st = M.lib().morph_rle_rect_noalloc(M.ERODE, ctypes.byref(d), ctypes.byref(s), 3, 3, 1, 1, None)
    assert st == M.MORPH_EINVAL
    assert b"65536" in M.lib().morph_last_error()
