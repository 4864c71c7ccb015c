"""morph_rle_rect_noalloc — the entry point for callers that may not allocate
device memory (its scratch is a fixed array inside the library).

Checked through the C ABI against the oracle (plain erosion / dilation of the
decoded image, encoded again) and against the regular RLE entry point (which
uses a caller workspace), bit for bit, on calls in a row: rectangles with a
between-line pass and without one (sh = 1, the run pass alone), a full letter
page, and a narrow image at the scratch's 65536-row limit (its run counts are
summed by the multi-segment prefix sum).  This file is collected last so that
a run stopping at the first failure has already run every other test; it also
passes alone in a fresh process, where its first call is the one that sets up
the scratch address on the device."""
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


def run_case(img, op, sw, sh, ox, oy, compare_workspace=True):
    H, W = img.shape
    src = rle_of(img)
    cap = H * ((W + 1) // 2)
    got = M.Rle.empty(W, H, cap)
    noalloc(op, got, src, sw, sh, ox, oy)
    assert M.sync_status() == M.MORPH_OK
    g_rp, g_runs = got.to_numpy()
    o_rp, o_runs = oracle.rle_apply(op, *oracle.rle_encode(img), W, H, sw, sh, ox, oy, mode="separable")
    assert np.array_equal(g_rp, o_rp), (op, sw, sh, ox, oy, W, H)
    assert np.array_equal(g_runs.reshape(-1, 2), o_runs.reshape(-1, 2)), (op, sw, sh, ox, oy, W, H)
    assert int(got.n_runs.item()) == o_rp[-1]
    if compare_workspace:
        ref = M.Rle.empty(W, H, cap)
        M.morph_rect(op, ref, src, sw, sh, ox, oy)
        assert M.sync_status() == M.MORPH_OK
        r_rp, r_runs = ref.to_numpy()
        assert np.array_equal(g_rp, r_rp) and np.array_equal(g_runs, r_runs)


def test_noalloc_matches_the_oracle_and_the_workspace_entry_point_on_calls_in_a_row():
    cases = [
        (synth.text_page(640, 480, 501, 0.15, glyph=(4, 9, 6, 12), gap=(2, 5))[0], "erode", 5, 3, 2, 1),
        (synth.random_bits((300, 777), 502, 0.6), "dilate", 3, 7, 0, 6),
        # no between-line pass: the run pass (count, scan, write) alone
        (synth.random_bits((257, 1001), 503, 0.55), "erode", 9, 1, 4, 0),
        (synth.random_bits((130, 333), 504, 0.3), "dilate", 13, 1, 12, 0),
        # a vertical bar: between-line pass, trivial run pass
        (synth.random_bits((199, 520), 505, 0.7), "dilate", 1, 15, 0, 7),
    ]
    for img, op, sw, sh, ox, oy in cases:  # calls in a row, different inputs and ops
        run_case(img, op, sw, sh, ox, oy)


def test_noalloc_on_a_letter_page():
    img, _ = synth.config2_page()
    for op, sw, sh in (("erode", 7, 7), ("dilate", 51, 1), ("erode", 1, 31)):
        run_case(img, op, sw, sh, sw // 2, sh // 2)


def test_noalloc_at_the_scratch_row_limit():
    """65536 rows of 64 pixels: the per-row counts fill the whole fixed
    scratch and are summed by the multi-segment prefix sum."""
    img = synth.random_bits((65536, 64), 506, 0.5)
    run_case(img, "dilate", 3, 1, 1, 0, compare_workspace=False)
    run_case(img, "erode", 3, 3, 1, 1, compare_workspace=False)


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
