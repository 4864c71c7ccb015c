"""RLE path and conversions against the oracle, bit for bit (run lists are
canonical, so row_ptr and every run must match exactly)."""
import numpy as np
import pytest
import torch

import oracle
from paper_0712_0121_gb300 import synth

pytestmark = pytest.mark.gpu

M = pytest.importorskip("paper_0712_0121_gb300.morph")
from gpu_helpers import NCORES, rle_op, to_rle, unpack_words  # noqa: E402

OPS = ("erode", "dilate", "open", "close")


def assert_rle_equal(dst, ref_rp, ref_runs, what=""):
    rp, runs = dst.to_numpy()
    assert np.array_equal(rp, ref_rp), "row_ptr differs %s (first row %s)" % (
        what, np.argwhere(rp != ref_rp)[:3].ravel().tolist())
    assert np.array_equal(runs, ref_runs), "runs differ %s" % what
    assert int(dst.n_runs.item()) == int(ref_rp[-1])


# ------------------------------------------------------------ conversions

@pytest.mark.parametrize("W,H", [(1, 1), (31, 3), (32, 5), (33, 4), (64, 7), (65, 9), (200, 50),
                                 (1000, 33), (5000, 3)])
@pytest.mark.parametrize("word_bits", [32, 64])
def test_bitmap_to_rle_and_back(W, H, word_bits):
    for k, p in enumerate((0.5, 0.97, 0.03)):
        img = synth.random_bits((H, W), 3000 + W + k, p)
        rle = to_rle(img, word_bits)
        assert M.sync_status() == M.MORPH_OK
        rp, runs = oracle.rle_encode(img)
        assert_rle_equal(rle, rp, runs)
        back = M.Packed.empty(W, H, word_bits)
        back.words.fill_(-1)
        M.rle_to_bitmap(back, rle)
        assert np.array_equal(unpack_words(back.words, W), img)
        raw = back.words.cpu().numpy().view(np.uint8).reshape(H, -1)
        assert not np.unpackbits(raw, axis=1, bitorder="little")[:, W:].any()


def test_conversion_worst_case_and_full_rows():
    H, W = 6, 4099
    alt = np.zeros((H, W), np.uint8)
    alt[:, ::2] = 1
    full = np.ones((H, W), np.uint8)
    for img in (alt, full, np.zeros((H, W), np.uint8)):
        rle = to_rle(img)
        rp, runs = oracle.rle_encode(img)
        assert_rle_equal(rle, rp, runs)


def test_conversion_max_width_rows():
    img = synth.random_bits((3, 65535), 17, 0.5)
    img[:, -1] = 1
    rle = to_rle(img)
    rp, runs = oracle.rle_encode(img)
    assert_rle_equal(rle, rp, runs)
    back = M.Packed.empty(65535, 3, 64)
    M.rle_to_bitmap(back, rle)
    assert np.array_equal(unpack_words(back.words, 65535), img)


def test_capacity_overflow_is_reported_not_written():
    img = synth.random_bits((20, 300), 21, 0.5)
    rp, runs = oracle.rle_encode(img)
    need = int(rp[-1])
    dst = M.Rle.empty(300, 20, need - 1)
    sentinel = torch.full_like(dst.runs, 7)
    dst.runs.copy_(sentinel)
    M.rle_from_bitmap(dst, M.pack(img))
    assert M.sync_status() == M.MORPH_ECAPACITY
    assert int(dst.n_runs.item()) == need
    assert np.array_equal(dst.row_ptr.cpu().numpy(), rp)
    assert torch.equal(dst.runs, sentinel)
    assert M.sync_status() == M.MORPH_OK  # the latch was cleared


def test_config_pages_round_trip():
    for img in (synth.config1_page()[0], synth.config2_page()[0], synth.config3_page("halftone")[0]):
        rle = to_rle(img)
        rp, runs = oracle.rle_encode(img)
        assert_rle_equal(rle, rp, runs)


# -------------------------------------------------------------- RLE ops

def check_rle(op, img, sw, sh, ox, oy, mode="brute"):
    dst, st = rle_op(op, img, sw, sh, ox, oy)
    assert st == M.MORPH_OK
    H, W = img.shape
    rp, runs = oracle.rle_encode(oracle.apply(op, img, sw, sh, ox, oy, mode=mode, threads=NCORES))
    assert_rle_equal(dst, rp, runs, "%s %dx%d o=(%d,%d) W=%d H=%d" % (op, sw, sh, ox, oy, W, H))


def test_config1_rle():
    img, _ = synth.config1_page()
    for op in ("erode", "dilate"):
        for sw, sh in ((3, 3), (11, 1), (1, 11)):
            check_rle(op, img, sw, sh, sw // 2, sh // 2)


@pytest.mark.parametrize("op", OPS)
@pytest.mark.parametrize("W,H", [(1, 1), (2, 40), (37, 1), (31, 17), (64, 70), (130, 67), (333, 129)])
def test_rle_ragged_sizes(op, W, H):
    img = synth.random_bits((H, W), 4000 + W * 3 + H, 0.6)
    for sw, sh, ox, oy in [(3, 3, 1, 1), (2, 5, 0, 4), (6, 2, 5, 1), (7, 1, 3, 0), (1, 4, 0, 1),
                           (1, 1, 0, 0)]:
        check_rle(op, img, sw, sh, ox, oy)


@pytest.mark.parametrize("op", OPS)
def test_rle_structuring_elements(op):
    img = synth.text_page(301, 257, 78, 0.2, glyph=(4, 9, 5, 11), gap=(1, 5))[0]
    for sw, sh in [(3, 3), (4, 4), (9, 2), (2, 9), (15, 15), (31, 31), (101, 1), (1, 61), (300, 2),
                   (2, 300)]:
        for ox, oy in {(sw // 2, sh // 2), (0, 0), (sw - 1, sh - 1)}:
            check_rle(op, img, sw, sh, ox, oy, mode="separable")


def test_rle_wide_rows():
    img = synth.random_bits((40, 20000), 31, 0.85)
    for op in OPS:
        check_rle(op, img, 5, 3, 2, 1, mode="separable")


def test_rle_capacity_overflow():
    img = synth.random_bits((30, 100), 41, 0.5)
    ref = oracle.rle_encode(oracle.dilate(img, 1, 3))[1].shape[0]
    dst, st = rle_op("dilate", img, 1, 3, 0, 1, capacity=ref - 1)
    assert st == M.MORPH_ECAPACITY
    assert int(dst.n_runs.item()) == ref


@pytest.mark.parametrize("op", ["open", "close"])
def test_config2_rle_full_page(op):
    img, _ = synth.config2_page()
    for sw, sh in ((3, 3), (15, 15), (51, 51), (1, 51), (51, 1)):
        check_rle(op, img, sw, sh, sw // 2, sh // 2, mode="separable")


@pytest.mark.parametrize("kind", ["blank", "text", "halftone", "noise"])
def test_config3_rle_full_page(kind):
    img, _ = synth.config3_page(kind)
    for op, sw, sh in (("dilate", 101, 1), ("dilate", 1, 61), ("open", 5, 5)):
        check_rle(op, img, sw, sh, sw // 2, sh // 2, mode="separable")


@pytest.mark.parametrize("H", [8192, 8193, 12289, 70001])
def test_tall_images_multi_cta_scan(H):
    # above 8192 rows the row offsets come from the multi-CTA scan: segment
    # boundaries, a ragged last segment and many segments
    img = synth.random_bits((H, 130), 5000 + H, 0.7)
    rle = to_rle(img)
    rp, runs = oracle.rle_encode(img)
    assert_rle_equal(rle, rp, runs)
    for op in ("erode", "close"):
        check_rle(op, img, 5, 3, 2, 1, mode="separable")


def test_tall_capacity_overflow():
    img = synth.random_bits((20000, 100), 43, 0.5)
    ref = oracle.rle_encode(oracle.dilate(img, 1, 3))[1].shape[0]
    dst, st = rle_op("dilate", img, 1, 3, 0, 1, capacity=ref - 1)
    assert st == M.MORPH_ECAPACITY
    assert int(dst.n_runs.item()) == ref
