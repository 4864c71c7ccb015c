"""Packed path (fused tile kernel) against the oracle, bit for bit.

Sizes span several tiles, ragged word tails (W not a multiple of 32/64), both
word formats, every origin class, SEs larger than the image, constant and
worst-case images, and the full-size pages of the benchmark workloads.
"""
import numpy as np
import pytest

import oracle
from paper_0712_0121_gb300 import synth

pytestmark = pytest.mark.gpu

M = pytest.importorskip("paper_0712_0121_gb300.morph")
from gpu_helpers import NCORES, packed_op, padding_bits_zero  # noqa: E402

OPS = ("erode", "dilate", "open", "close")


def check(op, img, sw, sh, ox, oy, word_bits=64, dst_word_bits=None, mode="brute"):
    got, dst = packed_op(op, img, sw, sh, ox, oy, word_bits, dst_word_bits)
    ref = oracle.apply(op, img, sw, sh, ox, oy, mode=mode, threads=NCORES)
    assert padding_bits_zero(dst.words, img.shape[1]), "padding bits not cleared"
    if not np.array_equal(got, ref):
        bad = np.argwhere(got != ref)
        pytest.fail("%s %dx%d o=(%d,%d) W=%d H=%d: %d pixels differ, first %s" % (
            op, sw, sh, ox, oy, img.shape[1], img.shape[0], len(bad), bad[:5].tolist()))


def test_config1_text_512():
    img, _ = synth.config1_page()
    for op in ("erode", "dilate"):
        for sw, sh in ((3, 3), (11, 1), (1, 11)):
            check(op, img, sw, sh, sw // 2, sh // 2, word_bits=32)


@pytest.mark.parametrize("op", OPS)
@pytest.mark.parametrize("W,H", [(1, 1), (1, 37), (45, 1), (31, 17), (33, 70), (64, 9), (65, 130),
                                 (200, 67), (333, 211)])
def test_ragged_sizes_all_ops(op, W, H):
    img = synth.random_bits((H, W), 1000 + W * 7 + H, 0.62)
    for sw, sh, ox, oy in [(3, 3, 1, 1), (2, 5, 0, 4), (6, 2, 5, 1), (7, 1, 3, 0), (1, 4, 0, 1)]:
        check(op, img, sw, sh, ox, oy, word_bits=64 if (W + H) % 2 else 32)


@pytest.mark.parametrize("op", OPS)
def test_structuring_elements_and_origins(op):
    img = synth.text_page(301, 257, 77, 0.2, glyph=(4, 9, 5, 11), gap=(1, 5))[0]
    ses = [(3, 3), (4, 4), (5, 5), (9, 2), (2, 9), (15, 15), (31, 31), (33, 3), (64, 1), (65, 1),
           (1, 61), (101, 1), (129, 3), (257, 1)]
    for sw, sh in ses:
        for ox, oy in {(sw // 2, sh // 2), (0, 0), (sw - 1, sh - 1), (0, sh - 1), (sw - 1, 0)}:
            check(op, img, sw, sh, ox, oy, mode="separable")


def test_se_larger_than_image():
    img = synth.random_bits((23, 40), 5, 0.9)
    for op in OPS:
        for sw, sh, ox, oy in [(100, 3, 50, 1), (3, 100, 1, 99), (300, 300, 0, 299), (81, 47, 40, 23)]:
            check(op, img, sw, sh, ox, oy)


def test_constant_and_worst_case_images():
    H, W = 41, 130
    alt = np.zeros((H, W), np.uint8)
    alt[:, ::2] = 1
    checker = (np.add.outer(np.arange(H), np.arange(W)) % 2).astype(np.uint8)
    for img in (np.zeros((H, W), np.uint8), np.ones((H, W), np.uint8), alt, checker):
        for op in OPS:
            for sw, sh, ox, oy in [(3, 3, 1, 1), (2, 2, 0, 1), (5, 1, 2, 0), (1, 6, 0, 2)]:
                check(op, img, sw, sh, ox, oy, word_bits=32)


def test_mixed_word_formats_and_strides():
    img = synth.random_bits((50, 150), 8, 0.7)
    for src_b, dst_b in ((32, 64), (64, 32)):
        check("open", img, 5, 3, 2, 1, word_bits=src_b, dst_word_bits=dst_b)
    got, _ = packed_op("close", img, 4, 4, 1, 2, 64, 64, stride_pad=3)
    assert np.array_equal(got, oracle.closing(img, 4, 4, 1, 2))


def test_wide_rows_use_column_strips():
    """Rows wider than one CTA covers (> 16384 pixels) split into strips with
    halo words; results must not change at strip seams."""
    img = synth.random_bits((9, 20011), 9, 0.8)
    for op in OPS:
        for sw, sh, ox, oy in [(3, 3, 1, 1), (65, 2, 10, 1), (7, 5, 6, 0)]:
            check(op, img, sw, sh, ox, oy, mode="separable")


@pytest.mark.parametrize("op", ["open", "close"])
def test_config2_full_page(op):
    img, _ = synth.config2_page()
    for sw, sh in ((3, 3), (7, 7), (15, 15), (31, 31), (51, 51), (1, 51), (51, 1)):
        check(op, img, sw, sh, sw // 2, sh // 2, mode="separable")


@pytest.mark.parametrize("kind", ["blank", "text", "halftone", "noise"])
def test_config3_full_page(kind):
    img, _ = synth.config3_page(kind)
    for op, sw, sh in (("dilate", 101, 1), ("dilate", 1, 61), ("open", 5, 5)):
        check(op, img, sw, sh, sw // 2, sh // 2, mode="separable")


def test_vertical_windows_of_every_height_class():
    """Window heights on both sides of the register-window / van Herk-Gil-
    Werman switch, block boundaries that do not line up with the row chunks,
    and heights past the shared-memory limit of the van Herk rings."""
    img = synth.random_bits((613, 170), 31, 0.85)
    for op in OPS:
        for sh in (2, 4, 5, 8, 9, 16, 17, 33, 64, 65, 99, 150, 250):
            for oy in sorted({0, sh // 2, sh - 1}):
                check(op, img, 3, sh, 1, oy, mode="separable")


def test_rows_wider_than_one_cta_split_into_strips():
    img = synth.random_bits((7, 70001), 12, 0.9)
    for op in OPS:
        for sw, sh, ox, oy in [(3, 3, 1, 1), (129, 4, 64, 2), (40, 7, 3, 6), (1, 5, 0, 2)]:
            check(op, img, sw, sh, ox, oy, mode="separable")
