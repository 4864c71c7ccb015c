"""Arbitrary structuring elements (section "Morphology with Arbitrary
Masks") on the packed path and on RLE images, through the C ABI, bit for bit
against the oracle's pixel-at-a-time definition: random elements with gaps
and origins outside the element, discs, full rectangles (which must equal the
rectangle path), ragged sizes, both word formats, wide elements, runs
touching the line ends, and the errors."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_0712_0121_gb300 import synth

pytestmark = pytest.mark.gpu

M = pytest.importorskip("paper_0712_0121_gb300.morph")
from gpu_helpers import NCORES, packed_op, padding_bits_zero, unpack_words  # noqa: E402

OPS = ("erode", "dilate", "open", "close")


def mask_op(op, img, mask, ox, oy, word_bits=64, dst_word_bits=None, stride_pad=0):
    H, W = img.shape
    src = M.pack(img, word_bits, stride=(W + word_bits - 1) // word_bits + stride_pad)
    dwb = dst_word_bits or word_bits
    dst = M.Packed.empty(W, H, dwb, stride=(W + dwb - 1) // dwb + stride_pad)
    dst.words.fill_(-1)  # every output bit must be written
    M.morph_mask(op, dst, src, mask, ox, oy)
    torch.cuda.synchronize()
    assert M.sync_status() == M.MORPH_OK
    return unpack_words(dst.words, W), dst


def check(op, img, mask, ox, oy, **kw):
    got, dst = mask_op(op, img, mask, ox, oy, **kw)
    ref = oracle.apply_mask(op, img, mask, ox, oy, threads=NCORES)
    W = img.shape[1]
    dwb = kw.get("dst_word_bits") or kw.get("word_bits", 64)
    cover = (W + dwb - 1) // dwb  # words of a row (stride padding beyond is not the image's)
    assert padding_bits_zero(dst.words[:, :cover], W), "padding bits not cleared"
    if not np.array_equal(got, ref):
        bad = np.argwhere(got != ref)
        pytest.fail("%s mask %s o=(%d,%d) W=%d H=%d: %d pixels differ, first %s" % (
            op, mask.shape, ox, oy, img.shape[1], img.shape[0], len(bad), bad[:5].tolist()))


def rand_mask(rng, mh, mw, p):
    m = (rng.random((mh, mw)) < p).astype(np.uint8)
    if not m.any():
        m[rng.integers(mh), rng.integers(mw)] = 1
    return m


@pytest.mark.parametrize("op", OPS)
@pytest.mark.parametrize("W,H", [(1, 1), (33, 7), (64, 40), (100, 129), (517, 61)])
def test_random_masks_ragged_sizes(op, W, H):
    rng = np.random.default_rng(W * 7 + H)
    img = synth.random_bits((H, W), 6000 + W + H, 0.6 if op in ("erode", "open") else 0.2)
    for k in range(4):
        m = rand_mask(rng, 1 + (k * 5) % 9, 1 + (k * 7) % 13, 0.5)
        ox, oy = int(rng.integers(m.shape[1])), int(rng.integers(m.shape[0]))
        check(op, img, m, ox, oy, word_bits=(32, 64)[k % 2], dst_word_bits=(64, 32)[k % 2])


@pytest.mark.parametrize("op", OPS)
def test_discs_on_a_text_page(op):
    img = synth.text_page(700, 520, 91, 0.15, glyph=(5, 12, 7, 14), gap=(2, 6), ncols=2)[0]
    for r in (1, 2, 5, 9, 14):
        d = oracle.disc_mask(r)
        check(op, img, d, r, r)


@pytest.mark.parametrize("op", OPS)
def test_full_rectangle_mask_equals_rectangle_path(op):
    img = synth.text_page(300, 257, 78, 0.2, glyph=(4, 9, 5, 11), gap=(1, 5))[0]
    for sw, sh, ox, oy in [(3, 3, 1, 1), (7, 2, 0, 1), (1, 9, 0, 8), (15, 15, 14, 0), (40, 1, 20, 0)]:
        got, _ = mask_op(op, img, np.ones((sh, sw), np.uint8), ox, oy)
        rect, _ = packed_op(op, img, sw, sh, ox, oy)
        assert np.array_equal(got, rect), (op, sw, sh, ox, oy)


def test_one_pixel_and_origin_outside_the_element():
    img = synth.random_bits((50, 90), 77, 0.5)
    one = np.zeros((3, 3), np.uint8)
    one[1, 1] = 1
    got, _ = mask_op("erode", img, one, 1, 1)
    assert np.array_equal(got, img)
    ring = np.ones((5, 5), np.uint8)
    ring[1:4, 1:4] = 0  # the origin (2, 2) is not in the element
    for op in OPS:
        check(op, img, ring, 2, 2)


def test_wide_and_tall_elements_and_strides():
    img = synth.text_page(1200, 300, 12, 0.3, glyph=(4, 12, 6, 14), gap=(2, 6), ncols=2)[0]
    bar = np.ones((1, 301), np.uint8)         # reaches 150 pixels each side
    check("dilate", img, bar, 150, 0)
    check("erode", img, bar, 0, 0, stride_pad=3)
    tall = np.zeros((61, 3), np.uint8)
    tall[:, 1] = 1
    tall[::7, 0] = 1
    check("close", img, tall, 1, 30, word_bits=32)
    bigger = np.ones((400, 1500), np.uint8)    # larger than the image
    check("erode", img, bigger, 700, 200)
    check("dilate", img, bigger, 3, 390)


def test_config2_page_disc_close():
    img, _ = synth.config2_page()
    d = oracle.disc_mask(8)
    check("close", img, d, 8, 8)


def test_errors():
    img = synth.random_bits((20, 30), 3, 0.5)
    src, dst = M.pack(img, 64), M.Packed.empty(30, 20, 64)
    with pytest.raises(M.MorphError):
        M.morph_mask("erode", dst, src, np.zeros((3, 3), np.uint8))      # no pixel
    with pytest.raises(M.MorphError):
        M.morph_mask("erode", dst, src, np.ones((3, 3), np.uint8), 3, 0)  # origin outside
    stripes = np.zeros((1, 4100), np.uint8)
    with pytest.raises(M.MorphError):
        M.morph_mask("erode", dst, src, stripes)                          # wider than 4096
    many = np.zeros((64, 64), np.uint8)
    many[:, ::2] = 1                                                      # 2048 runs
    with pytest.raises(M.MorphError):
        M.morph_mask("erode", dst, src, many)
    lib = M.lib()
    m = np.ones((3, 9), np.uint8)
    mp = m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    need = lib.morph_mask_workspace_size(2, ctypes.byref(dst.desc()), ctypes.byref(src.desc()),
                                         mp, 9, 3, 4, 1)
    assert need > 0
    st = lib.morph_mask(2, ctypes.byref(dst.desc()), ctypes.byref(src.desc()), mp, 9, 3, 4, 1,
                        None, 0, None)
    assert st == M.MORPH_ENOMEM
    assert M.sync_status() == M.MORPH_OK


# ------------------------------------------------------------- RLE images

def rle_mask_op(op, img, mask, ox, oy, capacity=None):
    H, W = img.shape
    rp, runs = oracle.rle_encode(img)
    src = M.Rle.from_numpy(rp, runs, W)
    dst = M.Rle.empty(W, H, capacity if capacity is not None else H * ((W + 1) // 2))
    M.morph_mask(op, dst, src, mask, ox, oy)
    return dst


def check_rle(op, img, mask, ox, oy):
    dst = rle_mask_op(op, img, mask, ox, oy)
    assert M.sync_status() == M.MORPH_OK
    g_rp, g_runs = dst.to_numpy()
    o_rp, o_runs = oracle.rle_encode(oracle.apply_mask(op, img, mask, ox, oy, threads=NCORES))
    assert np.array_equal(g_rp, o_rp), (op, mask.shape, ox, oy, img.shape)
    assert np.array_equal(g_runs.reshape(-1, 2), np.asarray(o_runs).reshape(-1, 2)), (op, mask.shape, ox, oy)
    assert int(dst.n_runs.item()) == o_rp[-1]


@pytest.mark.parametrize("op", OPS)
@pytest.mark.parametrize("W,H", [(1, 1), (33, 7), (64, 40), (100, 129), (517, 61)])
def test_rle_random_masks_ragged_sizes(op, W, H):
    rng = np.random.default_rng(W * 11 + H)
    img = synth.random_bits((H, W), 6100 + W + H, 0.6 if op in ("erode", "open") else 0.2)
    for k in range(4):
        m = rand_mask(rng, 1 + (k * 5) % 9, 1 + (k * 7) % 13, 0.5)
        ox, oy = int(rng.integers(m.shape[1])), int(rng.integers(m.shape[0]))
        check_rle(op, img, m, ox, oy)


@pytest.mark.parametrize("op", OPS)
def test_rle_discs_on_a_text_page(op):
    img = synth.text_page(700, 520, 92, 0.15, glyph=(5, 12, 7, 14), gap=(2, 6), ncols=2)[0]
    for r in (1, 3, 9, 14):
        check_rle(op, img, oracle.disc_mask(r), r, r)


def test_rle_runs_at_the_line_ends_and_origin_outside():
    img = synth.random_bits((60, 97), 78, 0.5)
    img[:, 0] = 1
    img[:, -1] = 1            # runs that touch both ends of every line
    img[10] = 1               # a full line
    img[20] = 0               # an empty line
    ring = np.ones((5, 5), np.uint8)
    ring[1:4, 1:4] = 0        # the origin (2, 2) is not in the element
    bar = np.ones((1, 201), np.uint8)   # wider than the image
    tall = np.ones((81, 1), np.uint8)   # taller than the image
    for op in OPS:
        check_rle(op, img, ring, 2, 2)
        check_rle(op, img, bar, 100, 0)
        check_rle(op, img, tall, 0, 40)


def test_rle_full_rectangle_mask_equals_the_rectangle_path():
    img = synth.text_page(300, 257, 79, 0.2, glyph=(4, 9, 5, 11), gap=(1, 5))[0]
    rp, runs = oracle.rle_encode(img)
    src = M.Rle.from_numpy(rp, runs, 300)
    for op in OPS:
        for sw, sh, ox, oy in [(3, 3, 1, 1), (7, 2, 0, 1), (15, 15, 14, 0)]:
            a = rle_mask_op(op, img, np.ones((sh, sw), np.uint8), ox, oy)
            b = M.Rle.empty(300, 257, 257 * 151)
            M.morph_rect(op, b, src, sw, sh, ox, oy)
            assert M.sync_status() == M.MORPH_OK
            (arp, aruns), (brp, bruns) = a.to_numpy(), b.to_numpy()
            assert np.array_equal(arp, brp) and np.array_equal(aruns, bruns), (op, sw, sh)


def test_rle_config2_page_disc_open():
    img, _ = synth.config2_page()
    check_rle("open", img, oracle.disc_mask(6), 6, 6)


def test_rle_mask_capacity_and_format_errors():
    img = synth.random_bits((30, 64), 5, 0.5)
    dst = rle_mask_op("dilate", img, np.ones((1, 3), np.uint8), 1, 0, capacity=3)
    assert M.sync_status() == M.MORPH_ECAPACITY
    rp, runs = oracle.rle_encode(img)
    src = M.Rle.from_numpy(rp, runs, 64)
    with pytest.raises(M.MorphError):
        M.morph_mask("erode", M.Packed.empty(64, 30, 64), src, np.ones((3, 3), np.uint8))  # mixed formats
    del dst
