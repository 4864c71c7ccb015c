"""Transposition of packed and RLE images on the GPU against the oracle
(section "Efficient Transpose"), bit for bit, and the uses the paper makes of
it: vertical run-length statistics and between-line operations done as
within-line ones on the transpose."""
import numpy as np
import pytest
import torch

import oracle
from paper_0712_0121_gb300 import synth

pytestmark = pytest.mark.gpu

M = pytest.importorskip("paper_0712_0121_gb300.morph")
from gpu_helpers import to_rle, unpack_words  # noqa: E402


def row_bits(t: torch.Tensor, word_bits: int, width: int) -> np.ndarray:
    """All bits of each row's words (stride padding words left out)."""
    nw = (width + word_bits - 1) // word_bits
    return unpack_words(t[:, :nw].contiguous(), nw * word_bits)


@pytest.mark.parametrize("H,W", [(1, 1), (1, 300), (300, 1), (31, 33), (32, 32), (33, 65),
                                 (257, 300), (1000, 2550), (70, 9000)])
@pytest.mark.parametrize("wb_src,wb_dst,pad", [(64, 64, 0), (32, 64, 1), (64, 32, 3), (32, 32, 0)])
def test_packed_transpose(H, W, wb_src, wb_dst, pad):
    img = synth.random_bits((H, W), 6000 + H + W, 0.45)
    src = M.pack(img, wb_src, stride=(W + wb_src - 1) // wb_src + pad)
    dst = M.Packed.empty(H, W, wb_dst, stride=(H + wb_dst - 1) // wb_dst + pad)
    dst.words.fill_(-1)  # every word of every output row must be written
    M.transpose(dst, src)
    torch.cuda.synchronize()
    bits = row_bits(dst.words, wb_dst, H)
    assert np.array_equal(bits[:, :H], oracle.transpose(img))
    assert not bits[:, H:].any(), "padding bits of the transpose must be 0"


def test_packed_transpose_ignores_input_padding():
    H, W = 40, 70
    img = synth.random_bits((H, W), 5, 0.5)
    src = M.pack(img, 64)
    src.words[:, -1] |= torch.tensor(-1 << (W % 64), dtype=torch.int64, device="cuda")
    dst = M.Packed.empty(H, W, 64)
    M.transpose(dst, src)
    torch.cuda.synchronize()
    assert np.array_equal(unpack_words(dst.words, H), img.T)


def rle_t(img):
    H, W = img.shape
    src = to_rle(img)
    rp, runs = oracle.rle_encode(img)
    trp, truns = oracle.rle_transpose(rp, runs, W, H)
    dst = M.Rle.empty(H, W, max(1, int(trp[-1])))
    M.rle_transpose(dst, src)
    assert M.sync_status() == M.MORPH_OK
    grp, gruns = dst.to_numpy()
    assert np.array_equal(grp, trp)
    assert np.array_equal(gruns, truns)
    return dst


@pytest.mark.parametrize("H,W,p", [(1, 1, 1.0), (5, 300, 0.5), (300, 5, 0.5), (130, 257, 0.3),
                                   (26400, 64, 0.02)])
def test_rle_transpose(H, W, p):
    rle_t(synth.random_bits((H, W), 7000 + H + W, p))


def test_rle_transpose_page_and_back():
    page, _ = synth.document_page(2550, 3300, synth.seed_for(2, 3), 0.08)
    t = rle_t(page)
    back = M.Rle.empty(2550, 3300, 3300 * 1275)
    M.rle_transpose(back, t)
    assert M.sync_status() == M.MORPH_OK
    rp, runs = oracle.rle_encode(page)
    grp, gruns = back.to_numpy()
    assert np.array_equal(grp, rp) and np.array_equal(gruns, runs)


def test_vertical_run_length_statistics():
    """Vertical run lengths = horizontal run lengths of the transpose."""
    page, _ = synth.document_page(2550, 3300, synth.seed_for(2, 4), 0.08)
    t = rle_t(page)
    b, w = M.run_length_hist(t)
    rp, runs = oracle.rle_encode(page.T.copy())
    b_ref, w_ref = oracle.run_length_hist(rp, runs, 3300, 2550)
    assert np.array_equal(b.cpu().numpy(), b_ref) and np.array_equal(w.cpu().numpy(), w_ref)


@pytest.mark.parametrize("op,h", [("erode", 9), ("dilate", 15)])
def test_between_line_operation_through_transposes(op, h):
    """The paper's "rlet" strategy: a 1 x h operation as the h x 1 operation
    of the transpose, transposed back; equal to the direct RLE operation."""
    page, _ = synth.document_page(1700, 2200, synth.seed_for(4, 1), 0.1)
    H, W = page.shape
    src = to_rle(page)
    t = M.Rle.empty(H, W, W * ((H + 1) // 2))
    M.rle_transpose(t, src)
    t2 = M.Rle.empty(H, W, W * ((H + 1) // 2))
    M.morph_rect(op, t2, t, h, 1, h // 2, 0)
    via = M.Rle.empty(W, H, H * ((W + 1) // 2))
    M.rle_transpose(via, t2)
    direct = M.Rle.empty(W, H, H * ((W + 1) // 2))
    M.morph_rect(op, direct, src, 1, h, 0, h // 2)
    assert M.sync_status() == M.MORPH_OK
    ref = oracle.apply(op, page, 1, h, 0, h // 2)
    rp, runs = oracle.rle_encode(ref)
    for img in (via, direct):
        grp, gruns = img.to_numpy()
        assert np.array_equal(grp, rp) and np.array_equal(gruns, runs)
