"""Morphology with sheared line elements on the GPU against the oracle
(section "Morphology with Lines at Arbitrary Orientations"), bit for bit."""
import numpy as np
import pytest
import torch

import oracle
from paper_0712_0121_gb300 import synth

pytestmark = pytest.mark.gpu

M = pytest.importorskip("paper_0712_0121_gb300.morph")
from gpu_helpers import unpack_words  # noqa: E402

OPS = ("erode", "dilate", "open", "close")


def run(op, img, shift, L, o, horizontal, wb_src=64, wb_dst=64):
    H, W = img.shape
    src = M.pack(img, wb_src)
    dst = M.Packed.empty(W, H, wb_dst)
    dst.words.fill_(-1)
    M.sheared_line(op, dst, src, shift, L, o, horizontal)
    assert M.sync_status() == M.MORPH_OK
    nw = (W + wb_dst - 1) // wb_dst
    bits = unpack_words(dst.words[:, :nw].contiguous(), nw * wb_dst)
    assert not bits[:, W:].any(), "padding bits must be 0"
    return bits[:, :W]


@pytest.mark.parametrize("op", OPS)
@pytest.mark.parametrize("slope", [0.0, 0.3, -0.45, 1.0, -1.0, 0.07])
@pytest.mark.parametrize("horizontal", [False, True])
def test_random_images(op, slope, horizontal):
    H, W = 97, 130
    img = synth.random_bits((H, W), 800 + int(slope * 100) + horizontal, 0.6)
    shift = synth.line_shifts(W if horizontal else H, slope)
    for L, o in [(9, 4), (16, 3), (1, 0)]:
        got = run(op, img, shift, L, o, horizontal)
        ref = oracle.sheared_line(op, img, shift, L, o, horizontal)
        assert np.array_equal(got, ref), (op, slope, horizontal, L, o)


@pytest.mark.parametrize("wb_src,wb_dst", [(32, 64), (64, 32)])
def test_word_sizes_and_ragged_sizes(wb_src, wb_dst):
    for (H, W) in [(1, 1), (5, 33), (70, 65), (33, 200)]:
        img = synth.random_bits((H, W), H * 3 + W, 0.5)
        for horizontal in (False, True):
            shift = synth.line_shifts(W if horizontal else H, -0.7)
            got = run("close", img, shift, 5, 2, horizontal, wb_src, wb_dst)
            assert np.array_equal(got, oracle.sheared_line("close", img, shift, 5, 2, horizontal))


def test_page_with_angle_helper():
    page, _ = synth.document_page(1700, 2200, synth.seed_for(4, 2), 0.1)
    H, W = page.shape
    for angle in (30.0, 75.0, -20.0, 135.0):
        shift, L, o, horizontal = M.line_element(angle, 12, W, H)
        got = run("open", page, shift, L, o, horizontal)
        assert np.array_equal(got, oracle.sheared_line("open", page, shift, L, o, horizontal)), angle
