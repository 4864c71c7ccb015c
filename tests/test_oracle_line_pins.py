"""Pins of the sheared-line oracle (section "Morphology with Lines at
Arbitrary Orientations"): no shear is the vertical line rectangle, a shear
of one pixel per line is the anti-diagonal element of the arbitrary-mask
oracle, and any shear equals the paper's procedure written out with numpy
canvases (skew, axis-parallel line by the rectangle oracle, skew back)."""
import numpy as np
import pytest

import oracle
from paper_0712_0121_gb300 import synth

OPS = ("erode", "dilate", "open", "close")


def rand_img(seed, H, W, p):
    return (np.random.default_rng(seed).random((H, W)) < p).astype(np.uint8)


@pytest.mark.parametrize("op", OPS)
def test_no_shear_is_the_vertical_rectangle(op):
    img = rand_img(1, 37, 29, 0.6)
    for L, o in [(1, 0), (5, 2), (8, 0), (9, 8)]:
        got = oracle.sheared_line(op, img, np.zeros(37, np.int32), L, o)
        assert np.array_equal(got, oracle.apply(op, img, 1, L, 0, o)), (op, L, o)


@pytest.mark.parametrize("op", ("erode", "dilate"))
def test_unit_shear_is_the_antidiagonal_element(op):
    img = rand_img(2, 31, 40, 0.6)
    H = img.shape[0]
    for L, o in [(3, 1), (7, 3), (6, 0)]:
        mask = np.zeros((L, L), np.uint8)
        mask[np.arange(L), L - 1 - np.arange(L)] = 1
        got = oracle.sheared_line(op, img, np.arange(H, dtype=np.int32), L, o)
        ref = oracle.apply_mask(op, img, mask, L - 1 - o, o)
        assert np.array_equal(got, ref), (op, L, o)


def skew_procedure(op, img, shift, L, o):
    """The paper's steps with explicit canvases: rows moved right by
    shift - min(shift) into a wider canvas filled with the value that the
    clipped window ignores, the vertical line applied by the rectangle
    oracle, rows moved back."""
    H, W = img.shape
    s = shift - shift.min()
    Wc = W + int(s.max())

    def stage(x, dil):
        canvas = np.full((H, Wc), 0 if dil else 1, np.uint8)
        for y in range(H):
            canvas[y, s[y]:s[y] + W] = x[y]
        r = oracle.apply("dilate" if dil else "erode", canvas, 1, L, 0, o)
        return np.stack([r[y, s[y]:s[y] + W] for y in range(H)])
    if op == "erode":
        return stage(img, 0)
    if op == "dilate":
        return stage(img, 1)
    if op == "open":
        return stage(stage(img, 0), 1)
    return stage(stage(img, 1), 0)


@pytest.mark.parametrize("op", OPS)
@pytest.mark.parametrize("slope", [0.3, -0.45, 0.99, -1.0, 0.07])
def test_any_shear_matches_the_skew_procedure(op, slope):
    img = rand_img(int(abs(slope) * 100) + len(op), 45, 52, 0.55)
    H = img.shape[0]
    shift = synth.line_shifts(H, slope)
    for L, o in [(7, 3), (12, 4), (1, 0)]:
        got = oracle.sheared_line(op, img, shift, L, o)
        assert np.array_equal(got, skew_procedure(op, img, shift, L, o)), (op, slope, L, o)


def test_horizontal_lines_are_the_transposed_case():
    img = rand_img(5, 33, 47, 0.6)
    shift = synth.line_shifts(47, -0.6)
    got = oracle.sheared_line("erode", img, shift, 9, 4, horizontal=True)
    ref = skew_procedure("erode", img.T.copy(), shift, 9, 4).T
    assert np.array_equal(got, ref)
