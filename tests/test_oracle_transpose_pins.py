"""Pins of the transposition oracle (section "Efficient Transpose"):
numpy's transpose, transposing twice, the closed form of a single run, and
the paper's use of it for between-line operations (an erosion by a 1 x h
rectangle equals the transpose of the erosion by h x 1 of the transpose)."""
import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("H,W", [(1, 1), (1, 40), (37, 1), (33, 65), (100, 257)])
def test_matches_numpy_and_is_an_involution(H, W):
    img = (np.random.default_rng(H * 7 + W).random((H, W)) < 0.4).astype(np.uint8)
    t = oracle.transpose(img)
    assert t.shape == (W, H)
    assert np.array_equal(t, img.T)
    assert np.array_equal(oracle.transpose(t), img)


def test_single_run_becomes_a_column():
    H, W, y, s, e = 9, 30, 4, 7, 19
    img = np.zeros((H, W), np.uint8)
    img[y, s:e] = 1
    rp, runs = oracle.rle_encode(img)
    trp, truns = oracle.rle_transpose(rp, runs, W, H)
    assert trp.shape == (W + 1,)
    counts = np.diff(trp)
    assert counts.tolist() == [1 if s <= x < e else 0 for x in range(W)]
    assert truns.tolist() == [[y, y + 1]] * (e - s)


@pytest.mark.parametrize("h", [2, 5, 9])
def test_vertical_erosion_through_transposes(h):
    img = (np.random.default_rng(h).random((40, 53)) < 0.7).astype(np.uint8)
    via = oracle.transpose(oracle.erode(oracle.transpose(img), h, 1, h // 2, 0))
    assert np.array_equal(via, oracle.erode(img, 1, h, 0, h // 2))
