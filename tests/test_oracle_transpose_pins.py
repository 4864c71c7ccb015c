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


# The sweep (open column intervals merged with each line, no pixel decoded)
# against numpy's transpose of the decoded image, on shapes and densities that
# exercise every relation between an open interval and a run: inside,
# overlapping either end, covering, touching, disjoint.
@pytest.mark.parametrize("H,W,dens", [(1, 1, 0.5), (1, 40, 0.5), (37, 1, 0.5), (33, 65, 0.4),
                                      (100, 257, 0.1), (64, 64, 0.9), (200, 31, 0.5)])
def test_sweep_equals_the_transposed_bitmap(H, W, dens):
    img = (np.random.default_rng(H * 13 + W).random((H, W)) < dens).astype(np.uint8)
    rp, runs = oracle.rle_encode(img)
    trp, truns = oracle.rle_transpose_sweep(rp, runs, W, H)
    erp, eruns = oracle.rle_encode(np.ascontiguousarray(img.T))
    assert np.array_equal(trp, erp) and np.array_equal(truns, eruns)
    # and transposing back gives the input's runs
    brp, bruns = oracle.rle_transpose_sweep(trp, truns, H, W)
    assert np.array_equal(brp, rp) and np.array_equal(bruns, runs)


def test_sweep_on_document_pages_and_blocks():
    from paper_0712_0121_gb300 import synth
    img = synth.document_page(600, 400, 11, 0.08)[0]
    rp, runs = oracle.rle_encode(img)
    trp, truns = oracle.rle_transpose_sweep(rp, runs, 600, 400)
    assert np.array_equal(oracle.rle_decode(trp, truns, 400, 600), img.T)
    # coherent shapes: a filled rectangle is one run per covered column, a
    # staircase one run per column whose length is its step
    H, W = 12, 20
    img = np.zeros((H, W), np.uint8)
    img[3:9, 5:15] = 1
    trp, truns = oracle.rle_transpose_sweep(*oracle.rle_encode(img), W, H)
    assert np.diff(trp).tolist() == [1 if 5 <= x < 15 else 0 for x in range(W)]
    assert truns.tolist() == [[3, 9]] * 10
    stair = np.zeros((H, W), np.uint8)
    for y in range(H):
        stair[y, y:y + 4] = 1                 # run [y, y + 4) on line y
    trp, truns = oracle.rle_transpose_sweep(*oracle.rle_encode(stair), W, H)
    for x in range(W):                        # column x is set on lines max(0, x-3) .. min(x, H-1)
        lo, hi = max(0, x - 3), min(x, H - 1)
        want = [[lo, hi + 1]] if lo <= hi else []
        assert truns[trp[x]:trp[x + 1]].tolist() == want, x


def test_sweep_of_empty_and_full_images():
    for H, W in ((0, 5), (7, 0), (4, 6)):
        empty = np.zeros((H, W), np.uint8)
        trp, truns = oracle.rle_transpose_sweep(*oracle.rle_encode(empty), W, H)
        assert trp.shape == (W + 1,) and not trp.any() and truns.shape == (0, 2)
    full = np.ones((5, 9), np.uint8)
    trp, truns = oracle.rle_transpose_sweep(*oracle.rle_encode(full), 9, 5)
    assert np.diff(trp).tolist() == [1] * 9 and truns.tolist() == [[0, 5]] * 9


def test_sweep_rejects_non_canonical_runs():
    rp = np.array([0, 2], np.int32)
    for bad in ([[0, 3], [3, 5]], [[4, 6], [1, 2]], [[2, 2], [4, 5]], [[0, 3], [5, 11]]):
        with pytest.raises(ValueError):
            oracle.rle_transpose_sweep(rp, np.array(bad, np.uint16), 10, 1)
