"""Pins of the arbitrary-mask oracle (section "Morphology with Arbitrary
Masks") against what the mathematics fixes: a full-rectangle mask is the
rectangle operation (an independent oracle function), a one-pixel mask is a
shift with the clipped-window fill, dilation is the dual of erosion by the
reflected element, erosion by a union of elements is the AND of the
erosions, opening never adds a pixel, and the pixel-at-a-time definition
equals the paper's run-at-a-time loop."""
import numpy as np
import pytest

import oracle


def rand_img(rng, H, W, p):
    return (rng.random((H, W)) < p).astype(np.uint8)


def rand_mask(rng, mh, mw, p):
    m = (rng.random((mh, mw)) < p).astype(np.uint8)
    if not m.any():
        m[rng.integers(mh), rng.integers(mw)] = 1
    return m


@pytest.mark.parametrize("H,W,sw,sh", [(17, 23, 3, 3), (9, 40, 7, 2), (30, 5, 1, 6), (6, 6, 9, 11)])
def test_full_rectangle_mask_is_the_rectangle_operation(H, W, sw, sh):
    rng = np.random.default_rng(H * 100 + W)
    img = rand_img(rng, H, W, 0.6)
    full = np.ones((sh, sw), np.uint8)
    for ox, oy in {(0, 0), (sw // 2, sh // 2), (sw - 1, sh - 1)}:
        assert np.array_equal(oracle.erode_mask(img, full, ox, oy), oracle.erode(img, sw, sh, ox, oy))
        assert np.array_equal(oracle.dilate_mask(img, full, ox, oy), oracle.dilate(img, sw, sh, ox, oy))


def test_one_pixel_mask_is_a_shift():
    rng = np.random.default_rng(5)
    img = rand_img(rng, 13, 19, 0.5)
    H, W = img.shape
    m = np.zeros((5, 7), np.uint8)
    for (i, j, ox, oy) in [(3, 2, 3, 2), (6, 0, 1, 3), (0, 4, 5, 0)]:
        m[:] = 0
        m[j, i] = 1
        dx, dy = i - ox, j - oy
        # erosion: E(x, y) = I(x+dx, y+dy) inside, 1 outside
        want_e = np.ones_like(img)
        want_d = np.zeros_like(img)
        for y in range(H):
            for x in range(W):
                if 0 <= x + dx < W and 0 <= y + dy < H:
                    want_e[y, x] = img[y + dy, x + dx]
                if 0 <= x - dx < W and 0 <= y - dy < H:
                    want_d[y, x] = img[y - dy, x - dx]
        assert np.array_equal(oracle.erode_mask(img, m, ox, oy), want_e)
        assert np.array_equal(oracle.dilate_mask(img, m, ox, oy), want_d)
        if dx == 0 and dy == 0:
            assert np.array_equal(want_e, img)


def test_dilation_is_the_dual_of_erosion_by_the_reflected_mask():
    rng = np.random.default_rng(6)
    for k in range(6):
        img = rand_img(rng, 15 + k, 21, 0.4)
        m = rand_mask(rng, 1 + k, 2 + 2 * k, 0.5)
        ox, oy = int(rng.integers(m.shape[1])), int(rng.integers(m.shape[0]))
        r, rx, ry = oracle.reflect_mask(m, ox, oy)
        assert np.array_equal(oracle.dilate_mask(img, m, ox, oy), 1 - oracle.erode_mask(1 - img, r, rx, ry))


def test_erosion_by_a_union_is_the_and_of_erosions():
    rng = np.random.default_rng(7)
    for k in range(5):
        img = rand_img(rng, 25, 31, 0.7)
        a = rand_mask(rng, 5, 6, 0.3)
        b = rand_mask(rng, 5, 6, 0.3)
        ox, oy = 2, 3
        assert np.array_equal(oracle.erode_mask(img, a | b, ox, oy),
                              oracle.erode_mask(img, a, ox, oy) & oracle.erode_mask(img, b, ox, oy))
        assert np.array_equal(oracle.dilate_mask(img, a | b, ox, oy),
                              oracle.dilate_mask(img, a, ox, oy) | oracle.dilate_mask(img, b, ox, oy))


def test_opening_removes_and_closing_adds_only():
    rng = np.random.default_rng(8)
    img = rand_img(rng, 40, 50, 0.5)
    d = oracle.disc_mask(3)
    assert not (oracle.apply_mask("open", img, d, 3, 3) > img).any()
    assert not (oracle.apply_mask("close", img, d, 3, 3) < img).any()


@pytest.mark.parametrize("H,W", [(1, 1), (1, 37), (29, 1), (33, 47)])
def test_pixel_at_a_time_equals_run_at_a_time(H, W):
    rng = np.random.default_rng(H * 31 + W)
    for k in range(8):
        img = rand_img(rng, H, W, [0.2, 0.5, 0.9][k % 3])
        m = rand_mask(rng, 1 + k % 5, 1 + (3 * k) % 9, 0.45)
        ox, oy = int(rng.integers(m.shape[1])), int(rng.integers(m.shape[0]))
        for op in ("erode", "dilate", "open", "close"):
            assert np.array_equal(oracle.apply_mask(op, img, m, ox, oy, mode="brute"),
                                  oracle.apply_mask(op, img, m, ox, oy, mode="runs")), (op, k)


def test_mask_runs_and_disc():
    d = oracle.disc_mask(2)
    assert d.tolist() == [[0, 0, 1, 0, 0], [0, 1, 1, 1, 0], [1, 1, 1, 1, 1], [0, 1, 1, 1, 0], [0, 0, 1, 0, 0]]
    assert oracle.mask_runs(d) == [(0, 2, 1), (1, 1, 3), (2, 0, 5), (3, 1, 3), (4, 2, 1)]
    assert oracle.mask_runs([[1, 0, 1, 1]]) == [(0, 0, 1), (0, 2, 2)]
    with pytest.raises(ValueError):
        oracle.erode_mask(np.zeros((3, 3), np.uint8), np.zeros((2, 2), np.uint8), 0, 0)
