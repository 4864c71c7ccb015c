"""Pins of the connected-component and run-length-statistics oracle (sections
"Connected Component Extraction and Statistics" and "Other Operations")
against what does not depend on it: a breadth-first flood fill over pixels
written here, scipy's pixel labelling (renumbered in raster order), closed
forms (empty, full, checkerboard, diagonal, stripes), per-label statistics
gathered with numpy from the painted label image, and run lengths read off
the bitmap's transitions with numpy."""
from collections import deque

import numpy as np
import pytest

import oracle


def rand_img(rng, H, W, p):
    return (rng.random((H, W)) < p).astype(np.uint8)


def paint_labels(labels, row_ptr, runs, W, H):
    """Label image: -1 on background, the run's label on its pixels."""
    out = np.full((H, W), -1, np.int64)
    for y in range(H):
        for k in range(row_ptr[y], row_ptr[y + 1]):
            out[y, runs[k, 0]:runs[k, 1]] = labels[k]
    return out


def flood_fill(img, conn):
    """Pixel labels by breadth-first search, numbered in the raster order of
    each component's first pixel (-1 on background)."""
    H, W = img.shape
    lab = np.full((H, W), -1, np.int64)
    if conn == 4:
        nb = [(-1, 0), (1, 0), (0, -1), (0, 1)]
    else:
        nb = [(dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1) if dy or dx]
    n = 0
    for y in range(H):
        for x in range(W):
            if img[y, x] and lab[y, x] < 0:
                lab[y, x] = n
                q = deque([(y, x)])
                while q:
                    cy, cx = q.popleft()
                    for dy, dx in nb:
                        yy, xx = cy + dy, cx + dx
                        if 0 <= yy < H and 0 <= xx < W and img[yy, xx] and lab[yy, xx] < 0:
                            lab[yy, xx] = n
                            q.append((yy, xx))
                n += 1
    return lab, n


def raster_renumber(lab):
    """Renumber non-negative labels by first appearance in raster order."""
    out = np.full(lab.shape, -1, np.int64)
    flat = lab.ravel()
    seen = {}
    for v in flat:
        if v >= 0 and v not in seen:
            seen[v] = len(seen)
    for v, k in seen.items():
        out[lab == v] = k
    return out, len(seen)


def oracle_pixel_labels(img, conn):
    H, W = img.shape
    rp, ru = oracle.rle_encode(img)
    labels, n = oracle.rle_components(rp, ru, H, conn)
    return paint_labels(labels, rp, ru, W, H), n


@pytest.mark.parametrize("conn", [4, 8])
def test_all_3x3_images_match_flood_fill(conn):
    for code in range(512):
        img = ((code >> np.arange(9)) & 1).astype(np.uint8).reshape(3, 3)
        got, n = oracle_pixel_labels(img, conn)
        want, m = flood_fill(img, conn)
        assert n == m and np.array_equal(got, want), (code, conn)


@pytest.mark.parametrize("conn", [4, 8])
@pytest.mark.parametrize("H,W,p", [(7, 9, 0.5), (12, 31, 0.45), (25, 40, 0.6), (1, 50, 0.5), (50, 1, 0.5)])
def test_random_images_match_flood_fill(conn, H, W, p):
    rng = np.random.default_rng(H * 1000 + W + conn)
    for _ in range(4):
        img = rand_img(rng, H, W, p)
        got, n = oracle_pixel_labels(img, conn)
        want, m = flood_fill(img, conn)
        assert n == m and np.array_equal(got, want)


@pytest.mark.parametrize("conn", [4, 8])
def test_matches_scipy_label_on_a_page_sized_image(conn):
    nd = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(77 + conn)
    img = rand_img(rng, 300, 517, 0.42)
    structure = np.ones((3, 3), int) if conn == 8 else None
    lab, m = nd.label(img, structure=structure)
    want, m2 = raster_renumber(np.where(img > 0, lab - 1, -1))
    got, n = oracle_pixel_labels(img, conn)
    assert n == m == m2
    assert np.array_equal(got, want)


@pytest.mark.parametrize("conn", [4, 8])
def test_closed_forms(conn):
    H, W = 9, 14
    # empty image: no runs, no component
    rp, ru = oracle.rle_encode(np.zeros((H, W), np.uint8))
    labels, n = oracle.rle_components(rp, ru, H, conn)
    assert n == 0 and labels.size == 0
    # full image: one component, the whole box
    full = np.ones((H, W), np.uint8)
    rp, ru = oracle.rle_encode(full)
    labels, n = oracle.rle_components(rp, ru, H, conn)
    assert n == 1 and not labels.any()
    st = oracle.rle_component_stats(labels, n, rp, ru, H)
    assert st.tolist() == [[0, 0, W, H, W * H, H * W * (W - 1) // 2, W * H * (H - 1) // 2]]
    # checkerboard: every pixel alone under 4-connectivity, one component under 8
    yy, xx = np.mgrid[0:H, 0:W]
    cb = ((yy + xx) % 2 == 0).astype(np.uint8)
    rp, ru = oracle.rle_encode(cb)
    labels, n = oracle.rle_components(rp, ru, H, conn)
    assert n == (int(cb.sum()) if conn == 4 else 1)
    # anti-diagonal: pixels touch only at corners
    d = np.zeros((8, 8), np.uint8)
    d[np.arange(8), 7 - np.arange(8)] = 1
    rp, ru = oracle.rle_encode(d)
    assert oracle.rle_components(rp, ru, 8, conn)[1] == (8 if conn == 4 else 1)
    # vertical stripes two columns apart: one component per stripe, numbered left to right
    st_img = np.zeros((H, W), np.uint8)
    st_img[:, ::3] = 1
    rp, ru = oracle.rle_encode(st_img)
    labels, n = oracle.rle_components(rp, ru, H, conn)
    assert n == len(range(0, W, 3))
    assert labels.reshape(H, -1).tolist() == [list(range(n))] * H


def test_u_shape_merges_late():
    """Two arms that join only at the bottom line: the merge happens after
    both arms were labelled apart, so the relabelling must reach back."""
    img = np.zeros((6, 7), np.uint8)
    img[:, 0] = 1
    img[:, 6] = 1
    img[5, :] = 1
    img[0:3, 3] = 1  # a separate bar in the middle
    rp, ru = oracle.rle_encode(img)
    labels, n = oracle.rle_components(rp, ru, 6, 4)
    assert n == 2
    pix = paint_labels(labels, rp, ru, 7, 6)
    assert pix[0, 0] == pix[0, 6] == pix[5, 3] == 0 and pix[0, 3] == 1


@pytest.mark.parametrize("conn", [4, 8])
def test_stats_match_numpy(conn):
    rng = np.random.default_rng(9 + conn)
    img = rand_img(rng, 60, 83, 0.5)
    H, W = img.shape
    rp, ru = oracle.rle_encode(img)
    labels, n = oracle.rle_components(rp, ru, H, conn)
    st = oracle.rle_component_stats(labels, n, rp, ru, H)
    pix = paint_labels(labels, rp, ru, W, H)
    ys, xs = np.nonzero(pix >= 0)
    lab = pix[ys, xs]
    assert np.array_equal(st[:, 4], np.bincount(lab, minlength=n))
    assert np.array_equal(st[:, 5], np.bincount(lab, weights=xs, minlength=n).astype(np.int64))
    assert np.array_equal(st[:, 6], np.bincount(lab, weights=ys, minlength=n).astype(np.int64))
    for c in range(n):
        sel = lab == c
        assert st[c, :4].tolist() == [xs[sel].min(), ys[sel].min(), xs[sel].max() + 1, ys[sel].max() + 1]


def numpy_run_lengths(img):
    """(black, white) histograms from the transitions of each padded row."""
    H, W = img.shape
    black = np.zeros(W + 1, np.int64)
    white = np.zeros(W + 1, np.int64)
    for row in img.astype(np.int8):
        for val, hist in ((1, black), (0, white)):
            m = np.concatenate([[0], (row == val).astype(np.int8), [0]])
            d = np.diff(m)
            starts, ends = np.nonzero(d == 1)[0], np.nonzero(d == -1)[0]
            np.add.at(hist, ends - starts, 1)
    return black, white


@pytest.mark.parametrize("H,W,p", [(1, 1, 0.5), (20, 33, 0.3), (40, 64, 0.7), (7, 300, 0.05)])
def test_run_length_hist_matches_numpy(H, W, p):
    rng = np.random.default_rng(H + W)
    img = rand_img(rng, H, W, p)
    rp, ru = oracle.rle_encode(img)
    black, white = oracle.run_length_hist(rp, ru, W, H)
    nb, nw = numpy_run_lengths(img)
    assert np.array_equal(black, nb) and np.array_equal(white, nw)
    assert int((np.arange(W + 1) * (black + white)).sum()) == W * H


def test_run_length_hist_closed_forms():
    H, W = 5, 12
    rp, ru = oracle.rle_encode(np.zeros((H, W), np.uint8))
    b, w = oracle.run_length_hist(rp, ru, W, H)
    assert not b.any() and w[W] == H and w.sum() == H
    rp, ru = oracle.rle_encode(np.ones((H, W), np.uint8))
    b, w = oracle.run_length_hist(rp, ru, W, H)
    assert not w.any() and b[W] == H and b.sum() == H
    # "0110" repeated: black runs of 2, white runs of 2 inside, 1 at each end
    row = np.tile(np.array([0, 1, 1, 0], np.uint8), 3)
    rp, ru = oracle.rle_encode(np.tile(row, (H, 1)))
    b, w = oracle.run_length_hist(rp, ru, W, H)
    assert b[2] == 3 * H and b.sum() == 3 * H
    assert w[2] == 2 * H and w[1] == 2 * H and w.sum() == 4 * H
