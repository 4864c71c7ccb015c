"""Pins of the CPU oracle against things other than itself.

What fixes the result here:
  * a second, structurally different brute force: whole-image shifted AND / OR
    with padding (the paper's pixel-at-a-time ``bits_and`` loop, section
    "Morphology with Arbitrary Masks"), exhaustively on every 4x4 image;
  * the paper's run-list algorithms (section "Within-Line Morphological
    Operations": open1d, complement, close1d, erode1d, dilate1d), written here
    from their description with the stated readings;
  * closed forms (single pixel, rectangle, identity, constant images);
  * invariants of the operators (duality, separability, exact composition of
    segments, idempotence, (anti-)extensivity, monotonicity);
  * scipy.ndimage (a library routine) where it is installed;
  * the paper's worked TransitionSink example and its RLE size facts
    (``tests/golden``).
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_0712_0121_gb300 import synth
from conftest import read_golden


# ----------------------------------------------------------------- helpers

def shifted_and_or(imgs, sw, sh, ox, oy, dilate):
    """Whole-image shifted AND (erosion: pixel (x+i-ox, y+j-oy) moved onto
    (x, y), outside = 1) or OR (dilation: pixel (x-i+ox, y-j+oy), outside = 0)
    over every mask pixel (i, j).  imgs: uint8[n, H, W]."""
    n, H, W = imgs.shape
    m = max(sw, sh) + 1
    fill = 0 if dilate else 1
    P = np.full((n, H + 2 * m, W + 2 * m), fill, dtype=np.uint8)
    P[:, m:m + H, m:m + W] = imgs
    acc = np.full((n, H, W), fill, dtype=np.uint8)
    for i in range(sw):
        for j in range(sh):
            if dilate:
                dx, dy = -i + ox, -j + oy
                acc |= P[:, m + dy:m + dy + H, m + dx:m + dx + W]
            else:
                dx, dy = i - ox, j - oy
                acc &= P[:, m + dy:m + dy + H, m + dx:m + dx + W]
    return acc


def runs_of_row(row):
    """Maximal runs [s, e) of a 0/1 row (plain scan)."""
    runs, x, W = [], 0, len(row)
    while x < W:
        if row[x]:
            s = x
            while x < W and row[x]:
                x += 1
            runs.append((s, x))
        else:
            x += 1
    return runs


def paint(runs, W):
    row = np.zeros(W, dtype=np.uint8)
    for s, e in runs:
        row[s:e] = 1
    return row


# The paper's run-list algorithms, half-open runs on a row of W pixels.
def open1d(runs, u):
    """Keep runs of width >= u."""
    return [(s, e) for s, e in runs if e - s >= u]


def complement(runs, W):
    """Gaps between runs, including the border gaps, within [0, W)."""
    out, last = [], 0
    for s, e in runs:
        if s > last:
            out.append((last, s))
        last = e
    if last < W:
        out.append((last, W))
    return out


def close1d(runs, u, W):
    return complement(open1d(complement(runs, W), u), W)


def erode1d(runs, u, o, W):
    """Shrink each run by o on the left and u-1-o on the right; an end on the
    image border stays (clipped window); drop empty runs."""
    out = []
    for s, e in runs:
        s2 = s if s == 0 else s + o
        e2 = e if e == W else e - (u - 1 - o)
        if s2 < e2:
            out.append((s2, e2))
    return out


def dilate1d(runs, u, o, W):
    """complement, erode1d with the reflected origin, complement."""
    return complement(erode1d(complement(runs, W), u, u - 1 - o, W), W)


def doc(W, H, seed, density=0.12):
    return synth.text_page(W, H, seed, density, glyph=(3, 7, 4, 9), gap=(1, 4))[0]


# ------------------------------------------------------ exhaustive 4 x 4

ALL_4x4 = ((np.arange(1 << 16)[:, None] >> np.arange(16)[None, :]) & 1).astype(np.uint8).reshape(-1, 4, 4)


@pytest.mark.parametrize("sw,sh", list(itertools.product(range(1, 5), range(1, 5))))
def test_exhaustive_4x4_erode_dilate(sw, sh):
    for ox in range(sw):
        for oy in range(sh):
            for op, dil in (("erode", False), ("dilate", True)):
                got = oracle.rect_batch(ALL_4x4, sw, sh, ox, oy, op)
                ref = shifted_and_or(ALL_4x4, sw, sh, ox, oy, dil)
                assert np.array_equal(got, ref), (op, sw, sh, ox, oy)


@pytest.mark.parametrize("sw,sh", [(1, 2), (2, 1), (2, 2), (3, 2), (2, 3), (3, 3), (4, 4), (1, 4)])
def test_exhaustive_4x4_open_close(sw, sh):
    for ox in range(sw):
        for oy in range(sh):
            e = shifted_and_or(ALL_4x4, sw, sh, ox, oy, False)
            d = shifted_and_or(ALL_4x4, sw, sh, ox, oy, True)
            op_ref = shifted_and_or(e, sw, sh, ox, oy, True)
            cl_ref = shifted_and_or(d, sw, sh, ox, oy, False)
            assert np.array_equal(oracle.rect_batch(ALL_4x4, sw, sh, ox, oy, "open"), op_ref)
            assert np.array_equal(oracle.rect_batch(ALL_4x4, sw, sh, ox, oy, "close"), cl_ref)


def test_shifted_reference_on_larger_images():
    """The two brute forces agree on larger random and document images too
    (SE larger than the image included)."""
    imgs = np.stack([synth.random_bits((13, 29), 100 + k, 0.55) for k in range(3)]
                    + [doc(29, 13, 7)])
    for sw, sh, ox, oy in [(5, 3, 0, 2), (7, 1, 6, 0), (1, 6, 0, 3), (8, 8, 3, 4), (40, 2, 13, 1),
                           (3, 20, 1, 19)]:
        for op, dil in (("erode", False), ("dilate", True)):
            got = oracle.rect_batch(imgs, sw, sh, ox, oy, op)
            assert np.array_equal(got, shifted_and_or(imgs, sw, sh, ox, oy, dil)), (op, sw, sh)


# ------------------------------------------------------- separable mode

@pytest.mark.parametrize("op", ["erode", "dilate", "open", "close"])
def test_separable_mode_equals_brute_force(op):
    img = doc(97, 71, 11)
    rnd = synth.random_bits((40, 77), 12, 0.7)
    for a in (img, rnd):
        for sw, sh, ox, oy in [(3, 3, 1, 1), (4, 2, 0, 1), (11, 1, 5, 0), (1, 11, 0, 5), (6, 9, 5, 0),
                               (31, 7, 2, 6), (101, 1, 50, 0)]:
            ref = oracle.apply(op, a, sw, sh, ox, oy, mode="brute")
            got = oracle.apply(op, a, sw, sh, ox, oy, mode="separable", threads=2)
            assert np.array_equal(ref, got), (op, sw, sh, ox, oy)


# ---------------------------------------------------------- scipy routine

def test_scipy_ndimage_cross_check():
    ndi = pytest.importorskip("scipy.ndimage")
    for k in range(4):
        img = synth.random_bits((23, 31), 200 + k, 0.5 + 0.1 * k)
        for sw, sh in [(1, 1), (2, 1), (1, 2), (2, 2), (3, 3), (4, 5), (6, 2)]:
            for ox in range(sw):
                for oy in range(sh):
                    st = np.ones((sh, sw), bool)
                    org = (oy - sh // 2, ox - sw // 2)
                    e = ndi.binary_erosion(img.astype(bool), structure=st, border_value=1, origin=org)
                    d = ndi.binary_dilation(img.astype(bool), structure=st, border_value=0, origin=org)
                    assert np.array_equal(oracle.erode(img, sw, sh, ox, oy), e.astype(np.uint8))
                    assert np.array_equal(oracle.dilate(img, sw, sh, ox, oy), d.astype(np.uint8))


# ------------------------------------------------------------ closed forms

def test_identity_and_constants():
    img = doc(41, 23, 3)
    for op in ("erode", "dilate", "open", "close"):
        assert np.array_equal(oracle.apply(op, img, 1, 1, 0, 0), img)
    ones = np.ones((9, 13), np.uint8)
    zeros = np.zeros((9, 13), np.uint8)
    for op in ("erode", "dilate", "open", "close"):
        for sw, sh, ox, oy in [(3, 3, 1, 1), (20, 2, 0, 1), (2, 30, 1, 29)]:
            assert np.array_equal(oracle.apply(op, ones, sw, sh, ox, oy), ones)
            assert np.array_equal(oracle.apply(op, zeros, sw, sh, ox, oy), zeros)


def test_single_pixel_dilation_is_rectangle():
    W, H = 30, 20
    for (px, py), (sw, sh, ox, oy) in itertools.product([(0, 0), (12, 7), (29, 19), (3, 18)],
                                                        [(5, 3, 1, 2), (1, 7, 0, 0), (9, 1, 8, 0)]):
        img = np.zeros((H, W), np.uint8)
        img[py, px] = 1
        ref = np.zeros_like(img)
        # Minkowski addition: the point spreads to p + (i - ox, j - oy)
        x0, x1 = max(0, px - ox), min(W - 1, px + sw - 1 - ox)
        y0, y1 = max(0, py - oy), min(H - 1, py + sh - 1 - oy)
        ref[y0:y1 + 1, x0:x1 + 1] = 1
        assert np.array_equal(oracle.dilate(img, sw, sh, ox, oy), ref)


def test_interior_rectangle_erosion():
    W, H = 40, 30
    img = np.zeros((H, W), np.uint8)
    x0, x1, y0, y1 = 8, 31, 5, 22
    img[y0:y1, x0:x1] = 1
    for sw, sh, ox, oy in [(3, 3, 1, 1), (5, 2, 0, 1), (7, 7, 6, 2), (1, 9, 0, 4)]:
        ref = np.zeros_like(img)
        ref[y0 + oy:y1 - (sh - 1 - oy), x0 + ox:x1 - (sw - 1 - ox)] = 1
        assert np.array_equal(oracle.erode(img, sw, sh, ox, oy), ref)


# --------------------------------------------------------------- invariants

CASES = [(3, 3, 1, 1), (4, 3, 0, 2), (5, 5, 4, 0), (2, 7, 1, 3), (11, 1, 5, 0), (1, 11, 0, 10)]


@pytest.mark.parametrize("sw,sh,ox,oy", CASES)
def test_duality(sw, sh, ox, oy):
    img = doc(53, 37, 5)
    d = oracle.dilate(img, sw, sh, ox, oy)
    e_ref = oracle.erode(1 - img, sw, sh, sw - 1 - ox, sh - 1 - oy)
    assert np.array_equal(d, 1 - e_ref)


@pytest.mark.parametrize("sw,sh,ox,oy", CASES)
def test_separability(sw, sh, ox, oy):
    img = doc(53, 37, 6, 0.3)
    for op in ("erode", "dilate"):
        h = oracle.apply(op, img, sw, 1, ox, 0)
        assert np.array_equal(oracle.apply(op, img, sw, sh, ox, oy), oracle.apply(op, h, 1, sh, 0, oy))


def test_segment_composition_is_exact():
    """E_{B1+B2} = E_B2 o E_B1 for segments whose origins lie inside them
    (Minkowski sum of segments, origins add) — also at the borders."""
    img = synth.random_bits((17, 61), 9, 0.8)
    for (a, oa), (b, ob) in [((3, 1), (4, 0)), ((5, 4), (2, 1)), ((7, 0), (7, 6)), ((1, 0), (9, 3))]:
        for op in ("erode", "dilate"):
            two = oracle.apply(op, oracle.apply(op, img, a, 1, oa, 0), b, 1, ob, 0)
            one = oracle.apply(op, img, a + b - 1, 1, oa + ob, 0)
            assert np.array_equal(one, two), (op, a, oa, b, ob)


@pytest.mark.parametrize("sw,sh,ox,oy", CASES)
def test_idempotence_and_extensivity(sw, sh, ox, oy):
    img = doc(47, 39, 8, 0.2)
    o = oracle.opening(img, sw, sh, ox, oy)
    c = oracle.closing(img, sw, sh, ox, oy)
    assert np.array_equal(oracle.opening(o, sw, sh, ox, oy), o)
    assert np.array_equal(oracle.closing(c, sw, sh, ox, oy), c)
    assert np.all(o <= img) and np.all(img <= c)
    assert np.all(oracle.erode(img, sw, sh, ox, oy) <= img)
    assert np.all(img <= oracle.dilate(img, sw, sh, ox, oy))


def test_monotone_in_the_structuring_element():
    img = doc(47, 39, 10, 0.25)
    small, big = (3, 2, 1, 1), (5, 4, 2, 1)  # small rectangle inside big, same origin point
    assert np.all(oracle.erode(img, *big) <= oracle.erode(img, *small))
    assert np.all(oracle.dilate(img, *small) <= oracle.dilate(img, *big))


# --------------------------------------------- paper's run-list algorithms

def test_rows_against_paper_run_algorithms():
    W = 73
    rows = np.concatenate([synth.random_bits((60, W), 31, 0.65), doc(W, 40, 32, 0.4)])
    for u in (1, 2, 3, 4, 7, 12):
        for o in range(u):
            e = oracle.erode(rows, u, 1, o, 0)
            d = oracle.dilate(rows, u, 1, o, 0)
            for y in range(rows.shape[0]):
                r = runs_of_row(rows[y])
                assert np.array_equal(e[y], paint(erode1d(r, u, o, W), W)), (u, o, y)
                assert np.array_equal(d[y], paint(dilate1d(r, u, o, W), W)), (u, o, y)


def test_open1d_and_close1d_on_interior_runs():
    """A u x 1 opening deletes the runs shorter than u and keeps the others
    untouched; a closing fills the gaps shorter than u (interior runs / gaps,
    since the clipped window treats runs touching the border as unbounded)."""
    W = 80
    rows = synth.random_bits((120, W), 41, 0.6)
    rows_o = rows.copy()
    rows_o[:, 0] = rows_o[:, -1] = 0
    rows_c = rows.copy()
    rows_c[:, 0] = rows_c[:, -1] = 1
    for u in (2, 3, 5, 8):
        for o in range(u):
            op = oracle.opening(rows_o, u, 1, o, 0)
            cl = oracle.closing(rows_c, u, 1, o, 0)
            for y in range(rows.shape[0]):
                assert np.array_equal(op[y], paint(open1d(runs_of_row(rows_o[y]), u), W))
                assert np.array_equal(cl[y], paint(close1d(runs_of_row(rows_c[y]), u, W), W))


# ------------------------------------------------------------------- RLE

def test_rle_round_trip_and_canonical():
    for img in (doc(301, 57, 50), synth.random_bits((31, 257), 51, 0.5), np.ones((3, 64), np.uint8),
                np.zeros((4, 65), np.uint8)):
        rp, runs = oracle.rle_encode(img)
        H, W = img.shape
        for y in range(H):
            rr = runs[rp[y]:rp[y + 1]].astype(int)
            assert [tuple(r) for r in rr] == runs_of_row(img[y])
            assert np.all(rr[:, 0] < rr[:, 1]) if len(rr) else True
            assert np.all(rr[1:, 0] > rr[:-1, 1]) if len(rr) > 1 else True
        assert np.array_equal(oracle.rle_decode(rp, runs, W, H), img)


def test_rle_decode_rejects_non_canonical():
    rp = np.array([0, 2], np.int32)
    with pytest.raises(ValueError):
        oracle.rle_decode(rp, np.array([[1, 4], [4, 6]], np.uint16), 10, 1)  # touching
    with pytest.raises(ValueError):
        oracle.rle_decode(rp, np.array([[5, 7], [1, 2]], np.uint16), 10, 1)  # unsorted
    with pytest.raises(ValueError):
        oracle.rle_decode(np.array([0, 1], np.int32), np.array([[3, 3]], np.uint16), 10, 1)  # empty


def test_golden_transition_sink():
    g = read_golden("transition_sink.txt")
    seq = [t.split() for t in g["transitions"].split("|")]
    want = g["runs"].split()
    for xs in ([2, 5, 9, 14, 20], [0, 1, 2, 3, 4], [7, 8, 30, 31, 32]):
        name = {"x%d" % i: x for i, x in enumerate(xs)}
        W = xs[-1] + 3
        row = np.zeros((1, W), np.uint8)
        for k, (sym, val) in enumerate(seq):
            end = name[seq[k + 1][0]] if k + 1 < len(seq) else W
            row[0, name[sym]:end] = 1 if val == "T" else 0
        rp, runs = oracle.rle_encode(row)
        assert [tuple(int(v) for v in r) for r in runs] == [(name[want[0]], name[want[1]])]


def test_golden_rle_size_facts():
    g = read_golden("rle_size_facts.txt")
    W = 4096
    row = (np.arange(W) % 2 == 0).astype(np.uint8)[None, :]
    rp, runs = oracle.rle_encode(row)
    rle_bytes = runs.shape[0] * 4
    assert rle_bytes == int(g["worst_case_vs_packed"]) * (W // 8)
    assert rle_bytes == int(g["worst_case_vs_unpacked"]) * W
    f = int(g["scale_factor"])
    img = doc(200, 150, 77, 0.15)
    big = np.repeat(np.repeat(img, f, axis=0), f, axis=1)
    n_small = oracle.rle_encode(img)[1].shape[0]
    n_big = oracle.rle_encode(big)[1].shape[0]
    assert n_big == int(g["rle_growth"]) * n_small
    assert big.size // 8 == int(g["packed_growth"]) * (img.size // 8)


def test_rle_apply_is_definition():
    img = doc(90, 40, 60, 0.3)
    rp, runs = oracle.rle_encode(img)
    for op in ("erode", "dilate", "open", "close"):
        rp2, runs2 = oracle.rle_apply(op, rp, runs, 90, 40, 5, 3, 2, 1)
        assert np.array_equal(oracle.rle_decode(rp2, runs2, 90, 40), oracle.apply(op, img, 5, 3, 2, 1))
