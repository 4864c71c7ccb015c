"""Connected components, component statistics and run-length histograms of
RLE images on the GPU against the oracle (section "Connected Component
Extraction and Statistics"; run-length statistics of section "Other
Operations").  The labelling is unique (components numbered in the raster
order of their first run), so labels, counts and statistics must match
exactly."""
import numpy as np
import pytest
import torch

import oracle
from paper_0712_0121_gb300 import synth

pytestmark = pytest.mark.gpu

M = pytest.importorskip("paper_0712_0121_gb300.morph")
from gpu_helpers import to_rle  # noqa: E402


def check_components(img, conn, stats=True, capacity_extra=0):
    H, W = img.shape
    rle = to_rle(img)
    if capacity_extra:
        big = M.Rle.empty(W, H, rle.capacity + capacity_extra)
        M.rle_from_bitmap(big, M.pack(img, 64))
        rle = big
    rp, runs = oracle.rle_encode(img)
    want, n = oracle.rle_components(rp, runs, H, conn)
    want_stats = bool(stats)
    # exactly as many records as components (no capacity error)
    rec = torch.empty((max(n, 1), 7), dtype=torch.int64, device="cuda") if want_stats else False
    labels, st, nc = M.rle_components(rle, conn, stats=rec)
    assert M.sync_status() == M.MORPH_OK
    assert int(nc.item()) == n
    got = labels[: int(rp[-1])].cpu().numpy()
    assert np.array_equal(got, want), "first differing run %s" % np.argwhere(got != want)[:3].ravel()
    if want_stats:
        ref = oracle.rle_component_stats(want, n, rp, runs, H)
        assert np.array_equal(st[:n].cpu().numpy(), ref)
    return n


@pytest.mark.parametrize("conn", [4, 8])
@pytest.mark.parametrize("H,W,p", [(1, 1, 1.0), (1, 70, 0.5), (70, 1, 0.5), (37, 53, 0.5),
                                   (300, 517, 0.42), (257, 2000, 0.55), (1030, 333, 0.6)])
def test_random_images(conn, H, W, p):
    img = synth.random_bits((H, W), 4000 + H + W + conn, p)
    check_components(img, conn)


@pytest.mark.parametrize("conn", [4, 8])
def test_closed_forms(conn):
    H, W = 40, 90
    assert check_components(np.zeros((H, W), np.uint8), conn) == 0
    assert check_components(np.ones((H, W), np.uint8), conn) == 1
    yy, xx = np.mgrid[0:H, 0:W]
    cb = ((yy + xx) % 2 == 0).astype(np.uint8)
    assert check_components(cb, conn) == (int(cb.sum()) if conn == 4 else 1)


@pytest.mark.parametrize("conn", [4, 8])
def test_document_and_halftone_pages(conn):
    page, _ = synth.document_page(2550, 3300, synth.seed_for(2, 0), 0.08)
    check_components(page, conn)
    # one giant component per blob region: long union chains, many runs per label
    ht, _ = synth.halftone_page(1200, 900, synth.seed_for(3, 2))
    check_components(ht, conn)


def test_spare_capacity_and_no_stats():
    img = synth.random_bits((64, 300), 99, 0.5)
    check_components(img, 4, stats=False, capacity_extra=1000)
    check_components(img, 8, stats=True, capacity_extra=1000)


def test_too_many_components_latches_capacity():
    img = synth.random_bits((50, 80), 7, 0.3)
    H, W = img.shape
    rle = to_rle(img)
    rp, runs = oracle.rle_encode(img)
    want, n = oracle.rle_components(rp, runs, H, 4)
    assert n > 10
    stats = torch.empty((10, 7), dtype=torch.int64, device="cuda")
    labels, st, nc = M.rle_components(rle, 4, stats=stats)
    assert M.sync_status() == M.MORPH_ECAPACITY
    assert int(nc.item()) == n
    assert np.array_equal(labels[: int(rp[-1])].cpu().numpy(), want)
    ref = oracle.rle_component_stats(want, n, rp, runs, H)
    assert np.array_equal(st.cpu().numpy(), ref[:10])


def test_tall_stack():
    """Eight letter pages stacked (26400 rows: the per-line scan runs as
    three launches), every label and record against the oracle."""
    pages = [synth.document_page(2550, 3300, synth.seed_for(2, k), 0.08)[0] for k in range(4)]
    img = np.concatenate(pages * 2, axis=0)  # 26400 rows
    H, W = img.shape
    check_components(img, 8)


@pytest.mark.parametrize("H,W,p", [(1, 1, 0.5), (3, 5000, 0.001), (40, 64, 0.7), (500, 2550, 0.08),
                                   (20, 3000, 0.5)])
def test_run_length_hist(H, W, p):
    img = synth.random_bits((H, W), 5000 + H + W, p)
    rle = to_rle(img)
    rp, runs = oracle.rle_encode(img)
    b_ref, w_ref = oracle.run_length_hist(rp, runs, W, H)
    b, w = M.run_length_hist(rle)
    assert np.array_equal(b.cpu().numpy(), b_ref)
    assert np.array_equal(w.cpu().numpy(), w_ref)


def test_run_length_hist_pages():
    for img in (synth.document_page(2550, 3300, synth.seed_for(2, 1), 0.08)[0],
                np.zeros((7, 4000), np.uint8), np.ones((9, 3000), np.uint8)):
        H, W = img.shape
        rle = to_rle(img)
        rp, runs = oracle.rle_encode(img)
        b_ref, w_ref = oracle.run_length_hist(rp, runs, W, H)
        b, w = M.run_length_hist(rle)
        assert np.array_equal(b.cpu().numpy(), b_ref)
        assert np.array_equal(w.cpu().numpy(), w_ref)


@pytest.mark.parametrize("conn", [4, 8])
def test_crowded_lines(conn):
    """Lines with more runs than a band keeps in shared memory (alternating
    pixels: 4500 runs per line) and bands cut into several sub-bands (about
    a thousand runs per line): the seams inside a band are joined in global
    memory."""
    H, W = 70, 9000
    img = np.zeros((H, W), np.uint8)
    img[:, ::2] = 1
    noise = synth.random_bits((H, W), 31 + conn, 0.3)
    img[10:40] |= noise[10:40]
    check_components(img, conn)
    check_components(synth.random_bits((200, 4000), 77 + conn, 0.5), conn)
