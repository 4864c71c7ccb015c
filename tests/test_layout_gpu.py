"""Layout analysis on the GPU (section "Document Analysis Performance")
against the same steps composed from the oracle: white-run histograms along
the lines and along the columns, the gap estimates, the dilation by the
estimated rectangle, the 8-connected components and their records."""
import numpy as np
import pytest
import torch

import oracle
from paper_0712_0121_gb300 import synth

pytestmark = pytest.mark.gpu

M = pytest.importorskip("paper_0712_0121_gb300.morph")


def gap_estimate(white, lmax, pct):
    """Smallest L in [1, lmax] whose white runs of length <= L are at least
    pct percent of those of length <= lmax; 0 if there are none."""
    counts = np.asarray(white[1:lmax + 1], dtype=np.int64)
    total = int(counts.sum())
    if total == 0:
        return 0
    cum = np.cumsum(counts)
    return int(np.nonzero(cum * 100 >= pct * total)[0][0]) + 1


def oracle_layout(page, pct):
    H, W = page.shape
    rp, runs = oracle.rle_encode(page)
    _, wh = oracle.run_length_hist(rp, runs, W, H)
    rpt, runst = oracle.rle_encode(oracle.transpose(page))
    _, wv = oracle.run_length_hist(rpt, runst, H, W)
    th = gap_estimate(wh, max(W // 16, 1), pct)
    tv = gap_estimate(wv, max(H // 16, 1), pct)
    d = oracle.dilate(page, th + 1, tv + 1, (th + 1) // 2, (tv + 1) // 2, mode="separable")
    rpd, runsd = oracle.rle_encode(d)
    lab, n = oracle.rle_components(rpd, runsd, H, 8)
    return (th, tv), oracle.rle_component_stats(lab, n, rpd, runsd, H)


def check(page, pct=90):
    boxes, n, gaps = M.layout_boxes(M.pack(page, 64), pct)
    assert M.sync_status() == M.MORPH_OK
    ref_gaps, ref = oracle_layout(page, pct)
    assert gaps == ref_gaps
    k = int(n.item())
    assert k == ref.shape[0]
    assert np.array_equal(boxes[:k].cpu().numpy(), ref)
    return gaps, k


@pytest.mark.parametrize("seed", [0, 1])
def test_letter_pages(seed):
    page, _ = synth.document_page(2550, 3300, synth.seed_for(2, seed), 0.08)
    gaps, k = check(page)
    assert gaps[0] > 0 and gaps[1] > 0 and k > 0


@pytest.mark.parametrize("pct", [50, 99])
def test_coverage_and_small_pages(pct):
    page, _ = synth.document_page(1700, 2200, synth.seed_for(4, 3), 0.12)
    check(page, pct)
    check(synth.random_bits((90, 130), 12, 0.2), pct)


def test_blank_and_full_pages():
    assert check(np.zeros((64, 100), np.uint8)) == ((0, 0), 0)
    assert check(np.ones((40, 70), np.uint8)) == ((0, 0), 1)
