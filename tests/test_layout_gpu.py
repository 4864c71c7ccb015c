"""Layout analysis on the GPU (section "Document Analysis Performance")
against the oracle's pipeline (oracle.layout_boxes, pinned on its own):
white-run histograms along the lines and along the columns, the gap
estimates, the dilation by the estimated rectangle, the 8-connected
components and their records."""
import numpy as np
import pytest
import torch

import oracle
from paper_0712_0121_gb300 import synth

pytestmark = pytest.mark.gpu

M = pytest.importorskip("paper_0712_0121_gb300.morph")


def check(page, pct=90):
    boxes, n, gaps = M.layout_boxes(M.pack(page, 64), pct)
    assert M.sync_status() == M.MORPH_OK
    ref_gaps, ref = oracle.layout_boxes(page, pct)
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
