"""Pins of the layout-analysis oracle (section "Document Analysis
Performance"): the gap rule on histograms worked out by hand (one length
only, the exact percentage threshold, pct = 100, no runs, runs longer than
1/16 of the line left out), and the whole pipeline on a page whose gaps,
blocks and block records are worked out by hand (tests/golden/layout_page.txt)."""
import numpy as np
import pytest

import oracle
from conftest import read_golden


def hist(n, **counts):
    h = np.zeros(n, np.int64)
    for k, v in counts.items():
        h[int(k[1:])] = v
    return h


def test_gap_of_one_length_is_that_length():
    for pct in (1, 50, 90, 100):
        assert oracle.layout_gap(hist(20, L3=7), 16, pct) == 3


def test_gap_threshold_is_inclusive():
    h = hist(5, L1=9, L2=1)
    assert oracle.layout_gap(h, 4, 90) == 1   # 9 of 10 runs = 90 %
    assert oracle.layout_gap(h, 4, 91) == 2
    assert oracle.layout_gap(h, 4, 100) == 2


def test_gap_at_full_coverage_is_the_longest_counted_run():
    assert oracle.layout_gap(hist(8, L1=1, L5=1), 6, 100) == 5
    assert oracle.layout_gap(hist(8, L1=1, L5=1), 6, 50) == 1


def test_gap_without_counted_runs_is_zero():
    assert oracle.layout_gap(np.zeros(10, np.int64), 9, 90) == 0
    # a histogram of length-0 entries only (never produced, but not a run)
    assert oracle.layout_gap(hist(10, L0=5), 9, 90) == 0


def test_runs_longer_than_the_cap_are_left_out():
    h = hist(20, L1=1, L10=100)
    assert oracle.layout_gap(h, 8, 90) == 1
    assert oracle.layout_gap(h, 10, 90) == 10
    # lengths beyond the histogram's end count as zero
    assert oracle.layout_gap(hist(3, L2=4), 8, 90) == 2


def golden_page():
    g = read_golden("layout_page.txt")
    W, H = (int(v) for v in g["size"].split())
    gw, gh = (int(v) for v in g["glyph"].split())
    page = np.zeros((H, W), np.uint8)
    for key in ("block_a", "block_b"):
        xs, ys = g[key].split("|")
        for y in ys.split():
            for x in xs.split():
                page[int(y):int(y) + gh, int(x):int(x) + gw] = 1
    return g, page


def box_record(x0, y0, x1, y1):
    xs, ys = np.arange(x0, x1), np.arange(y0, y1)
    w, h = x1 - x0, y1 - y0
    return [x0, y0, x1, y1, w * h, h * int(xs.sum()), w * int(ys.sum())]


def test_pipeline_on_a_page_worked_out_by_hand():
    g, page = golden_page()
    gaps, rec = oracle.layout_boxes(page, 90)
    assert gaps == tuple(int(v) for v in g["gaps"].split())
    want = [box_record(*(int(v) for v in g[k].split())) for k in ("box_a", "box_b")]
    assert rec.tolist() == want


@pytest.mark.parametrize("pct", [1, 100])
def test_pipeline_gaps_do_not_depend_on_pct_when_one_length_is_counted(pct):
    g, page = golden_page()
    gaps, rec = oracle.layout_boxes(page, pct)
    assert gaps == (2, 4) and rec.shape == (2, 7)


def test_pipeline_on_blank_and_full_pages():
    gaps, rec = oracle.layout_boxes(np.zeros((32, 48), np.uint8))
    assert gaps == (0, 0) and rec.shape == (0, 7)
    gaps, rec = oracle.layout_boxes(np.ones((32, 48), np.uint8))
    assert gaps == (0, 0) and rec.tolist() == [box_record(0, 0, 48, 32)]
