"""Host logic of the line-element entry point (no GPU): the skew table,
length and orientation that ``morph_line_element`` (through
``morph.line_element``) derives from an angle, checked geometrically by
dilating one pixel with the oracle — the pixels reached lie along the
intended line (angle counterclockwise from the x axis, image rows growing
downwards) within the rounding of the skew — and equal to the oracle's
table, whose own pins are exact tables worked out by hand."""
import math

import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module")
def M():
    from paper_0712_0121_gb300 import build
    build.build_morph()
    from paper_0712_0121_gb300 import morph
    return morph


@pytest.mark.parametrize("angle", [0.0, 10.0, 30.0, 45.0, 60.0, 80.0, 90.0, 100.0, 135.0, -20.0, 170.0])
def test_dilated_pixel_follows_the_angle(M, angle):
    r = 10
    W = H = 61
    shift, L, o, horizontal = M.line_element(angle, r, W, H)
    assert L == 2 * o + 1
    img = np.zeros((H, W), np.uint8)
    img[30, 30] = 1
    out = oracle.sheared_line("dilate", img, shift, L, o, horizontal)
    ys, xs = np.nonzero(out)
    assert len(xs) == L, "a line of L pixels"
    a = math.radians(angle)
    # unit direction of the line in image coordinates (y down)
    dx, dy = math.cos(a), -math.sin(a)
    for x, y in zip(xs, ys):
        px, py = x - 30, y - 30
        dist = abs(px * dy - py * dx)       # distance from the ideal line
        assert dist <= 1.0 + 1e-9, (angle, x, y, dist)
        assert abs(px * dx + py * dy) <= r + 1.0  # within the half length (+ rounding)


def test_axis_choice_and_lengths(M):
    s, L, o, h = M.line_element(90.0, 12, 50, 40)
    assert not h and L == 25 and not s.any() and s.shape == (40,)
    s, L, o, h = M.line_element(0.0, 12, 50, 40)
    assert h and L == 25 and not s.any() and s.shape == (50,)
    s, L, o, h = M.line_element(45.0, 12, 50, 40)
    assert h and L == 2 * round(12 * math.cos(math.radians(45))) + 1
    assert s.tolist() == list(range(50))


@pytest.mark.parametrize("angle", [-89.0, -60.0, -45.0, -30.0, 0.5, 22.5, 45.0, 67.5, 91.0, 225.0])
def test_equals_the_oracle_table(M, angle):
    for r, W, H in [(5, 33, 21), (40, 400, 129)]:
        s, L, o, h = M.line_element(angle, r, W, H)
        ts, tL, to, th = oracle.line_table(angle, r, W, H)
        assert np.array_equal(s, ts) and (L, o, h) == (tL, to, th)
