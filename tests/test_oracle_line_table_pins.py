"""Pins of the oracle's line-element table (section "Morphology with Lines
at Arbitrary Orientations"): exact tables worked out by hand at 0, 45, 90,
135, 170, -20, 60 and -75 degrees (tests/golden/line_tables.txt), and the
geometry of the element they give — one dilated pixel spreads along the
intended line."""
import math

import numpy as np
import pytest

import oracle
from conftest import read_golden


def golden():
    out = {}
    for k, v in read_golden("line_tables.txt").items():
        f = [p.strip() for p in v.split("|")]
        out[k] = (float(f[0]), int(f[1]), int(f[2]), int(f[3]), bool(int(f[4])), int(f[5]),
                  [int(s) for s in f[6].split()])
    return out


@pytest.mark.parametrize("key", sorted(golden()))
def test_tables_worked_out_by_hand(key):
    angle, r, W, H, horizontal, L, table = golden()[key]
    shift, length, origin, hz = oracle.line_table(angle, r, W, H)
    assert hz == horizontal
    assert length == L and origin == L // 2
    assert shift.tolist() == table


def test_table_length_follows_the_axis():
    assert oracle.line_table(30, 5, 17, 9)[0].shape == (17,)
    assert oracle.line_table(60, 5, 17, 9)[0].shape == (9,)


def test_angles_a_half_turn_apart_give_the_same_element():
    for a in (-80.0, -45.0, -10.0, 0.0, 33.0, 45.0, 71.5):
        s1, L1, o1, h1 = oracle.line_table(a, 9, 40, 30)
        s2, L2, o2, h2 = oracle.line_table(a + 180.0, 9, 40, 30)
        assert (L1, o1, h1) == (L2, o2, h2) and np.array_equal(s1, s2)


def test_mirrored_angles_mirror_the_table():
    # reflecting the angle about the x axis negates the skew (rounding
    # ties aside: no entry of these tables is a tie)
    for a in (10.0, 30.0, 60.0, 80.0):
        s1, L1, _, h1 = oracle.line_table(a, 9, 40, 30)
        s2, L2, _, h2 = oracle.line_table(-a, 9, 40, 30)
        assert L1 == L2 and h1 == h2
        assert np.array_equal(s1, -s2)


@pytest.mark.parametrize("angle", [0.0, 10.0, 30.0, 45.0, 60.0, 80.0, 90.0, 100.0, 135.0, -20.0, 170.0])
def test_dilated_pixel_follows_the_angle(angle):
    r, W, H = 10, 61, 61
    shift, L, o, horizontal = oracle.line_table(angle, r, W, H)
    img = np.zeros((H, W), np.uint8)
    img[30, 30] = 1
    ys, xs = np.nonzero(oracle.sheared_line("dilate", img, shift, L, o, horizontal))
    assert len(xs) == L
    a = math.radians(angle)
    dx, dy = math.cos(a), -math.sin(a)  # image rows grow downwards
    for x, y in zip(xs, ys):
        px, py = x - 30, y - 30
        assert abs(px * dy - py * dx) <= 1.0 + 1e-9
        assert abs(px * dx + py * dy) <= r + 1.0


def test_bad_arguments():
    for args in ((float("nan"), 3, 5, 5), (10.0, -1, 5, 5), (10.0, 3, 0, 5)):
        with pytest.raises(ValueError):
            oracle.line_table(*args)
