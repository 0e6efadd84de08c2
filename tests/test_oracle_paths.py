"""Pins for the oracle's discretised segments (Sec. 2.2 and Sec. 3.1)."""
import json
import os
from fractions import Fraction

import pytest

import oracle
from tests.independent import segment_geometric

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _domain(W, H):
    """The half-domain D of Eq. (segments): [-W+1,-1]x[1,H-1] united with [0,W-1]x[0,H-1]."""
    for dx in range(-W + 1, 0):
        for dy in range(1, H):
            yield dx, dy
    for dx in range(0, W):
        for dy in range(0, H):
            yield dx, dy


@pytest.mark.parametrize("W,H", [(2, 2), (3, 3), (5, 5), (10, 10), (4, 7), (6, 9), (3, 11)])
def test_storage_count_matches_paper_formula(W, H):
    # Sec. 3.1: the number of stored pixel indices M, general (W <= H) and square forms.
    total = sum(len(oracle.segment(dx, dy)) for dx, dy in _domain(W, H))
    m_def = sum(max(i, j) for i in range(1, W + 1) for j in range(1, H + 1)) + \
        sum(max(i, j) for i in range(2, W + 1) for j in range(2, H + 1))
    m_general = Fraction(W * (3 * H * H + 3 * H + W * W - 1), 3) - Fraction(W * (W + 1), 2) \
        - Fraction(H * (H + 1), 2) + 1
    assert total == m_def == m_general
    if W == H:
        assert total == Fraction(4 * W ** 3 - 4 * W + 3, 3)


@pytest.mark.parametrize("W,H", [(2, 2), (5, 5), (4, 7), (16, 9)])
def test_domain_cardinality(W, H):
    # Sec. 2.2: |D| = 2HW - H - W + 1, and D is exactly the canonical half of
    # the window rx = W-1, ry = H-1 (dy > 0, or dy == 0 and dx >= 0).
    D = set(_domain(W, H))
    assert len(D) == 2 * H * W - H - W + 1
    canon = {(dx, dy) for dx in range(-W + 1, W) for dy in range(-H + 1, H)
             if dy > 0 or (dy == 0 and dx >= 0)}
    assert D == canon
    n_full, n_canon, base = oracle.window_sizes(W - 1, H - 1)
    assert n_canon == len(D) and n_full == 2 * n_canon - 1


def test_paper_operation_count_100():
    # Sec. 6.3 prints 6.716e9 comparisons for one standard evaluation at
    # 100x100: W*H translations times the pixels of the segments in [0,W-1]^2.
    W = H = 100
    ops = W * H * sum(len(oracle.segment(dx, dy)) for dx in range(W) for dy in range(H))
    g = GOLDEN["lpf_ops_standard_100x100"]
    assert abs(ops - g["value"]) <= 1e-3 * 1e9  # one unit of the last printed digit


def test_segments_match_geometric_rule():
    # Independent exact-rational statement of the nearest-pixel rule, all
    # vectors with |dx|,|dy| <= 12 (both halves).
    for dx in range(-12, 13):
        for dy in range(-12, 13):
            got = [tuple(p) for p in oracle.segment(dx, dy).tolist()]
            assert got == segment_geometric(dx, dy), (dx, dy)


def test_segment_properties():
    r = 20
    for dx in range(-r, r + 1):
        for dy in range(-r, r + 1):
            s = oracle.segment(dx, dy).tolist()
            a = max(abs(dx), abs(dy))
            assert len(s) == a + 1                      # both end pixels, one per major step
            pts = {tuple(p) for p in s}
            assert len(pts) == a + 1                    # no repeated pixel
            assert (0, 0) in pts and (dx, dy) in pts    # end pixels
            for (x0, y0), (x1, y1) in zip(s, s[1:]):    # 8-connected
                assert max(abs(x1 - x0), abs(y1 - y0)) == 1
            # every pixel within half a pixel of the ideal line along the minor axis
            for x, y in s:
                if a == 0:
                    continue
                if abs(dx) >= abs(dy):
                    assert abs(Fraction(y) - Fraction(x * dy, dx)) <= Fraction(1, 2)
                else:
                    assert abs(Fraction(x) - Fraction(y * dx, dy)) <= Fraction(1, 2)
            # point symmetry: the segment of v is the segment of -v seen from v
            m = {(x + dx, y + dy) for x, y in oracle.segment(-dx, -dy).tolist()}
            assert m == pts


def test_prefix_property_along_rays():
    # Multiples of a direction share their segments as prefixes: S(j u) is the
    # first part of S(k u) for j < k (a consequence of the rounding rule that
    # the enhanced evaluation of Sec. 3.2 relies on).
    for ux, uy in [(1, 0), (0, 1), (2, 1), (3, -1), (1, 3), (5, 2), (-4, 3)]:
        if not (uy > 0 or (uy == 0 and ux >= 0)):
            continue
        longest = oracle.segment(8 * ux, 8 * uy).tolist()
        for j in range(1, 8):
            s = oracle.segment(j * ux, j * uy).tolist()
            assert longest[: len(s)] == s


@pytest.mark.parametrize("r", [5, 12])
def test_segment_pixels_within_half_a_step_of_the_line(r):
    # Sec. 2.2's rounding keeps every pixel of S(v) within a/2 of the line
    # along v, a = max(|dx|, |dy|): |sy dx - sx dy| <= a/2.  So two pixels of
    # one segment differ by a vector within a of that line, inside the
    # segment's box -- the bound the annealer uses to rule out translations
    # whose segment holds both exchanged pixels.
    for dx in range(-r, r + 1):
        for dy in range(0, r + 1):
            if dy == 0 and dx < 0:
                continue
            a = max(abs(dx), dy)
            s = oracle.segment(dx, dy).astype(int)
            cross = s[:, 1] * dx - s[:, 0] * dy
            assert 2 * abs(cross).max() <= a
            d = s[:, None, :] - s[None, :, :]
            assert (abs(d[..., 0]) <= abs(dx)).all() and (abs(d[..., 1]) <= dy).all()
            assert (abs(d[..., 1] * dx - d[..., 0] * dy) <= a).all()
