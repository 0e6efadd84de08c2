"""Sec. 5 (Fig. unicity): with Bresenham segments, the discretised lineal
path function of both phases does not determine a 2 x 8 periodic cell --
there are cells with equal volume fractions, identical L2 of both phases and
different S2.  Brute force over all 12,870 cells with eight phase-1 pixels,
full domain (rx = 7, ry = 1)."""
import itertools

import numpy as np

import oracle


def test_two_by_eight_cells_with_equal_lpf_and_different_s2():
    H, W = 2, 8
    groups = {}
    for ones in itertools.combinations(range(H * W), H * W // 2):
        c = np.zeros(H * W, np.uint8)
        c[list(ones)] = 1
        c = c.reshape(H, W)
        groups.setdefault(oracle.lpf_full(c, W - 1, H - 1).tobytes(), []).append(c)
    found = 0
    for cells in groups.values():
        s2 = {np.round(oracle.s2_direct(c, 1) * H * W).astype(np.int64).tobytes() for c in cells}
        if len(s2) > 1:
            found += 1
    assert found > 0
