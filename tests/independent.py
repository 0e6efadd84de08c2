"""Second, independent restatements used to pin the oracle.

Nothing here is shared with the oracle's C code or with the CUDA library:
segments come from the geometric statement (nearest pixel to the ideal line,
exact rationals), counts from a vectorised product over shifted images.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def segment_geometric(dx: int, dy: int):
    """Pixels of the segment (0,0)->(dx,dy) from the geometric statement.

    For v in the half-domain D (dy > 0, or dy == 0 and dx >= 0): walk the axis
    with the larger extent one pixel at a time; along the other axis take the
    pixel whose centre is nearest the ideal line (exact rational arithmetic);
    on an exact tie take the pixel farther from the start.  Outside D the
    segment is the one of -v seen from its other end.
    """
    if not (dy > 0 or (dy == 0 and dx >= 0)):
        return [(sx + dx, sy + dy) for sx, sy in segment_geometric(-dx, -dy)]
    ax, ay = abs(dx), abs(dy)
    a, b = max(ax, ay), min(ax, ay)
    gx = -1 if dx < 0 else 1
    gy = -1 if dy < 0 else 1
    pts = []
    for i in range(a + 1):
        if a == 0:
            m = 0
        else:
            ideal = Fraction(i * b, a)
            lo = ideal.numerator // ideal.denominator
            hi = lo if ideal.denominator == 1 else lo + 1
            dlo, dhi = ideal - lo, hi - ideal
            m = hi if dhi <= dlo else lo  # tie -> farther from the start
        pts.append((gx * i, gy * m) if ax >= ay else (gx * m, gy * i))
    return pts


def counts_by_products(img: np.ndarray, seg, phase: int) -> int:
    """#x with img[(x + s) mod] == phase for every s in seg, as a product of
    shifted indicator images."""
    chi = (img == phase).astype(np.int64)
    acc = np.ones_like(chi)
    for sx, sy in seg:
        acc *= np.roll(chi, shift=(-sy, -sx), axis=(0, 1))
    return int(acc.sum())


def lpf_full_by_products(img: np.ndarray, rx: int, ry: int) -> np.ndarray:
    n_full = (2 * rx + 1) * (2 * ry + 1)
    out = np.zeros((2, n_full), np.int64)
    k = 0
    for dy in range(-ry, ry + 1):
        for dx in range(-rx, rx + 1):
            seg = segment_geometric(dx, dy)
            for p in (0, 1):
                out[p, k] = counts_by_products(img, seg, p)
            k += 1
    return out


def axis_count_by_runs(img: np.ndarray, z: int, phase: int, axis: int) -> int:
    """count_phase((z,0)) (axis=1, along rows) or ((0,z)) (axis=0, columns)
    from periodic run lengths: a maximal run of length l in a line of
    length n gives max(0, l - z) starts; a line entirely in the phase gives n."""
    a = img if axis == 1 else img.T
    total = 0
    for line in a:
        n = len(line)
        inph = line == phase
        if inph.all():
            total += n
            continue
        if not inph.any():
            continue
        # rotate so that the line starts right after an out-of-phase pixel
        k = int(np.flatnonzero(~inph)[0])
        rot = np.roll(inph, -(k + 1))
        run = 0
        for v in rot:
            if v:
                run += 1
            else:
                total += max(0, run - z)
                run = 0
        total += max(0, run - z)
    return total
