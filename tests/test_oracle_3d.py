"""Pins of the oracle's 3D extension (Sec. 2 remark on 3D media, Sec. 6.3
volumes): the segment rule restated with exact rationals, brute force by
products of shifted indicator volumes, the 2D case embedded, point symmetry,
L(0) = volume fraction, and axis-aligned counts from an independent
run-length tally."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth


def _canonical3(dx, dy, dz):
    return dz > 0 or (dz == 0 and (dy > 0 or (dy == 0 and dx >= 0)))


def _nearest_away(num: Fraction) -> int:
    """Nearest integer to num >= 0, an exact half rounded up (away from 0)."""
    f = num.numerator // num.denominator
    return f + 1 if num - f >= Fraction(1, 2) else f


def _segment3_rational(dx, dy, dz):
    """The 3D segment restated: step i moves round(i d_j / a) along each
    axis, exact halves away from the start; outside the half-domain the
    segment of -v seen from the other end."""
    if not _canonical3(dx, dy, dz):
        return [(x + dx, y + dy, z + dz) for x, y, z in _segment3_rational(-dx, -dy, -dz)]
    d = (dx, dy, dz)
    a = max(abs(c) for c in d)
    if a == 0:
        return [(0, 0, 0)]
    pts = []
    for i in range(a + 1):
        pts.append(tuple((1 if c >= 0 else -1) * _nearest_away(Fraction(i * abs(c), a)) for c in d))
    return pts


def test_segments_match_the_rational_statement_and_are_26_connected():
    r = 5
    for dz in range(-r, r + 1):
        for dy in range(-r, r + 1):
            for dx in range(-r, r + 1):
                s = oracle.segment3(dx, dy, dz)
                assert len(s) == max(abs(dx), abs(dy), abs(dz)) + 1
                assert [tuple(p) for p in s] == _segment3_rational(dx, dy, dz)
                pts = {tuple(p) for p in s}
                assert (0, 0, 0) in pts and (dx, dy, dz) in pts
                if len(s) > 1:
                    steps = np.abs(np.diff(s, axis=0))
                    assert steps.max() == 1 and (steps.max(axis=1) == 1).all()


def test_the_2d_segment_is_embedded():
    for dy in range(-7, 8):
        for dx in range(-7, 8):
            s3 = oracle.segment3(dx, dy, 0)
            s2 = oracle.segment(dx, dy)
            np.testing.assert_array_equal(s3[:, :2], s2)
            assert not s3[:, 2].any()


def _brute_counts(vol, rx, ry, rz):
    """Counts by products of shifted indicator volumes (np.roll), segments
    from the rational statement."""
    n_full, _, _ = oracle.window_sizes3(rx, ry, rz)
    out = np.zeros((2, n_full), np.int64)
    for dz in range(-rz, rz + 1):
        for dy in range(-ry, ry + 1):
            for dx in range(-rx, rx + 1):
                k = oracle.full_index3(dx, dy, dz, rx, ry, rz)
                for p in (0, 1):
                    m = np.ones(vol.shape, bool)
                    for sx, sy, sz in _segment3_rational(dx, dy, dz):
                        m &= np.roll(vol == p, shift=(-sz, -sy, -sx), axis=(0, 1, 2))
                    out[p, k] = int(m.sum())
    return out


@pytest.mark.parametrize("shape,window,seed", [((4, 4, 4), (3, 3, 3), 1), ((5, 6, 7), (3, 2, 4), 2),
                                                ((3, 8, 5), (4, 3, 2), 3)])
def test_counts_equal_brute_force(shape, window, seed):
    vol = (np.random.default_rng(seed).random(shape) < 0.55).astype(np.uint8)
    rx, ry, rz = window
    np.testing.assert_array_equal(oracle.lpf_full3(vol, rx, ry, rz), _brute_counts(vol, rx, ry, rz))


def test_symmetry_volume_fraction_and_planar_vectors():
    vol = synth.boolean_spheres(12, 14, 16, 2.5, 18, seed=4)
    rx, ry, rz = 6, 5, 4
    c = oracle.lpf_full3(vol, rx, ry, rz)
    n_full, _, base = oracle.window_sizes3(rx, ry, rz)
    np.testing.assert_array_equal(c, c[:, ::-1])                      # L(v) = L(-v)
    assert c[1, base] == int(vol.sum()) and c[0, base] == vol.size - int(vol.sum())
    # a volume constant along z: vectors with dz = 0 count D times the 2D counts
    img = synth.random_binary(14, 16, 0.45, 5)
    flat = np.repeat(img[None], 7, axis=0)
    c3 = oracle.lpf_full3(flat, 5, 4, 3)
    c2 = oracle.lpf_full(img, 5, 4)
    for dy in range(-4, 5):
        for dx in range(-5, 6):
            k3 = oracle.full_index3(dx, dy, 0, 5, 4, 3)
            k2 = oracle.full_index(dx, dy, 5, 4)
            assert c3[0, k3] == 7 * c2[0, k2] and c3[1, k3] == 7 * c2[1, k2]


def test_axis_aligned_counts_from_run_lengths():
    vol = (np.random.default_rng(8).random((11, 5, 6)) < 0.6).astype(np.uint8)
    D = vol.shape[0]
    for p in (0, 1):
        for z in range(0, D):
            expect = 0
            for y in range(vol.shape[1]):
                for x in range(vol.shape[2]):
                    col = vol[:, y, x] == p
                    if col.all():
                        expect += D
                        continue
                    start = int(np.argmin(col))  # a voxel outside the phase: runs do not wrap past it
                    run = 0
                    for k in range(1, D + 1):
                        if col[(start + k) % D]:
                            run += 1
                        else:
                            expect += max(0, run - z)
                            run = 0
            assert oracle.count3(vol, 0, 0, z, p) == expect
