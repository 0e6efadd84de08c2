"""Pins for the oracle's lineal-path counts (Sec. 2.2, Alg. 1 of Sec. 3.1)."""
import numpy as np
import pytest

import oracle
import synth
from tests.independent import axis_count_by_runs, lpf_full_by_products


@pytest.mark.parametrize("n,seed", [(4, 0), (4, 1), (4, 2), (8, 3), (8, 4), (5, 5), (7, 6)])
def test_brute_force_tiny_full_domain(n, seed):
    # Independent restatement (exact-rational segments, product of shifted
    # indicator images) on every vector of the paper's full domain.
    img = synth.random_binary(n, n, 0.55, seed)
    got = oracle.lpf_full(img, n - 1, n - 1)
    ref = lpf_full_by_products(img, n - 1, n - 1)
    np.testing.assert_array_equal(got, ref)


def test_brute_force_rectangular():
    img = synth.random_binary(6, 9, 0.6, 11)
    np.testing.assert_array_equal(oracle.lpf_full(img, 4, 3), lpf_full_by_products(img, 4, 3))


def test_zero_vector_is_volume_fraction():
    # Eq. (l2zero): L(0) = phi, i.e. count_p(0) = number of pixels of phase p,
    # and the two phases add up to W*H.
    img = synth.disks_64()
    n_full, _, base = oracle.window_sizes(6, 6)
    c = oracle.lpf_full(img, 6, 6)
    assert c[1, base] == int(img.sum())
    assert c[0, base] == img.size - int(img.sum())


@pytest.mark.parametrize("z", [1, 2, 3, 5, 8, 13, 21, 31])
def test_axis_aligned_by_run_lengths(z):
    # Axis-aligned segments: count from an independent run-length tally.
    img = synth.disks_64()
    got = oracle.count_list(img, [(z, 0), (0, z), (-z, 0), (0, -z)])
    for p in (0, 1):
        assert got[0, p] == axis_count_by_runs(img, z, p, axis=1)
        assert got[2, p] == axis_count_by_runs(img, z, p, axis=1)
        assert got[1, p] == axis_count_by_runs(img, z, p, axis=0)
        assert got[3, p] == axis_count_by_runs(img, z, p, axis=0)


@pytest.mark.parametrize("s", [2, 5, 10])
def test_chess_closed_form(s):
    # Chess pattern with s x s squares (Tab. comptime, microstructure A): a
    # horizontal segment of length z < s fits in a square in s - z of the 2s
    # positions of every period, so L_p((z,0)) = (s - z)/(2s); 0 for z >= s.
    W = H = 4 * s * 2
    img = synth.chess(H, W, s)
    for z in range(0, 2 * s + 1):
        c = oracle.count_list(img, [(z, 0), (0, z)])
        expect = max(0, s - z) * W * H // (2 * s)
        assert c[0, 0] == c[0, 1] == c[1, 0] == c[1, 1] == expect


@pytest.mark.parametrize("s", [3, 10])
def test_chess_diagonals_closed_form(s):
    # Along (k, k) the segment is the exact diagonal: from (x, y) both
    # coordinates cross a square edge at the same steps (the colour is kept)
    # exactly when x = y (mod s); along (-k, k) exactly when
    # x mod s + y mod s = s - 1.  Either way N/s starts, for every k >= s.
    n = 10 * s
    img = synth.chess(n, n, s)
    vecs = [(k, k) for k in (s, s + 1, 2 * s + 3, n - 1)] + [(-k, k) for k in (s, 2 * s - 1, n - 1)]
    c = oracle.count_list(img, vecs)
    np.testing.assert_array_equal(c.sum(axis=1), np.full(len(vecs), n * n // s))
    # Shorter diagonals (k < s): with a = x mod s, b = y mod s the colour is
    # kept when neither coordinate reaches an edge within k steps ((s - k)^2
    # residue pairs) or both reach it at the same step (a = b >= s - k: k
    # pairs), so the two phases together count N ((s - k)^2 + k) / s^2.
    for k in range(1, s):
        assert oracle.count_list(img, [(k, k)]).sum() == n * n * ((s - k) ** 2 + k) // (s * s), k


def test_point_symmetry_exact():
    # Eq. (symmetry): L(v) = L(-v); the oracle evaluates both halves directly.
    img = synth.disks_64()
    c = oracle.lpf_full(img, 20, 14)
    np.testing.assert_array_equal(c, c[:, ::-1])


def test_complement_swaps_phases():
    img = synth.random_binary(24, 20, 0.45, 3)
    a = oracle.lpf_full(img, 9, 7)
    b = oracle.lpf_full(1 - img, 9, 7)
    np.testing.assert_array_equal(a[0], b[1])
    np.testing.assert_array_equal(a[1], b[0])


def test_translation_invariance():
    img = synth.disks_64()
    a = oracle.lpf_full(img, 10, 10)
    b = oracle.lpf_full(np.roll(img, (7, -19), axis=(0, 1)), 10, 10)
    np.testing.assert_array_equal(a, b)


def test_monotone_along_nested_segments():
    # Sec. 3.2: a segment containing a shorter one can only have a smaller
    # count (the basis of the enhanced evaluation's zero test).
    img = synth.disks_64()
    for ux, uy in [(1, 0), (0, 1), (1, 1), (2, 1), (-3, 2), (1, 4)]:
        c = oracle.count_list(img, [(k * ux, k * uy) for k in range(0, 10)])
        assert (np.diff(c, axis=0) <= 0).all()


def test_counts_bounded_and_vanish():
    # Eq. (l2lim): the lineal path vanishes for long segments in a medium
    # without long-range order; on the 64x64 disks image both phases are far below phi at |v|=32.
    img = synth.disks_64()
    c = oracle.count_list(img, [(32, 0), (0, 32), (32, 32), (-32, 17)])
    assert (c[:, 1] < 0.05 * img.sum()).all()


def test_selected_translations_variant():
    # Monte-Carlo variant (Sec. 3): all translations selected gives the exact
    # counts; a single selected translation gives 0/1 per vector, checked by
    # the independent product formula at that translation; counts are
    # additive over disjoint selections.
    img = synth.random_binary(11, 9, 0.55, 8)
    rx, ry = 5, 4
    full = oracle.lpf_full(img, rx, ry)
    np.testing.assert_array_equal(oracle.lpf_full_selected(img, rx, ry, np.ones_like(img)), full)
    rng = np.random.default_rng(3)
    sel = (rng.random(img.shape) < 0.3).astype(np.uint8)
    a = oracle.lpf_full_selected(img, rx, ry, sel)
    b = oracle.lpf_full_selected(img, rx, ry, 1 - sel)
    np.testing.assert_array_equal(a + b, full)
    one = np.zeros_like(img)
    one[4, 7] = 1
    c = oracle.lpf_full_selected(img, rx, ry, one)
    assert set(np.unique(c)) <= {0, 1}
    from tests.independent import segment_geometric
    k = 0
    for dy in range(-ry, ry + 1):
        for dx in range(-rx, rx + 1):
            pts = segment_geometric(dx, dy)
            for p in (0, 1):
                inside = all(img[(4 + sy) % 11, (7 + sx) % 9] == p for sx, sy in pts)
                assert c[p, k] == int(inside)
            k += 1
