"""Pins for the oracle's swap deltas (Sec. 4 operator) and Eq. (LSE)."""
import numpy as np
import pytest

import oracle
import synth
from tests.independent import lpf_full_by_products


def _canon(c, rx, ry):
    _, _, base = oracle.window_sizes(rx, ry)
    return c[:, base:]


def _pairs(img, k, seed, allow_same=True):
    rng = np.random.default_rng(seed)
    H, W = img.shape
    flat = img.reshape(-1)
    ones = np.flatnonzero(flat == 1)
    zeros = np.flatnonzero(flat == 0)
    out = [(int(rng.choice(ones)), int(rng.choice(zeros))) for _ in range(k)]
    if allow_same:
        out.append((int(ones[0]), int(ones[1])))
        out.append((int(zeros[0]), int(zeros[-1])))
        out.append((int(zeros[3]), int(ones[2])))  # reversed order is still an exchange
    return np.array(out, np.int32)


def test_delta_matches_independent_recount():
    img = synth.random_binary(9, 8, 0.5, 21)
    rx, ry = 5, 6
    pairs = _pairs(img, 6, 1)
    d = oracle.delta_swap(img, rx, ry, pairs)
    before = _canon(lpf_full_by_products(img, rx, ry), rx, ry)
    for k, (a, b) in enumerate(pairs):
        im2 = img.copy().reshape(-1)
        im2[a], im2[b] = im2[b], im2[a]
        after = _canon(lpf_full_by_products(im2.reshape(img.shape), rx, ry), rx, ry)
        np.testing.assert_array_equal(d[k], after - before)


def test_same_phase_pair_is_identity_and_inverse_cancels():
    img = synth.disks_64()[:32, :32].copy()
    rx = ry = 8
    pairs = _pairs(img, 5, 2)
    d = oracle.delta_swap(img, rx, ry, pairs)
    flat = img.reshape(-1)
    for k, (a, b) in enumerate(pairs):
        if flat[a] == flat[b]:
            assert not d[k].any()
            continue
        im2 = flat.copy()
        im2[a], im2[b] = im2[b], im2[a]
        back = oracle.delta_swap(im2.reshape(img.shape), rx, ry, [(b, a)])
        np.testing.assert_array_equal(back[0], -d[k])
        # phase 0 and phase 1 counts at v = 0 are unchanged by an exchange
        assert d[k][0, 0] == 0 and d[k][1, 0] == 0


def test_objective_zero_at_own_descriptor_and_delta_is_sum_of_squares():
    # Eq. (LSE) with the target equal to the image's own descriptor is 0; the
    # change after a swap is then the squared change of the descriptor.
    # W*H is a power of two, so the normalised descriptor is exact in float32.
    rx, ry = 5, 7
    img = synth.random_binary(16, 16, 0.4, 5)
    H, W = img.shape
    counts = lpf_full_by_products(img, rx, ry)
    target = (counts / float(H * W)).astype(np.float32)
    assert oracle.objective(target, counts, rx, ry, H, W) == 0.0
    pairs = _pairs(img, 4, 3)
    d = oracle.delta_swap(img, rx, ry, pairs)
    de = oracle.delta_objective(target, counts, d, rx, ry, H, W)
    for k in range(len(pairs)):
        expect = float(((d[k].astype(np.float64) / (H * W)) ** 2).sum())
        assert de[k] == pytest.approx(expect, rel=1e-12, abs=1e-18)


def test_objective_definition_on_hand_example():
    # Two vectors per phase in the canonical half of rx=1, ry=0: (0,0) and (1,0).
    rx, ry, H, W = 1, 0, 2, 2
    target = np.zeros((2, 3), np.float32)
    target[0] = [9.0, 0.5, 0.25]   # index 0 is the mirrored (-1,0): not part of D
    target[1] = [9.0, 0.75, 0.0]
    counts = np.zeros((2, 3), np.int64)
    counts[0] = [7, 2, 1]
    counts[1] = [7, 2, 2]
    e = (0.5 - 0.5) ** 2 + (0.25 - 0.25) ** 2 + (0.75 - 0.5) ** 2 + (0.0 - 0.5) ** 2
    assert oracle.objective(target, counts, rx, ry, H, W) == pytest.approx(e, rel=1e-15)
    d = np.zeros((1, 2, 2), np.int64)
    d[0, 1, 1] = -2
    de = oracle.delta_objective(target, counts, d, rx, ry, H, W)
    assert de[0] == pytest.approx(-(0.5 ** 2), rel=1e-15)
    # single-phase errors (the L2^b / L2^w compressions of Sec. 6, Tab. mutual):
    # phase 0 contributes nothing here, phase 1 everything; the change of -2
    # sits in phase 1
    assert oracle.objective(target, counts, rx, ry, H, W, phases=1) == 0.0
    assert oracle.objective(target, counts, rx, ry, H, W, phases=2) == pytest.approx(e, rel=1e-15)
    assert oracle.delta_objective(target, counts, d, rx, ry, H, W, phases=1)[0] == 0.0
    assert oracle.delta_objective(target, counts, d, rx, ry, H, W, phases=2)[0] == pytest.approx(-(0.5 ** 2), rel=1e-15)
