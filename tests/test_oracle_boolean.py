"""Boolean-disk pin for the oracle's counts.

For N disk centres placed independently and uniformly on the torus, the
pixels of a segment are all uncovered exactly when no centre falls in the
union U of the radius-R disks around their centres, so the expected void
lineal path is (1 - |U| / (W H))^N.  For axis-aligned and diagonal
segments |U| is close to the stadium area pi R^2 + 2 R |v|, which gives the
closed form L(v) = exp(-lambda (pi R^2 + 2 R |v|)) with lambda = N / (W H).
"""
import math

import numpy as np
import pytest

import oracle
import synth

R = 5.0
SIZE = 2048
SEEDS = list(range(100, 116))
VECS = [(0, 0), (1, 0), (2, 0), (4, 0), (8, 0), (16, 0), (0, 4), (0, 16),
        (2, 2), (5, 5), (11, 11), (-6, 6)]


def _union_area(seg, R, h=1.0 / 32):
    pts = np.asarray(seg, dtype=np.float64)
    lo = pts.min(axis=0) - R - h
    hi = pts.max(axis=0) + R + h
    xs = np.arange(lo[0], hi[0], h) + h / 2
    ys = np.arange(lo[1], hi[1], h) + h / 2
    X, Y = np.meshgrid(xs, ys)
    cov = np.zeros(X.shape, bool)
    for px, py in pts:
        cov |= (X - px) ** 2 + (Y - py) ** 2 <= R * R
    return cov.sum() * h * h


@pytest.fixture(scope="module")
def sample():
    n = synth.disks_for_fraction(SIZE, SIZE, R, 0.4)
    per_seed = []
    for s in SEEDS:
        img = synth.boolean_disks(SIZE, SIZE, R, n, seed=s)
        c = oracle.count_list(img, VECS)
        per_seed.append(c[:, 0] / float(SIZE * SIZE))
    return n, np.array(per_seed)


def test_void_lineal_path_exact_expectation(sample):
    n, L = sample
    mean = L.mean(axis=0)
    sem = L.std(axis=0, ddof=1) / math.sqrt(len(SEEDS))
    for k, (dx, dy) in enumerate(VECS):
        seg = oracle.segment(dx, dy).tolist()
        expect = (1.0 - _union_area(seg, R) / (SIZE * SIZE)) ** n
        assert abs(mean[k] - expect) <= 4.0 * sem[k] + 2e-4, ((dx, dy), mean[k], expect)


def test_void_lineal_path_closed_form(sample):
    n, L = sample
    lam = n / float(SIZE * SIZE)
    mean = L.mean(axis=0)
    for k, (dx, dy) in enumerate(VECS):
        if not (dx == 0 or dy == 0 or abs(dx) == abs(dy)):
            continue
        length = math.hypot(dx, dy)
        closed = math.exp(-lam * (math.pi * R * R + 2 * R * length))
        assert abs(mean[k] - closed) <= 2e-3, ((dx, dy), mean[k], closed)
