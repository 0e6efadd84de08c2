"""Pins for the annealer oracle: Philox-4x32-10 known answers, interfacial
pixel lists, proposal draws, and the stage schedule of Alg. 3."""
import json
import math
import os

import numpy as np

import oracle
import synth
from oracle import sa

KAT = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "philox_kat.json")))


def test_philox_known_answers():
    for v in KAT["vectors"]:
        got = sa.philox4x32_10([int(x, 16) for x in v["ctr"]], [int(x, 16) for x in v["key"]])
        assert ["%08x" % g for g in got] == v["out"]


def test_interfacial_lists_by_brute_force():
    cell = synth.random_binary(9, 13, 0.4, 2)
    l1, l0 = sa.interfacial_lists(cell)
    H, W = cell.shape
    e1, e0 = [], []
    for y in range(H):
        for x in range(W):
            v = cell[y, x]
            nb = [cell[(y - 1) % H, x], cell[(y + 1) % H, x], cell[y, (x - 1) % W], cell[y, (x + 1) % W]]
            if any(n != v for n in nb):
                (e1 if v else e0).append(y * W + x)
    assert l1.tolist() == e1 and l0.tolist() == e0


def test_proposals_are_interfacial_and_uniform():
    cell = synth.clustered_disks(64, 64, 0.3, seed=5)
    pairs, u = sa.propose(cell, 0, 4000, seed=11)
    l1, l0 = sa.interfacial_lists(cell)
    flat = cell.reshape(-1)
    assert (flat[pairs[:, 0]] == 1).all() and (flat[pairs[:, 1]] == 0).all()
    assert np.isin(pairs[:, 0], l1).all() and np.isin(pairs[:, 1], l0).all()
    assert 0.0 < u.min() and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.02
    # counter-based: candidate n does not depend on how many were drawn before
    p2, u2 = sa.propose(cell, 1234, 3, seed=11)
    np.testing.assert_array_equal(p2, pairs[1234:1237])
    np.testing.assert_array_equal(u2, u[1234:1237])


def test_schedule_every_move_accepted_reaches_t_min():
    # Tab. annealing: with T_mult = (T_min/T_max)^(s_max/N_step), a run in
    # which every attempt is accepted ends each stage after s_max acceptances,
    # so after N_step evaluations T = T_min.
    cell = synth.random_binary(8, 8, 0.5, 1)
    rx = ry = 2
    counts = oracle.lpf_full(cell, rx, ry)
    target = (counts / 64.0).astype(np.float32)
    out, n_acc, T = sa.anneal(cell, target, counts, rx, ry, n_step=40, c_max=1000, s_max=4, t_max=1e30,
                              t_min_ratio=0.01, seed=3)
    assert n_acc == 40
    assert math.isclose(T, 1e28, rel_tol=1e-12)


def test_schedule_no_move_accepted_stages_by_attempts():
    # Target = the cell's own descriptor: e = 0 and every exchange raises it;
    # with T negligible nothing is accepted and each stage ends after c_max
    # attempts, so T = T_max * T_mult^(N_step / c_max).
    cell = synth.random_binary(8, 8, 0.5, 1)
    rx = ry = 2
    counts = oracle.lpf_full(cell, rx, ry)
    target = (counts / 64.0).astype(np.float32)
    t_max = 1e-200
    out, n_acc, T = sa.anneal(cell, target, counts, rx, ry, n_step=40, c_max=8, s_max=4, t_max=t_max,
                              t_min_ratio=0.01, seed=3)
    assert n_acc == 0 and (out == cell).all()
    assert math.isclose(T, t_max * (0.01 ** (4 / 40)) ** 5, rel_tol=1e-12)


def test_anneal_reduces_error():
    orig = synth.clustered_disks(48, 48, 0.3, seed=9)
    rx = ry = 6
    target = (oracle.lpf_full(orig, rx, ry) / float(orig.size)).astype(np.float32)
    cell = synth.exact_fraction_shuffle(24, 24, int(round(0.3 * 576)), seed=4)
    counts = oracle.lpf_full(cell, rx, ry)
    e0 = oracle.objective(target, counts, rx, ry, 24, 24)
    out, n_acc, T = sa.anneal(cell, target, counts, rx, ry, n_step=600, c_max=60, s_max=6, t_max=1e-6,
                              t_min_ratio=0.01, seed=2)
    e1 = oracle.objective(target, oracle.lpf_full(out, rx, ry), rx, ry, 24, 24)
    assert n_acc > 0 and e1 < e0
    assert out.sum() == cell.sum()  # exchanges keep the volume fraction


def test_monte_carlo_annealing_with_every_translation_is_the_exact_one():
    # Sec. 3 opening: with N = W*H sampled positions the Monte-Carlo descriptor
    # is the exact one, so the annealing runs coincide step for step.
    H = W = 10
    rx = ry = 3
    cell = synth.exact_fraction_shuffle(H, W, 35, seed=2)
    orig = synth.clustered_disks(20, 20, 0.35, seed=3)
    target = (oracle.lpf_full(orig, rx, ry) / float(orig.size)).astype(np.float32)
    counts = oracle.lpf_full(cell, rx, ry)
    kw = dict(n_step=120, c_max=20, s_max=4, t_max=1e-3, t_min_ratio=0.01, seed=5)
    a = sa.anneal(cell, target, counts, rx, ry, **kw)
    b = sa.anneal(cell, target, counts, rx, ry, sel=np.ones((H, W), np.uint8), **kw)
    np.testing.assert_array_equal(a[0], b[0])
    assert a[1] == b[1] and a[1] > 0
