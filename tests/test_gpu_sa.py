"""GPU annealer (Sec. 4, Alg. 3): proposals, trajectories and bookkeeping
against the oracle."""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import sa as osa

pytestmark = pytest.mark.gpu


def _setup(H, W, r, frac=0.3, seed=4, orig_seed=9):
    orig = synth.clustered_disks(2 * H, 2 * W, frac, seed=orig_seed)
    target = (oracle.lpf_full(orig, r, r) / float(orig.size)).astype(np.float32)
    cell = synth.exact_fraction_shuffle(H, W, int(round(frac * H * W)), seed=seed)
    return cell, target


def _run_to_end(lpf, ann, chunk=64):
    while True:
        lpf.lpf_sa_run(ann, chunk)
        st = lpf.lpf_sa_read(ann)
        if st["done"]:
            return st


def test_proposals_match_oracle(gpu_lib):
    cell, target = _setup(64, 64, 10)
    p = gpu_lib.lpf_build_paths(10, 10)
    d_cell = torch.from_numpy(cell).cuda()
    ann = gpu_lib.lpf_sa_create(d_cell, p, torch.from_numpy(target).cuda(), n_step=10000, t_max=1e-5,
                                k_max=512, seed=0x1234567890ABCDEF)
    pairs, u = gpu_lib.lpf_sa_propose(ann, 512)
    ref_pairs, ref_u = osa.propose(cell, 0, 512, seed=0x1234567890ABCDEF)
    np.testing.assert_array_equal(pairs.cpu().numpy(), ref_pairs)
    np.testing.assert_array_equal(u.cpu().numpy(), ref_u)
    # after some batches the draws continue from the run's evaluation counter
    gpu_lib.lpf_sa_run(ann, 5)
    st = gpu_lib.lpf_sa_read(ann)
    pairs, u = gpu_lib.lpf_sa_propose(ann, 64)
    ref_pairs, ref_u = osa.propose(d_cell.cpu().numpy(), st["n_eval"], 64, seed=0x1234567890ABCDEF)
    np.testing.assert_array_equal(pairs.cpu().numpy(), ref_pairs)
    np.testing.assert_array_equal(u.cpu().numpy(), ref_u)


@pytest.mark.parametrize("kmin,kmax,H,W", [(1, 1, 24, 24), (8, 64, 24, 24), (32, 4096, 24, 24), (1, 1, 20, 28),
                                            (8, 64, 28, 20)])
def test_trajectory_equals_sequential_oracle(gpu_lib, kmin, kmax, H, W):
    # (non-square cells take the other branch of the counts' sheared layout)
    r = 6
    cell, target = _setup(H, W, r)
    n_step, c_max, s_max = 600, 60, 6
    # a temperature where some uphill moves pass: median uphill change of the start
    counts0 = oracle.lpf_full(cell, r, r)
    pairs, _ = osa.propose(cell, 0, 200, seed=7)
    de = oracle.delta_objective(target, counts0, oracle.delta_swap(cell, r, r, pairs), r, r, H, W)
    t_max = float(np.median(de[de > 0]))
    p = gpu_lib.lpf_build_paths(r, r)
    d_cell = torch.from_numpy(cell).cuda()
    counts = torch.empty((2, p.n_full), dtype=torch.int64, device="cuda")
    ann = gpu_lib.lpf_sa_create(d_cell, p, torch.from_numpy(target).cuda(), counts, n_step=n_step, c_max=c_max,
                                s_max=s_max, t_max=t_max, k_min=kmin, k_max=kmax, seed=7)
    st = _run_to_end(gpu_lib, ann)
    assert st["n_eval"] == n_step
    ref_cell, ref_acc, ref_T = osa.anneal(cell, target, counts0, r, r, n_step, c_max, s_max, t_max, 0.01, seed=7)
    got = d_cell.cpu().numpy()
    assert st["n_accept"] == ref_acc
    np.testing.assert_array_equal(got, ref_cell)
    assert st["temperature"] == pytest.approx(ref_T, rel=1e-9)
    # bookkeeping: the incrementally updated counts are the exact counts of the final cell
    np.testing.assert_array_equal(counts.cpu().numpy(), oracle.lpf_full(got, r, r))
    e_inc = st["error"]
    e_new = gpu_lib.lpf_sa_recompute_error(ann)
    assert e_new == pytest.approx(oracle.objective(target, oracle.lpf_full(got, r, r), r, r, H, W), rel=1e-12)
    assert abs(e_inc - e_new) <= 1e-5 * abs(e_new) + 1e-12


def test_annealing_128_cell_reduces_error_and_is_deterministic(gpu_lib):
    # The compression workload at reduced length: 128x128 cell, |v| <= 64,
    # target from a 512x512 clustered-disk original.
    orig = synth.clustered_512()
    r = 64
    p = gpu_lib.lpf_build_paths(r, r)
    d_orig = torch.from_numpy(orig).cuda()
    c_orig = gpu_lib.lpf_full(d_orig, p)
    target = (c_orig.double() / float(orig.size)).float()
    cell0 = synth.exact_fraction_shuffle(128, 128, int(round(orig.mean() * 128 * 128)), seed=5)
    finals = []
    for _ in range(2):
        d_cell = torch.from_numpy(cell0).cuda()
        counts = torch.empty((2, p.n_full), dtype=torch.int64, device="cuda")
        ann = gpu_lib.lpf_sa_create(d_cell, p, target, counts, n_step=20000, seed=99)
        e0 = gpu_lib.lpf_sa_read(ann)["error"]
        st = _run_to_end(gpu_lib, ann, chunk=256)
        assert st["error"] < 0.5 * e0
        assert gpu_lib.lpf_paths_status(p) == 0
        # thousands of accepted exchanges later, the counts the run kept
        # current (from its per-translation phase-0 counts) are the exact
        # counts of its cell; its error, a running sum of float32 changes,
        # stays within a small relative drift of the recomputed one
        assert st["n_accept"] > 5000
        assert torch.equal(counts, gpu_lib.lpf_full(d_cell, p))
        e_new = gpu_lib.lpf_sa_recompute_error(ann)
        assert abs(st["error"] - e_new) <= 1e-3 * abs(e_new)
        finals.append(d_cell.cpu().numpy())
    np.testing.assert_array_equal(finals[0], finals[1])
    assert finals[0].sum() == cell0.sum()


def test_wide_window_annealer_keeps_exact_counts(gpu_lib):
    # A 128x128 cell against a window of 100: the vector chunks hold more
    # segment pixels than the block keeps in registers, so every accepted
    # exchange updates the phase-0 counts by reading them again; after the
    # run the counts it kept are the exact counts of its cell.
    r = 100
    orig = synth.clustered_disks(256, 256, 0.3, seed=12)
    p = gpu_lib.lpf_build_paths(r, r)
    c_orig = gpu_lib.lpf_full(torch.from_numpy(orig).cuda(), p)
    target = (c_orig.double() / float(orig.size)).float()
    cell0 = synth.exact_fraction_shuffle(128, 128, int(round(orig.mean() * 128 * 128)), seed=3)
    d_cell = torch.from_numpy(cell0).cuda()
    counts = torch.empty((2, p.n_full), dtype=torch.int64, device="cuda")
    ann = gpu_lib.lpf_sa_create(d_cell, p, target, counts, n_step=3000, seed=5)
    st = _run_to_end(gpu_lib, ann, chunk=256)
    assert st["n_eval"] == 3000 and st["n_accept"] > 500
    assert gpu_lib.lpf_paths_status(p) == 0
    assert torch.equal(counts, gpu_lib.lpf_full(d_cell, p))
    assert d_cell.sum().item() == cell0.sum()


def test_run_continues_after_the_handle_serves_another_width(gpu_lib):
    # The swap-delta tables of a paths handle belong to one cell width; a
    # swap-delta call on another width re-bakes them.  An annealing run on the
    # handle takes its own width's tables again before its next launch and
    # carries on with exact counts.
    r = 20
    p = gpu_lib.lpf_build_paths(r, r)
    orig = synth.clustered_disks(128, 128, 0.3, seed=21)
    target = (gpu_lib.lpf_full(torch.from_numpy(orig).cuda(), p).double() / float(orig.size)).float()
    cell0 = synth.exact_fraction_shuffle(64, 64, int(round(orig.mean() * 64 * 64)), seed=4)
    d_cell = torch.from_numpy(cell0).cuda()
    counts = torch.empty((2, p.n_full), dtype=torch.int64, device="cuda")
    ann = gpu_lib.lpf_sa_create(d_cell, p, target, counts, n_step=4000, seed=8)
    gpu_lib.lpf_sa_run(ann, 64)
    other = synth.clustered_disks(48, 48, 0.3, seed=22)
    d_other = torch.from_numpy(other).cuda()
    pairs = torch.from_numpy(synth.swap_candidates(other, 8, seed=1)).cuda()
    dc, _ = gpu_lib.lpf_delta_swap(d_other, p, pairs)
    np.testing.assert_array_equal(dc.cpu().numpy(), oracle.delta_swap(other, r, r, pairs.cpu().numpy()))
    st = _run_to_end(gpu_lib, ann, chunk=128)
    assert st["n_eval"] == 4000
    assert gpu_lib.lpf_paths_status(p) == 0
    assert torch.equal(counts, gpu_lib.lpf_full(d_cell, p))
