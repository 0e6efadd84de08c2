"""Failure detection on the GPU without a fault: a bounded device-side wait
is made to run out, and the kernel must report it through its status word;
an annealing run is left in a consistent state (the run then continues and
still equals the sequential oracle's)."""
import time

import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import sa as osa

pytestmark = pytest.mark.gpu


def test_grid_barrier_timeout_is_reported_and_harmless(gpu_lib):
    H = W = 24
    r = 6
    orig = synth.clustered_disks(2 * H, 2 * W, 0.3, seed=9)
    target = (oracle.lpf_full(orig, r, r) / float(orig.size)).astype(np.float32)
    cell = synth.exact_fraction_shuffle(H, W, int(round(0.3 * H * W)), seed=4)
    n_step, c_max, s_max, t_max = 400, 40, 4, 2e-4
    p = gpu_lib.lpf_build_paths(r, r)
    d_cell = torch.from_numpy(cell).cuda()
    counts = torch.empty((2, p.n_full), dtype=torch.int64, device="cuda")
    ann = gpu_lib.lpf_sa_create(d_cell, p, torch.from_numpy(target).cuda(), counts, n_step=n_step, c_max=c_max,
                                s_max=s_max, t_max=t_max, k_min=1, k_max=64, seed=3)
    gpu_lib.lpf_sa_run(ann, 5)
    st1 = gpu_lib.lpf_sa_read(ann)
    cell1, counts1 = d_cell.cpu().numpy(), counts.cpu().numpy()
    t0 = time.time()
    rc = gpu_lib.lpf_sa_selftest_timeout(ann, -1)
    assert rc == 0, gpu_lib.lpf_strerror(rc)
    assert time.time() - t0 < 60
    st2 = gpu_lib.lpf_sa_read(ann)  # status cleared: no LpfError
    # the same state; the error is recomputed from the exact counts
    assert {k: v for k, v in st2.items() if k != "error"} == {k: v for k, v in st1.items() if k != "error"}
    assert abs(st2["error"] - st1["error"]) <= 1e-5 * abs(st1["error"])
    np.testing.assert_array_equal(d_cell.cpu().numpy(), cell1)
    np.testing.assert_array_equal(counts.cpu().numpy(), counts1)
    while not gpu_lib.lpf_sa_read(ann)["done"]:
        gpu_lib.lpf_sa_run(ann, 16)
    ref_cell, ref_acc, _ = osa.anneal(cell, target, oracle.lpf_full(cell, r, r), r, r, n_step, c_max, s_max, t_max,
                                      0.01, seed=3)
    np.testing.assert_array_equal(d_cell.cpu().numpy(), ref_cell)
    assert gpu_lib.lpf_sa_read(ann)["n_accept"] == ref_acc


@pytest.mark.parametrize("block", [0, 1])
def test_partial_grid_barrier_timeout_leaves_a_consistent_run(gpu_lib, block):
    # Only one block's barrier wait runs out.  block 0 (which keeps the run
    # state and the cell) gives up: the other blocks applied the batch to
    # their vector chunks' counts.  Block 1 gives up: block 0 applied the
    # batch to the cell, block 1's chunk missed it.  Either way the library
    # recounts from the cell, and the run still equals the sequential oracle.
    H = W = 24
    r = 6
    orig = synth.clustered_disks(2 * H, 2 * W, 0.3, seed=9)
    target = (oracle.lpf_full(orig, r, r) / float(orig.size)).astype(np.float32)
    cell = synth.exact_fraction_shuffle(H, W, int(round(0.3 * H * W)), seed=4)
    n_step, c_max, s_max, t_max = 400, 40, 4, 2e-4
    p = gpu_lib.lpf_build_paths(r, r)
    d_cell = torch.from_numpy(cell).cuda()
    counts = torch.empty((2, p.n_full), dtype=torch.int64, device="cuda")
    ann = gpu_lib.lpf_sa_create(d_cell, p, torch.from_numpy(target).cuda(), counts, n_step=n_step, c_max=c_max,
                                s_max=s_max, t_max=t_max, k_min=1, k_max=64, seed=3)
    gpu_lib.lpf_sa_run(ann, 5)
    st1 = gpu_lib.lpf_sa_read(ann)
    rc = gpu_lib.lpf_sa_selftest_timeout(ann, block)
    assert rc == 0, gpu_lib.lpf_strerror(rc)
    st2 = gpu_lib.lpf_sa_read(ann)
    assert st2["n_batches"] == st1["n_batches"] + (0 if block == 0 else 1)
    # counts agree with the cell again, and the error with the counts
    cell2 = d_cell.cpu().numpy()
    np.testing.assert_array_equal(counts.cpu().numpy(), oracle.lpf_full(cell2, r, r))
    e_ref = oracle.objective(target, oracle.lpf_full(cell2, r, r), r, r, H, W)
    assert abs(st2["error"] - e_ref) <= 1e-9 * max(1.0, abs(e_ref))
    while not gpu_lib.lpf_sa_read(ann)["done"]:
        gpu_lib.lpf_sa_run(ann, 16)
    ref_cell, ref_acc, _ = osa.anneal(cell, target, oracle.lpf_full(cell, r, r), r, r, n_step, c_max, s_max, t_max,
                                      0.01, seed=3)
    np.testing.assert_array_equal(d_cell.cpu().numpy(), ref_cell)
    assert gpu_lib.lpf_sa_read(ann)["n_accept"] == ref_acc


def test_walk_staging_timeout_is_reported(gpu_lib):
    # The self-test makes every walk block's wait for its staging copy expect
    # bytes no copy delivers; the bounded waits run out and the status says so.
    img = synth.disks_64()
    p = gpu_lib.lpf_build_paths(16, 16)
    d = torch.from_numpy(img).cuda()
    ref = gpu_lib.lpf_full(d, p).clone()
    assert gpu_lib.lpf_paths_status(p) == 0
    gpu_lib.lpf_paths_set_selftest(p, True)
    t0 = time.time()
    gpu_lib.lpf_full(d, p)
    assert gpu_lib.lpf_paths_status(p) == gpu_lib.LPF_ETIMEOUT
    assert time.time() - t0 < 60
    gpu_lib.lpf_paths_set_selftest(p, False)
    assert gpu_lib.lpf_paths_status(p) == 0
    assert torch.equal(gpu_lib.lpf_full(d, p), ref)
    assert gpu_lib.lpf_paths_status(p) == 0
