"""Failure detection on the GPU without a fault: a bounded device-side wait
is made to run out, and the kernel must report it through its status word
and leave the annealing run as it was (the run then continues and still
equals the sequential oracle's)."""
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
    rc = gpu_lib.lpf_sa_selftest_timeout(ann)
    assert rc == 0, gpu_lib.lpf_strerror(rc)
    assert time.time() - t0 < 60
    st2 = gpu_lib.lpf_sa_read(ann)  # status cleared: no LpfError
    assert st2 == st1
    np.testing.assert_array_equal(d_cell.cpu().numpy(), cell1)
    np.testing.assert_array_equal(counts.cpu().numpy(), counts1)
    while not gpu_lib.lpf_sa_read(ann)["done"]:
        gpu_lib.lpf_sa_run(ann, 16)
    ref_cell, ref_acc, _ = osa.anneal(cell, target, oracle.lpf_full(cell, r, r), r, r, n_step, c_max, s_max, t_max,
                                      0.01, seed=3)
    np.testing.assert_array_equal(d_cell.cpu().numpy(), ref_cell)
    assert gpu_lib.lpf_sa_read(ann)["n_accept"] == ref_acc
