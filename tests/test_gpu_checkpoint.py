"""Checkpoint / resume of an annealing run: a run saved part-way and resumed
in a new annealer ends exactly where the uninterrupted run ends."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


def test_resumed_run_equals_uninterrupted(gpu_lib, tmp_path):
    H = W = 24
    r = 6
    orig = synth.clustered_disks(2 * H, 2 * W, 0.3, seed=9)
    target = torch.from_numpy((oracle.lpf_full(orig, r, r) / float(orig.size)).astype(np.float32)).cuda()
    cell0 = synth.exact_fraction_shuffle(H, W, int(round(0.3 * H * W)), seed=4)
    p = gpu_lib.lpf_build_paths(r, r)
    kw = dict(n_step=800, c_max=80, s_max=8, t_max=2e-4, t_min_ratio=0.02, k_min=1, k_max=64, seed=21)
    d = torch.from_numpy(cell0).cuda()
    ann = gpu_lib.lpf_sa_create(d, p, target, **kw)
    gpu_lib.lpf_sa_run(ann, 30)
    path = str(tmp_path / "run.npz")
    gpu_lib.save_checkpoint(ann, path)
    mid = gpu_lib.lpf_sa_read(ann)
    assert 0 < mid["n_eval"] < kw["n_step"]
    while not gpu_lib.lpf_sa_read(ann)["done"]:
        gpu_lib.lpf_sa_run(ann, 16)
    end_a = gpu_lib.lpf_sa_read(ann)
    cell_a = d.cpu().numpy()

    res = gpu_lib.load_checkpoint(path, p, target, k_max=64, k_min=1)
    st = gpu_lib.lpf_sa_read(res)
    assert st["n_eval"] == mid["n_eval"] and st["temperature"] == mid["temperature"]
    while not gpu_lib.lpf_sa_read(res)["done"]:
        gpu_lib.lpf_sa_run(res, 16)
    end_b = gpu_lib.lpf_sa_read(res)
    np.testing.assert_array_equal(res.cell.cpu().numpy(), cell_a)
    for k in ("n_eval", "n_accept", "temperature", "next_batch"):
        assert end_a[k] == end_b[k], k
    np.testing.assert_array_equal(res.counts.cpu().numpy(), ann.counts.cpu().numpy())


def test_import_checks_parameters(gpu_lib):
    H = W = 16
    p = gpu_lib.lpf_build_paths(4, 4)
    target = torch.zeros((2, p.n_full), dtype=torch.float32, device="cuda")
    cell = torch.from_numpy(synth.exact_fraction_shuffle(H, W, 80, seed=1)).cuda()
    ann = gpu_lib.lpf_sa_create(cell, p, target, n_step=100, t_max=1e-3, seed=3)
    pr = gpu_lib.lpf_sa_export_progress(ann)
    pr["seed"] = 4
    with pytest.raises(gpu_lib.LpfError):
        gpu_lib.lpf_sa_import_progress(ann, pr)
