"""Ensemble of parallel cuts (Sec. 6.3: the descriptor of a volume averaged
over its cuts): the summed counts of the slices equal the oracle's counts of
each slice added up, exactly."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("D,H,W,r", [(12, 32, 32, 15), (5, 24, 40, 12)])
def test_ensemble_counts_are_the_sum_over_cuts(gpu_lib, D, H, W, r):
    vol = synth.boolean_spheres(D, H, W, 4.0, 12, seed=D)
    p = gpu_lib.lpf_build_paths(r, r)
    got = gpu_lib.lpf_full_ensemble(torch.from_numpy(vol).cuda(), p).cpu().numpy()
    ref = sum(oracle.lpf_full(vol[z], r, r) for z in range(D))
    np.testing.assert_array_equal(got, ref)
    # cuts in another direction of the same volume: same ensemble size, and
    # the zero vector counts every voxel once
    got_y = gpu_lib.lpf_full_ensemble(torch.from_numpy(np.ascontiguousarray(vol.transpose(1, 0, 2))).cuda(),
                                      gpu_lib.lpf_build_paths(r, min(r, D - 1))).cpu().numpy()
    _, _, base = oracle.window_sizes(r, min(r, D - 1))
    assert got_y[1, base] == int(vol.sum()) and got_y[0, base] == vol.size - int(vol.sum())
