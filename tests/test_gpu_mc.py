"""GPU Monte-Carlo variant (Sec. 3): counts over selected translations
against the oracle, on the canonical half D that the paper evaluates."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("H,W,rx,ry,frac,seed", [(40, 50, 20, 15, 0.1, 1), (64, 64, 32, 32, 0.5, 2),
                                                 (33, 70, 69, 32, 0.02, 3), (100, 100, 99, 99, 0.01, 4)])
def test_selected_counts_match_oracle(gpu_lib, H, W, rx, ry, frac, seed):
    img = synth.squares(H, W, 4, 0.3, seed=seed) if seed % 2 else synth.clustered_disks(H, W, 0.35, seed=seed)
    rng = np.random.default_rng(seed)
    sel = np.zeros(H * W, np.uint8)
    sel[rng.choice(H * W, max(1, int(frac * H * W)), replace=False)] = 1
    sel = sel.reshape(H, W)
    p = gpu_lib.lpf_build_paths(rx, ry)
    got = gpu_lib.lpf_full_mc(torch.from_numpy(img).cuda(), p, torch.from_numpy(sel).cuda()).cpu().numpy()
    ref = oracle.lpf_full_selected(img, rx, ry, sel)
    _, _, base = oracle.window_sizes(rx, ry)
    np.testing.assert_array_equal(got[:, base:], ref[:, base:])
    np.testing.assert_array_equal(got[:, :base], got[:, base + 1:][:, ::-1])  # filled by symmetry
    assert got[0, base] + got[1, base] == sel.sum()


def test_all_selected_equals_exact(gpu_lib):
    img = synth.config1_image()
    p = gpu_lib.lpf_build_paths(32, 32)
    d = torch.from_numpy(img).cuda()
    a = gpu_lib.lpf_full_mc(d, p, torch.ones_like(d))
    b = gpu_lib.lpf_full(d, p)
    assert torch.equal(a, b)
