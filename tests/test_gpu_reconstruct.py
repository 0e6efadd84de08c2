"""Reconstruction from the full-domain lineal path function (Sec. 5, Fig.
chess): a random 20 x 20 cell annealed against the descriptor of a 100 x 100
chess of 10 x 10 squares (period 20) becomes that chess, up to a
translation, within 5e5 swap evaluations.

Schedule: Tab. annealing with c_max = 0.01 N_step, so that the stages end
after at most s_max = c_max attempts and the temperature reaches
T_min = 0.01 T_max by N_step (with c_max = 0.1 N_step most stages end by
c_max at the acceptance rates of this problem and T stays near T_max);
T_max = 0.1 x the automatic start temperature."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def test_chess_cell_recovered(gpu_lib):
    orig = synth.chess(100, 100, 10)
    r = 19
    p = gpu_lib.lpf_build_paths(r, r)
    c = gpu_lib.lpf_full(torch.from_numpy(orig).cuda(), p)
    target = (c.double() / float(orig.size)).float()
    cell0 = synth.exact_fraction_shuffle(20, 20, 200, seed=2)
    n_step = 500000
    kw = dict(n_step=n_step, c_max=n_step // 100, s_max=n_step // 100, seed=2)
    auto = gpu_lib.lpf_sa_read(gpu_lib.lpf_sa_create(torch.from_numpy(cell0).cuda(), p, target, **kw))["t_max"]
    d = torch.from_numpy(cell0).cuda()
    ann = gpu_lib.lpf_sa_create(d, p, target, t_max=0.1 * auto, **kw)
    e0 = gpu_lib.lpf_sa_read(ann)["error"]
    while True:
        gpu_lib.lpf_sa_run(ann, 256)
        st = gpu_lib.lpf_sa_read(ann)
        if st["done"] or st["error"] < 1e-12:
            break
    cell = d.cpu().numpy()
    chess20 = synth.chess(20, 20, 10)
    translates = [np.roll(chess20, (dy, dx), axis=(0, 1)) for dy in range(20) for dx in range(20)]
    recovered = any((cell == t).all() for t in translates)
    e = gpu_lib.lpf_sa_recompute_error(ann)
    assert recovered, (e0, e, st)
    assert e < 1e-12 and st["n_eval"] <= n_step
