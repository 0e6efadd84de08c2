"""GPU Monte-Carlo variant (Sec. 3): counts over selected translations
against the oracle, on the canonical half D that the paper evaluates."""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import sa as osa

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
    img = synth.disks_64()
    p = gpu_lib.lpf_build_paths(32, 32)
    d = torch.from_numpy(img).cuda()
    a = gpu_lib.lpf_full_mc(d, p, torch.ones_like(d))
    b = gpu_lib.lpf_full(d, p)
    assert torch.equal(a, b)


def _sel(H, W, n, seed):
    rng = np.random.default_rng(seed)
    sel = np.zeros(H * W, np.uint8)
    sel[rng.choice(H * W, n, replace=False)] = 1
    return sel.reshape(H, W)


@pytest.mark.parametrize("H,W,r,n,seed", [(24, 24, 8, 100, 1), (37, 45, 20, 10, 2), (50, 50, 49, 1000, 3)])
def test_selected_delta_matches_recount(gpu_lib, H, W, r, n, seed):
    # swap changes over the sampled translations = recount over them after
    # minus before; error changes with the descriptor count / N
    img = synth.squares(H, W, 4, 0.3, seed=seed)
    sel = _sel(H, W, n, seed + 10)
    flat = img.reshape(-1)
    rng = np.random.default_rng(seed)
    ones, zeros = np.flatnonzero(flat == 1), np.flatnonzero(flat == 0)
    pairs = np.array([(int(rng.choice(ones)), int(rng.choice(zeros))) for _ in range(12)] +
                     [(int(ones[0]), int(ones[1]))], np.int32)
    p = gpu_lib.lpf_build_paths(r, r)
    d_img, d_sel = torch.from_numpy(img).cuda(), torch.from_numpy(sel).cuda()
    counts = gpu_lib.lpf_full_mc(d_img, p, d_sel)
    orig = synth.squares(2 * H, 2 * W, 4, 0.3, seed=seed + 5)
    target = (oracle.lpf_full(orig, r, r) / float(orig.size)).astype(np.float32)
    dc, de = gpu_lib.lpf_delta_swap_mc(d_img, p, d_sel, torch.from_numpy(pairs).cuda(),
                                       target=torch.from_numpy(target).cuda(), counts=counts, want_de=True)
    dc, de = dc.cpu().numpy(), de.cpu().numpy().astype(np.float64)
    before = oracle.lpf_full_selected(img, r, r, sel)
    _, n_canon, base = oracle.window_sizes(r, r)
    ref = np.zeros((len(pairs), 2, n_canon), np.int64)
    for k, (a, b) in enumerate(pairs):
        after = flat.copy()
        after[a], after[b] = after[b], after[a]
        ref[k] = (oracle.lpf_full_selected(after.reshape(H, W), r, r, sel) - before)[:, base:]
    np.testing.assert_array_equal(dc, ref)
    de_ref = oracle.delta_objective(target, counts.cpu().numpy(), ref, r, r, n, 1)  # descriptor count / N
    t = target[:, base:].astype(np.float64)
    c = before[:, base:].astype(np.float64)
    x = ref.astype(np.float64) / n
    mag = np.abs(x * (x - 2 * (t - c / n)[None])).sum(axis=(1, 2))
    tol = (2 * n_canon / 8 + 8 + 1024 + 8) * 2.0 ** -24 * mag + 1e-12
    assert (np.abs(de - de_ref) <= tol).all()


@pytest.mark.parametrize("kmin,kmax", [(1, 1), (4, 64)])
def test_monte_carlo_annealing_equals_sequential_oracle(gpu_lib, kmin, kmax):
    H = W = 20
    r = 6
    orig = synth.squares(40, 40, 4, 0.3, seed=3)
    sel_o = _sel(40, 40, 400, 7)
    target = (oracle.lpf_full_selected(orig, r, r, sel_o) / 400.0).astype(np.float32)
    cell = synth.exact_fraction_shuffle(H, W, 120, seed=4)
    sel = _sel(H, W, 150, 8)
    n_step, c_max, s_max = 400, 40, 4
    counts0 = oracle.lpf_full_selected(cell, r, r, sel)
    t_max = 1e-3
    p = gpu_lib.lpf_build_paths(r, r)
    d_cell = torch.from_numpy(cell).cuda()
    counts = torch.empty((2, p.n_full), dtype=torch.int64, device="cuda")
    ann = gpu_lib.lpf_sa_create_mc(d_cell, p, torch.from_numpy(sel).cuda(), torch.from_numpy(target).cuda(), counts,
                                   n_step=n_step, c_max=c_max, s_max=s_max, t_max=t_max, k_min=kmin, k_max=kmax,
                                   seed=9)
    _, _, base = oracle.window_sizes(r, r)
    # the Monte-Carlo counts are defined on the half-domain D (the other half
    # is filled by symmetry, which does not hold for a sample of starts)
    np.testing.assert_array_equal(counts.cpu().numpy()[:, base:], counts0[:, base:])
    e0 = gpu_lib.lpf_sa_read(ann)["error"]
    assert e0 == pytest.approx(oracle.objective(target, counts0, r, r, 150, 1), rel=1e-12)
    while not gpu_lib.lpf_sa_read(ann)["done"]:
        gpu_lib.lpf_sa_run(ann, 32)
    st = gpu_lib.lpf_sa_read(ann)
    ref_cell, ref_acc, _ = osa.anneal(cell, target, counts0, r, r, n_step, c_max, s_max, t_max, 0.01, seed=9, sel=sel)
    got = d_cell.cpu().numpy()
    assert st["n_accept"] == ref_acc and ref_acc > 0
    np.testing.assert_array_equal(got, ref_cell)
    np.testing.assert_array_equal(counts.cpu().numpy()[:, base:], oracle.lpf_full_selected(got, r, r, sel)[:, base:])
