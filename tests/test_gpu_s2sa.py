"""GPU parity of the two-point-probability objective (Sec. 2.1, Eq. (S2dis);
Eq. (LSE) on S2 for the compressions of Sec. 6): exact counts, swap changes,
error changes and annealing trajectories against the oracle, plus
single-phase lineal-path annealing (the L2^w / L2^b rows of Tab. mutual)."""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import sa as osa

pytestmark = pytest.mark.gpu


def _cut(s2_orig, H, W):
    """Target per cell offset (y, x): the original's S2 at the centred offset
    (y or y - H, x or x - W), the cut of a descriptor to the cell (Sec. 6)."""
    H0, W0 = s2_orig.shape
    ys = np.array([y if y < H - (H + 1) // 2 else y - H for y in range(H)]) % H0
    xs = np.array([x if x < W - (W + 1) // 2 else x - W for x in range(W)]) % W0
    return s2_orig[np.ix_(ys, xs)].astype(np.float32)


def _s2_target(H, W, frac=0.3, seed=9):
    orig = synth.clustered_disks(2 * H, 2 * W, frac, seed=seed)
    return _cut(oracle.s2_direct(orig, 1), H, W)


@pytest.mark.parametrize("H,W,seed", [(1, 7, 0), (5, 3, 1), (16, 16, 2), (37, 45, 3), (64, 64, 4), (50, 50, 5),
                                      (33, 97, 6)])
def test_s2_counts_exact(gpu_lib, H, W, seed):
    img = synth.random_binary(H, W, 0.4, seed)
    got = gpu_lib.s2_counts(torch.from_numpy(img).cuda())
    np.testing.assert_array_equal(got.cpu().numpy(), oracle.s2_counts(img))


def test_s2_counts_chess_closed_form(gpu_lib):
    # chess with s x s squares on a 4s period: C(dx, 0) = WH (s - |dx|)/(2s) for
    # |dx| <= s along a row, by the same argument as for the lineal path
    s = 6
    img = synth.chess(48, 48, s)
    C = gpu_lib.s2_counts(torch.from_numpy(img).cuda()).cpu().numpy()
    for dx in range(0, s + 1):
        assert C[0, dx] == 48 * 48 * (s - dx) // (2 * s)


def _pairs(img, k, seed):
    rng = np.random.default_rng(seed)
    flat = img.reshape(-1)
    ones = np.flatnonzero(flat == 1)
    zeros = np.flatnonzero(flat == 0)
    out = [(int(rng.choice(ones)), int(rng.choice(zeros))) for _ in range(k)]
    out += [(int(zeros[1]), int(ones[1])),   # reversed order: still an exchange
            (int(ones[0]), int(ones[-1])),   # same phase: identity
            (int(ones[3]), int(ones[3])),    # a == b: identity
            (int(ones[0]), int(ones[0]) + 1 if flat[int(ones[0]) + 1] == 0 else int(zeros[0]))]
    rng.shuffle(out)
    return np.array(out, np.int32)


def _tolerance(target, counts, dcounts, H, W):
    # float32 terms x (x - 2 delta), each with a few roundings, summed
    # sequentially in groups of at most H*W/256 per thread, then 5 shuffle
    # levels, 8 warps and the chunks
    N = float(H * W)
    d = target.astype(np.float64).reshape(-1) - counts.reshape(-1) / N
    x = dcounts.reshape(len(dcounts), -1).astype(np.float64) / N
    mag = np.abs(x * (x - 2 * d[None])).sum(axis=1)
    seq = H * W / 256 + 5 + 8 + 64 + 8
    return seq * 2.0 ** -24 * mag + 1e-12


@pytest.mark.parametrize("H,W,seed", [(16, 16, 0), (37, 45, 1), (50, 50, 2), (128, 128, 3), (9, 130, 4)])
def test_s2_delta_matches_oracle(gpu_lib, H, W, seed):
    img = synth.clustered_disks(H, W, 0.3, seed=seed) if min(H, W) >= 16 else synth.random_binary(H, W, 0.4, seed)
    pairs = _pairs(img, 20, seed)
    target = _s2_target(H, W, seed=seed + 20)
    d_img = torch.from_numpy(img).cuda()
    counts = gpu_lib.s2_counts(d_img)
    dc, de = gpu_lib.s2_delta_swap(d_img, torch.from_numpy(pairs).cuda(), target=torch.from_numpy(target).cuda(),
                                   counts=counts, want_de=True)
    dc = dc.cpu().numpy()
    de = de.cpu().numpy().astype(np.float64)
    C0 = oracle.s2_counts(img)
    flat = img.reshape(-1)
    ref_dc = np.zeros_like(dc)
    for k, (a, b) in enumerate(pairs):
        after = flat.copy()
        after[a], after[b] = after[b], after[a]
        ref_dc[k] = oracle.s2_counts(after.reshape(H, W)) - C0
    np.testing.assert_array_equal(dc, ref_dc)
    ref_de = oracle.s2_delta_objective(img, target, pairs)
    tol = _tolerance(target, C0, ref_dc, H, W)
    err = np.abs(de - ref_de)
    assert (err <= tol).all(), (err.max(), tol[err.argmax()])
    same = flat[pairs[:, 0]] == flat[pairs[:, 1]]
    assert not dc[same].any() and (de[same] == 0).all()
    # the zero offset never changes (volume fraction kept), and C(d) = C(-d) is kept
    assert not dc[:, 0, 0].any()
    np.testing.assert_array_equal(dc[:, 1:, 1:], dc[:, 1:, 1:][:, ::-1, ::-1])


def test_s2_delta_bad_index_gives_nan(gpu_lib):
    img = synth.random_binary(12, 12, 0.4, 1)
    flat = img.reshape(-1)
    good = (int(np.flatnonzero(flat == 1)[0]), int(np.flatnonzero(flat == 0)[0]))
    pairs = np.array([good, (-1, 3), (5, 144), good], np.int32)
    d_img = torch.from_numpy(img).cuda()
    counts = gpu_lib.s2_counts(d_img)
    target = torch.zeros((12, 12), dtype=torch.float32, device="cuda")
    _, de = gpu_lib.s2_delta_swap(d_img, torch.from_numpy(pairs).cuda(), target=target, counts=counts,
                                  want_dcounts=False, want_de=True)
    de = de.cpu().numpy()
    assert np.isfinite(de[[0, 3]]).all() and de[0] == de[3]
    assert np.isnan(de[[1, 2]]).all()


def _run_to_end(lpf, ann, chunk=64):
    while True:
        lpf.lpf_sa_run(ann, chunk)
        st = lpf.lpf_sa_read(ann)
        if st["done"]:
            return st


@pytest.mark.parametrize("kmin,kmax", [(1, 1), (8, 64), (16, 2048)])
def test_s2_trajectory_equals_sequential_oracle(gpu_lib, kmin, kmax):
    H = W = 20
    target = _s2_target(H, W)
    cell = synth.exact_fraction_shuffle(H, W, int(round(0.3 * H * W)), seed=4)
    n_step, c_max, s_max = 500, 50, 5
    pairs, _ = osa.propose(cell, 0, 200, seed=11)
    de = oracle.s2_delta_objective(cell, target, pairs)
    t_max = float(np.median(de[de > 0]))
    d_cell = torch.from_numpy(cell).cuda()
    counts = torch.empty((H, W), dtype=torch.int64, device="cuda")
    ann = gpu_lib.s2_sa_create(d_cell, torch.from_numpy(target).cuda(), counts, n_step=n_step, c_max=c_max,
                               s_max=s_max, t_max=t_max, k_min=kmin, k_max=kmax, seed=11)
    # proposals are the lineal-path annealer's
    p_gpu, u_gpu = gpu_lib.lpf_sa_propose(ann, 64)
    p_ref, u_ref = osa.propose(cell, 0, 64, seed=11)
    np.testing.assert_array_equal(p_gpu.cpu().numpy(), p_ref)
    np.testing.assert_array_equal(u_gpu.cpu().numpy(), u_ref)
    st = _run_to_end(gpu_lib, ann)
    assert st["n_eval"] == n_step
    ref_cell, ref_acc, ref_T = osa.anneal(cell, target, np.zeros((2, 1), np.int64), 0, 0, n_step, c_max, s_max,
                                          t_max, 0.01, seed=11, objective="s2")
    got = d_cell.cpu().numpy()
    assert st["n_accept"] == ref_acc
    np.testing.assert_array_equal(got, ref_cell)
    assert st["temperature"] == pytest.approx(ref_T, rel=1e-9)
    np.testing.assert_array_equal(counts.cpu().numpy(), oracle.s2_counts(got))
    e_new = gpu_lib.lpf_sa_recompute_error(ann)
    e_ref = float(((target.astype(np.float64) - oracle.s2_counts(got) / (H * W)) ** 2).sum())
    assert e_new == pytest.approx(e_ref, rel=1e-12)
    assert abs(st["error"] - e_new) <= 1e-5 * abs(e_new) + 1e-12


@pytest.mark.parametrize("phases", [1, 2])
def test_single_phase_lineal_trajectory(gpu_lib, phases):
    H = W = 24
    r = 6
    orig = synth.clustered_disks(2 * H, 2 * W, 0.3, seed=9)
    target = (oracle.lpf_full(orig, r, r) / float(orig.size)).astype(np.float32)
    cell = synth.exact_fraction_shuffle(H, W, int(round(0.3 * H * W)), seed=4)
    n_step, c_max, s_max = 500, 50, 5
    counts0 = oracle.lpf_full(cell, r, r)
    pairs, _ = osa.propose(cell, 0, 200, seed=7)
    de = oracle.delta_objective(target, counts0, oracle.delta_swap(cell, r, r, pairs), r, r, H, W, phases)
    t_max = float(np.median(de[de > 0]))
    p = gpu_lib.lpf_build_paths(r, r)
    d_cell = torch.from_numpy(cell).cuda()
    counts = torch.empty((2, p.n_full), dtype=torch.int64, device="cuda")
    ann = gpu_lib.lpf_sa_create(d_cell, p, torch.from_numpy(target).cuda(), counts, n_step=n_step, c_max=c_max,
                                s_max=s_max, t_max=t_max, k_min=4, k_max=256, seed=7, phases=phases)
    e0 = gpu_lib.lpf_sa_read(ann)["error"]
    assert e0 == pytest.approx(oracle.objective(target, counts0, r, r, H, W, phases), rel=1e-12)
    st = _run_to_end(gpu_lib, ann)
    ref_cell, ref_acc, ref_T = osa.anneal(cell, target, counts0, r, r, n_step, c_max, s_max, t_max, 0.01, seed=7,
                                          phases=phases)
    got = d_cell.cpu().numpy()
    assert st["n_accept"] == ref_acc
    np.testing.assert_array_equal(got, ref_cell)
    np.testing.assert_array_equal(counts.cpu().numpy(), oracle.lpf_full(got, r, r))
    e_new = gpu_lib.lpf_sa_recompute_error(ann)
    assert e_new == pytest.approx(oracle.objective(target, oracle.lpf_full(got, r, r), r, r, H, W, phases),
                                  rel=1e-12)


def test_s2_annealing_128_reduces_error_and_auto_temperature(gpu_lib):
    # 128x128 cell against the S2 of the 512x512 clustered-disk original, cut
    # to the cell's centred offsets; automatic T_max.
    orig = synth.clustered_512()
    s2o = gpu_lib.s2_fft(torch.from_numpy(orig).cuda(), 1).cpu().numpy()
    target = torch.from_numpy(_cut(s2o, 128, 128)).cuda()
    cell0 = synth.exact_fraction_shuffle(128, 128, int(round(orig.mean() * 128 * 128)), seed=5)
    finals = []
    for _ in range(2):
        d_cell = torch.from_numpy(cell0).cuda()
        ann = gpu_lib.s2_sa_create(d_cell, target, n_step=20000, seed=3)
        st0 = gpu_lib.lpf_sa_read(ann)
        assert st0["t_max"] > 0 and math.isfinite(st0["t_max"])
        st = _run_to_end(gpu_lib, ann, chunk=256)
        assert st["error"] < 0.5 * st0["error"]
        finals.append(d_cell.cpu().numpy())
        np.testing.assert_array_equal(ann.counts.cpu().numpy(), oracle.s2_counts(finals[-1]))
    np.testing.assert_array_equal(finals[0], finals[1])
    assert finals[0].sum() == cell0.sum()
