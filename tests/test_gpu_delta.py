"""GPU parity of lpf_delta_swap (count changes and error changes) against the
CPU oracle's recount-after-minus-before and its double-precision Eq. (LSE)."""
import os

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


def _pairs(img, k, seed):
    rng = np.random.default_rng(seed)
    flat = img.reshape(-1)
    ones = np.flatnonzero(flat == 1)
    zeros = np.flatnonzero(flat == 0)
    out = [(int(rng.choice(ones)), int(rng.choice(zeros))) for _ in range(k)]
    out += [(int(zeros[1]), int(ones[1])),   # reversed order: still an exchange
            (int(ones[0]), int(ones[-1])),   # same phase: identity
            (int(zeros[0]), int(zeros[2])),
            (int(ones[3]), int(ones[3]))]    # a == b: identity
    rng.shuffle(out)
    return np.array(out, np.int32)


def _target(rx, ry, seed):
    ref = synth.clustered_disks(96, 96, 0.3, seed=seed)
    c = oracle.lpf_full(ref, rx, ry)
    return (c / float(ref.size)).astype(np.float32)


def _de_tolerance(target, counts, dcounts, rx, ry, H, W, n_chunks=1024):
    """Bound of the float32 evaluation: every term x*(x - 2d) carries a few
    rounding errors, and the terms are summed sequentially in groups of at
    most n_canon*2/8 + 8 + n_chunks (per warp, across warps, across chunks)."""
    _, n_canon, base = oracle.window_sizes(rx, ry)
    N = float(H * W)
    t = target[:, base:].astype(np.float64)
    c = counts[:, base:].astype(np.float64)
    d = t - c / N
    x = dcounts.astype(np.float64) / N
    terms = x * (x - 2 * d[None])
    mag = np.abs(terms).sum(axis=(1, 2))
    seq = 2 * n_canon / 8 + 8 + n_chunks
    return (seq + 8) * 2.0 ** -24 * mag + 1e-12


CASES = [
    ("cell 32x32 r8", lambda: synth.random_binary(32, 32, 0.3, 1), 8, 8),
    ("ragged 45x37 rx20 ry15", lambda: synth.clustered_disks(37, 45, 0.3, seed=2), 20, 15),
    ("full domain 9x8", lambda: synth.random_binary(8, 9, 0.5, 3), 8, 7),
    ("disks 64x64 r32", lambda: synth.disks_64(), 32, 32),
]


@pytest.mark.parametrize("name,make,rx,ry", CASES, ids=[c[0] for c in CASES])
def test_delta_counts_and_error_match_oracle(gpu_lib, name, make, rx, ry):
    img = make()
    H, W = img.shape
    pairs = _pairs(img, 24, 5)
    p = gpu_lib.lpf_build_paths(rx, ry)
    d_img = torch.from_numpy(img).cuda()
    counts = gpu_lib.lpf_full(d_img, p)
    target = _target(rx, ry, 9)
    dc, de = gpu_lib.lpf_delta_swap(d_img, p, torch.from_numpy(pairs).cuda(),
                                    target=torch.from_numpy(target).cuda(), counts=counts, want_de=True)
    torch.cuda.synchronize()
    assert gpu_lib.lpf_paths_status(p) == 0
    ref = oracle.delta_swap(img, rx, ry, pairs)
    np.testing.assert_array_equal(dc.cpu().numpy(), ref)
    counts_h = counts.cpu().numpy()
    de_ref = oracle.delta_objective(target, counts_h, ref, rx, ry, H, W)
    tol = _de_tolerance(target, counts_h, ref, rx, ry, H, W)
    err = np.abs(de.cpu().numpy().astype(np.float64) - de_ref)
    assert (err <= tol).all(), (err.max(), tol[err.argmax()])
    # identities are exactly zero
    flat = img.reshape(-1)
    same = flat[pairs[:, 0]] == flat[pairs[:, 1]]
    assert not dc.cpu().numpy()[same].any() and (de.cpu().numpy()[same] == 0).all()


def test_error_only_and_determinism(gpu_lib):
    img = synth.clustered_disks(64, 64, 0.3, seed=4)
    rx = ry = 24
    pairs = torch.from_numpy(_pairs(img, 200, 6)).cuda()
    p = gpu_lib.lpf_build_paths(rx, ry)
    d_img = torch.from_numpy(img).cuda()
    counts = gpu_lib.lpf_full(d_img, p)
    target = torch.from_numpy(_target(rx, ry, 10)).cuda()
    _, de1 = gpu_lib.lpf_delta_swap(d_img, p, pairs, target=target, counts=counts, want_dcounts=False, want_de=True)
    dc, de2 = gpu_lib.lpf_delta_swap(d_img, p, pairs, target=target, counts=counts, want_de=True)
    _, de3 = gpu_lib.lpf_delta_swap(d_img, p, pairs, target=target, counts=counts, want_dcounts=False, want_de=True)
    assert torch.equal(de1, de2) and torch.equal(de1, de3)  # bitwise reproducible


def test_clustered_128_cell_full_batch_64_candidates(gpu_lib):
    # The swap-delta workload: the 128x128 clustered cell, |v| <= 64, K = 4096
    # candidates in one launch; 64 of them (the first, the last, identities,
    # same-phase and reversed pairs, and random ones) against the oracle's
    # recount stored by tests/golden/make_lpf_goldens.py.
    g = np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "lpf_delta_clustered_128.npz"))
    cell = synth.clustered_cell_128()
    rx = ry = 64
    pairs, sample, ref = g["pairs"], g["sample"], g["dcounts"].astype(np.int64)
    p = gpu_lib.lpf_build_paths(rx, ry)
    d_img = torch.from_numpy(cell).cuda()
    counts = gpu_lib.lpf_full(d_img, p)
    counts_h = counts.cpu().numpy()
    np.testing.assert_array_equal(counts_h, g["counts"])
    target = (counts_h / float(cell.size) * 0.9).astype(np.float32)
    dc, de = gpu_lib.lpf_delta_swap(d_img, p, torch.from_numpy(pairs).cuda(),
                                    target=torch.from_numpy(target).cuda(), counts=counts, want_de=True)
    assert gpu_lib.lpf_paths_status(p) == 0
    dc = dc.cpu().numpy()
    de = de.cpu().numpy()
    np.testing.assert_array_equal(dc[sample], ref)
    de_ref = oracle.delta_objective(target, counts_h, ref, rx, ry, 128, 128)
    tol = _de_tolerance(target, counts_h, ref, rx, ry, 128, 128)
    assert (np.abs(de[sample] - de_ref) <= tol).all()
    # a swap changes no count at v = 0, and every change is bounded by the
    # number of translations through the two pixels
    assert not dc[:, :, 0].any()
    _, ptr, _ = gpu_lib.lpf_paths_export(p)
    L1 = np.diff(ptr)
    assert (np.abs(dc) <= 2 * L1[None, None, :]).all()
