"""Pixels outside {0, 1}: checked mode reports them (LPF_EPIXEL), unchecked
mode reads every nonzero byte as phase 1 (the header's stated behaviour).

The oracle's definition (Sec. 2.2) covers two-phase images only, so the
unchecked case is compared with the oracle on the image with every nonzero
byte replaced by 1.  Nothing here faults: a bad pixel only sets a status bit.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


def _with_twos(img, seed=3, n=7):
    rng = np.random.default_rng(seed)
    out = img.copy()
    ones = np.flatnonzero(out.reshape(-1) == 1)
    out.reshape(-1)[rng.choice(ones, n, replace=False)] = 2
    return out


def test_checked_mode_reports_a_pixel_of_value_two(gpu_lib):
    img = synth.disks_64()[:40, :56].copy()
    bad = _with_twos(img)
    p = gpu_lib.lpf_build_paths(10, 9)
    gpu_lib.lpf_set_checked(p, True)
    c = gpu_lib.lpf_full(torch.from_numpy(img).cuda(), p)
    assert gpu_lib.lpf_paths_status(p) == 0                       # a clean image raises nothing
    np.testing.assert_array_equal(c.cpu().numpy(), oracle.lpf_full(img, 10, 9))
    gpu_lib.lpf_full(torch.from_numpy(bad).cuda(), p)
    assert gpu_lib.lpf_paths_status(p) == gpu_lib.LPF_EPIXEL
    assert gpu_lib.lpf_paths_status(p) == 0                       # reported once, then cleared
    # swap deltas read the image too
    pairs = torch.tensor([[0, 1], [5, 17]], dtype=torch.int32, device="cuda")
    gpu_lib.lpf_delta_swap(torch.from_numpy(bad).cuda(), p, pairs, want_dcounts=True, want_de=False)
    assert gpu_lib.lpf_paths_status(p) == gpu_lib.LPF_EPIXEL
    # a byte of 255 is caught as well
    worst = img.copy()
    worst[3, 4] = 255
    gpu_lib.lpf_full(torch.from_numpy(worst).cuda(), p)
    assert gpu_lib.lpf_paths_status(p) == gpu_lib.LPF_EPIXEL


def test_unchecked_mode_reads_nonzero_as_phase_one(gpu_lib):
    img = synth.ellipses(48, 72, 0.35, seed=5)
    bad = _with_twos(img, n=25)
    p = gpu_lib.lpf_build_paths(20, 13)
    c = gpu_lib.lpf_full(torch.from_numpy(bad).cuda(), p)
    assert gpu_lib.lpf_paths_status(p) == 0
    np.testing.assert_array_equal(c.cpu().numpy(), oracle.lpf_full((bad != 0).astype(np.uint8), 20, 13))
    # swap deltas agree: a pair (2, 0) is a phase-1 / phase-0 exchange, (2, 1) the identity
    flat = bad.reshape(-1)
    two = int(np.flatnonzero(flat == 2)[0])
    one = int(np.flatnonzero(flat == 1)[0])
    zero = int(np.flatnonzero(flat == 0)[0])
    pairs = np.array([[two, zero], [two, one]], np.int32)
    dc = gpu_lib.lpf_delta_swap(torch.from_numpy(bad).cuda(), p, torch.from_numpy(pairs).cuda(), want_dcounts=True,
                                want_de=False)[0]
    ref = oracle.delta_swap((bad != 0).astype(np.uint8), 20, 13, pairs)
    np.testing.assert_array_equal(dc.cpu().numpy(), ref)
    assert not ref[1].any()


def test_checked_mode_of_the_allocation_free_variant(gpu_lib):
    lib = gpu_lib.load()
    img = synth.disks_64()
    bad = _with_twos(img)
    p = gpu_lib.lpf_build_paths(16, 16)
    gpu_lib.lpf_set_checked(p, True)
    d_bad = torch.from_numpy(bad).cuda()
    gpu_lib.lpf_full(torch.from_numpy(img).cuda(), p)             # set-up: program on the device
    assert gpu_lib.lpf_paths_status(p) == 0
    out = torch.empty((2, p.n_full), dtype=torch.int64, device="cuda")
    rc = lib.lpf_full_noalloc(ctypes.c_void_p(d_bad.data_ptr()), 64, 64, ctypes.c_void_p(p.handle),
                              ctypes.c_void_p(out.data_ptr()),
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    assert gpu_lib.lpf_paths_status(p) == gpu_lib.LPF_EPIXEL
    assert gpu_lib.lpf_paths_status(p) == 0
