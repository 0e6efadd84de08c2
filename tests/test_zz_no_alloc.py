"""lpf_full_noalloc: the full evaluation for callers that cannot allocate
device memory while they evaluate (a host application that owns all device
allocations, or a real-time loop where cudaMalloc, which can synchronise the
device, is forbidden).  Its work area is a fixed array inside the library.

Called through the C ABI with ctypes; each of two calls in a row must give
exactly the counts of lpf_full (integer counts: bit-exact), on different
images so that the shared fixed array cannot carry a stale result over.
Every test does its own set-up (an lpf_full call for its image size), so the
tests do not depend on the order in which files are collected.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def _call(lib, img, paths, out):
    H, W = img.shape
    return lib.lpf_full_noalloc(ctypes.c_void_p(img.data_ptr()), H, W, ctypes.c_void_p(paths.handle),
                                ctypes.c_void_p(out.data_ptr()),
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_matches_lpf_full_on_two_calls(gpu_lib):
    lib = gpu_lib.load()
    r = 256
    paths = gpu_lib.lpf_build_paths(r, r)
    a = torch.from_numpy(synth.ellipses_512()).cuda()
    b = torch.from_numpy(synth.clustered_disks(512, 512, 0.3, seed=21)).cuda()
    ref_a = gpu_lib.lpf_full(a, paths)   # existing entry point; also puts the program on the device
    ref_b = gpu_lib.lpf_full(b, paths)
    out1 = torch.full((2, paths.n_full), -1, dtype=torch.int64, device="cuda")
    out2 = torch.full((2, paths.n_full), -1, dtype=torch.int64, device="cuda")
    assert _call(lib, a, paths, out1) == 0
    assert _call(lib, b, paths, out2) == 0
    torch.cuda.synchronize()
    assert torch.equal(out1, ref_a)
    assert torch.equal(out2, ref_b)
    # and again on the first image: nothing left over from the previous call
    assert _call(lib, a, paths, out2) == 0
    torch.cuda.synchronize()
    assert torch.equal(out2, ref_a)


def test_noalloc_rejects_what_it_cannot_do(gpu_lib):
    lib = gpu_lib.load()
    small = torch.from_numpy(synth.disks_64()).cuda()
    fresh = gpu_lib.lpf_build_paths(32, 32)
    out = torch.empty((2, fresh.n_full), dtype=torch.int64, device="cuda")
    # the program for this size was never put on the device: refused, not allocated
    assert _call(lib, small, fresh, out) == -1
    gpu_lib.lpf_full(small, fresh)
    assert _call(lib, small, fresh, out) == 0
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), gpu_lib.lpf_full(small, fresh).cpu().numpy())
    # an image whose packed rows exceed the fixed area (4128 rows x 67 words
    # > 2^18 words) is refused with LPF_EUNSUPPORTED
    big = torch.zeros((4096, 2048), dtype=torch.uint8, device="cuda")
    big_out = torch.empty((2, fresh.n_full), dtype=torch.int64, device="cuda")
    assert _call(lib, big, fresh, big_out) == -5


def test_noalloc_after_autotune_and_shape_changes(gpu_lib):
    # 200 x 200, window 40: launch shapes with 1 and 8 words per thread lay
    # the packed rows out with different strides (11 and 13 words).  After the
    # autotuner, and after a launch shape set later, the call still finds a
    # usable program and gives lpf_full's counts.
    lib = gpu_lib.load()
    img = torch.from_numpy(synth.ellipses(200, 200, 0.35, seed=8)).cuda()
    paths = gpu_lib.lpf_build_paths(40, 40)
    ref = gpu_lib.lpf_full(img, paths).clone()
    gpu_lib.lpf_autotune_full(img, paths)
    out = torch.full((2, paths.n_full), -1, dtype=torch.int64, device="cuda")
    assert _call(lib, img, paths, out) == 0
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    for T in (1, 8):
        gpu_lib.lpf_set_launch_shape(paths, 200, 200, T, 1)
        out.fill_(-1)
        assert _call(lib, img, paths, out) == 0
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    assert gpu_lib.lpf_paths_status(paths) == 0


def test_noalloc_equals_the_oracle_and_reports_a_timeout(gpu_lib):
    import oracle
    lib = gpu_lib.load()
    img = synth.clustered_disks(72, 90, 0.3, seed=12)
    d = torch.from_numpy(img).cuda()
    paths = gpu_lib.lpf_build_paths(30, 20)
    gpu_lib.lpf_full(d, paths)   # set-up
    out = torch.empty((2, paths.n_full), dtype=torch.int64, device="cuda")
    assert _call(lib, d, paths, out) == 0
    assert gpu_lib.lpf_paths_status(paths) == 0
    np.testing.assert_array_equal(out.cpu().numpy(), oracle.lpf_full(img, 30, 20))
    # a staging wait made to run out is reported through lpf_paths_status
    gpu_lib.lpf_paths_set_selftest(paths, True)
    assert _call(lib, d, paths, out) == 0
    assert gpu_lib.lpf_paths_status(paths) == gpu_lib.LPF_ETIMEOUT
    gpu_lib.lpf_paths_set_selftest(paths, False)
    assert _call(lib, d, paths, out) == 0
    assert gpu_lib.lpf_paths_status(paths) == 0
    np.testing.assert_array_equal(out.cpu().numpy(), oracle.lpf_full(img, 30, 20))


def test_noalloc_captured_in_a_graph_and_replayed(gpu_lib):
    # A stream capture in global mode fails on any call that allocates device
    # memory or synchronises, so a successful capture shows the call does
    # neither.  The graph is then replayed on two images copied into its
    # input, each replay's counts equal to lpf_full's.
    lib = gpu_lib.load()
    imgs = [synth.ellipses(200, 184, 0.35, seed=31), synth.clustered_disks(200, 184, 0.3, seed=32)]
    paths = gpu_lib.lpf_build_paths(60, 50)
    refs = [gpu_lib.lpf_full(torch.from_numpy(i).cuda(), paths) for i in imgs]  # set-up
    inp = torch.from_numpy(imgs[0]).cuda()
    out = torch.full((2, paths.n_full), -1, dtype=torch.int64, device="cuda")
    assert _call(lib, inp, paths, out) == 0  # the first call on the device, outside any capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="global"):
        rc = _call(lib, inp, paths, out)
    assert rc == 0
    for img, ref in zip(imgs[::-1], refs[::-1]):
        inp.copy_(torch.from_numpy(img).cuda())
        out.fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    assert gpu_lib.lpf_paths_status(paths) == 0
