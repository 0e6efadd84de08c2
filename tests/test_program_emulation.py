"""Host side of the walk, checked on the CPU: the programs the library builds
and bakes (prefix trees of the x-major segments and of the transposed y-major
segments, pieces with prologues, skip words, pixel pairs) are walked by a C++
emulation of the kernels' semantics (tests/walk_emulator.cpp) over the image
and its transpose and compared with the oracle entry by entry."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def emulator(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("emu") / "libwalkemu.so")
    src = [os.path.join(ROOT, "tests", "walk_emulator.cpp"),
           os.path.join(ROOT, "paper_1601_04359_gb300", "csrc", "lpf_paths.cpp")]
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", out] + src, check=True)
    lib = ctypes.CDLL(out)
    lib.emulate_walk.restype = ctypes.c_int
    lib.emulate_walk.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    lib.emulate_walk_sel.restype = ctypes.c_int
    lib.emulate_walk_sel.argtypes = [ctypes.c_void_p, ctypes.c_void_p] + [ctypes.c_int] * 5 + [ctypes.c_void_p,
                                                                                               ctypes.c_void_p]
    lib.emulate_walk3.restype = ctypes.c_int
    lib.emulate_walk3.argtypes = [ctypes.c_void_p] + [ctypes.c_int] * 7 + [ctypes.c_void_p, ctypes.c_void_p]
    return lib


def _walk(lib, img, rx, ry, standard, T):
    img = np.ascontiguousarray(img, np.uint8)
    H, W = img.shape
    counts = np.zeros((2, (2 * rx + 1) * (2 * ry + 1)), np.int64)
    stats = np.zeros(4, np.int64)
    rc = lib.emulate_walk(img.ctypes.data, H, W, rx, ry, int(standard), T, counts.ctypes.data, stats.ctypes.data)
    assert rc == 0
    return counts, stats


CASES = [
    ("chess 40 full domain", lambda: synth.chess(40, 40, 10), 39, 39),
    ("chess 33x65 rx=64", lambda: synth.chess(33, 65, 10), 64, 32),
    ("squares 64 window 30x20", lambda: synth.squares(64, 64, 4, 0.2, seed=7), 30, 20),
    ("random 50x70", lambda: synth.random_binary(50, 70, 0.5, 3), 12, 9),
    ("foam crop 37x45 full domain", lambda: synth.foam(100, 100, 0.75, seed=5)[:37, :45].copy(), 36, 36),
    ("ellipses 96 window 60", lambda: synth.ellipses(96, 96, 0.35, seed=2), 60, 60),
    ("all zeros", lambda: np.zeros((20, 20), np.uint8), 19, 19),
    ("all ones 20x33", lambda: np.ones((20, 33), np.uint8), 19, 19),
]


@pytest.mark.parametrize("name,make,rx,ry", CASES, ids=[c[0] for c in CASES])
def test_baked_programs_walk_to_the_oracle_counts(emulator, name, make, rx, ry):
    img = make()
    ref = oracle.lpf_full(img, rx, ry)
    for T in (1, 2):
        got, stats = _walk(emulator, img, rx, ry, standard=False, T=T)
        np.testing.assert_array_equal(got, ref, err_msg=f"tree T={T}")
        assert 0 < stats[0] <= stats[1] or img.sum() == 0
    got, _ = _walk(emulator, img, rx, ry, standard=True, T=1)
    np.testing.assert_array_equal(got, ref, err_msg="standard")


def test_skips_and_pairs_are_exercised(emulator):
    # chess: most subtrees die early (skips, little walked); near-horizontal
    # segments read the same staged words for several pixels (pairs)
    img = synth.chess(40, 40, 10)
    _, stats = _walk(emulator, img, 39, 39, standard=False, T=1)
    walked, nominal, skips, pairs = (int(x) for x in stats)
    assert skips > 0 and walked < 0.6 * nominal
    assert pairs > 0
    _, stats = _walk(emulator, np.ones((20, 33), np.uint8), 19, 19, standard=False, T=2)
    assert stats[0] == stats[1] and stats[2] == 0  # nothing to skip when every segment fits


def test_wide_tiles(emulator):
    # 4 and 8 words per thread: wider staged rows, other pixel pairs
    img = synth.ellipses(40, 200, 0.35, seed=5)
    ref = oracle.lpf_full(img, 70, 25)
    for T in (4, 8):
        got, stats = _walk(emulator, img, 70, 25, standard=False, T=T)
        np.testing.assert_array_equal(got, ref, err_msg=f"T={T}")
        assert stats[3] > 0


@pytest.mark.parametrize("shape,window,T", [((6, 20, 24), (7, 5, 3), 1), ((9, 33, 40), (12, 9, 4), 2),
                                            ((5, 40, 70), (20, 6, 2), 4)])
def test_volume_programs_walk_to_the_oracle_counts(emulator, shape, window, T):
    # The 3D program (prefix tree of 3D segments) baked for the slice layout:
    # slices of 32-row bands extended by ry rows above and below, the next rz
    # slices staged with them.
    vol = synth.boolean_spheres(*shape, 3.0, 14, seed=sum(shape))
    D, H, W = vol.shape
    rx, ry, rz = window
    counts = np.zeros((2, (2 * rx + 1) * (2 * ry + 1) * (2 * rz + 1)), np.int64)
    stats = np.zeros(4, np.int64)
    v = np.ascontiguousarray(vol)
    assert emulator.emulate_walk3(v.ctypes.data, D, H, W, rx, ry, rz, T, counts.ctypes.data, stats.ctypes.data) == 0
    np.testing.assert_array_equal(counts, oracle.lpf_full3(vol, rx, ry, rz))
    assert 0 < stats[0] <= stats[1]


@pytest.mark.parametrize("H,W,rx,ry,frac,seed", [(40, 50, 20, 15, 0.1, 1), (33, 70, 69, 32, 0.05, 3),
                                                 (30, 30, 29, 29, 0.3, 4)])
def test_selected_start_translations(emulator, H, W, rx, ry, frac, seed):
    # The Monte-Carlo variant counts only selected start pixels: a segment of
    # the transposed tree must start where the image's segment starts (a
    # vector with dx < 0 runs to y' < 0 over the transposed image).
    img = synth.squares(H, W, 4, 0.3, seed=seed)
    rng = np.random.default_rng(seed)
    sel = np.zeros(H * W, np.uint8)
    sel[rng.choice(H * W, max(1, int(frac * H * W)), replace=False)] = 1
    sel = sel.reshape(H, W)
    counts = np.zeros((2, (2 * rx + 1) * (2 * ry + 1)), np.int64)
    stats = np.zeros(4, np.int64)
    assert emulator.emulate_walk_sel(img.ctypes.data, sel.ctypes.data, H, W, rx, ry, 2, counts.ctypes.data,
                                     stats.ctypes.data) == 0
    _, _, base = oracle.window_sizes(rx, ry)
    np.testing.assert_array_equal(counts[:, base:], oracle.lpf_full_selected(img, rx, ry, sel)[:, base:])
