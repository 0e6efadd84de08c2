"""Host-side checks of the C ABI: the library loads, exports every declared
symbol, and its host-only entry points (path tables) work without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_1601_04359_gb300 as lpf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if not f.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", f)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names |= set(re.findall(r"\b((?:lpf|s2)_[a-z0-9_]+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol():
    lib = lpf.load()
    names = _declared()
    assert {"lpf_full", "lpf_build_paths", "s2_fft", "s2_sa_create", "lpf_sa_create_mc"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_build_paths_tables_match_oracle_segments():
    for rx, ry in [(0, 0), (3, 2), (12, 12), (7, 19)]:
        p = lpf.lpf_build_paths(rx, ry)
        n_full, n_canon, base = oracle.window_sizes(rx, ry)
        assert (p.n_full, p.n_canon, p.base) == (n_full, n_canon, base)
        vec, ptr, off = lpf.lpf_paths_export(p)
        for c in range(n_canon):
            k = base + c
            dy, dx = k // (2 * rx + 1) - ry, k % (2 * rx + 1) - rx
            assert tuple(vec[c]) == (dx, dy)
            np.testing.assert_array_equal(off[ptr[c]:ptr[c + 1]], oracle.segment(dx, dy))


def test_prefix_program_statistics():
    # The prefix tree visits far fewer pixels than the segments hold.
    p = lpf.lpf_build_paths(64, 64)
    st = lpf.lpf_paths_stats(p)
    assert p.n_offsets == 366081
    assert st["n_tree_nodes"] < 0.25 * p.n_offsets
    assert 1 <= st["stack_depth"] <= 24 and st["n_pieces"] >= 1


def test_invalid_arguments_rejected_on_host():
    lib = lpf.load()
    h = ctypes.c_void_p()
    assert lib.lpf_build_paths(-1, 3, ctypes.byref(h)) == -1
    assert lib.lpf_build_paths(4096, 3, ctypes.byref(h)) == -1
    assert lib.lpf_build_paths(3, 3, None) == -1
    p = lpf.lpf_build_paths(4, 4)
    # null image / counts and a window wider than the image: rejected before any CUDA call
    assert lib.lpf_full(None, 8, 8, p.handle, None, None) == -1
    assert lib.lpf_full(ctypes.c_void_p(16), 8, 4, p.handle, ctypes.c_void_p(16), None) == -1
    assert lib.lpf_full(ctypes.c_void_p(16), 0, 8, p.handle, ctypes.c_void_p(16), None) == -1
    assert lpf.lpf_strerror(-1) == "invalid argument"


def test_newer_entry_points_reject_bad_arguments_on_host():
    lib = lpf.load()
    p = lpf.lpf_build_paths(4, 4)
    v = ctypes.c_void_p(16)
    h = ctypes.c_void_p()
    prm = lpf.SaParams(100, 10, 1, 1e-3, 0.01, 64, 1, 1, 3)
    assert lib.s2_counts(None, 8, 8, v, None) == -1
    assert lib.s2_delta_swap(v, 8, 8, v, -1, None, None, None, None, None) == -1
    assert lib.s2_sa_create(v, 1, 8, v, v, ctypes.byref(prm), None, ctypes.byref(h)) == -1   # H < 2
    assert lib.lpf_full_ensemble(None, 2, 8, 8, p.handle, v, None) == -1
    assert lib.lpf_full_ensemble(v, 0, 8, 8, p.handle, v, None) == -1
    assert lib.lpf_sa_create_mc(v, 8, 8, p.handle, None, v, v, ctypes.byref(prm), None, ctypes.byref(h)) == -1
    assert lib.lpf_sa_import_progress(None, None, None) == -1
    assert lib.lpf_sa_export_progress(None, None, None) == -1
    assert lib.lpf_sa_selftest_timeout(None, -1, None) == -1
    assert lib.lpf_set_checked(None, 1) == -1
    assert lib.lpf_set_checked(p.handle, 2) == -1
    assert lib.lpf_paths_set_selftest(None, 1) == -1
    assert lib.lpf_batch_work(None, v, v, None) == -1
    assert lpf.lpf_strerror(-6).startswith("pixel value")
    bad = lpf.SaParams(100, 10, 1, 1e-3, 0.01, 64, 1, 1, 7)   # phases outside {0..3}
    assert lib.lpf_sa_create(v, 8, 8, p.handle, v, v, ctypes.byref(bad), None, ctypes.byref(h)) == -1


def test_readme_c_example_compiles_and_links(tmp_path):
    # The C example of the README, compiled against include/lpf.h and linked
    # with the built library and the CUDA runtime (not run: no GPU needed).
    import shutil
    import subprocess
    gcc, nvcc = shutil.which("gcc"), shutil.which("nvcc")
    if gcc is None or nvcc is None:
        pytest.skip("gcc or the CUDA toolkit not available")
    cuda = os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    cudart = [d for d in ("lib64", "lib", "targets/x86_64-linux/lib", "targets/sbsa-linux/lib")
              if os.path.exists(os.path.join(cuda, d, "libcudart.so"))]
    if not cudart:
        pytest.skip("libcudart.so not found")
    readme = open(os.path.join(ROOT, "README.md")).read()
    blocks = re.findall(r"```c\n(.*?)```", readme, flags=re.S)
    assert len(blocks) == 1
    src = tmp_path / "example.c"
    src.write_text(blocks[0])
    libdir = os.path.dirname(lpf.load()._name)
    r = subprocess.run([gcc, "-std=c11", "-Wall", "-Werror", str(src), "-o", str(tmp_path / "example"),
                        "-I", os.path.join(ROOT, "include"), "-I", os.path.join(cuda, "include"),
                        "-L", libdir, "-llpf", "-L", os.path.join(cuda, cudart[0]), "-lcudart"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
