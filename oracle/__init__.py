"""CPU oracle for the lineal path function (LPF) of arXiv:1601.04359.

TEST INFRASTRUCTURE ONLY.  The oracle is the correctness definition the CUDA
library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it; the library never does,
and the two share no code.

The arithmetic lives in ``lpf_oracle.c`` (plain C, Alg. 1 of Sec. 3.1 with its
early break, one vector at a time; OpenMP only spreads whole vectors over
cores).  This module marshals numpy arrays to it through ctypes.

Functions and the passages they follow:
  segment(dx, dy)            Sec. 2.2, Bresenham segment (tie reading in the C file)
  lpf_full(img, rx, ry)      Sec. 2.2 definition + Alg. 1, every vector of the window
  count_list(img, vecs)      same, for selected vectors
  delta_swap(img, rx, ry, pairs)   Sec. 4 pixel-exchange operator, by recount
  objective(target, counts, ...)   Eq. (LSE), double precision
  delta_objective(...)             Eq. (LSE) after minus before, double precision
  s2_direct(img, phase)            Eq. (S2dis), direct double sum
  lpf_full_selected(img, rx, ry, sel)   Sec. 3 Monte-Carlo variant (selected translations)
  s2_counts(img), s2_delta_objective(img, target, pairs)   Eq. (S2dis) counts; Eq. (LSE) on S2, by recount
  segment3(dx, dy, dz), lpf_full3(vol, rx, ry, rz), count3(vol, dx, dy, dz, phase)
                             3D extension (Sec. 2 remark, Sec. 6.3): the 2D tie rule per minor axis
Parity status: every function above is pinned by ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        i32, i64, p = ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
        lib.lpfo_num_threads.restype = i32
        lib.lpfo_set_num_threads.argtypes = [i32]
        lib.lpfo_segment.argtypes = [i32, i32, p, p]
        lib.lpfo_segment.restype = i32
        lib.lpfo_count.argtypes = [p, i32, i32, i32, i32, i32]
        lib.lpfo_count.restype = i64
        lib.lpfo_lpf_full.argtypes = [p, i32, i32, i32, i32, p]
        lib.lpfo_count_list.argtypes = [p, i32, i32, p, p, i32, p]
        lib.lpfo_delta_swap.argtypes = [p, i32, i32, i32, i32, p, i32, p]
        lib.lpfo_objective.argtypes = [p, p, i32, i32, i32, i32, i32]
        lib.lpfo_objective.restype = ctypes.c_double
        lib.lpfo_delta_objective.argtypes = [p, p, p, i32, i32, i32, i32, i32, i32, p]
        lib.lpfo_s2_direct.argtypes = [p, i32, i32, i32, p]
        lib.lpfo_lpf_full_sel.argtypes = [p, i32, i32, i32, i32, p, p]
        lib.lpfo_s2_counts.argtypes = [p, i32, i32, p]
        lib.lpfo_s2_delta_objective.argtypes = [p, i32, i32, p, p, i32, p]
        lib.lpfo_segment3.argtypes = [i32, i32, i32, p, p, p]
        lib.lpfo_segment3.restype = i32
        lib.lpfo_count3.argtypes = [p, i32, i32, i32, i32, i32, i32, i32]
        lib.lpfo_count3.restype = i64
        lib.lpfo_lpf_full3.argtypes = [p, i32, i32, i32, i32, i32, i32, p]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def num_threads() -> int:
    """Threads the oracle's OpenMP loops use."""
    return int(_load().lpfo_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the oracle's later OpenMP loops (for timing it on one core)."""
    _load().lpfo_set_num_threads(int(n))


def window_sizes(rx: int, ry: int):
    """(n_full, n_canon, base) of the window |dx|<=rx, |dy|<=ry."""
    n_full = (2 * rx + 1) * (2 * ry + 1)
    base = (n_full - 1) // 2
    return n_full, n_full - base, base


def full_index(dx: int, dy: int, rx: int, ry: int) -> int:
    return (dy + ry) * (2 * rx + 1) + (dx + rx)


def segment(dx: int, dy: int) -> np.ndarray:
    """Pixel offsets [(sx, sy), ...] of the segment (0,0) -> (dx, dy)."""
    n = max(abs(dx), abs(dy)) + 1
    sx = np.zeros(n, np.int32)
    sy = np.zeros(n, np.int32)
    m = _load().lpfo_segment(int(dx), int(dy), _ptr(sx), _ptr(sy))
    assert m == n
    return np.stack([sx, sy], axis=1)


def _img(img) -> np.ndarray:
    a = np.ascontiguousarray(img, dtype=np.uint8)
    assert a.ndim == 2
    return a


def lpf_full(img, rx: int, ry: int) -> np.ndarray:
    """int64 [2][(2ry+1)(2rx+1)] counts of phases 0 and 1, every vector evaluated."""
    a = _img(img)
    H, W = a.shape
    if not (0 <= rx < W and 0 <= ry < H):
        raise ValueError("window must satisfy 0 <= rx < W and 0 <= ry < H")
    n_full, _, _ = window_sizes(rx, ry)
    out = np.zeros((2, n_full), np.int64)
    _load().lpfo_lpf_full(_ptr(a), H, W, rx, ry, _ptr(out))
    return out


def lpf_full_selected(img, rx: int, ry: int, sel) -> np.ndarray:
    """Counts over the selected translations only (Monte-Carlo variant of Sec. 3)."""
    a = _img(img)
    H, W = a.shape
    s = np.ascontiguousarray(sel, dtype=np.uint8)
    assert s.shape == a.shape
    n_full, _, _ = window_sizes(rx, ry)
    out = np.zeros((2, n_full), np.int64)
    _load().lpfo_lpf_full_sel(_ptr(a), H, W, rx, ry, _ptr(s), _ptr(out))
    return out


def count(img, dx: int, dy: int, phase: int) -> int:
    a = _img(img)
    H, W = a.shape
    return int(_load().lpfo_count(_ptr(a), H, W, int(dx), int(dy), int(phase)))


def count_list(img, vecs) -> np.ndarray:
    """int64 [n][2] counts (phase 0, phase 1) for vectors vecs = [(dx, dy), ...]."""
    a = _img(img)
    H, W = a.shape
    v = np.ascontiguousarray(np.asarray(vecs, dtype=np.int32).reshape(-1, 2))
    dx = np.ascontiguousarray(v[:, 0])
    dy = np.ascontiguousarray(v[:, 1])
    out = np.zeros((len(v), 2), np.int64)
    _load().lpfo_count_list(_ptr(a), H, W, _ptr(dx), _ptr(dy), len(v), _ptr(out))
    return out


def delta_swap(img, rx: int, ry: int, pairs) -> np.ndarray:
    """int64 [K][2][n_canon]: canonical-half counts after exchanging each pair minus before."""
    a = _img(img)
    H, W = a.shape
    pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    K = len(pr)
    _, n_canon, _ = window_sizes(rx, ry)
    out = np.zeros((K, 2, n_canon), np.int64)
    _load().lpfo_delta_swap(_ptr(a), H, W, rx, ry, _ptr(pr), K, _ptr(out))
    return out


def objective(target, counts, rx: int, ry: int, H: int, W: int, phases: int = 3) -> float:
    """Eq. (LSE) over the phases in the bit mask `phases` (bit p: phase p)."""
    t = np.ascontiguousarray(target, dtype=np.float32)
    c = np.ascontiguousarray(counts, dtype=np.int64)
    return float(_load().lpfo_objective(_ptr(t), _ptr(c), rx, ry, H, W, int(phases)))


def delta_objective(target, counts, dcounts, rx: int, ry: int, H: int, W: int, phases: int = 3) -> np.ndarray:
    t = np.ascontiguousarray(target, dtype=np.float32)
    c = np.ascontiguousarray(counts, dtype=np.int64)
    d = np.ascontiguousarray(dcounts, dtype=np.int64)
    K = d.shape[0]
    out = np.zeros(K, np.float64)
    _load().lpfo_delta_objective(_ptr(t), _ptr(c), _ptr(d), K, rx, ry, H, W, int(phases), _ptr(out))
    return out


def s2_counts(img) -> np.ndarray:
    """int64 [H][W] phase-1 autocorrelation counts (W*H * S2, exact)."""
    a = _img(img)
    H, W = a.shape
    out = np.zeros((H, W), np.int64)
    _load().lpfo_s2_counts(_ptr(a), H, W, _ptr(out))
    return out


def s2_delta_objective(img, target, pairs) -> np.ndarray:
    """float64 [K]: change of sum_d (t[d] - C[d]/(W H))^2 for each exchange, by recount."""
    a = _img(img)
    H, W = a.shape
    t = np.ascontiguousarray(target, dtype=np.float32)
    pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    out = np.zeros(len(pr), np.float64)
    _load().lpfo_s2_delta_objective(_ptr(a), H, W, _ptr(t), _ptr(pr), len(pr), _ptr(out))
    return out


def s2_direct(img, phase: int) -> np.ndarray:
    a = _img(img)
    H, W = a.shape
    out = np.zeros((H, W), np.float64)
    _load().lpfo_s2_direct(_ptr(a), H, W, int(phase), _ptr(out))
    return out


def window_sizes3(rx: int, ry: int, rz: int):
    """(n_full, n_canon, base) of the 3D window |dx|<=rx, |dy|<=ry, |dz|<=rz."""
    n_full = (2 * rx + 1) * (2 * ry + 1) * (2 * rz + 1)
    base = (n_full - 1) // 2
    return n_full, n_full - base, base


def full_index3(dx: int, dy: int, dz: int, rx: int, ry: int, rz: int) -> int:
    return ((dz + rz) * (2 * ry + 1) + (dy + ry)) * (2 * rx + 1) + (dx + rx)


def segment3(dx: int, dy: int, dz: int) -> np.ndarray:
    """Voxel offsets [(sx, sy, sz), ...] of the 3D segment (0,0,0) -> (dx, dy, dz)."""
    n = max(abs(dx), abs(dy), abs(dz)) + 1
    out = np.zeros((3, n), np.int32)
    m = _load().lpfo_segment3(int(dx), int(dy), int(dz), _ptr(out[0]), _ptr(out[1]), _ptr(out[2]))
    assert m == n
    return np.ascontiguousarray(out.T)


def _vol(vol) -> np.ndarray:
    a = np.ascontiguousarray(vol, dtype=np.uint8)
    assert a.ndim == 3
    return a


def count3(vol, dx: int, dy: int, dz: int, phase: int) -> int:
    a = _vol(vol)
    D, H, W = a.shape
    return int(_load().lpfo_count3(_ptr(a), D, H, W, int(dx), int(dy), int(dz), int(phase)))


def lpf_full3(vol, rx: int, ry: int, rz: int) -> np.ndarray:
    """int64 [2][(2rz+1)(2ry+1)(2rx+1)] counts of a periodic volume vol[z][y][x]."""
    a = _vol(vol)
    D, H, W = a.shape
    if not (0 <= rx < W and 0 <= ry < H and 0 <= rz < D):
        raise ValueError("window must satisfy 0 <= rx < W, 0 <= ry < H, 0 <= rz < D")
    n_full, _, _ = window_sizes3(rx, ry, rz)
    out = np.zeros((2, n_full), np.int64)
    _load().lpfo_lpf_full3(_ptr(a), D, H, W, rx, ry, rz, _ptr(out))
    return out
