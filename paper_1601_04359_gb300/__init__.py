"""Python binding of liblpf, the GB300 (sm_103a) lineal-path-function library.

Every function here marshals arguments to the C ABI declared in
``include/lpf.h`` and returns; all computation runs in the library's CUDA
kernels.  PyTorch is used only to own device memory and to name streams.
There is no CPU fallback: if the library cannot be loaded or a call fails,
an exception is raised.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

__all__ = [
    "load", "LpfError", "Paths", "lpf_build_paths", "lpf_paths_info", "lpf_paths_export", "lpf_paths_stats",
    "lpf_paths_work",
    "lpf_full", "lpf_full_standard", "lpf_paths_status", "lpf_paths_set_timer", "lpf_delta_swap",
    "lpf_full_mc", "lpf_autotune_full", "lpf_set_launch_shape", "lpf_strerror", "SaParams", "SaStats",
    "Annealer", "lpf_sa_create", "lpf_sa_run", "lpf_sa_read", "lpf_sa_recompute_error", "lpf_sa_propose",
    "lpf_sa_selftest_timeout", "lpf_delta_swap_mc", "lpf_sa_create_mc", "lpf_full_ensemble", "SaProgress",
    "lpf_sa_export_progress", "lpf_sa_import_progress", "save_checkpoint", "load_checkpoint",
    "lpf_cnn_set_loss", "s2_fft", "s2_counts", "s2_delta_swap", "s2_sa_create", "Cnn", "lpf_cnn_create",
    "lpf_cnn_set_params", "lpf_cnn_get_params", "lpf_cnn_forward", "lpf_cnn_gradients", "lpf_cnn_train_step",
    "lpf_sa_set_proposer", "Batch", "lpf_batch_create", "lpf_batch_run", "lpf_batch_autotune",
    "lpf_batch_status", "lpf_batch_work", "lpf_set_checked", "lpf_paths_set_selftest", "LPF_EPIXEL", "LPF_ETIMEOUT",
    "lpf_build_paths_3d", "lpf_full_3d",
]

LPF_ETIMEOUT = -4
LPF_EPIXEL = -6

_lib = None
LIB_PATH = _build.LIB


class SaParams(ctypes.Structure):
    """lpf_sa_params of include/lpf.h."""
    _fields_ = [("n_step", ctypes.c_int64), ("c_max", ctypes.c_int64), ("s_max", ctypes.c_int64),
                ("t_max", ctypes.c_double), ("t_min_ratio", ctypes.c_double), ("k_max", ctypes.c_int32),
                ("k_min", ctypes.c_int32), ("seed", ctypes.c_uint64), ("phases", ctypes.c_int32)]


class SaStats(ctypes.Structure):
    """lpf_sa_stats of include/lpf.h."""
    _fields_ = [("n_eval", ctypes.c_int64), ("n_accept", ctypes.c_int64), ("n_batches", ctypes.c_int64),
                ("n_candidates", ctypes.c_int64), ("temperature", ctypes.c_double), ("error", ctypes.c_double),
                ("t_max", ctypes.c_double), ("next_batch", ctypes.c_int32), ("done", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class SaProgress(ctypes.Structure):
    """lpf_sa_progress of include/lpf.h."""
    _fields_ = [("n_eval", ctypes.c_int64), ("n_accept", ctypes.c_int64), ("n_batches", ctypes.c_int64),
                ("n_candidates", ctypes.c_int64), ("c_stage", ctypes.c_int64), ("s_stage", ctypes.c_int64),
                ("temperature", ctypes.c_double), ("error", ctypes.c_double), ("p_est", ctypes.c_double),
                ("t_max", ctypes.c_double), ("next_batch", ctypes.c_int32), ("done", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("n_step", ctypes.c_int64), ("c_max", ctypes.c_int64),
                ("s_max", ctypes.c_int64), ("t_min_ratio", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class LpfError(RuntimeError):
    def __init__(self, code: int, what: str):
        detail = ""
        if code == -3 and _lib is not None:
            detail = " [" + _lib.lpf_last_error_message().decode() + "]"
        super().__init__(f"{what}: {lpf_strerror(code)} ({code}){detail}")
        self.code = code


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load liblpf.so (building it in-tree first when it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"liblpf not built: {path}")
    lib = ctypes.CDLL(path)
    i32, i64, p = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
    P64 = ctypes.POINTER(ctypes.c_int64)
    P32 = ctypes.POINTER(ctypes.c_int32)
    sig = {
        "lpf_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "lpf_last_error_message": (ctypes.c_char_p, []),
        "lpf_build_paths": (ctypes.c_int, [i32, i32, ctypes.POINTER(p)]),
        "lpf_paths_info": (ctypes.c_int, [p, P64, P64, P64]),
        "lpf_paths_export": (ctypes.c_int, [p, p, p, p]),
        "lpf_paths_stats": (ctypes.c_int, [p, P64, P32, P32]),
        "lpf_paths_work": (ctypes.c_int, [p, P64, P64]),
        "lpf_paths_free": (None, [p]),
        "lpf_full": (ctypes.c_int, [p, i32, i32, p, p, p]),
        "lpf_full_standard": (ctypes.c_int, [p, i32, i32, p, p, p]),
        "lpf_paths_status": (ctypes.c_int, [p, p]),
        "lpf_paths_set_timer": (ctypes.c_int, [p, p, p]),
        "lpf_delta_swap": (ctypes.c_int, [p, i32, i32, p, p, i32, p, p, p, p, p]),
        "lpf_autotune_full": (ctypes.c_int, [p, i32, i32, p, p, p, P32, P32]),
        "lpf_set_launch_shape": (ctypes.c_int, [p, i32, i32, i32, i32]),
        "lpf_full_noalloc": (ctypes.c_int, [p, i32, i32, p, p, p]),
        "lpf_full_mc": (ctypes.c_int, [p, i32, i32, p, p, p, p]),
        "s2_fft": (ctypes.c_int, [p, i32, i32, i32, p, p]),
        "s2_counts": (ctypes.c_int, [p, i32, i32, p, p]),
        "lpf_cnn_set_loss": (ctypes.c_int, [p, i32, ctypes.c_float]),
        "lpf_sa_export_progress": (ctypes.c_int, [p, ctypes.POINTER(SaProgress), p]),
        "lpf_sa_import_progress": (ctypes.c_int, [p, ctypes.POINTER(SaProgress), p]),
        "lpf_full_ensemble": (ctypes.c_int, [p, i32, i32, i32, p, p, p]),
        "lpf_delta_swap_mc": (ctypes.c_int, [p, i32, i32, p, p, p, i32, p, p, p, p, p]),
        "lpf_sa_create_mc": (ctypes.c_int, [p, i32, i32, p, p, p, p, ctypes.POINTER(SaParams), p, ctypes.POINTER(p)]),
        "lpf_sa_selftest_timeout": (ctypes.c_int, [p, i32, p]),
        "lpf_set_checked": (ctypes.c_int, [p, i32]),
        "lpf_build_paths_3d": (ctypes.c_int, [i32, i32, i32, ctypes.POINTER(p)]),
        "lpf_full_3d": (ctypes.c_int, [p, i32, i32, i32, p, p, p]),
        "lpf_paths_set_selftest": (ctypes.c_int, [p, i32]),
        "s2_delta_swap": (ctypes.c_int, [p, i32, i32, p, i32, p, p, p, p, p]),
        "s2_sa_create": (ctypes.c_int, [p, i32, i32, p, p, ctypes.POINTER(SaParams), p, ctypes.POINTER(p)]),
        "lpf_cnn_create": (ctypes.c_int, [i32, i32, ctypes.c_uint64, ctypes.POINTER(p)]),
        "lpf_cnn_num_params": (ctypes.c_int64, [p]),
        "lpf_cnn_set_params": (ctypes.c_int, [p, p, i64]),
        "lpf_cnn_get_params": (ctypes.c_int, [p, p, i64]),
        "lpf_cnn_forward": (ctypes.c_int, [p, p, p, p]),
        "lpf_cnn_gradients": (ctypes.c_int, [p, p, p, p, i32, p, p, p]),
        "lpf_cnn_train_step": (ctypes.c_int, [p, p, i32, p, p, i32, ctypes.c_float, p, p]),
        "lpf_cnn_free": (None, [p]),
        "lpf_sa_set_proposer": (ctypes.c_int, [p, p, ctypes.c_float, ctypes.c_float, i32]),
        "lpf_batch_create": (ctypes.c_int, [i32, p, p, p, p, p, p, ctypes.POINTER(p)]),
        "lpf_batch_run": (ctypes.c_int, [p, i32, p]),
        "lpf_batch_autotune": (ctypes.c_int, [p, p, p, p, p, p, p]),
        "lpf_batch_status": (ctypes.c_int, [p, p]),
        "lpf_batch_work": (ctypes.c_int, [p, p, p, p]),
        "lpf_batch_free": (None, [p]),
        "lpf_sa_create": (ctypes.c_int, [p, i32, i32, p, p, p, ctypes.POINTER(SaParams), p, ctypes.POINTER(p)]),
        "lpf_sa_run": (ctypes.c_int, [p, i32, p]),
        "lpf_sa_read": (ctypes.c_int, [p, ctypes.POINTER(SaStats), p]),
        "lpf_sa_recompute_error": (ctypes.c_int, [p, ctypes.POINTER(ctypes.c_double), p]),
        "lpf_sa_propose": (ctypes.c_int, [p, i32, p, p, p]),
        "lpf_sa_free": (None, [p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def lpf_strerror(code: int) -> str:
    return load().lpf_strerror(int(code)).decode()


def _check(rc: int, what: str):
    if rc != 0:
        raise LpfError(rc, what)


def _stream_ptr(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dev_ptr(t, dtype_name: str, what: str) -> int:
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what} must be a CUDA tensor")
    if str(t.dtype) != f"torch.{dtype_name}":
        raise TypeError(f"{what} must be {dtype_name}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    return t.data_ptr()


class Paths:
    """Owning wrapper of an ``lpf_paths*`` handle (freed on garbage collection)."""

    def __init__(self, handle: int, rx: int, ry: int, rz: int | None = None):
        self.handle = handle
        self.rx, self.ry = rx, ry
        self.rz = rz
        self.dims = 2 if rz is None else 3
        self.n_full, self.n_canon, self.n_offsets = lpf_paths_info(self)
        self.base = (self.n_full - 1) // 2

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            _lib.lpf_paths_free(h)
            self.handle = None


def lpf_build_paths(rx: int, ry: int) -> Paths:
    h = ctypes.c_void_p()
    _check(load().lpf_build_paths(int(rx), int(ry), ctypes.byref(h)), "lpf_build_paths")
    return Paths(h.value, int(rx), int(ry))


def lpf_paths_info(paths: Paths):
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(load().lpf_paths_info(paths.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "lpf_paths_info")
    return a.value, b.value, c.value


def lpf_paths_export(paths: Paths):
    """(vec [n_canon][dims] int16, ptr [n_canon+1] int64, off [n_offsets][dims] int16); dims = 2 or 3."""
    vec = np.zeros((paths.n_canon, paths.dims), np.int16)
    ptr = np.zeros(paths.n_canon + 1, np.int64)
    off = np.zeros((paths.n_offsets, paths.dims), np.int16)
    _check(load().lpf_paths_export(paths.handle, vec.ctypes.data, ptr.ctypes.data, off.ctypes.data),
           "lpf_paths_export")
    return vec, ptr, off


def lpf_paths_stats(paths: Paths):
    a, b, c = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
    _check(load().lpf_paths_stats(paths.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
           "lpf_paths_stats")
    return {"n_tree_nodes": a.value, "stack_depth": b.value, "n_pieces": c.value}


def lpf_paths_work(paths: Paths):
    """(executed, nominal) pixel words ANDed by the walk warps in the last
    full evaluation with this handle, with and without the zero-count skip."""
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(load().lpf_paths_work(paths.handle, ctypes.byref(a), ctypes.byref(b)), "lpf_paths_work")
    return a.value, b.value


def lpf_full(img, paths: Paths, counts=None, stream=None):
    """Counts of both phases for every vector: int64 CUDA tensor [2][n_full]."""
    import torch
    H, W = img.shape
    if counts is None:
        counts = torch.empty((2, paths.n_full), dtype=torch.int64, device=img.device)
    _check(load().lpf_full(_dev_ptr(img, "uint8", "img"), H, W, paths.handle,
                           _dev_ptr(counts, "int64", "counts"), _stream_ptr(stream)), "lpf_full")
    return counts


def lpf_build_paths_3d(rx: int, ry: int, rz: int) -> Paths:
    """Segments of every vector |dx|<=rx, |dy|<=ry, |dz|<=rz of a volume (3D extension)."""
    h = ctypes.c_void_p()
    _check(load().lpf_build_paths_3d(int(rx), int(ry), int(rz), ctypes.byref(h)), "lpf_build_paths_3d")
    return Paths(h.value, int(rx), int(ry), int(rz))


def lpf_full_3d(vol, paths: Paths, counts=None, stream=None):
    """Counts of both phases of a periodic volume (uint8 CUDA tensor [D][H][W]) for every vector."""
    import torch
    D, H, W = vol.shape
    if counts is None:
        counts = torch.empty((2, paths.n_full), dtype=torch.int64, device=vol.device)
    _check(load().lpf_full_3d(_dev_ptr(vol, "uint8", "vol"), D, H, W, paths.handle,
                              _dev_ptr(counts, "int64", "counts"), _stream_ptr(stream)), "lpf_full_3d")
    return counts


def lpf_full_mc(img, paths: Paths, sel, counts=None, stream=None):
    """Counts over the selected translations only (sel: uint8 CUDA tensor H x W)."""
    import torch
    H, W = img.shape
    if counts is None:
        counts = torch.empty((2, paths.n_full), dtype=torch.int64, device=img.device)
    _check(load().lpf_full_mc(_dev_ptr(img, "uint8", "img"), H, W, paths.handle, _dev_ptr(sel, "uint8", "sel"),
                              _dev_ptr(counts, "int64", "counts"), _stream_ptr(stream)), "lpf_full_mc")
    return counts


def lpf_autotune_full(img, paths: Paths, counts=None, stream=None):
    """Pick the fastest walk-kernel launch shape for this image size; returns (T, BB)."""
    import torch
    H, W = img.shape
    if counts is None:
        counts = torch.empty((2, paths.n_full), dtype=torch.int64, device=img.device)
    t, b = ctypes.c_int32(), ctypes.c_int32()
    _check(load().lpf_autotune_full(_dev_ptr(img, "uint8", "img"), H, W, paths.handle,
                                    _dev_ptr(counts, "int64", "counts"), _stream_ptr(stream),
                                    ctypes.byref(t), ctypes.byref(b)), "lpf_autotune_full")
    return t.value, b.value


def lpf_set_launch_shape(paths: Paths, H: int, W: int, T: int, BB: int):
    _check(load().lpf_set_launch_shape(paths.handle, int(H), int(W), int(T), int(BB)), "lpf_set_launch_shape")


def lpf_set_checked(paths: Paths, on: bool = True):
    """Checked mode: kernels that read an image flag pixels other than 0/1 (lpf_paths_status -> LPF_EPIXEL)."""
    _check(load().lpf_set_checked(paths.handle, int(bool(on))), "lpf_set_checked")


def lpf_paths_set_selftest(paths: Paths, on: bool = True):
    """Failure-detection self-test of the walk kernel's staging wait (tests only)."""
    _check(load().lpf_paths_set_selftest(paths.handle, int(bool(on))), "lpf_paths_set_selftest")


def lpf_full_ensemble(imgs, paths: Paths, counts=None, stream=None):
    """Summed counts of the images imgs (uint8 CUDA [n][H][W]); divide by n*H*W for the ensemble average."""
    import torch
    n, H, W = imgs.shape
    if counts is None:
        counts = torch.empty((2, paths.n_full), dtype=torch.int64, device=imgs.device)
    _check(load().lpf_full_ensemble(_dev_ptr(imgs, "uint8", "imgs"), n, H, W, paths.handle,
                                    _dev_ptr(counts, "int64", "counts"), _stream_ptr(stream)), "lpf_full_ensemble")
    return counts


def lpf_full_standard(img, paths: Paths, counts=None, stream=None):
    import torch
    H, W = img.shape
    if counts is None:
        counts = torch.empty((2, paths.n_full), dtype=torch.int64, device=img.device)
    _check(load().lpf_full_standard(_dev_ptr(img, "uint8", "img"), H, W, paths.handle,
                                    _dev_ptr(counts, "int64", "counts"), _stream_ptr(stream)),
           "lpf_full_standard")
    return counts


def lpf_delta_swap(img, paths: Paths, pairs, dcounts=None, target=None, counts=None, de=None,
                   want_dcounts: bool = True, want_de: bool = False, stream=None):
    """Count changes (int32 [K][2][n_canon]) and/or error changes (float32 [K])
    for candidate exchanges pairs (int32 CUDA tensor [K][2])."""
    import torch
    H, W = img.shape
    K = int(pairs.shape[0])
    if want_dcounts and dcounts is None:
        dcounts = torch.empty((K, 2, paths.n_canon), dtype=torch.int32, device=img.device)
    if want_de and de is None:
        de = torch.empty(K, dtype=torch.float32, device=img.device)
    _check(load().lpf_delta_swap(
        _dev_ptr(img, "uint8", "img"), H, W, paths.handle, _dev_ptr(pairs, "int32", "pairs"), K,
        _dev_ptr(dcounts, "int32", "dcounts") if dcounts is not None else None,
        _dev_ptr(target, "float32", "target") if target is not None else None,
        _dev_ptr(counts, "int64", "counts") if counts is not None else None,
        _dev_ptr(de, "float32", "de") if de is not None else None,
        _stream_ptr(stream)), "lpf_delta_swap")
    return dcounts, de


def lpf_delta_swap_mc(img, paths: Paths, sel, pairs, target=None, counts=None, want_dcounts: bool = True,
                      want_de: bool = False, stream=None):
    """lpf_delta_swap restricted to the translations sampled in sel (uint8 CUDA [H][W])."""
    import torch
    H, W = img.shape
    K = int(pairs.shape[0])
    dcounts = torch.empty((K, 2, paths.n_canon), dtype=torch.int32, device=img.device) if want_dcounts else None
    de = torch.empty(K, dtype=torch.float32, device=img.device) if want_de else None
    _check(load().lpf_delta_swap_mc(
        _dev_ptr(img, "uint8", "img"), H, W, paths.handle, _dev_ptr(sel, "uint8", "sel"),
        _dev_ptr(pairs, "int32", "pairs"), K,
        _dev_ptr(dcounts, "int32", "dcounts") if dcounts is not None else None,
        _dev_ptr(target, "float32", "target") if target is not None else None,
        _dev_ptr(counts, "int64", "counts") if counts is not None else None,
        _dev_ptr(de, "float32", "de") if de is not None else None,
        _stream_ptr(stream)), "lpf_delta_swap_mc")
    return dcounts, de


def lpf_paths_set_timer(paths: Paths, ev_start=None, ev_stop=None):
    """Record torch.cuda.Event pair around the dominant kernel of later calls."""
    a = ev_start.cuda_event if ev_start is not None else None
    b = ev_stop.cuda_event if ev_stop is not None else None
    _check(load().lpf_paths_set_timer(paths.handle, a, b), "lpf_paths_set_timer")


class Batch:
    """Owning wrapper of an lpf_batch* (keeps the bound tensors and handles alive)."""

    def __init__(self, handle, imgs, paths, counts, arrays):
        self.handle = handle
        self.imgs, self.paths, self.counts = imgs, paths, counts
        self._arrays = arrays

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            _lib.lpf_batch_free(h)
            self.handle = None


def _batch_arrays(imgs, paths, counts):
    n = len(imgs)
    ptrs = (ctypes.c_void_p * n)(*[_dev_ptr(t, "uint8", "img") for t in imgs])
    Hs = (ctypes.c_int32 * n)(*[int(t.shape[0]) for t in imgs])
    Ws = (ctypes.c_int32 * n)(*[int(t.shape[1]) for t in imgs])
    hs = (ctypes.c_void_p * n)(*[p.handle for p in paths])
    cs = (ctypes.c_void_p * n)(*[_dev_ptr(c, "int64", "counts") for c in counts])
    return ptrs, Hs, Ws, hs, cs


def lpf_batch_create(imgs, paths, counts=None, words_per_thread=None) -> Batch:
    """Bind CUDA uint8 images, their paths handles and int64 count buffers."""
    import torch
    if counts is None:
        counts = [torch.empty((2, p.n_full), dtype=torch.int64, device=t.device) for t, p in zip(imgs, paths)]
    arrays = _batch_arrays(imgs, paths, counts)
    wpt = None
    if words_per_thread is not None:
        wpt = (ctypes.c_int32 * len(imgs))(*[int(x) for x in words_per_thread])
    h = ctypes.c_void_p()
    _check(load().lpf_batch_create(len(imgs), *arrays, wpt, ctypes.byref(h)), "lpf_batch_create")
    return Batch(h.value, list(imgs), list(paths), counts, arrays)


def lpf_batch_run(batch: Batch, use_graph: bool = True, stream=None):
    _check(load().lpf_batch_run(batch.handle, 1 if use_graph else 0, _stream_ptr(stream)), "lpf_batch_run")
    return batch.counts


def lpf_batch_autotune(batch: Batch, stream=None):
    n = len(batch.imgs)
    chosen = (ctypes.c_int32 * n)()
    ptrs, Hs, Ws, _, cs = batch._arrays
    _check(load().lpf_batch_autotune(batch.handle, ptrs, Hs, Ws, cs, _stream_ptr(stream), chosen),
           "lpf_batch_autotune")
    return list(chosen)


def lpf_batch_status(batch: Batch, stream=None) -> int:
    return int(load().lpf_batch_status(batch.handle, _stream_ptr(stream)))


def lpf_batch_work(batch: Batch, stream=None):
    """Per image of the last run: (executed, nominal) pixel words ANDed by the
    walk warps, with and without the zero-count skip (numpy int64 arrays)."""
    import numpy as np
    n = len(batch.imgs)
    ex, nom = np.zeros(n, np.int64), np.zeros(n, np.int64)
    _check(load().lpf_batch_work(batch.handle, ex.ctypes.data, nom.ctypes.data, _stream_ptr(stream)),
           "lpf_batch_work")
    return ex, nom


class Annealer:
    """Owning wrapper of an lpf_sa* run (keeps its device buffers alive)."""

    def __init__(self, handle, cell, paths, target, counts):
        self.handle = handle
        self.cell, self.paths, self.target, self.counts = cell, paths, target, counts

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            _lib.lpf_sa_free(h)
            self.handle = None


def _sa_params(n_step, c_max, s_max, t_max, t_min_ratio, k_max, k_min, seed, phases) -> SaParams:
    return SaParams(int(n_step), int(c_max if c_max is not None else max(1, n_step // 10)),
                    int(s_max if s_max is not None else max(1, n_step // 100)), float(t_max), float(t_min_ratio),
                    int(k_max), int(k_min), int(seed), int(phases))


def lpf_sa_create(cell, paths: Paths, target, counts=None, n_step=1_000_000, c_max=None, s_max=None,
                  t_max=0.0, t_min_ratio=0.01, k_max=4096, k_min=1, seed=1, phases=3, stream=None) -> Annealer:
    """Start an annealing run on the CUDA uint8 cell (modified in place).
    phases: bit mask of the phases in the lineal-path error (3 both, 2 phase 1, 1 phase 0)."""
    import torch
    H, W = cell.shape
    if counts is None:
        counts = torch.empty((2, paths.n_full), dtype=torch.int64, device=cell.device)
    prm = _sa_params(n_step, c_max, s_max, t_max, t_min_ratio, k_max, k_min, seed, phases)
    h = ctypes.c_void_p()
    _check(load().lpf_sa_create(_dev_ptr(cell, "uint8", "cell"), H, W, paths.handle,
                                _dev_ptr(target, "float32", "target"), _dev_ptr(counts, "int64", "counts"),
                                ctypes.byref(prm), _stream_ptr(stream), ctypes.byref(h)), "lpf_sa_create")
    return Annealer(h.value, cell, paths, target, counts)


def lpf_sa_run(sa: Annealer, n_batches: int, stream=None):
    _check(load().lpf_sa_run(sa.handle, int(n_batches), _stream_ptr(stream)), "lpf_sa_run")


def lpf_sa_read(sa: Annealer, stream=None) -> dict:
    st = SaStats()
    _check(load().lpf_sa_read(sa.handle, ctypes.byref(st), _stream_ptr(stream)), "lpf_sa_read")
    return st.as_dict()


def lpf_sa_recompute_error(sa: Annealer, stream=None) -> float:
    e = ctypes.c_double()
    _check(load().lpf_sa_recompute_error(sa.handle, ctypes.byref(e), _stream_ptr(stream)), "lpf_sa_recompute_error")
    return e.value


def lpf_cnn_set_loss(net, kind: str = "squared", beta: float = 1.0):
    """Training loss of the network: "squared" (default) or "listwise"."""
    _check(load().lpf_cnn_set_loss(net.handle, {"squared": 0, "listwise": 1}[kind], float(beta)), "lpf_cnn_set_loss")


def lpf_sa_export_progress(sa: Annealer, stream=None) -> dict:
    pr = SaProgress()
    _check(load().lpf_sa_export_progress(sa.handle, ctypes.byref(pr), _stream_ptr(stream)), "lpf_sa_export_progress")
    return pr.as_dict()


def lpf_sa_import_progress(sa: Annealer, progress: dict, stream=None):
    pr = SaProgress(**{k: progress[k] for k, _ in SaProgress._fields_})
    _check(load().lpf_sa_import_progress(sa.handle, ctypes.byref(pr), _stream_ptr(stream)), "lpf_sa_import_progress")


def save_checkpoint(sa: Annealer, path: str, stream=None):
    """Write the run's cell and progress to an .npz file (the counts follow
    from the cell and are recomputed on resume)."""
    import numpy as np
    pr = lpf_sa_export_progress(sa, stream)
    np.savez(path, cell=sa.cell.cpu().numpy(), **{k: np.asarray(v) for k, v in pr.items()})


def load_checkpoint(path: str, paths: Paths, target, k_max=4096, k_min=1, phases=3, stream=None) -> Annealer:
    """Resume a lineal-path run from save_checkpoint's file: an annealer on
    the saved cell with the saved parameters and progress."""
    import numpy as np
    import torch
    z = np.load(path)
    pr = {k: z[k].item() for k, _ in SaProgress._fields_}
    cell = torch.from_numpy(z["cell"]).to(target.device)
    ann = lpf_sa_create(cell, paths, target, n_step=pr["n_step"], c_max=pr["c_max"], s_max=pr["s_max"],
                        t_max=pr["t_max"], t_min_ratio=pr["t_min_ratio"], k_max=k_max, k_min=k_min, seed=pr["seed"],
                        phases=phases, stream=stream)
    lpf_sa_import_progress(ann, pr, stream)
    return ann


def lpf_sa_selftest_timeout(sa: Annealer, block: int = -1, stream=None) -> int:
    """Status code of the annealer's timeout check (0: the bounded grid-barrier
    wait of every block (block=-1) or of one block ran out, was reported, and
    the run state was made consistent again)."""
    return int(load().lpf_sa_selftest_timeout(sa.handle, int(block), _stream_ptr(stream)))


def lpf_sa_propose(sa: Annealer, k: int, stream=None):
    import torch
    pairs = torch.empty((k, 2), dtype=torch.int32, device=sa.cell.device)
    u = torch.empty(k, dtype=torch.float32, device=sa.cell.device)
    _check(load().lpf_sa_propose(sa.handle, int(k), pairs.data_ptr(), u.data_ptr(), _stream_ptr(stream)),
           "lpf_sa_propose")
    return pairs, u


def s2_fft(img, phase: int, out=None, stream=None):
    """Two-point probability of `phase`: float32 CUDA tensor [H][W]."""
    import torch
    H, W = img.shape
    if out is None:
        out = torch.empty((H, W), dtype=torch.float32, device=img.device)
    _check(load().s2_fft(_dev_ptr(img, "uint8", "img"), H, W, int(phase), _dev_ptr(out, "float32", "s2"),
                         _stream_ptr(stream)), "s2_fft")
    return out


def lpf_sa_create_mc(cell, paths: Paths, sel, target, counts=None, n_step=1_000_000, c_max=None, s_max=None,
                     t_max=0.0, t_min_ratio=0.01, k_max=4096, k_min=1, seed=1, phases=3, stream=None) -> Annealer:
    """Annealing run on the Monte-Carlo lineal path function of the translations sampled in sel."""
    import torch
    H, W = cell.shape
    if counts is None:
        counts = torch.empty((2, paths.n_full), dtype=torch.int64, device=cell.device)
    prm = _sa_params(n_step, c_max, s_max, t_max, t_min_ratio, k_max, k_min, seed, phases)
    h = ctypes.c_void_p()
    _check(load().lpf_sa_create_mc(_dev_ptr(cell, "uint8", "cell"), H, W, paths.handle, _dev_ptr(sel, "uint8", "sel"),
                                   _dev_ptr(target, "float32", "target"), _dev_ptr(counts, "int64", "counts"),
                                   ctypes.byref(prm), _stream_ptr(stream), ctypes.byref(h)), "lpf_sa_create_mc")
    ann = Annealer(h.value, cell, paths, target, counts)
    ann.sel = sel
    return ann


def s2_counts(img, out=None, stream=None):
    """Exact phase-1 autocorrelation counts (W*H * S2): int64 CUDA tensor [H][W]."""
    import torch
    H, W = img.shape
    if out is None:
        out = torch.empty((H, W), dtype=torch.int64, device=img.device)
    _check(load().s2_counts(_dev_ptr(img, "uint8", "img"), H, W, _dev_ptr(out, "int64", "counts"),
                            _stream_ptr(stream)), "s2_counts")
    return out


def s2_delta_swap(img, pairs, target=None, counts=None, want_dcounts: bool = True, want_de: bool = False,
                  dcounts=None, de=None, stream=None):
    """S2 count changes (int32 [K][H][W]) and/or S2 error changes (float32 [K])
    for candidate exchanges pairs (int32 CUDA tensor [K][2])."""
    import torch
    H, W = img.shape
    K = int(pairs.shape[0])
    if want_dcounts and dcounts is None:
        dcounts = torch.empty((K, H, W), dtype=torch.int32, device=img.device)
    if want_de and de is None:
        de = torch.empty(K, dtype=torch.float32, device=img.device)
    _check(load().s2_delta_swap(
        _dev_ptr(img, "uint8", "img"), H, W, _dev_ptr(pairs, "int32", "pairs"), K,
        _dev_ptr(dcounts, "int32", "dcounts") if dcounts is not None else None,
        _dev_ptr(target, "float32", "target") if target is not None else None,
        _dev_ptr(counts, "int64", "counts") if counts is not None else None,
        _dev_ptr(de, "float32", "de") if de is not None else None,
        _stream_ptr(stream)), "s2_delta_swap")
    return dcounts, de


def s2_sa_create(cell, target, counts=None, n_step=1_000_000, c_max=None, s_max=None, t_max=0.0, t_min_ratio=0.01,
                 k_max=4096, k_min=1, seed=1, stream=None) -> Annealer:
    """Start an annealing run on the S2 error (target float32 [H][W] per cell offset)."""
    import torch
    H, W = cell.shape
    if counts is None:
        counts = torch.empty((H, W), dtype=torch.int64, device=cell.device)
    prm = _sa_params(n_step, c_max, s_max, t_max, t_min_ratio, k_max, k_min, seed, 0)
    h = ctypes.c_void_p()
    _check(load().s2_sa_create(_dev_ptr(cell, "uint8", "cell"), H, W, _dev_ptr(target, "float32", "target"),
                               _dev_ptr(counts, "int64", "counts"), ctypes.byref(prm), _stream_ptr(stream),
                               ctypes.byref(h)), "s2_sa_create")
    return Annealer(h.value, cell, None, target, counts)


class Cnn:
    """Owning wrapper of an lpf_cnn* (the learned swap proposer)."""

    def __init__(self, handle, H, W):
        self.handle = handle
        self.H, self.W = H, W
        self.n_params = int(load().lpf_cnn_num_params(handle))

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            _lib.lpf_cnn_free(h)
            self.handle = None


def lpf_cnn_create(H: int, W: int, seed: int = 0) -> Cnn:
    h = ctypes.c_void_p()
    _check(load().lpf_cnn_create(int(H), int(W), int(seed), ctypes.byref(h)), "lpf_cnn_create")
    return Cnn(h.value, int(H), int(W))


def lpf_cnn_set_params(cnn: Cnn, params: np.ndarray):
    a = np.ascontiguousarray(params, dtype=np.float32)
    _check(load().lpf_cnn_set_params(cnn.handle, a.ctypes.data, a.size), "lpf_cnn_set_params")


def lpf_cnn_get_params(cnn: Cnn) -> np.ndarray:
    a = np.zeros(cnn.n_params, np.float32)
    _check(load().lpf_cnn_get_params(cnn.handle, a.ctypes.data, a.size), "lpf_cnn_get_params")
    return a


def lpf_cnn_forward(cnn: Cnn, cell, stream=None):
    import torch
    out = torch.empty((cnn.H, cnn.W, 2), dtype=torch.float32, device=cell.device)
    _check(load().lpf_cnn_forward(cnn.handle, _dev_ptr(cell, "uint8", "cell"), out.data_ptr(), _stream_ptr(stream)),
           "lpf_cnn_forward")
    return out


def lpf_cnn_gradients(cnn: Cnn, cell, pairs, y, stream=None):
    import torch
    g = torch.empty(cnn.n_params, dtype=torch.float32, device=cell.device)
    loss = torch.empty(1, dtype=torch.float32, device=cell.device)
    _check(load().lpf_cnn_gradients(cnn.handle, _dev_ptr(cell, "uint8", "cell"), _dev_ptr(pairs, "int32", "pairs"),
                                    _dev_ptr(y, "float32", "y"), int(pairs.shape[0]), g.data_ptr(), loss.data_ptr(),
                                    _stream_ptr(stream)), "lpf_cnn_gradients")
    return g, loss


def lpf_cnn_train_step(cnn: Cnn, cells, pairs, y, lr: float, stream=None):
    """One Adam step on snapshots cells [B][H][W] with pairs [B][n][2], y [B][n]."""
    import torch
    loss = torch.empty(1, dtype=torch.float32, device=cells.device)
    B, n = int(pairs.shape[0]), int(pairs.shape[1])
    _check(load().lpf_cnn_train_step(cnn.handle, _dev_ptr(cells, "uint8", "cells"), B,
                                     _dev_ptr(pairs, "int32", "pairs"), _dev_ptr(y, "float32", "y"), n, float(lr),
                                     loss.data_ptr(), _stream_ptr(stream)), "lpf_cnn_train_step")
    return loss


def lpf_sa_set_proposer(sa: "Annealer", cnn, epsilon: float = 0.4, tau: float = 0.35, refresh: int = 16):
    _check(load().lpf_sa_set_proposer(sa.handle, cnn.handle if cnn is not None else None, float(epsilon),
                                      float(tau), int(refresh)), "lpf_sa_set_proposer")
    sa.cnn = cnn


def lpf_paths_status(paths: Paths, stream=None) -> int:
    return int(load().lpf_paths_status(paths.handle, _stream_ptr(stream)))
