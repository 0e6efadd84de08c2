"""Write the oracle's full lineal-path counts of the two headline workloads.

This script calls only ``oracle/`` (the plain C restatement of Alg. 1 of
Sec. 3.1) and ``synth/`` (the seeded input generators).  Nothing here comes
from the CUDA library.  Outputs, next to this file:

  lpf_ellipses_512_r256.npz
      512x512 overlapping ellipses (fraction 0.35, seed 2), window
      |dx|, |dy| <= 256, both phases.  ``counts`` = the oracle's whole
      [2][513*513] table as uint32 (every count is at most 512*512, so the
      conversion is exact), ``sha256`` = digest of the same table as
      little-endian int64 (the layout ``lpf_full`` returns).

  lpf_mixed_sizes_batch_256.json
      the 256 images of ``synth.mixed_sizes_batch(256, seed=4)`` (H, W in
      48..256, windows r = floor(W/2), floor(H/2)): per image H, W, rx, ry,
      the per-phase sums of the counts and the sha256 of the oracle's
      [2][(2ry+1)(2rx+1)] int64 table.

  lpf_delta_clustered_128.npz
      the swap-delta workload: the 128x128 clustered cell, window 64, the
      4096 candidates of ``synth.swap_candidates(cell, 4096, seed=0)`` with
      four of them replaced by identities (a == b, two phase-1 pixels, two
      phase-0 pixels) and one reversed pair (phase-0 pixel first).
      ``pairs`` int32 [4096][2], ``sample`` the 64 candidate indices
      recounted (first, last, the five special ones, 57 more at random),
      ``dcounts`` int16 [64][2][n_canon] the oracle's count changes (every
      change is at most 2*65 in magnitude), ``counts`` int32 [2][n_full]
      the oracle's counts of the cell.

Usage: python tests/golden/make_lpf_goldens.py [ellipses_512] [mixed_batch] [delta_128]
(about 20, 45 and 15 minutes on 8 cores).
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

ELLIPSES = os.path.join(HERE, "lpf_ellipses_512_r256.npz")
MIXED = os.path.join(HERE, "lpf_mixed_sizes_batch_256.json")
DELTA = os.path.join(HERE, "lpf_delta_clustered_128.npz")
DELTA_SPECIAL = (100, 101, 102, 103, 104)  # identity, two same-phase pairs, a == b, reversed


def table_sha256(counts: np.ndarray) -> str:
    """Digest of a counts table as little-endian int64, row-major."""
    return hashlib.sha256(np.ascontiguousarray(counts, dtype="<i8").tobytes()).hexdigest()


def ellipses_512() -> None:
    img = synth.ellipses_512()
    t = time.time()
    counts = oracle.lpf_full(img, 256, 256)
    assert counts.max() <= 512 * 512 and counts.min() >= 0
    np.savez_compressed(ELLIPSES, counts=counts.astype(np.uint32), sha256=np.array(table_sha256(counts)),
                        rx=256, ry=256)
    print(f"ellipses_512: {time.time() - t:.0f} s, {oracle.num_threads()} threads -> {ELLIPSES}")


def mixed_batch() -> None:
    imgs = synth.mixed_sizes_batch(256, seed=4)
    out = []
    t = time.time()
    for k, img in enumerate(imgs):
        H, W = img.shape
        rx, ry = W // 2, H // 2
        c = oracle.lpf_full(img, rx, ry)
        out.append({"H": H, "W": W, "rx": rx, "ry": ry, "sum0": int(c[0].sum()), "sum1": int(c[1].sum()),
                    "sha256": table_sha256(c)})
        if k % 32 == 31:
            print(f"mixed_batch: {k + 1} images, {time.time() - t:.0f} s", flush=True)
    with open(MIXED, "w") as f:
        json.dump({"workload": "synth.mixed_sizes_batch(256, seed=4), windows floor(W/2), floor(H/2)",
                   "digest": "sha256 of the oracle's int64 [2][(2ry+1)(2rx+1)] counts, little-endian",
                   "images": out}, f, indent=0)
    print(f"mixed_batch: {time.time() - t:.0f} s -> {MIXED}")


def delta_pairs(cell: np.ndarray) -> np.ndarray:
    """The 4096 candidates of the swap-delta workload with the special ones planted."""
    pairs = synth.swap_candidates(cell, 4096, seed=0)
    flat = cell.reshape(-1)
    ones, zeros = np.flatnonzero(flat == 1), np.flatnonzero(flat == 0)
    pairs[100] = (ones[0], ones[0])            # a == b
    pairs[101] = (ones[1], ones[2])            # both phase 1
    pairs[102] = (zeros[0], zeros[5])          # both phase 0
    pairs[103] = (zeros[7], zeros[7])          # a == b on phase 0
    pairs[104] = (pairs[104, 1], pairs[104, 0])  # phase-0 pixel first
    return pairs


def delta_128() -> None:
    cell = synth.clustered_cell_128()
    pairs = delta_pairs(cell)
    rng = np.random.default_rng(11)
    rest = [int(i) for i in rng.choice(np.arange(1, 4095), 80, replace=False) if i not in DELTA_SPECIAL][:57]
    sample = np.array(sorted({0, 4095, *DELTA_SPECIAL, *rest}), np.int64)
    assert len(sample) == 64
    t = time.time()
    d = oracle.delta_swap(cell, 64, 64, pairs[sample])
    assert np.abs(d).max() <= 2 * 65
    counts = oracle.lpf_full(cell, 64, 64)
    np.savez_compressed(DELTA, pairs=pairs, sample=sample, dcounts=d.astype(np.int16),
                        counts=counts.astype(np.int32), rx=64, ry=64)
    print(f"delta_128: {time.time() - t:.0f} s -> {DELTA}")


if __name__ == "__main__":
    which = sys.argv[1:] or ["ellipses_512", "mixed_batch", "delta_128"]
    for w in which:
        {"ellipses_512": ellipses_512, "mixed_batch": mixed_batch, "delta_128": delta_128}[w]()
