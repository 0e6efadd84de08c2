"""Run one named workload a few times, for capture under a profiler.

    python -m paper_1601_04359_gb300.profile_case lpf_full_512 [--repeat N] [--shape T BB]

Each workload does one warm-up call (which also uploads tables) and then
`repeat` calls, so a profiler can skip the first launch of a kernel and
capture the next ones.  No timing is printed: numbers taken under a profiler
are not benchmark values.
"""
import argparse
import os
import sys

import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import paper_1601_04359_gb300 as lpf  # noqa: E402
import synth  # noqa: E402


def lpf_full_512(repeat, shape=None):
    img = torch.from_numpy(synth.ellipses_512()).cuda()
    p = lpf.lpf_build_paths(256, 256)
    if shape:
        lpf.lpf_set_launch_shape(p, 512, 512, shape[0], shape[1])
    c = lpf.lpf_full(img, p)
    for _ in range(repeat):
        lpf.lpf_full(img, p, c)
    torch.cuda.synchronize()
    assert lpf.lpf_paths_status(p) == 0


def lpf_full_512_standard(repeat, shape=None):
    img = torch.from_numpy(synth.ellipses_512()).cuda()
    p = lpf.lpf_build_paths(256, 256)
    c = lpf.lpf_full_standard(img, p)
    for _ in range(repeat):
        lpf.lpf_full_standard(img, p, c)
    torch.cuda.synchronize()


def delta_128(repeat, shape=None):
    """lpf_delta_swap, 128x128 clustered cell, |v| <= 64, 4096 candidates, error changes."""
    import numpy as np
    cell = synth.clustered_512()[:128, :128].copy()
    p = lpf.lpf_build_paths(64, 64)
    d = torch.from_numpy(cell).cuda()
    counts = lpf.lpf_full(d, p)
    target = (counts.double() / cell.size).float() * 0.9
    rng = np.random.default_rng(0)
    flat = cell.reshape(-1)
    pairs = np.stack([rng.choice(np.flatnonzero(flat == 1), 4096), rng.choice(np.flatnonzero(flat == 0), 4096)], 1)
    pairs = torch.from_numpy(pairs.astype(np.int32)).cuda()
    for _ in range(1 + repeat):
        lpf.lpf_delta_swap(d, p, pairs, target=target, counts=counts, want_dcounts=False, want_de=True)
    torch.cuda.synchronize()


def sa_128(repeat, shape=None):
    """Annealing batches on the 128x128 compression workload (one persistent launch of the batches)."""
    orig = synth.clustered_512()
    p = lpf.lpf_build_paths(64, 64)
    c = lpf.lpf_full(torch.from_numpy(orig).cuda(), p)
    target = (c.double() / float(orig.size)).float()
    cell = torch.from_numpy(synth.exact_fraction_shuffle(128, 128, int(round(orig.mean() * 128 * 128)), seed=5)).cuda()
    ann = lpf.lpf_sa_create(cell, p, target, n_step=10 ** 6, seed=1)
    lpf.lpf_sa_run(ann, 8 + repeat)
    torch.cuda.synchronize()


WORKLOADS = {"lpf_full_512": lpf_full_512, "lpf_full_512_standard": lpf_full_512_standard, "delta_128": delta_128,
             "sa_128": sa_128}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workload", choices=sorted(WORKLOADS))
    ap.add_argument("--repeat", type=int, default=2)
    ap.add_argument("--shape", type=int, nargs=2, metavar=("T", "BB"),
                    help="walk-kernel launch shape (lpf_full workloads; default: the built-in choice)")
    a = ap.parse_args()
    lpf.load()
    WORKLOADS[a.workload](a.repeat, a.shape)


if __name__ == "__main__":
    main()
