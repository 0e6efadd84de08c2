"""Run one named workload a few times, for capture under a profiler.

    python -m paper_1601_04359_gb300.profile_case lpf_full_512 [--repeat N]

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


def lpf_full_512(repeat):
    img = torch.from_numpy(synth.config2_image()).cuda()
    p = lpf.lpf_build_paths(256, 256)
    c = lpf.lpf_full(img, p)
    for _ in range(repeat):
        lpf.lpf_full(img, p, c)
    torch.cuda.synchronize()
    assert lpf.lpf_paths_status(p) == 0


def lpf_full_512_standard(repeat):
    img = torch.from_numpy(synth.config2_image()).cuda()
    p = lpf.lpf_build_paths(256, 256)
    c = lpf.lpf_full_standard(img, p)
    for _ in range(repeat):
        lpf.lpf_full_standard(img, p, c)
    torch.cuda.synchronize()


WORKLOADS = {"lpf_full_512": lpf_full_512, "lpf_full_512_standard": lpf_full_512_standard}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workload", choices=sorted(WORKLOADS))
    ap.add_argument("--repeat", type=int, default=2)
    a = ap.parse_args()
    lpf.load()
    WORKLOADS[a.workload](a.repeat)


if __name__ == "__main__":
    main()
