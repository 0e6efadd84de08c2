"""Time of one evaluation of the lineal path function of both phases over the
full vector domain of an image (rx = W - 1, ry = H - 1), the measurement of
Sec. 3.2 / Tab. comptime, on the media of that table:

    chess    -- chess pattern of 10 x 10 px squares
    squares  -- equal-sized 4 x 4 px squares, phase-1 fraction 0.2 (the paper
                gives none), seed 7
    foam     -- stand-in for the metal-foam image (not available): the
                top-left n x n crop of a 500 x 500 foam-like medium (pores of
                radius 2-8 px, porosity 0.75, seed 5)

at 10^2 ... 500^2 px.  As in the table, the one-time setup (segment
generation and upload; here the prefix-tree build, shared by the media of
one size, and the launch-shape autotune) is excluded and reported apart, and
each time is the mean of `reps` evaluations after two warm-up calls.  Three
times per case:

    tree     -- lpf_full, image and counts resident on the device
    e2e      -- lpf_full with the image copied from pinned host memory before
                and the counts copied back after, inside the timed region
    standard -- lpf_full_standard (every segment walked from scratch, the
                paper's "standard" order without shared work), device-resident

Counts of lpf_full and lpf_full_standard are compared for equality on every
case.  The inputs fit in L2 (at most 250 KB image, 16 MB counts), as they
would inside an annealing loop; no flush between evaluations.

    python -m paper_1601_04359_gb300.comptime [--sizes 10 20 50 100 200 500] [--media chess squares foam]
"""
import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import paper_1601_04359_gb300 as lpf  # noqa: E402

# Tab. comptime, seconds: (GPU standard, CPU standard, GPU enhanced, CPU enhanced)
# on a Quadro 4000 (GPU) and one core of a Xeon E5-2620 (CPU).  The foam row at
# 500^2 prints "445.2.1" for the enhanced GPU time, read as 445.2.
PAPER = {
    "chess": {10: (2.4e-3, 0.59e-3, 2.4e-3, 0.39e-3), 20: (11.9e-3, 11.9e-3, 11.1e-3, 7.8e-3),
              50: (0.15, 0.55, 0.10, 0.24), 100: (2.1, 7.0, 0.26, 0.27),
              200: (32.6, 110.9, 2.0, 1.0), 500: (318.4, 1071.1, 16.3, 6.4)},
    "squares": {10: (2.5e-3, 0.71e-3, 2.5e-3, 0.38e-3), 20: (12.9e-3, 16.0e-3, 12.5e-3, 8.2e-3),
                50: (0.16, 0.81, 0.13, 0.36), 100: (2.5, 16.1, 1.7, 7.2),
                200: (41.9, 256.3, 20.8, 78.0), 500: (411.6, 2544.0, 205.1, 789.1)},
    "foam": {10: (2.4e-3, 0.73e-3, 2.4e-3, 0.65e-3), 20: (12.0e-3, 13.8e-3, 11.9e-3, 9.7e-3),
             50: (0.17, 1.31, 0.15, 0.67), 100: (2.8, 31.9, 2.22, 17.2),
             200: (48.3, 577.9, 32.9, 241.7), 500: (542.1, 7911.7, 445.2, 3884.2)},
}

_FOAM = {}


def medium(name: str, n: int):
    import synth
    if name == "chess":
        return synth.chess(n, n, 10)
    if name == "squares":
        return synth.squares(n, n, 4, 0.2, seed=7)
    if name == "foam":
        if "big" not in _FOAM:
            _FOAM["big"] = synth.foam(500, 500, 0.75, seed=5)
        return _FOAM["big"][:n, :n].copy()
    raise ValueError(name)


def _mean_ms(fn, reps, stream):
    import torch
    for _ in range(2):
        fn()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    torch.cuda.synchronize()
    for a, b in ev:
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev) / reps


def case(name: str, n: int, paths, reps: int = 5, standard: bool = True):
    import torch
    img = medium(name, n)
    stream = torch.cuda.current_stream()
    t0 = time.time()
    d_img = torch.from_numpy(img).cuda()
    counts = torch.empty((2, paths.n_full), dtype=torch.int64, device="cuda")
    shape = lpf.lpf_autotune_full(d_img, paths, counts)
    torch.cuda.synchronize()
    setup_s = time.time() - t0

    tree_ms = _mean_ms(lambda: lpf.lpf_full(d_img, paths, counts), reps, stream)
    executed, nominal = lpf.lpf_paths_work(paths)
    h_img = torch.from_numpy(img).pin_memory()
    h_counts = torch.empty((2, paths.n_full), dtype=torch.int64).pin_memory()

    def e2e():
        d_img.copy_(h_img, non_blocking=True)
        lpf.lpf_full(d_img, paths, counts)
        h_counts.copy_(counts, non_blocking=True)
    e2e_ms = _mean_ms(e2e, reps, stream)
    row = {"medium": name, "dim": n, "fraction": float(img.mean()), "n_vec_half": paths.n_canon,
           "n_tree_nodes": lpf.lpf_paths_stats(paths)["n_tree_nodes"], "autotune_s": setup_s, "shape": shape,
           "tree_ms": tree_ms, "walked_share": executed / nominal if nominal else 1.0, "e2e_ms": e2e_ms,
           "tests_per_s": 2.0 * n * n * paths.n_full / (tree_ms / 1e3)}
    if standard:
        c_std = torch.empty_like(counts)
        row["standard_ms"] = _mean_ms(lambda: lpf.lpf_full_standard(d_img, paths, c_std), reps, stream)
        row["standard_equal"] = bool(torch.equal(c_std, counts))
    assert lpf.lpf_paths_status(paths) == 0
    assert torch.equal(h_counts, counts.cpu())
    p = PAPER.get(name, {}).get(n)
    if p:
        row["paper_s"] = {"gpu_std": p[0], "cpu_std": p[1], "gpu_enh": p[2], "cpu_enh": p[3]}
        # speed-ups of the e2e time over the paper's fastest GPU and CPU variants
        row["x_paper_gpu"] = min(p[0], p[2]) / (e2e_ms / 1e3)
        row["x_paper_cpu"] = min(p[1], p[3]) / (e2e_ms / 1e3)
    return row


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--sizes", type=int, nargs="+", default=[10, 20, 50, 100, 200, 500])
    ap.add_argument("--media", nargs="+", default=["chess", "squares", "foam"], choices=list(PAPER))
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--no-standard", action="store_true")
    a = ap.parse_args()
    lpf.load()
    rows = []
    for n in a.sizes:
        t0 = time.time()
        paths = lpf.lpf_build_paths(n - 1, n - 1)
        build_s = time.time() - t0
        for m in a.media:
            r = case(m, n, paths, a.reps, not a.no_standard)
            r["paths_build_s"] = build_s
            print(json.dumps(r), file=sys.stderr, flush=True)
            rows.append(r)
        del paths
    print(json.dumps(rows))


if __name__ == "__main__":
    main()
