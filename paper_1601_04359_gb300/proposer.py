"""Learned swap proposer: data collection, training and evaluation.

Orchestration only -- every step runs in the library's kernels (annealing
batches, exact swap deltas, network forward/backward and Adam).

Data: while a uniform-proposal annealing run progresses, every `gap` batches
the current cell is copied and the next `n` candidates the annealer would
draw are evaluated exactly (lpf_delta_swap); their error changes, standardised
within the snapshot (y = -(de - mean) / std, clipped to [-3, 3]), are the
targets of the additive pair score s1[a] + s0[b].

Training data come from uniform-proposal runs with seeds distinct from the
evaluation seeds (an optional second round adds candidates drawn by runs that
already use the network; measured, it lowers the gain).

Evaluation (swaps to target error), two protocols.  First crossing: for each
evaluation seed, a uniform run of N evaluations reaches error e_U; the
model-proposal run (same initial cell, seed and temperature schedule, the
schedule of an N-evaluation run) is followed until its error first falls to
e_U; the ratio of evaluations is the gain, reported as the median over seeds.
Own budget: annealers with a budget of N/k evaluations (each with the
schedule of its budget) end at e_M(k) with the network's proposals and at
e_u(k) with uniform ones; a seed's gain is the largest k such that every
budget N/j, j <= k, reached e_M(j) <= e_U; the control's the same for e_u.

    python -m paper_1601_04359_gb300.proposer --evaluate [--n-step 100000]
    python -m paper_1601_04359_gb300.proposer --evaluate-budget [--ks 2 3 4 6]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import paper_1601_04359_gb300 as lpf  # noqa: E402


def annealing_problem(r: int = 64, cell_size: int = 128, seed: int = 5, orig_size: int = 512):
    """The compression workload: target = lineal path function (|v| <= r) of a
    clustered-disk original (the 512x512 one of the annealing workload, or
    an orig_size^2 one with fraction 0.3); random initial cell with its fraction."""
    import torch

    import synth
    orig = synth.clustered_512() if orig_size == 512 else synth.clustered_disks(orig_size, orig_size, 0.3, seed=9)
    paths = lpf.lpf_build_paths(r, r)
    c = lpf.lpf_full(torch.from_numpy(orig).cuda(), paths)
    target = (c.double() / float(orig.size)).float()
    n1 = int(round(orig.mean() * cell_size * cell_size))
    cell0 = synth.exact_fraction_shuffle(cell_size, cell_size, n1, seed=seed)
    return paths, target, cell0


def collect(paths, target, cell0, n_step: int, seed: int, snapshots: int, n: int, t_max: float = 0.0,
            net=None, eps: float = 0.1, tau: float = 1.0, spacing: str = "evals"):
    """Run an annealer (uniform proposals, or the network's when `net` is
    given) and log `snapshots` snapshots of the next `n` candidates it would
    draw, each evaluated exactly.  spacing = "evals": snapshots evenly spaced
    in evaluations; "early": spaced by n_step / (2 snapshots) batches, which
    puts more of them where batches are short (early, high acceptance).
    Returns (cells, pairs, y, t_max)."""
    import torch
    d_cell = torch.from_numpy(cell0).cuda()
    ann = lpf.lpf_sa_create(d_cell, paths, target, n_step=n_step, t_max=t_max, seed=seed)
    if net is not None:
        lpf.lpf_sa_set_proposer(ann, net, epsilon=eps, tau=tau, refresh=16)
    H, W = cell0.shape
    cells = torch.empty((snapshots, H, W), dtype=torch.uint8, device="cuda")
    pairs = torch.empty((snapshots, n, 2), dtype=torch.int32, device="cuda")
    ys = torch.empty((snapshots, n), dtype=torch.float32, device="cuda")
    t_used = lpf.lpf_sa_read(ann)["t_max"]
    k = 0
    gap = max(1, n_step // (2 * snapshots))
    for k in range(snapshots):
        if spacing == "early":
            lpf.lpf_sa_run(ann, gap)
        else:
            goal = (k * n_step) // snapshots
            while lpf.lpf_sa_read(ann)["n_eval"] < goal:
                lpf.lpf_sa_run(ann, 16)
        cells[k].copy_(d_cell)
        p, _ = lpf.lpf_sa_propose(ann, n)
        _, de = lpf.lpf_delta_swap(d_cell, paths, p, target=target, counts=ann.counts, want_dcounts=False,
                                   want_de=True)
        de = de.double()
        sd = de.std().clamp_min(1e-30)
        ys[k] = (-(de - de.mean()) / sd).clamp(-3.0, 3.0).float()
        pairs[k] = p
    return cells, pairs, ys, t_used


def train(net, cells, pairs, ys, epochs: int = 4, batch: int = 8, lr: float = 1e-3, seed: int = 0):
    import torch
    rng = np.random.default_rng(seed)
    N = cells.shape[0]
    losses = []
    for _ in range(epochs):
        order = torch.from_numpy(rng.permutation(N)).cuda()
        for i in range(0, N - batch + 1, batch):
            idx = order[i:i + batch]
            loss = lpf.lpf_cnn_train_step(net, cells[idx].contiguous(), pairs[idx].contiguous(), ys[idx].contiguous(),
                                          lr)
            losses.append(loss)
    return [float(x.item()) for x in losses]


def run_until(paths, target, cell0, n_step: int, seed: int, t_max: float, net=None, eps: float = 0.1,
              tau: float = 1.0, target_error: float | None = None, chunk: int = 64, refresh: int = 16):
    """Anneal; return (evaluations when the error first reached target_error
    (or None), final stats, seconds)."""
    import torch
    d_cell = torch.from_numpy(cell0).cuda()
    ann = lpf.lpf_sa_create(d_cell, paths, target, n_step=n_step, t_max=t_max, seed=seed)
    if net is not None:
        lpf.lpf_sa_set_proposer(ann, net, epsilon=eps, tau=tau, refresh=refresh)
    hit = None
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    while True:
        lpf.lpf_sa_run(ann, chunk)
        st = lpf.lpf_sa_read(ann)
        if target_error is not None and hit is None and st["error"] <= target_error:
            hit = st["n_eval"]
            break
        if st["done"]:
            break
    dt = time.perf_counter() - t0
    return hit, st, dt


def evaluate(n_step: int = 100000, train_seeds=(11, 12, 13), eval_seeds=(21, 22, 23, 24, 25), snapshots: int = 256,
             n: int = 64, epochs: int = 8, taus=(0.35,), epss=(0.4,), on_policy: bool = False,
             spacing: str = "early", refreshes=(16,), loss: str = "squared", beta: float = 1.0,
             r: int = 64, cell_size: int = 128, orig_size: int = 512, net_seed: int = 3):
    """Swaps-to-target gain of the learned proposer (median over eval seeds)."""
    import torch

    import synth
    C = cell_size
    paths, target, cell0 = annealing_problem(r=r, cell_size=C, orig_size=orig_size)
    n1 = int(cell0.sum())
    cells0 = {s: synth.exact_fraction_shuffle(C, C, n1, seed=1000 + s) for s in eval_seeds}
    # uniform reference runs
    ref = {}
    t_max = None
    for s in eval_seeds:
        _, st_u, dt_u = run_until(paths, target, cells0[s], n_step, s, t_max=t_max or 0.0)
        t_max = t_max or st_u["t_max"]
        ref[s] = (st_u["error"], dt_u, st_u["n_eval"] / dt_u)
    net = lpf.lpf_cnn_create(C, C, seed=net_seed)
    lpf.lpf_cnn_set_loss(net, loss, beta)
    t0 = time.perf_counter()
    data = [collect(paths, target, synth.exact_fraction_shuffle(C, C, n1, seed=s), n_step, s, snapshots, n,
                    t_max=t_max, spacing=spacing) for s in train_seeds]
    cells = torch.cat([d[0] for d in data])
    pairs = torch.cat([d[1] for d in data])
    ys = torch.cat([d[2] for d in data])
    losses = train(net, cells, pairs, ys, epochs=epochs)
    rounds = 1
    if on_policy:
        # second round: candidates drawn by the annealer while it uses the network
        data2 = [collect(paths, target, synth.exact_fraction_shuffle(C, C, n1, seed=s + 100), n_step, s + 100,
                         snapshots, n, t_max=t_max, net=net, eps=epss[0], tau=taus[0], spacing=spacing)
                 for s in train_seeds]
        cells = torch.cat([cells] + [d[0] for d in data2])
        pairs = torch.cat([pairs] + [d[1] for d in data2])
        ys = torch.cat([ys] + [d[2] for d in data2])
        losses += train(net, cells, pairs, ys, epochs=max(1, epochs // 2), seed=1)
        rounds = 2
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    runs = []
    for refresh in refreshes:
        for tau in taus:
            for eps in epss:
                per_seed = []
                for s in eval_seeds:
                    e_u = ref[s][0]
                    hit, st_m, dt_m = run_until(paths, target, cells0[s], n_step, s, t_max=t_max, net=net, eps=eps,
                                                tau=tau, target_error=e_u, refresh=refresh)
                    per_seed.append({"seed": s, "uniform_error": e_u, "model_evals": hit,
                                     "ratio": (n_step / hit) if hit else None, "model_seconds": dt_m})
                ratios = sorted(r["ratio"] or 0.0 for r in per_seed)
                runs.append({"refresh": refresh, "tau": tau, "epsilon": eps, "median_ratio": ratios[len(ratios) // 2],
                             "per_seed": per_seed})
    best = max(runs, key=lambda r: r["median_ratio"])
    return {
        "workload": f"{C}x{C} cell, |v|<=%d, target from {orig_size}x{orig_size} clustered disks (f=0.3)" % r,
        "n_step_uniform": n_step, "uniform": {str(s): {"error": v[0], "seconds": v[1], "evals_per_s": v[2]}
                                              for s, v in ref.items()},
        "train_seeds": list(train_seeds), "eval_seeds": list(eval_seeds), "rounds": rounds, "spacing": spacing,
        "runs": runs, "best": {"refresh": best["refresh"], "tau": best["tau"], "epsilon": best["epsilon"],
                               "median_ratio": best["median_ratio"]},
        "train_snapshots": int(cells.shape[0]), "train_candidates_per_snapshot": n, "epochs": epochs,
        "loss": loss, "beta": beta,
        "train_and_collect_seconds": t_train, "loss_first": losses[0] if losses else None,
        "loss_last": float(np.mean(losses[-8:])) if losses else None, "t_max": t_max,
    }


def _budget_gain(ks, err, e_ref) -> int:
    """Largest k of ks (ascending) such that the runs with every budget N/j,
    j <= k in ks, ended at or below e_ref (1 if the smallest k already fails)."""
    gain = 1
    for k in sorted(ks):
        if err[k] > e_ref:
            break
        gain = k
    return gain


def evaluate_budget(n_step: int = 100000, ks=(2, 3, 4, 6), train_seeds=(11, 12, 13),
                    eval_seeds=(21, 22, 23, 24, 25, 26, 27), snapshots: int = 256, n: int = 64, epochs: int = 8,
                    tau: float = 0.35, eps: float = 0.4, r: int = 64, cell_size: int = 128, orig_size: int = 512,
                    net_seed: int = 3):
    """Swaps-to-target gain with each annealer run to its own budget.

    For each evaluation seed a uniform-proposal annealer with a budget of
    N = n_step evaluations ends at error e_U; annealers with a budget of N/k
    (their own temperature schedule, same initial cell, seed and initial
    temperature) end at e_M(k) with the network's proposals and at e_u(k)
    with uniform ones (the control).  The seed's gain is the largest k in
    ks such that e_M(j) <= e_U for every j <= k in ks (1 if none); the
    control's gain is the same with e_u.  Reported: the medians over the
    evaluation seeds."""
    import torch

    import synth
    C = cell_size
    paths, target, cell0 = annealing_problem(r=r, cell_size=C, orig_size=orig_size)
    n1 = int(cell0.sum())
    cells0 = {s: synth.exact_fraction_shuffle(C, C, n1, seed=1000 + s) for s in eval_seeds}
    e_full = {}
    t_max = None
    t0 = time.perf_counter()
    for s in eval_seeds:
        _, st, _ = run_until(paths, target, cells0[s], n_step, s, t_max=t_max or 0.0)
        t_max = t_max or st["t_max"]
        e_full[s] = st["error"]
    net = lpf.lpf_cnn_create(C, C, seed=net_seed)
    data = [collect(paths, target, synth.exact_fraction_shuffle(C, C, n1, seed=s), n_step, s, snapshots, n,
                    t_max=t_max, spacing="early") for s in train_seeds]
    train(net, torch.cat([d[0] for d in data]), torch.cat([d[1] for d in data]), torch.cat([d[2] for d in data]),
          epochs=epochs)
    per_seed = []
    for s in eval_seeds:
        row = {"seed": s, "uniform_error": e_full[s], "model_error": {}, "uniform_k_error": {}}
        for k in ks:
            _, st_m, _ = run_until(paths, target, cells0[s], n_step // k, s, t_max=t_max, net=net, eps=eps, tau=tau)
            _, st_u, _ = run_until(paths, target, cells0[s], n_step // k, s, t_max=t_max)
            row["model_error"][k] = st_m["error"]
            row["uniform_k_error"][k] = st_u["error"]
        row["gain"] = _budget_gain(ks, row["model_error"], e_full[s])
        row["control_gain"] = _budget_gain(ks, row["uniform_k_error"], e_full[s])
        per_seed.append(row)
    gains = sorted(r_["gain"] for r_ in per_seed)
    control = sorted(r_["control_gain"] for r_ in per_seed)
    return {
        "workload": f"{C}x{C} cell, |v|<={r}, target from {orig_size}x{orig_size} clustered disks (f=0.3)",
        "n_step_uniform": n_step, "ks": list(ks), "tau": tau, "epsilon": eps, "train_seeds": list(train_seeds),
        "eval_seeds": list(eval_seeds), "median_gain": gains[len(gains) // 2],
        "median_control_gain": control[len(control) // 2], "per_seed": per_seed,
        "seconds": time.perf_counter() - t0,
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--evaluate", action="store_true", help="first-crossing protocol (one schedule of N)")
    ap.add_argument("--evaluate-budget", action="store_true", help="own-budget protocol (schedules of N/k)")
    ap.add_argument("--ks", type=int, nargs="+", default=[2, 3, 4, 6])
    ap.add_argument("--n-step", type=int, default=100000)
    ap.add_argument("--snapshots", type=int, default=256)
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--train-seeds", type=int, nargs="+", default=[11, 12, 13])
    ap.add_argument("--eval-seeds", type=int, nargs="+", default=[21, 22, 23, 24, 25])
    ap.add_argument("--tau", type=float, nargs="+", default=[0.35])
    ap.add_argument("--eps", type=float, nargs="+", default=[0.4])
    ap.add_argument("--on-policy", action="store_true")
    ap.add_argument("--spacing", choices=["evals", "early"], default="early")
    ap.add_argument("--refresh", type=int, nargs="+", default=[16])
    ap.add_argument("--loss", choices=["squared", "listwise"], default="squared")
    ap.add_argument("--beta", type=float, default=1.0, help="listwise target temperature")
    ap.add_argument("--r", type=int, default=64, help="window radius")
    ap.add_argument("--cell", type=int, default=128, help="cell size")
    ap.add_argument("--orig", type=int, default=512, help="original size (512: the annealing workload's image)")
    a = ap.parse_args()
    lpf.load()
    if a.evaluate:
        print(json.dumps(evaluate(n_step=a.n_step, train_seeds=tuple(a.train_seeds), eval_seeds=tuple(a.eval_seeds),
                                  snapshots=a.snapshots, epochs=a.epochs, taus=tuple(a.tau), epss=tuple(a.eps),
                                  on_policy=a.on_policy, spacing=a.spacing, refreshes=tuple(a.refresh),
                                  loss=a.loss, beta=a.beta, r=a.r, cell_size=a.cell, orig_size=a.orig)),
              flush=True)
    if a.evaluate_budget:
        print(json.dumps(evaluate_budget(n_step=a.n_step, ks=tuple(a.ks), train_seeds=tuple(a.train_seeds),
                                         eval_seeds=tuple(a.eval_seeds), snapshots=a.snapshots, epochs=a.epochs,
                                         tau=a.tau[0], eps=a.eps[0], r=a.r, cell_size=a.cell, orig_size=a.orig)),
              flush=True)


if __name__ == "__main__":
    main()
