"""Descriptor comparison by annealing (Sec. 5 Fig. chess, Sec. 6 Tab. mutual)
on synthetic media, with the two-point probability S2 and the lineal path
function of both phases (L2), of phase 1 only (L2^w: phase 1 is the white
squares) or of phase 0 only (L2^b) as the objective.

chess  -- reconstruction: a random 20x20 cell annealed against the
          descriptor of a 100x100 chess of 10x10 squares (full vector domain
          of the cell, rx = ry = 19); the cell should become the chess up to
          a translation.  Sweeps the initial temperature as a multiple of
          the automatic one (an average uphill move accepted with
          probability 1/2), because the stage rule
          T_mult = (T_min/T_max)^(s_max/N_step) reaches T_min only if every
          stage ends after s_max acceptances in a row.
mutual -- compression: 4x4 white squares (phase 1, fraction 0.2: the paper
          gives none) on a 100x100 original, 50x50 cells annealed on each
          descriptor cut to the cell (L2: window rx = ry = 49; S2: the
          centred offsets of the cell), and every result scored by both
          e(S2) and e(L2) of Eq. (LSE1), next to the random start.

    python -m paper_1601_04359_gb300.compression chess [--n-step N] [--seeds K] [--scales ...] [--c-frac ...]
    python -m paper_1601_04359_gb300.compression mutual [--n-step N] [--t-scale s] [--c-frac f]
"""
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

DESCRIPTORS = {"S2": None, "L2": 3, "L2w": 2, "L2b": 1}   # lineal-path phase masks


def s2_cut(s2, H, W):
    """The cell's S2 target: entry (y, x) is the original's S2 at the centred
    offset (y or y - H, x or x - W), i.e. the descriptor cut to the cell."""
    import torch
    H0, W0 = s2.shape
    ys = torch.tensor([(y if y < H - (H + 1) // 2 else y - H) % H0 for y in range(H)], device=s2.device)
    xs = torch.tensor([(x if x < W - (W + 1) // 2 else x - W) % W0 for x in range(W)], device=s2.device)
    return s2[ys][:, xs].contiguous()


class Problem:
    """Targets of one original for H x W cells."""

    def __init__(self, orig: np.ndarray, H: int, W: int, r: int):
        import torch
        self.H, self.W = H, W
        self.paths = lpf.lpf_build_paths(r, r)
        d = torch.from_numpy(orig).cuda()
        self.t_l2 = (lpf.lpf_full(d, self.paths).double() / float(orig.size)).float()
        self.t_s2 = s2_cut(lpf.s2_fft(d, 1), H, W)
        self.t_s2_0 = s2_cut(lpf.s2_fft(d, 0), H, W)

    def errors(self, cell: np.ndarray):
        """(e(S2), e(L2)) of a cell, both phases (the paper's convention when no
        phase is named): Eq. (LSE1) over the cell's offsets for S2 and over the
        canonical half for L2.  S2 of phase 0 follows from phase 1 by Eq. (S2add)."""
        import torch
        d = torch.from_numpy(cell).cuda()
        n = float(cell.size)
        s1 = lpf.s2_counts(d).double() / n
        phi1 = float(cell.mean())
        s0 = s1 + (1.0 - phi1) ** 2 - phi1 ** 2
        e_s2 = float(((self.t_s2.double() - s1) ** 2).sum() + ((self.t_s2_0.double() - s0) ** 2).sum())
        base = self.paths.base
        c = lpf.lpf_full(d, self.paths).double() / n
        e_l2 = float(((self.t_l2.double()[:, base:] - c[:, base:]) ** 2).sum())
        return e_s2, e_l2

    def create(self, desc: str, d_cell, n_step: int, seed: int, t_max: float = 0.0, c_frac: float = 0.1,
               t_min_ratio: float = 0.01):
        kw = dict(n_step=n_step, c_max=max(1, int(c_frac * n_step)), s_max=max(1, n_step // 100), t_max=t_max,
                  t_min_ratio=t_min_ratio, seed=seed)
        if desc == "S2":
            return lpf.s2_sa_create(d_cell, self.t_s2, **kw)
        return lpf.lpf_sa_create(d_cell, self.paths, self.t_l2, phases=DESCRIPTORS[desc], **kw)

    def anneal(self, desc: str, cell0: np.ndarray, n_step: int, seed: int, t_scale: float = 1.0,
               t_limit: float = 600.0, c_frac: float = 0.1, t_min_ratio: float = 0.01):
        """Anneal a copy of cell0 (Tab. annealing: c_max = c_frac N_step,
        s_max = 0.01 N_step); stop at n_step, at zero error or after t_limit s."""
        import torch
        t_max = 0.0
        if t_scale != 1.0:
            probe = self.create(desc, torch.from_numpy(cell0).cuda(), n_step, seed)
            t_max = t_scale * lpf.lpf_sa_read(probe)["t_max"]
            del probe
        d = torch.from_numpy(cell0).cuda()
        ann = self.create(desc, d, n_step, seed, t_max, c_frac, t_min_ratio)
        st0 = lpf.lpf_sa_read(ann)
        torch.cuda.synchronize()
        t0 = time.time()
        while True:
            lpf.lpf_sa_run(ann, 256)
            st = lpf.lpf_sa_read(ann)
            if st["done"] or st["error"] < 1e-12 or time.time() - t0 > t_limit:
                break
        dt = time.time() - t0
        e_run = lpf.lpf_sa_recompute_error(ann)
        return d.cpu().numpy(), {"desc": desc, "seed": seed, "t_scale": t_scale, "c_frac": c_frac,
                                 "t_min_ratio": t_min_ratio, "t_max": st0["t_max"], "t_final": st["temperature"],
                                 "e0": st0["error"], "e_final": e_run, "n_eval": st["n_eval"],
                                 "n_accept": st["n_accept"], "seconds": dt, "evals_per_s": st["n_eval"] / dt}


def chess(n_step: int, seeds, scales, c_fracs=(0.1,), t_min_ratio: float = 0.01, descs=tuple(DESCRIPTORS)):
    import synth
    orig = synth.chess(100, 100, 10)
    pr = Problem(orig, 20, 20, 19)
    goal = synth.chess(20, 20, 10)
    translates = [np.roll(goal, (dy, dx), axis=(0, 1)) for dy in range(20) for dx in range(20)]
    rows = []
    for desc in descs:
        for cf in c_fracs:
            for sc in scales:
                for seed in seeds:
                    cell0 = synth.exact_fraction_shuffle(20, 20, 200, seed=seed)
                    cell, info = pr.anneal(desc, cell0, n_step, seed, sc, t_limit=120.0, c_frac=cf,
                                           t_min_ratio=t_min_ratio)
                    info["recovered"] = any((cell == t).all() for t in translates)
                    info["e_s2"], info["e_l2"] = pr.errors(cell)
                    rows.append(info)
                    print(json.dumps(info), file=sys.stderr, flush=True)
    return rows


def mutual(n_step: int, seed: int = 1, t_scale: float = 1.0, c_frac: float = 0.1, t_min_ratio: float = 0.01):
    import synth
    orig = synth.squares(100, 100, 4, 0.2, seed=7)
    pr = Problem(orig, 50, 50, 49)
    n1 = int(round(orig.mean() * 2500))
    cell0 = synth.exact_fraction_shuffle(50, 50, n1, seed=seed)
    e_s2, e_l2 = pr.errors(cell0)
    rows = [{"medium": "random", "e_s2": e_s2, "e_l2": e_l2}]
    for desc in DESCRIPTORS:
        cell, info = pr.anneal(desc, cell0, n_step, seed, t_scale, t_limit=300.0, c_frac=c_frac,
                               t_min_ratio=t_min_ratio)
        info["medium"] = desc + "-based"
        info["e_s2"], info["e_l2"] = pr.errors(cell)
        rows.append(info)
        print(json.dumps(info), file=sys.stderr, flush=True)
    return {"fraction": float(orig.mean()), "rows": rows}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["chess", "mutual"])
    ap.add_argument("--n-step", type=int, default=500000)
    ap.add_argument("--seeds", type=int, default=3)
    ap.add_argument("--scales", type=float, nargs="+", default=[1.0, 0.3, 0.1, 0.03])
    ap.add_argument("--t-scale", type=float, default=1.0)
    ap.add_argument("--c-frac", type=float, nargs="+", default=[0.1], help="c_max / N_step")
    ap.add_argument("--t-min-ratio", type=float, default=0.01)
    ap.add_argument("--desc", nargs="+", default=list(DESCRIPTORS), choices=list(DESCRIPTORS))
    a = ap.parse_args()
    lpf.load()
    if a.what == "chess":
        out = chess(a.n_step, list(range(1, a.seeds + 1)), a.scales, a.c_frac, a.t_min_ratio, a.desc)
    else:
        out = mutual(a.n_step, t_scale=a.t_scale, c_frac=a.c_frac[0], t_min_ratio=a.t_min_ratio)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
