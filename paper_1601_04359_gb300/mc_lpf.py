"""Error of the Monte-Carlo lineal path function versus the number of
sampled translations (Sec. 3 opening, Fig. MC_LP), on the two reproducible
microstructures of that figure: A, chess of 10x10 squares, and B, 4x4
squares (fraction 0.3, the paper does not give it), both 100x100 with the
full half-domain D.  For each N, the translations are a random
N-combination of the W*H positions (seeded), L~ = counts over them / N, and
e(L~) = sum over D of (L - L~)^2 per phase (Eq. LSE1), averaged over seeds.

    python -m paper_1601_04359_gb300.mc_lpf                   # error of L~ versus N
    python -m paper_1601_04359_gb300.mc_lpf reconstruction    # reconstruction driven by L~ (Fig. ComMicRec)
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import paper_1601_04359_gb300 as lpf  # noqa: E402


def error_curve(img, ns=(10, 30, 100, 300, 1000, 3000, 10000), seeds=5):
    import torch
    H, W = img.shape
    p = lpf.lpf_build_paths(W - 1, H - 1)
    d = torch.from_numpy(img).cuda()
    exact = lpf.lpf_full(d, p).double() / (H * W)
    base = p.base
    out = []
    for n in ns:
        errs = []
        for s in range(seeds):
            rng = np.random.default_rng(1000 * n + s)
            sel = np.zeros(H * W, np.uint8)
            sel[rng.choice(H * W, n, replace=False)] = 1
            c = lpf.lpf_full_mc(d, p, torch.from_numpy(sel.reshape(H, W)).cuda()).double() / n
            e = ((exact[:, base:] - c[:, base:]) ** 2).sum(dim=1)
            errs.append(e.cpu().numpy())
        errs = np.array(errs)
        out.append({"N": n, "e_phase0": float(errs[:, 0].mean()), "e_phase1": float(errs[:, 1].mean())})
    return out


def _sample(H, W, n, seed):
    rng = np.random.default_rng(seed)
    sel = np.zeros(H * W, np.uint8)
    sel[rng.choice(H * W, n, replace=False)] = 1
    return sel.reshape(H, W)


def reconstruction(img, ns=(10, 100, 1000, 2500), seeds=(1, 2), n_step=500000):
    """Fig. ComMicRec: reconstruct a cell of the original's size from the
    Monte-Carlo L~ of the original (its own random N-combination), annealing
    on the cell's L~ (a fixed random N-combination of its positions); N = W*H
    is the exact function.  Each final cell is scored by the exact L2 (both
    phases, half-domain D): e = sum (L_orig - L_cell)^2 and e / sum L_orig^2.
    Schedule: Tab. annealing with c_max = s_max = 0.01 N_step, T_max = 0.3 x
    the automatic start temperature."""
    import torch
    H, W = img.shape
    p = lpf.lpf_build_paths(W - 1, H - 1)
    d = torch.from_numpy(img).cuda()
    exact = lpf.lpf_full(d, p).double() / (H * W)
    base = p.base
    norm = float((exact[:, base:] ** 2).sum())
    out = []
    for n in ns:
        for seed in seeds:
            cell0 = torch.from_numpy(_exact_fraction(img, seed)).cuda()
            kw = dict(n_step=n_step, c_max=n_step // 100, s_max=n_step // 100, seed=seed)
            if n >= H * W:
                target = exact.float()
                make = lambda c, **k: lpf.lpf_sa_create(c, p, target, **k)
            else:
                so = torch.from_numpy(_sample(H, W, n, 1000 + seed)).cuda()
                target = (lpf.lpf_full_mc(d, p, so).double() / n).float()
                sc = torch.from_numpy(_sample(H, W, n, 2000 + seed)).cuda()
                make = lambda c, **k: lpf.lpf_sa_create_mc(c, p, sc, target, **k)
            auto = lpf.lpf_sa_read(make(cell0.clone(), **kw))["t_max"]
            cell = cell0.clone()
            ann = make(cell, t_max=0.3 * auto, **kw)
            while not lpf.lpf_sa_read(ann)["done"]:
                lpf.lpf_sa_run(ann, 256)
            fin = lpf.lpf_full(cell, p).double() / (H * W)
            e = float(((exact[:, base:] - fin[:, base:]) ** 2).sum())
            out.append({"N": n, "seed": seed, "e_exact": e, "relative": e / norm,
                        "equal_to_original_up_to_translation": _is_translate(cell.cpu().numpy(), img)})
            print(json.dumps(out[-1]), file=sys.stderr, flush=True)
    return out


def _exact_fraction(img, seed):
    import synth
    H, W = img.shape
    return synth.exact_fraction_shuffle(H, W, int(img.sum()), seed=seed)


def _is_translate(a, b):
    H, W = b.shape
    return any((np.roll(b, (dy, dx), axis=(0, 1)) == a).all() for dy in range(H) for dx in range(W))


def main():
    import synth
    lpf.load()
    if len(sys.argv) > 1 and sys.argv[1] == "reconstruction":
        res = {"A_chess_5_50": reconstruction(synth.chess(50, 50, 5)),
               "B_squares_4_50": reconstruction(synth.squares(50, 50, 4, 0.3, seed=7))}
    else:
        res = {"A_chess_10": error_curve(synth.chess(100, 100, 10)),
               "B_squares_4": error_curve(synth.squares(100, 100, 4, 0.3, seed=7))}
    print(json.dumps(res))


if __name__ == "__main__":
    main()
