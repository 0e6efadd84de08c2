"""Error of the Monte-Carlo lineal path function versus the number of
sampled translations (Sec. 3 opening, Fig. MC_LP), on the two reproducible
microstructures of that figure: A, chess of 10x10 squares, and B, 4x4
squares (fraction 0.3, the paper does not give it), both 100x100 with the
full half-domain D.  For each N, the translations are a random
N-combination of the W*H positions (seeded), L~ = counts over them / N, and
e(L~) = sum over D of (L - L~)^2 per phase (Eq. LSE1), averaged over seeds.

    python -m paper_1601_04359_gb300.mc_lpf
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


def main():
    import synth
    lpf.load()
    res = {"A_chess_10": error_curve(synth.chess(100, 100, 10)),
           "B_squares_4": error_curve(synth.squares(100, 100, 4, 0.3, seed=7))}
    print(json.dumps(res))


if __name__ == "__main__":
    main()
