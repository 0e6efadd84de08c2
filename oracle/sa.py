"""Oracle of the annealer (Sec. 4, Alg. 3): random draws, proposals and a
plain sequential annealing loop on the CPU oracle's counts.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Readings of the paper that this follows (its printed Alg. 3 is garbled):
  - one evaluation counter n runs to N_step; a temperature stage ends after
    c_max attempts or s_max acceptances, then T <- T * T_mult with
    T_mult = (T_min / T_max)^(s_max / N_step);
  - a candidate is accepted when Delta e <= 0 or U < exp(-Delta e / T);
  - the modification exchanges a phase-1 and a phase-0 pixel, both drawn
    uniformly among interfacial pixels (4-neighbourhood on the torus);
  - the random numbers of candidate n come from Philox-4x32-10 keyed by the
    run's seed: attempt j = 0, 1, ... uses counter (n mod 2^32, n div 2^32,
    j, 0); its words 0 and 1 each propose a pixel floor(r * H*W / 2^32), and
    the first proposal that has the wanted phase and is interfacial is kept
    (rejection sampling, i.e. uniform over the interfacial pixels of that
    phase); word 2 of attempt 0 gives U = ((r >> 8) + 1/2) / 2^24 evaluated in
    float32.  With no such pixel after 65536 attempts the candidate is the
    identity (0, 0).
"""
from __future__ import annotations

import math

import numpy as np

from . import delta_swap

MASK = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    """Philox-4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, "Parallel random
    numbers: as easy as 1, 2, 3", SC'11): each round multiplies words 0 and 2
    by the round multipliers, mixes the high halves with words 1 and 3 and the
    key, and the key is bumped by the Weyl constants between rounds."""
    M0, M1 = 0xD2511F53, 0xCD9E8D57
    W0, W1 = 0x9E3779B9, 0xBB67AE85
    c0, c1, c2, c3 = (int(x) & MASK for x in ctr)
    k0, k1 = (int(x) & MASK for x in key)
    for _ in range(10):
        p0 = M0 * c0
        p1 = M1 * c2
        hi0, lo0 = p0 >> 32, p0 & MASK
        hi1, lo1 = p1 >> 32, p1 & MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & MASK, lo1, (hi0 ^ c3 ^ k1) & MASK, lo0
        k0 = (k0 + W0) & MASK
        k1 = (k1 + W1) & MASK
    return c0, c1, c2, c3


def interfacial_lists(cell: np.ndarray):
    """Raster-order lists of interfacial phase-1 and phase-0 pixels (a pixel
    with a 4-neighbour of the other phase on the torus)."""
    c = np.asarray(cell)
    inter = np.zeros(c.shape, bool)
    for ax, sh in ((0, 1), (0, -1), (1, 1), (1, -1)):
        inter |= np.roll(c, sh, axis=ax) != c
    flat = c.reshape(-1)
    it = inter.reshape(-1)
    return np.flatnonzero(it & (flat == 1)), np.flatnonzero(it & (flat == 0))


def propose(cell: np.ndarray, n_eval: int, k: int, seed: int):
    """Candidates n_eval .. n_eval+k-1 drawn from `cell`: pairs int32 [k][2]
    (phase-1 pixel, phase-0 pixel) and uniforms float32 [k]."""
    c = np.asarray(cell)
    flat = c.reshape(-1)
    npix = flat.size
    l1, l0 = interfacial_lists(c)
    inter1 = np.zeros(npix, bool)
    inter0 = np.zeros(npix, bool)
    inter1[l1] = True
    inter0[l0] = True
    key = (seed & MASK, (seed >> 32) & MASK)
    pairs = np.zeros((k, 2), np.int32)
    u = np.zeros(k, np.float32)
    for i in range(k):
        n = n_eval + i
        a = b = -1
        for j in range(65536):
            r = philox4x32_10((n & MASK, (n >> 32) & MASK, j, 0), key)
            if j == 0:
                u[i] = (np.float32(r[2] >> 8) + np.float32(0.5)) * np.float32(1.0 / 16777216.0)
            if a < 0 and inter1[(r[0] * npix) >> 32]:
                a = (r[0] * npix) >> 32
            if b < 0 and inter0[(r[1] * npix) >> 32]:
                b = (r[1] * npix) >> 32
            if a >= 0 and b >= 0:
                break
        if a < 0 or b < 0:
            a = b = 0
        pairs[i] = (a, b)
    return pairs, u


def anneal(cell: np.ndarray, target: np.ndarray, counts: np.ndarray, rx: int, ry: int, n_step: int,
           c_max: int, s_max: int, t_max: float, t_min_ratio: float, seed: int, phases: int = 3,
           objective: str = "l2", sel=None):
    """Sequential Alg. 3 with the readings above; Delta e from the oracle's
    recount (double precision, rounded to float32 as the error change of a
    candidate).  objective "l2": Eq. (LSE) on the lineal path counts of the
    phases in the bit mask `phases` (counts int64 [2][n_full], target
    [2][n_full]); with `sel` (uint8 [H][W], the N sampled translations) the
    counts are those of the Monte-Carlo variant (Sec. 3 opening) and the
    descriptor is count / N; "s2": Eq. (LSE) on the phase-1 two-point
    probability over all W*H offsets of the cell (target [H*W]; counts and
    rx, ry unused).  Returns (final cell, n_accept, final T)."""
    from . import delta_objective, lpf_full_selected, s2_delta_objective
    cell = np.array(cell, np.uint8)
    counts = np.array(counts, np.int64)
    H, W = cell.shape
    n_full = (2 * rx + 1) * (2 * ry + 1)
    base = (n_full - 1) // 2
    T = t_max
    t_mult = t_min_ratio ** (s_max / n_step)
    c = s = 0
    n_accept = 0
    for n in range(n_step):
        pairs, u = propose(cell, n, 1, seed)
        if objective == "s2":
            de = np.float32(s2_delta_objective(cell, target, pairs)[0])
        elif sel is not None:
            a, b = pairs[0]
            after = cell.copy().reshape(-1)
            after[a], after[b] = after[b], after[a]
            d = (lpf_full_selected(after.reshape(H, W), rx, ry, sel) - counts)[:, base:][None]
            # normalisation by N: the oracle's objective divides by H*W, so pass N x 1
            de = np.float32(delta_objective(target, counts, d, rx, ry, int(np.count_nonzero(sel)), 1, phases)[0])
        else:
            d = delta_swap(cell, rx, ry, pairs)
            de = np.float32(delta_objective(target, counts, d, rx, ry, H, W, phases)[0])
        c += 1
        accept = de <= 0 or u[0] < np.float32(math.exp(-float(de) / T))
        if accept:
            s += 1
            n_accept += 1
            a, b = pairs[0]
            flat = cell.reshape(-1)
            flat[a], flat[b] = flat[b], flat[a]
            if objective != "s2":
                counts[:, base:] += d[0]
                counts[:, :base] = counts[:, base + 1:][:, ::-1]
        if c >= c_max or s >= s_max:
            T *= t_mult
            c = s = 0
    return cell, n_accept, T
