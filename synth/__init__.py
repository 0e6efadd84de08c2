"""Seeded synthetic two-phase microstructures (periodic, uint8 0/1 images).

These stand in for the paper's datasets (metal foam, epithelial cells,
trabecular bone, the particulate original), which are not available.  The
morphologies follow the kinds the paper uses (Sec. 3.2 and Sec. 6: chess
pattern, equal-sized squares, particle suspensions, clustered real-like media).

This module holds input generation only (random geometry and rasterisation);
it contains none of the lineal-path arithmetic, and both the oracle and the
CUDA library are fed from it.

Rasterisation convention: pixel (x, y) has its centre at (x + 1/2, y + 1/2);
it is phase 1 when that centre lies inside a particle, with distances taken
on the torus [0, W) x [0, H).
"""
from __future__ import annotations

import math

import numpy as np


def _torus_delta(d: np.ndarray, period: float) -> np.ndarray:
    return d - period * np.round(d / period)


def disks_fixed(H: int, W: int, R: float, centres: np.ndarray) -> np.ndarray:
    """Union of radius-R disks with the given continuous centres [(cx, cy), ...]."""
    img = np.zeros((H, W), np.uint8)
    if len(centres) == 0:
        return img
    r = int(math.ceil(R)) + 1
    offs = np.arange(-r, r + 1)
    cx = centres[:, 0]
    cy = centres[:, 1]
    bx = np.floor(cx).astype(np.int64)
    by = np.floor(cy).astype(np.int64)
    for oy in offs:
        py = by + oy
        dy = _torus_delta((py + 0.5) - cy, H)
        for ox in offs:
            px = bx + ox
            dx = _torus_delta((px + 0.5) - cx, W)
            hit = dx * dx + dy * dy <= R * R
            img[(py[hit] % H), (px[hit] % W)] = 1
    return img


def boolean_disks(H: int, W: int, R: float, n: int, seed: int) -> np.ndarray:
    """n disks of radius R, centres uniform on the torus (Boolean model)."""
    rng = np.random.default_rng(seed)
    centres = np.stack([rng.uniform(0, W, n), rng.uniform(0, H, n)], axis=1)
    return disks_fixed(H, W, R, centres)


def boolean_spheres(D: int, H: int, W: int, R: float, n: int, seed: int) -> np.ndarray:
    """Volume [D][H][W] of n balls of radius R, centres uniform on the 3-torus
    (Boolean model): a stand-in for a CT volume whose parallel cuts are
    averaged (Sec. 6.3).  Voxel (x, y, z) is phase 1 when its centre lies in a ball."""
    rng = np.random.default_rng(seed)
    c = np.stack([rng.uniform(0, W, n), rng.uniform(0, H, n), rng.uniform(0, D, n)], axis=1)
    z, y, x = np.mgrid[0:D, 0:H, 0:W].astype(np.float64) + 0.5
    vol = np.zeros((D, H, W), bool)
    for cx, cy, cz in c:
        dx = _torus_delta(x - cx, W)
        dy = _torus_delta(y - cy, H)
        dz = _torus_delta(z - cz, D)
        vol |= dx * dx + dy * dy + dz * dz <= R * R
    return vol.astype(np.uint8)


def disks_for_fraction(H: int, W: int, R: float, fraction: float) -> int:
    """Number of Boolean disks whose expected covered fraction is `fraction`."""
    return int(round(-math.log(1.0 - fraction) * W * H / (math.pi * R * R)))


def _stamp_ellipse(img, cx, cy, a, b, theta):
    H, W = img.shape
    r = int(math.ceil(max(a, b))) + 1
    ys = np.arange(int(math.floor(cy)) - r, int(math.floor(cy)) + r + 1)
    xs = np.arange(int(math.floor(cx)) - r, int(math.floor(cx)) + r + 1)
    X, Y = np.meshgrid(xs, ys)
    dx = _torus_delta(X + 0.5 - cx, W)
    dy = _torus_delta(Y + 0.5 - cy, H)
    c, s = math.cos(theta), math.sin(theta)
    u = c * dx + s * dy
    v = -s * dx + c * dy
    hit = (u / a) ** 2 + (v / b) ** 2 <= 1.0
    img[Y[hit] % H, X[hit] % W] = 1


def ellipses(H: int, W: int, fraction: float, seed: int, axes=(6.0, 20.0)) -> np.ndarray:
    """Overlapping ellipses, semi-axes ~ U[axes], orientation ~ U[0, pi), centres
    uniform; ellipses are added until the phase-1 fraction reaches `fraction`."""
    rng = np.random.default_rng(seed)
    img = np.zeros((H, W), np.uint8)
    target = fraction * H * W
    while img.sum(dtype=np.int64) < target:
        a = rng.uniform(*axes)
        b = rng.uniform(*axes)
        _stamp_ellipse(img, rng.uniform(0, W), rng.uniform(0, H), a, b, rng.uniform(0, math.pi))
    return img


def clustered_disks(H: int, W: int, fraction: float, seed: int, R: float = 5.0,
                    children: float = 8.0, spread: float = 12.0) -> np.ndarray:
    """Thomas cluster process: parent points uniform, a Poisson(children) number
    of children per parent displaced by N(0, spread^2), radius-R disks on the
    children; clusters are added until the phase-1 fraction reaches `fraction`."""
    rng = np.random.default_rng(seed)
    img = np.zeros((H, W), np.uint8)
    target = fraction * H * W
    while img.sum(dtype=np.int64) < target:
        px, py = rng.uniform(0, W), rng.uniform(0, H)
        k = max(1, rng.poisson(children))
        cs = np.stack([(px + rng.normal(0, spread, k)) % W, (py + rng.normal(0, spread, k)) % H], axis=1)
        img |= disks_fixed(H, W, R, cs)
    return img


def chess(H: int, W: int, s: int) -> np.ndarray:
    """Chess pattern of s x s squares (Tab. comptime, first microstructure)."""
    y, x = np.mgrid[0:H, 0:W]
    return (((x // s) + (y // s)) % 2).astype(np.uint8)


def squares(H: int, W: int, s: int, fraction: float, seed: int) -> np.ndarray:
    """Equal-sized s x s squares at uniform integer positions (overlap allowed),
    added until the phase-1 fraction reaches `fraction` (Tab. comptime, second
    microstructure; the paper does not give its fraction)."""
    rng = np.random.default_rng(seed)
    img = np.zeros((H, W), np.uint8)
    target = fraction * H * W
    ar = np.arange(s)
    while img.sum(dtype=np.int64) < target:
        x0, y0 = rng.integers(0, W), rng.integers(0, H)
        img[np.ix_((y0 + ar) % H, (x0 + ar) % W)] = 1
    return img


def _disks_radii(H: int, W: int, R: np.ndarray, centres: np.ndarray) -> np.ndarray:
    """Union of disks with per-disk radii R[i] and continuous centres[i]."""
    img = np.zeros((H, W), np.uint8)
    r = int(math.ceil(float(R.max()))) + 1
    bx = np.floor(centres[:, 0]).astype(np.int64)
    by = np.floor(centres[:, 1]).astype(np.int64)
    for oy in range(-r, r + 1):
        py = by + oy
        dy = _torus_delta((py + 0.5) - centres[:, 1], H)
        for ox in range(-r, r + 1):
            px = bx + ox
            dx = _torus_delta((px + 0.5) - centres[:, 0], W)
            hit = dx * dx + dy * dy <= R * R
            img[(py[hit] % H), (px[hit] % W)] = 1
    return img


def foam(H: int, W: int, porosity: float, seed: int, radii=(2.0, 8.0)) -> np.ndarray:
    """Foam-like medium: phase 1 is the solid left between pores, the pores
    being disks of radius uniform in `radii` at uniform centres, added in
    draw order until the pore fraction reaches `porosity` (a stand-in for the
    metal-foam image of Tab. comptime, third microstructure, which is not
    available)."""
    rng = np.random.default_rng(seed)
    pores = np.zeros((H, W), np.uint8)
    target = porosity * H * W
    while pores.sum(dtype=np.int64) < target:
        # a round of k pores while far from the target, one at a time near it
        k = 64 if (target - pores.sum(dtype=np.int64)) > 64 * math.pi * radii[1] ** 2 else 1
        R = rng.uniform(radii[0], radii[1], k)
        c = np.stack([rng.uniform(0, W, k), rng.uniform(0, H, k)], axis=1)
        pores |= _disks_radii(H, W, R, c)
    return (1 - pores).astype(np.uint8)


def random_binary(H: int, W: int, fraction: float, seed: int) -> np.ndarray:
    """Independent pixels, phase 1 with probability `fraction`."""
    rng = np.random.default_rng(seed)
    return (rng.random((H, W)) < fraction).astype(np.uint8)


def exact_fraction_shuffle(H: int, W: int, n_ones: int, seed: int) -> np.ndarray:
    """Random image with exactly n_ones phase-1 pixels, uniformly placed (the
    annealer's random initial image with the original's volume fraction)."""
    rng = np.random.default_rng(seed)
    flat = np.zeros(H * W, np.uint8)
    flat[rng.choice(H * W, size=n_ones, replace=False)] = 1
    return flat.reshape(H, W)


# ---- the named workloads ---------------------------------------------------

def disks_64() -> np.ndarray:
    """64x64 Boolean disks R=5, expected phase-1 fraction 0.4 (27 disks), seed 1."""
    return boolean_disks(64, 64, 5.0, disks_for_fraction(64, 64, 5.0, 0.4), seed=1)


def ellipses_512() -> np.ndarray:
    """512x512 overlapping ellipses, semi-axes 6-20 px, fraction 0.35, seed 2."""
    return ellipses(512, 512, 0.35, seed=2)


def clustered_512() -> np.ndarray:
    """512x512 clustered disks (Thomas process, R=5), fraction 0.30, seed 3."""
    return clustered_disks(512, 512, 0.30, seed=3)


def mixed_sizes_batch(n: int = 256, seed: int = 4):
    """n images, H, W ~ U{48..256} independently, morphology cycling
    disks / ellipses / clustered disks, fraction ~ U[0.2, 0.6]."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        H = int(rng.integers(48, 257))
        W = int(rng.integers(48, 257))
        f = float(rng.uniform(0.2, 0.6))
        s = int(rng.integers(0, 2**31 - 1))
        kind = i % 3
        if kind == 0:
            img = boolean_disks(H, W, 5.0, disks_for_fraction(H, W, 5.0, f), seed=s)
        elif kind == 1:
            img = ellipses(H, W, f, seed=s)
        else:
            img = clustered_disks(H, W, f, seed=s)
        out.append(img)
    return out


def swap_candidates(cell: np.ndarray, K: int, seed: int = 0) -> np.ndarray:
    """int32 [K][2] candidate exchanges of a two-phase cell: column 0 a
    phase-1 pixel, column 1 a phase-0 pixel (linear indices y*W + x), each
    uniform over its phase, independently (the candidate batch of the
    swap-delta workload)."""
    rng = np.random.default_rng(seed)
    flat = cell.reshape(-1)
    ones = np.flatnonzero(flat == 1)
    zeros = np.flatnonzero(flat == 0)
    return np.stack([rng.choice(ones, K), rng.choice(zeros, K)], axis=1).astype(np.int32)


def clustered_cell_128() -> np.ndarray:
    """128x128 crop of the 512x512 clustered-disk image (the swap-delta workload's cell)."""
    return clustered_512()[:128, :128].copy()
