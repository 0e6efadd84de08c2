"""Pins for the oracle's two-point probability (Sec. 2.1)."""
import numpy as np
import pytest

import oracle
import synth


@pytest.mark.parametrize("H,W,seed", [(16, 16, 0), (12, 20, 1), (33, 17, 2)])
def test_direct_sum_equals_fft_form(H, W, seed):
    # Eq. (S2dis) equals the FFT form 1/(WH) IDFT(DFT chi conj(DFT chi)) (Sec. 2.1),
    # here computed with numpy's FFT.
    img = synth.random_binary(H, W, 0.4, seed)
    for p in (0, 1):
        chi = (img == p).astype(np.float64)
        F = np.fft.fft2(chi)
        ref = np.real(np.fft.ifft2(np.conj(F) * F)) / (H * W)
        np.testing.assert_allclose(oracle.s2_direct(img, p), ref, atol=1e-12)


def test_asymptotics_and_two_phase_relation():
    img = synth.disks_64()
    H, W = img.shape
    phi1 = img.mean()
    phi0 = 1 - phi1
    s1 = oracle.s2_direct(img, 1)
    s0 = oracle.s2_direct(img, 0)
    assert s1[0, 0] == pytest.approx(phi1, abs=1e-15)           # Eq. (s2zero)
    assert s0[0, 0] == pytest.approx(phi0, abs=1e-15)
    np.testing.assert_allclose(s1 - s0, phi1 ** 2 - phi0 ** 2, atol=1e-12)   # Eq. (S2add)
    assert s1.sum() == pytest.approx(phi1 ** 2 * H * W, rel=1e-12)
    # Eq. (s2lim): far correlations approach phi^2 (disks of radius 5 on 64 px)
    assert abs(s1[32, 32] - phi1 ** 2) < 0.05


def test_s2_counts_and_delta_by_definition():
    # Counts = W*H * direct S2 (exact integers); the swap change of the S2
    # error equals the closed form of the count change,
    # dC(d) = -chi(a+d) - chi(a-d) + chi(b+d) + chi(b-d) + 2[d=0] - [d=b-a] - [d=a-b],
    # written here independently of the oracle's recount.
    img = synth.random_binary(9, 11, 0.4, 4)
    H, W = img.shape
    C = oracle.s2_counts(img)
    np.testing.assert_allclose(C, oracle.s2_direct(img, 1) * H * W, atol=1e-9)
    rng = np.random.default_rng(2)
    t = (C / (H * W) + rng.normal(0, 0.01, size=C.shape)).astype(np.float32)
    flat = img.reshape(-1)
    pairs = [(int(rng.choice(np.flatnonzero(flat == 1))), int(rng.choice(np.flatnonzero(flat == 0)))) for _ in range(6)]
    de = oracle.s2_delta_objective(img, t, pairs)
    chi = (img == 1).astype(np.int64)
    for k, (a, b) in enumerate(pairs):
        ay, ax, by, bx = a // W, a % W, b // W, b % W
        dC = np.zeros((H, W), np.int64)
        for dy in range(H):
            for dx in range(W):
                v = (-chi[(ay + dy) % H, (ax + dx) % W] - chi[(ay - dy) % H, (ax - dx) % W]
                     + chi[(by + dy) % H, (bx + dx) % W] + chi[(by - dy) % H, (bx - dx) % W])
                v += 2 if (dy == 0 and dx == 0) else 0
                v -= 1 if ((by - ay) % H == dy and (bx - ax) % W == dx) else 0
                v -= 1 if ((ay - by) % H == dy and (ax - bx) % W == dx) else 0
                dC[dy, dx] = v
        N = H * W
        e0 = ((t.astype(np.float64) - C / N) ** 2).sum()
        e1 = ((t.astype(np.float64) - (C + dC) / N) ** 2).sum()
        assert de[k] == pytest.approx(e1 - e0, rel=1e-12, abs=1e-15)
