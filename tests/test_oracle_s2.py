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
    img = synth.config1_image()
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
