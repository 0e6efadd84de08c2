"""GPU two-point probability (s2_fft) against the oracle's direct sum of
Eq. (S2dis).  Transforms run in double precision and the result is rounded
to float32, so the bound is half an ulp of float32 plus the double FFT's
rounding (a few 1e-16 times log2(WH) relative to the largest value)."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("H,W,seed", [(64, 64, 1), (37, 45, 2), (1, 9, 3), (16, 1, 4), (96, 130, 5)])
def test_s2_matches_direct_sum(gpu_lib, H, W, seed):
    img = synth.clustered_disks(H, W, 0.35, seed=seed) if min(H, W) > 8 else synth.random_binary(H, W, 0.5, seed)
    d = torch.from_numpy(img).cuda()
    for p in (0, 1):
        got = gpu_lib.s2_fft(d, p).cpu().numpy().astype(np.float64)
        ref = oracle.s2_direct(img, p)
        tol = 2.0 ** -24 * np.abs(ref) + 1e-12 * (1 + np.log2(H * W))
        assert (np.abs(got - ref) <= tol).all(), np.abs(got - ref).max()


def test_s2_properties_512(gpu_lib):
    img = synth.ellipses_512()
    d = torch.from_numpy(img).cuda()
    s1 = gpu_lib.s2_fft(d, 1).cpu().numpy().astype(np.float64)
    s0 = gpu_lib.s2_fft(d, 0).cpu().numpy().astype(np.float64)
    phi = img.mean()
    assert s1[0, 0] == pytest.approx(phi, rel=1e-6)                                   # Eq. (s2zero)
    np.testing.assert_allclose(s1 - s0, phi ** 2 - (1 - phi) ** 2, atol=1e-6)          # Eq. (S2add)
    assert s1.sum() == pytest.approx(phi ** 2 * img.size, rel=1e-5)
    # sampled entries against the direct sum, one offset at a time
    chi = (img == 1).astype(np.int64)
    for (y, x) in [(0, 1), (3, 250), (511, 7), (256, 256)]:
        ref = (chi * np.roll(chi, (-y, -x), axis=(0, 1))).sum() / img.size
        assert abs(s1[y, x] - ref) <= 2.0 ** -24 * ref + 1e-12
