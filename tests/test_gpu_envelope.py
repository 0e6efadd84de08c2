"""The size envelope of lpf_full: the largest supported widths and windows
against sampled oracle counts, and a clean LPF_EUNSUPPORTED beyond them."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


def _sampled_check(gpu_lib, img, rx, ry, n_vec, seed):
    p = gpu_lib.lpf_build_paths(rx, ry)
    c = gpu_lib.lpf_full(torch.from_numpy(img).cuda(), p).cpu().numpy()
    assert gpu_lib.lpf_paths_status(p) == 0
    rng = np.random.default_rng(seed)
    vecs = [(int(rng.integers(-rx, rx + 1)), int(rng.integers(0, ry + 1))) for _ in range(n_vec)]
    vecs += [(rx, ry), (-rx, ry), (rx, 0), (0, ry), (0, 0)]
    ref = oracle.count_list(img, vecs)
    for k, (dx, dy) in enumerate(vecs):
        idx = (dy + ry) * (2 * rx + 1) + (dx + rx)
        assert c[0, idx] == ref[k, 0] and c[1, idx] == ref[k, 1], (dx, dy)
    np.testing.assert_array_equal(c, c[:, ::-1])  # point symmetry
    assert c[1, (2 * rx + 1) * (2 * ry + 1) // 2] == int(img.sum())


def test_widest_image(gpu_lib):
    img = synth.random_binary(40, 4096, 0.6, 1)
    _sampled_check(gpu_lib, img, 200, 12, 24, 2)


def test_full_domain_300(gpu_lib):
    img = synth.clustered_disks(300, 300, 0.35, seed=3)
    _sampled_check(gpu_lib, img, 299, 299, 16, 4)


def test_beyond_the_envelope_is_refused(gpu_lib):
    p = gpu_lib.lpf_build_paths(8, 4)
    with pytest.raises(gpu_lib.LpfError) as e:
        gpu_lib.lpf_full(torch.zeros((16, 4100), dtype=torch.uint8, device="cuda"), p)
    assert e.value.code in (-1, -5)  # LPF_EINVAL or LPF_EUNSUPPORTED
    q = gpu_lib.lpf_build_paths(4, 1500)  # halo rows of 1500 x 130 words: far beyond shared memory
    with pytest.raises(gpu_lib.LpfError) as e:
        gpu_lib.lpf_full(torch.zeros((1600, 4096), dtype=torch.uint8, device="cuda"), q)
    assert e.value.code == -5
