"""The size envelope of lpf_full: the largest supported widths, heights and
windows against sampled oracle counts, and a clean LPF_EINVAL or
LPF_EUNSUPPORTED beyond them."""
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


def test_widest_and_tallest_images_at_the_size_limit(gpu_lib):
    # 8192 words of translations in a row on one side: the image's (wide) or
    # the transpose's (tall)
    _sampled_check(gpu_lib, synth.random_binary(40, 8192, 0.6, 5), 200, 12, 16, 6)
    _sampled_check(gpu_lib, synth.random_binary(8192, 40, 0.6, 7), 12, 200, 16, 8)


def test_full_domain_300(gpu_lib):
    img = synth.clustered_disks(300, 300, 0.35, seed=3)
    _sampled_check(gpu_lib, img, 299, 299, 16, 4)


def test_beyond_the_envelope_is_refused(gpu_lib):
    p = gpu_lib.lpf_build_paths(8, 4)
    for shape in ((16, 8193), (8193, 16)):
        with pytest.raises(gpu_lib.LpfError) as e:
            gpu_lib.lpf_full(torch.zeros(shape, dtype=torch.uint8, device="cuda"), p)
        assert e.value.code == -1  # LPF_EINVAL
    # halo rows of min(rx, ry) = 299 x 277 words of a 8192-wide row: beyond shared memory
    q = gpu_lib.lpf_build_paths(299, 299)
    with pytest.raises(gpu_lib.LpfError) as e:
        gpu_lib.lpf_full(torch.zeros((320, 8192), dtype=torch.uint8, device="cuda"), q)
    assert e.value.code == -5  # LPF_EUNSUPPORTED


def test_long_one_sided_windows_fit_on_the_transposed_side(gpu_lib):
    # a window 4 x 1500: the y-major vectors run along rows of the transposed
    # image, whose halo is min(rx, ry - 1) = 4 rows, so the image fits
    img = synth.random_binary(1600, 64, 0.7, 9)
    _sampled_check(gpu_lib, img, 4, 1500, 12, 10)
