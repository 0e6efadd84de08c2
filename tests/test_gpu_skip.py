"""The zero-count subtree skip of the walk kernels (the "enhanced" evaluation
of Sec. 3.2 applied to the prefix tree): counts stay exact while the warps
skip work, on the media and sizes of Tab. comptime."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


def _full(lpf, img, p, standard=False):
    d = torch.from_numpy(np.ascontiguousarray(img)).cuda()
    c = (lpf.lpf_full_standard if standard else lpf.lpf_full)(d, p)
    torch.cuda.synchronize()
    assert lpf.lpf_paths_status(p) == 0
    return c.cpu().numpy()


def test_work_counter(gpu_lib):
    p = gpu_lib.lpf_build_paths(47, 47)
    assert gpu_lib.lpf_paths_work(p) == (0, 0)
    # all ones: every phase-1 count is positive, nothing can be skipped
    _full(gpu_lib, np.ones((48, 48), np.uint8), p)
    ex, nom = gpu_lib.lpf_paths_work(p)
    assert nom > 0 and ex == nom
    # chess of 10 px squares on the full domain: most long segments cross a square
    c = _full(gpu_lib, synth.chess(48, 48, 10), p)
    ex, nom = gpu_lib.lpf_paths_work(p)
    assert 0 < ex < 0.8 * nom
    np.testing.assert_array_equal(c, oracle.lpf_full(synth.chess(48, 48, 10), 47, 47))
    # the standard program shares no work (more nominal work); a segment stops
    # once no translation of the tile is left (Alg. 1's early break, per warp)
    cs = _full(gpu_lib, synth.chess(48, 48, 10), p, standard=True)
    ex_s, nom_s = gpu_lib.lpf_paths_work(p)
    assert 0 < ex_s < nom_s and nom_s > nom
    np.testing.assert_array_equal(cs, c)


def _sampled(lpf, img, p, n_vec, seed):
    H, W = img.shape
    rx, ry = p.rx, p.ry
    c = _full(lpf, img, p)
    rng = np.random.default_rng(seed)
    vecs = [(int(rng.integers(-rx, rx + 1)), int(rng.integers(0, ry + 1))) for _ in range(n_vec)]
    vecs += [(0, 0), (1, 0), (0, 1), (1, 1), (10, 10), (-10, 10), (rx, ry), (-rx, ry), (rx, 0), (0, ry), (3, 2)]
    ref = oracle.count_list(img, vecs)
    for k, (dx, dy) in enumerate(vecs):
        i = (dy + ry) * (2 * rx + 1) + (dx + rx)
        assert c[0, i] == ref[k, 0] and c[1, i] == ref[k, 1], (dx, dy)
    np.testing.assert_array_equal(c, c[:, ::-1])
    assert c[1, c.shape[1] // 2] == int(img.sum()) and c[0, c.shape[1] // 2] == img.size - int(img.sum())
    return c


def test_comptime_500_full_domain(gpu_lib):
    # the largest case of Tab. comptime: 500 x 500, every vector of the half-domain
    p = gpu_lib.lpf_build_paths(499, 499)
    chess = synth.chess(500, 500, 10)
    c = _sampled(gpu_lib, chess, p, 24, 1)
    ex, nom = gpu_lib.lpf_paths_work(p)
    assert ex < 0.2 * nom
    # Closed form: along (k, k) the colour stays the same from (x, y) exactly when
    # x = y (mod 10) (both coordinates cross a square edge at the same step), and
    # along (-k, k) exactly when x mod 10 + y mod 10 = 9: 500^2 / 10 starts either way.
    for dx, dy in ((10, 10), (37, 37), (499, 499), (-10, 10), (-250, 250), (-499, 499)):
        i = (dy + 499) * 999 + (dx + 499)
        assert c[0, i] + c[1, i] == 25000, (dx, dy)
    _sampled(gpu_lib, synth.foam(500, 500, 0.75, seed=5), p, 24, 2)
    _sampled(gpu_lib, synth.squares(500, 500, 4, 0.2, seed=7), p, 24, 3)


def test_batch_with_skips(gpu_lib):
    imgs = [synth.chess(64, 64, 10), synth.chess(50, 70, 10), synth.squares(60, 60, 4, 0.2, seed=7),
            np.ones((40, 40), np.uint8), synth.foam(80, 80, 0.75, seed=5)]
    paths = [gpu_lib.lpf_build_paths(W - 1, H - 1) for H, W in (i.shape for i in imgs)]
    b = gpu_lib.lpf_batch_create([torch.from_numpy(i).cuda() for i in imgs], paths)
    counts = gpu_lib.lpf_batch_run(b, use_graph=True)
    torch.cuda.synchronize()
    assert gpu_lib.lpf_batch_status(b) == 0
    for img, p, c in zip(imgs, paths, counts):
        np.testing.assert_array_equal(c.cpu().numpy(), oracle.lpf_full(img, p.rx, p.ry))


def test_skip_with_a_selection_and_an_ensemble(gpu_lib):
    # The skip tests the tile's selected translations only (Monte-Carlo
    # variant), and each cut of an ensemble skips on its own.
    img = synth.chess(64, 96, 10)
    p = gpu_lib.lpf_build_paths(95, 63)
    sel = (np.random.default_rng(3).random(img.shape) < 0.1).astype(np.uint8)
    c = gpu_lib.lpf_full_mc(torch.from_numpy(img).cuda(), p, torch.from_numpy(sel).cuda())
    torch.cuda.synchronize()
    assert gpu_lib.lpf_paths_status(p) == 0
    # with a selection L(v) and L(-v) count different starts: the canonical half
    # is computed, the other half mirrors it
    base = p.base
    np.testing.assert_array_equal(c.cpu().numpy()[:, base:], oracle.lpf_full_selected(img, 95, 63, sel)[:, base:])
    ex, nom = gpu_lib.lpf_paths_work(p)
    assert 0 < ex < nom
    vol = np.stack([synth.chess(64, 96, 10), synth.squares(64, 96, 4, 0.2, seed=7), synth.foam(64, 96, 0.75, seed=5)])
    e = gpu_lib.lpf_full_ensemble(torch.from_numpy(vol).cuda(), p)
    torch.cuda.synchronize()
    ref = sum(oracle.lpf_full(v, 95, 63) for v in vol)
    np.testing.assert_array_equal(e.cpu().numpy(), ref)
