"""Batched evaluation of many images of uneven sizes against the oracle and
against per-image lpf_full."""
import hashlib
import json
import os

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


def _images(n, lo, hi, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        H, W = int(rng.integers(lo, hi + 1)), int(rng.integers(lo, hi + 1))
        f = float(rng.uniform(0.2, 0.6))
        s = int(rng.integers(0, 2 ** 31 - 1))
        out.append([synth.boolean_disks(H, W, 5.0, synth.disks_for_fraction(H, W, 5.0, f), seed=s),
                    synth.ellipses(H, W, f, seed=s), synth.clustered_disks(H, W, f, seed=s)][i % 3])
    return out


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_matches_oracle(gpu_lib, use_graph):
    imgs = _images(10, 33, 100, 3)
    paths = [gpu_lib.lpf_build_paths(min(W // 2, W - 1), min(H // 2, H - 1)) for H, W in (i.shape for i in imgs)]
    d = [torch.from_numpy(i).cuda() for i in imgs]
    b = gpu_lib.lpf_batch_create(d, paths)
    for _ in range(2):  # a second run on the same batch (graph replay) gives the same counts
        counts = gpu_lib.lpf_batch_run(b, use_graph=use_graph)
        torch.cuda.synchronize()
        assert gpu_lib.lpf_batch_status(b) == 0
        for img, p, c in zip(imgs, paths, counts):
            np.testing.assert_array_equal(c.cpu().numpy(), oracle.lpf_full(img, p.rx, p.ry))
        # the walked work of the run: every image walked some of its program, at
        # most all of it
        executed, nominal = gpu_lib.lpf_batch_work(b)
        assert (nominal > 0).all() and (executed > 0).all() and (executed <= nominal).all()


def test_batch_every_words_per_thread_choice(gpu_lib):
    imgs = _images(6, 40, 130, 5)
    paths = [gpu_lib.lpf_build_paths(W // 2, H // 2) for H, W in (i.shape for i in imgs)]
    d = [torch.from_numpy(i).cuda() for i in imgs]
    refs = [oracle.lpf_full(img, p.rx, p.ry) for img, p in zip(imgs, paths)]
    # (word-group counts G = ceil(words / T) of 1 to 4, including 3, which does
    # not divide a block's 8 warps; bands per group from 1 to 4)
    for T in (1, 2, 4, 8):
        choice = []
        for img in imgs:
            nw = (img.shape[1] + 31) // 32
            G = (nw + T - 1) // T
            choice.append(T if G <= 8 else 8)
        b = gpu_lib.lpf_batch_create(d, paths, words_per_thread=choice)
        counts = gpu_lib.lpf_batch_run(b, use_graph=False)
        for c, r in zip(counts, refs):
            np.testing.assert_array_equal(c.cpu().numpy(), r)


def test_mixed_sizes_batch_every_image_equals_the_oracle(gpu_lib):
    # 256 images, 48..256 px, windows r = size/2, autotuned, one graph launch
    # (the batched workload): every count of every image equals the oracle's,
    # compared through the digest of each image's whole table stored by
    # tests/golden/make_lpf_goldens.py; each image also equals its own lpf_full.
    gold = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                       "lpf_mixed_sizes_batch_256.json")))["images"]
    imgs = synth.mixed_sizes_batch(256, seed=4)
    paths = [gpu_lib.lpf_build_paths(W // 2, H // 2) for H, W in (i.shape for i in imgs)]
    d = [torch.from_numpy(i).cuda() for i in imgs]
    b = gpu_lib.lpf_batch_create(d, paths)
    chosen = gpu_lib.lpf_batch_autotune(b)
    assert set(chosen) <= {1, 2, 4, 8}
    counts = gpu_lib.lpf_batch_run(b, use_graph=True)
    torch.cuda.synchronize()
    assert gpu_lib.lpf_batch_status(b) == 0
    bad = []
    for k, (img, p, c, g) in enumerate(zip(imgs, paths, counts, gold)):
        assert (g["H"], g["W"], g["rx"], g["ry"]) == (img.shape[0], img.shape[1], p.rx, p.ry)
        h = c.cpu().numpy()
        if hashlib.sha256(np.ascontiguousarray(h, dtype="<i8").tobytes()).hexdigest() != g["sha256"]:
            bad.append(k)
        single = gpu_lib.lpf_full(d[k], gpu_lib.lpf_build_paths(p.rx, p.ry))
        assert torch.equal(c, single), k
    assert not bad, f"images differing from the oracle: {bad}"


def test_batch_keeps_its_programs_when_the_handles_are_used_alone(gpu_lib):
    # Evaluating a batch's handles on their own in another launch shape
    # uploads the handles' programs for another row stride; the batch keeps
    # its own copies and still gives the oracle's counts.
    imgs = [synth.ellipses(40, 96, 0.35, seed=1), synth.clustered_disks(64, 64, 0.3, seed=2)]
    paths = [gpu_lib.lpf_build_paths(W // 2, H // 2) for H, W in (i.shape for i in imgs)]
    d = [torch.from_numpy(i).cuda() for i in imgs]
    refs = [oracle.lpf_full(i, p.rx, p.ry) for i, p in zip(imgs, paths)]
    b = gpu_lib.lpf_batch_create(d, paths, words_per_thread=[8, 1])  # 8 and 2 staged words per row
    for img, p, dd, r in zip(imgs, paths, d, refs):
        H, W = img.shape
        gpu_lib.lpf_set_launch_shape(p, H, W, 4, 1)  # 4 staged words per row: another row stride
        np.testing.assert_array_equal(gpu_lib.lpf_full(dd, p).cpu().numpy(), r)
    for use_graph in (False, True):
        counts = gpu_lib.lpf_batch_run(b, use_graph=use_graph)
        torch.cuda.synchronize()
        assert gpu_lib.lpf_batch_status(b) == 0
        for c, r in zip(counts, refs):
            np.testing.assert_array_equal(c.cpu().numpy(), r)
