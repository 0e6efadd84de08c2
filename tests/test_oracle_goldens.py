"""The stored oracle tables (tests/golden/make_lpf_goldens.py, which calls
only the oracle) agree with the oracle run now on sampled entries, and with
their stored digests; they serve the full-size GPU parity tests."""
import hashlib
import json
import os

import numpy as np

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _sha(counts):
    return hashlib.sha256(np.ascontiguousarray(counts, dtype="<i8").tobytes()).hexdigest()


def test_ellipses_512_table():
    g = np.load(os.path.join(GOLDEN, "lpf_ellipses_512_r256.npz"))
    ref = g["counts"].astype(np.int64)
    assert ref.shape == (2, 513 * 513)
    assert _sha(ref) == str(g["sha256"])
    img = synth.ellipses_512()
    vecs = [(0, 0), (1, 0), (256, 0), (-256, 256), (17, -129), (-7, 200), (255, 3), (0, -256)]
    for (dx, dy), r in zip(vecs, oracle.count_list(img, vecs)):
        k = oracle.full_index(dx, dy, 256, 256)
        assert ref[0, k] == r[0] and ref[1, k] == r[1]
    np.testing.assert_array_equal(ref, ref[:, ::-1])  # Eq. (symmetry)


def test_mixed_sizes_batch_digests():
    d = json.load(open(os.path.join(GOLDEN, "lpf_mixed_sizes_batch_256.json")))
    imgs = synth.mixed_sizes_batch(256, seed=4)
    assert len(d["images"]) == len(imgs) == 256
    for k in (0, 1, 2, 77, 255):  # recomputed now: small images take a fraction of a second
        img, e = imgs[k], d["images"][k]
        assert img.shape == (e["H"], e["W"])
        if img.size > 120 * 120:
            continue
        c = oracle.lpf_full(img, e["rx"], e["ry"])
        assert _sha(c) == e["sha256"]
        assert int(c[0].sum()) == e["sum0"] and int(c[1].sum()) == e["sum1"]


def test_delta_clustered_128_sample():
    g = np.load(os.path.join(GOLDEN, "lpf_delta_clustered_128.npz"))
    cell = synth.clustered_cell_128()
    pairs, sample, dc = g["pairs"], g["sample"], g["dcounts"]
    assert pairs.shape == (4096, 2) and len(sample) == 64 and dc.shape[0] == 64
    assert {0, 4095, 100, 101, 102, 103, 104} <= set(sample.tolist())
    # identities change nothing; the reversed pair is the same exchange
    for j, k in enumerate(sample):
        if k in (100, 101, 102, 103):
            assert not dc[j].any()
    j0 = int(np.flatnonzero(sample == 0)[0])
    np.testing.assert_array_equal(dc[j0], oracle.delta_swap(cell, 64, 64, pairs[[0]])[0])
    np.testing.assert_array_equal(g["counts"][:, ::97], oracle.lpf_full(cell, 64, 64)[:, ::97])
