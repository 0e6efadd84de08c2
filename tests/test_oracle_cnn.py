"""Pins for the proposer network's CPU reference: parameter count, the
circular convolution against a direct loop, and every gradient against
central finite differences of the loss."""
import numpy as np
import pytest

import synth
from oracle import cnn


def test_parameter_count():
    assert cnn.n_params() == 9 * (2 * 32 + 32 * 64 + 64 * 48 + 48 * 32 + 32 * 2) + (32 + 64 + 48 + 32 + 2) == 61234


def test_circular_convolution_by_loops():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(5, 7, 3))
    w = rng.normal(size=(9, 3, 4))
    b = rng.normal(size=4)
    out = cnn.conv(x, w, b)
    H, W = 5, 7
    for y in range(H):
        for xx in range(W):
            for co in range(4):
                s = b[co]
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        tap = (dy + 1) * 3 + (dx + 1)
                        s += sum(x[(y + dy) % H, (xx + dx) % W, ci] * w[tap, ci, co] for ci in range(3))
                assert abs(out[y, xx, co] - s) < 1e-12


def test_gradients_by_central_differences():
    cell = synth.clustered_disks(12, 10, 0.4, seed=3)
    x = cnn.features(cell)
    params = cnn.init_params(5)
    rng = np.random.default_rng(1)
    params = [(w + 0.05 * rng.normal(size=w.shape), b + 0.05 * rng.normal(size=b.shape)) for w, b in params]
    a_idx = np.array([3, 17, 40, 88])
    b_idx = np.array([5, 60, 41, 100])
    y = np.array([0.3, -1.0, 0.7, 0.0])
    out, acts = cnn.forward(params, x)
    grads = cnn.backward(params, acts, cnn.loss_grad_out(out, a_idx, b_idx, y))
    eps = 1e-6
    for li, (w, b) in enumerate(params):
        for arr, garr in ((w, grads[li][0]), (b, grads[li][1])):
            flat = arr.reshape(-1)
            gflat = garr.reshape(-1)
            for j in rng.choice(flat.size, size=min(6, flat.size), replace=False):
                old = flat[j]
                flat[j] = old + eps
                lp = cnn.loss(cnn.forward(params, x)[0], a_idx, b_idx, y)
                flat[j] = old - eps
                lm = cnn.loss(cnn.forward(params, x)[0], a_idx, b_idx, y)
                flat[j] = old
                fd = (lp - lm) / (2 * eps)
                assert abs(fd - gflat[j]) <= 1e-6 * max(1.0, abs(fd)), (li, j, fd, gflat[j])


def test_listwise_gradient_by_central_differences():
    # d/ds of logsumexp(s) - sum q s is p - q; checked numerically through
    # the scores of the output map
    rng = np.random.default_rng(4)
    out = rng.normal(size=(6, 7, 2))
    a_idx = np.array([0, 9, 20, 33])
    b_idx = np.array([4, 9, 21, 40])
    y = np.array([1.0, -0.5, 2.0, 0.0])
    g = cnn.listwise_grad_out(out, a_idx, b_idx, y, 0.7)
    eps = 1e-6
    for idx in [(0, 0, 1), (1, 2, 1), (0, 4, 0), (1, 2, 0), (5, 5, 0), (3, 2, 1)]:
        o1, o2 = out.copy(), out.copy()
        o1[idx] += eps
        o2[idx] -= eps
        num = (cnn.listwise_loss(o1, a_idx, b_idx, y, 0.7) - cnn.listwise_loss(o2, a_idx, b_idx, y, 0.7)) / (2 * eps)
        assert abs(num - g[idx]) < 1e-8
    # equal scores and equal targets: zero gradient; the loss is then log n
    z = np.zeros_like(out)
    assert np.abs(cnn.listwise_grad_out(z, a_idx, b_idx, np.zeros(4), 1.0)).max() < 1e-15
    assert cnn.listwise_loss(z, a_idx, b_idx, np.zeros(4), 1.0) == pytest.approx(np.log(4))


def test_operand_rounding_hook():
    # The optional rounding hook is applied to the layer inputs only: the
    # identity gives the plain float64 network, and a rounding of the inputs
    # changes the output no more than the rounding's size allows.
    import numpy as np

    from oracle import cnn as ocnn
    params = ocnn.init_params(2)
    rng = np.random.default_rng(3)
    cell = (rng.random((12, 10)) < 0.4).astype(np.uint8)
    x = ocnn.features(cell)
    plain, _ = ocnn.forward(params, x)
    same, _ = ocnn.forward(params, x, rnd=lambda a: a)
    np.testing.assert_array_equal(plain, same)
    coarse, acts = ocnn.forward(params, x, rnd=lambda a: np.round(a * 256.0) / 256.0)
    assert 0 < np.abs(coarse - plain).max() < 0.05 * np.abs(plain).max()
    g = ocnn.loss_grad_out(coarse, np.array([3]), np.array([7]), np.array([0.5]))
    a = ocnn.backward(params, acts, g, rnd=lambda v: v)
    b = ocnn.backward(params, acts, g)
    for (wa, ba), (wb, bb) in zip(a, b):
        np.testing.assert_array_equal(wa, wb)
        np.testing.assert_array_equal(ba, bb)
