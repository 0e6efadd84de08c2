"""GPU proposer network against its float64 CPU reference.

The GPU uses bfloat16 copies of the weights; the reference is given the same
bfloat16-rounded values (in float64), so the remaining difference is float32
accumulation: a forward layer sums 9*Cin <= 576 products, so relative errors
stay at a few 1e-6 of the summed magnitudes; the tolerance below is 1e-4 of
the largest magnitude of each compared array.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import cnn as ocnn

pytestmark = pytest.mark.gpu


def _bf16_round(a):
    x = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    x = ((x + 0x7FFF + ((x >> 16) & 1)) >> 16) << 16  # round to nearest even
    return x.astype(np.uint32).view(np.float32).astype(np.float64)


def _flat(params):
    return np.concatenate([np.concatenate([w.reshape(-1), b]) for w, b in params]).astype(np.float32)


def _params_for_reference(params):
    return [(_bf16_round(w), np.asarray(b, np.float32).astype(np.float64)) for w, b in params]


def _setup(gpu_lib, H, W, seed):
    params = ocnn.init_params(seed)
    rng = np.random.default_rng(seed)
    params = [(w, 0.05 * rng.normal(size=b.shape)) for w, b in params]
    net = gpu_lib.lpf_cnn_create(H, W, seed)
    gpu_lib.lpf_cnn_set_params(net, _flat(params))
    return net, _params_for_reference(params)


def test_param_roundtrip(gpu_lib):
    net = gpu_lib.lpf_cnn_create(16, 16, 3)
    assert net.n_params == ocnn.n_params() == 61234
    p = np.random.default_rng(0).normal(size=net.n_params).astype(np.float32)
    gpu_lib.lpf_cnn_set_params(net, p)
    np.testing.assert_array_equal(gpu_lib.lpf_cnn_get_params(net), p)


@pytest.mark.parametrize("H,W", [(16, 16), (37, 23), (128, 128)])
def test_forward_matches_reference(gpu_lib, H, W):
    net, ref_params = _setup(gpu_lib, H, W, 1)
    cell = synth.clustered_disks(H, W, 0.35, seed=2)
    got = gpu_lib.lpf_cnn_forward(net, torch.from_numpy(cell).cuda()).cpu().numpy().astype(np.float64)
    ref, _ = ocnn.forward(ref_params, ocnn.features(cell))
    assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max()


@pytest.mark.parametrize("H,W", [(16, 16), (40, 28)])
def test_gradients_match_reference(gpu_lib, H, W):
    net, ref_params = _setup(gpu_lib, H, W, 4)
    cell = synth.clustered_disks(H, W, 0.4, seed=5)
    rng = np.random.default_rng(6)
    flat = cell.reshape(-1)
    a = rng.choice(np.flatnonzero(flat == 1), 12).astype(np.int32)
    b = rng.choice(np.flatnonzero(flat == 0), 12).astype(np.int32)
    y = rng.normal(size=12).astype(np.float32)
    pairs = np.stack([a, b], axis=1)
    g, loss = gpu_lib.lpf_cnn_gradients(net, torch.from_numpy(cell).cuda(), torch.from_numpy(pairs).cuda(),
                                        torch.from_numpy(y).cuda())
    x = ocnn.features(cell)
    out, acts = ocnn.forward(ref_params, x)
    grads = ocnn.backward(ref_params, acts, ocnn.loss_grad_out(out, a, b, y.astype(np.float64)))
    ref = np.concatenate([np.concatenate([dw.reshape(-1), db]) for dw, db in grads])
    got = g.cpu().numpy().astype(np.float64)
    assert abs(loss.item() - ocnn.loss(out, a, b, y.astype(np.float64))) <= 1e-4 * max(1.0, loss.item())
    # per layer: relative to that layer's largest gradient
    off = 0
    for (dw, db) in grads:
        n = dw.size + db.size
        seg_ref, seg_got = ref[off:off + n], got[off:off + n]
        assert np.abs(seg_got - seg_ref).max() <= 2e-3 * np.abs(seg_ref).max() + 1e-7
        off += n


def test_training_reduces_loss(gpu_lib):
    H = W = 32
    net = gpu_lib.lpf_cnn_create(H, W, 7)
    rng = np.random.default_rng(8)
    B, n = 4, 16
    cells = np.stack([synth.clustered_disks(H, W, 0.3, seed=10 + i) for i in range(B)])
    pairs = np.zeros((B, n, 2), np.int32)
    for i in range(B):
        flat = cells[i].reshape(-1)
        pairs[i, :, 0] = rng.choice(np.flatnonzero(flat == 1), n)
        pairs[i, :, 1] = rng.choice(np.flatnonzero(flat == 0), n)
    y = rng.normal(size=(B, n)).astype(np.float32)
    c, p, t = (torch.from_numpy(v).cuda() for v in (cells, pairs, y))
    first = gpu_lib.lpf_cnn_train_step(net, c, p, t, 1e-3).item()
    for _ in range(200):
        last = gpu_lib.lpf_cnn_train_step(net, c, p, t, 1e-3).item()
    assert last < 0.2 * first


@pytest.mark.parametrize("beta", [0.5, 2.0])
def test_listwise_gradients_match_reference(gpu_lib, beta):
    H = W = 24
    net, ref_params = _setup(gpu_lib, H, W, 8)
    gpu_lib.lpf_cnn_set_loss(net, "listwise", beta)
    cell = synth.clustered_disks(H, W, 0.4, seed=9)
    rng = np.random.default_rng(10)
    flat = cell.reshape(-1)
    a = rng.choice(np.flatnonzero(flat == 1), 16).astype(np.int32)
    b = rng.choice(np.flatnonzero(flat == 0), 16).astype(np.int32)
    y = rng.normal(size=16).astype(np.float32)
    pairs = np.stack([a, b], axis=1)
    g, loss = gpu_lib.lpf_cnn_gradients(net, torch.from_numpy(cell).cuda(), torch.from_numpy(pairs).cuda(),
                                        torch.from_numpy(y).cuda())
    out, acts = ocnn.forward(ref_params, ocnn.features(cell))
    yd = y.astype(np.float64)
    grads = ocnn.backward(ref_params, acts, ocnn.listwise_grad_out(out, a, b, yd, beta))
    assert abs(loss.item() - ocnn.listwise_loss(out, a, b, yd, beta)) <= 1e-4 * max(1.0, abs(loss.item()))
    ref = np.concatenate([np.concatenate([dw.reshape(-1), db]) for dw, db in grads])
    got = g.cpu().numpy().astype(np.float64)
    off = 0
    for (dw, db) in grads:
        n = dw.size + db.size
        seg_ref, seg_got = ref[off:off + n], got[off:off + n]
        assert np.abs(seg_got - seg_ref).max() <= 2e-3 * np.abs(seg_ref).max() + 1e-7
        off += n
