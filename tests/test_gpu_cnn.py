"""GPU proposer network against its float64 CPU reference.

The GPU convolutions run on tensor cores with bfloat16 operands and float32
accumulation: weights are stored as bfloat16, activations are rounded to
bfloat16 where they enter a product, gradients enter as two bfloat16 terms
(high and low part).  Two comparisons:

- against the reference given the same roundings (weights rounded, and the
  oracle's operand-rounding hook set to the same round-to-nearest-even for
  layer inputs): what remains is float32 accumulation order, the low-term
  residue of the gradients (2^-16 relative), and the rare activation whose
  float32 and float64 values round to neighbouring bfloat16 values (one
  bfloat16 ulp, 2^-8 relative, of one operand); tolerance 3e-3 of the
  largest magnitude (forward);
- the forward pass also against the plain float64 reference (only the
  weights rounded): the bfloat16 rounding of activations, BF16-scale
  tolerance 1e-2 of the largest magnitude.

Gradients are compared with the rounded reference only, at the BF16-scale
1e-2 of each layer's largest gradient: they are the gradients of the network
the library evaluates (bfloat16 activations).  Against the unrounded network
the first layer's gradients differ by a few percent, because the loss's
residuals s1[a] + s0[b] - y cancel and amplify the forward rounding.
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


def _per_layer_close(grads, ref, got, tol):
    """Each layer's gradients within tol of that layer's largest reference gradient."""
    off = 0
    for li, (dw, db) in enumerate(grads):
        n = dw.size + db.size
        seg_ref, seg_got = ref[off:off + n], got[off:off + n]
        err = np.abs(seg_got - seg_ref).max() / (np.abs(seg_ref).max() + 1e-30)
        print(f"layer {li}: rel grad err {err:.2e} (tol {tol:.0e})")
        assert err <= tol
        off += n


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
    ref, _ = ocnn.forward(ref_params, ocnn.features(cell), rnd=_bf16_round)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    plain, _ = ocnn.forward(ref_params, ocnn.features(cell))
    err_plain = np.abs(got - plain).max() / np.abs(plain).max()
    print(f"forward {H}x{W}: rel err {err:.2e} (rounded reference), {err_plain:.2e} (float64)")
    assert err <= 3e-3
    assert err_plain <= 1e-2


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
    got = g.cpu().numpy().astype(np.float64)
    for rnd, tol in ((_bf16_round, 1e-2),):
        out, acts = ocnn.forward(ref_params, x, rnd=rnd)
        grads = ocnn.backward(ref_params, acts, ocnn.loss_grad_out(out, a, b, y.astype(np.float64)), rnd=rnd)
        ref = np.concatenate([np.concatenate([dw.reshape(-1), db]) for dw, db in grads])
        assert abs(loss.item() - ocnn.loss(out, a, b, y.astype(np.float64))) <= tol * max(1.0, loss.item())
        _per_layer_close(grads, ref, got, tol)


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
    yd = y.astype(np.float64)
    got = g.cpu().numpy().astype(np.float64)
    # The listwise gradient p_i - q_i is a difference of nearly equal
    # probabilities: it amplifies the few activations whose float32 and
    # float64 values round to neighbouring bfloat16 values (measured up to
    # 1.6e-2 of a layer's largest gradient at beta = 0.5); tolerance 2e-2.
    for rnd, tol in ((_bf16_round, 2e-2),):
        out, acts = ocnn.forward(ref_params, ocnn.features(cell), rnd=rnd)
        grads = ocnn.backward(ref_params, acts, ocnn.listwise_grad_out(out, a, b, yd, beta), rnd=rnd)
        assert abs(loss.item() - ocnn.listwise_loss(out, a, b, yd, beta)) <= tol * max(1.0, abs(loss.item()))
        ref = np.concatenate([np.concatenate([dw.reshape(-1), db]) for dw, db in grads])
        _per_layer_close(grads, ref, got, tol)
