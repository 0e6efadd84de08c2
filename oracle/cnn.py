"""Oracle of the swap-proposal network: forward and backward of a small
convolutional network in float64 with numpy.

TEST INFRASTRUCTURE ONLY (see the package docstring).  The paper has no
learned part; this is the reference the library's CUDA kernels for the
proposer are checked against.

Network (every layer a 3x3 convolution with circular padding, i.e. the
periodic medium's wrap, followed by ReLU except the last):
  input  [2][H][W]  channel 0 = cell (0/1), channel 1 = interfacial mask (0/1)
  conv 2 -> 32, conv 32 -> 64, conv 64 -> 48, conv 48 -> 32, conv 32 -> 2
  output [2][H][W]  channel 0 = score of phase-0 pixels (the "b" of a swap),
                    channel 1 = score of phase-1 pixels (the "a" of a swap)
Weights W_l[tap][cin][cout] with tap = (dy+1)*3 + (dx+1), dy, dx in {-1,0,1};
out[y][x][co] = b[co] + sum_tap sum_ci in[(y+dy)%H][(x+dx)%W][ci] * W[tap][ci][co].

Operand rounding (optional): the network's arithmetic contract is bfloat16
weights and activations with float32 accumulation (gradients enter products
as two bfloat16 terms, close to float32).  Callers pass bfloat16-rounded
weights; `rnd`, when given, is applied to the layer inputs where they enter
a product (the forward convolutions and the weight-gradient products), so
that a comparison with the library isolates the order of float32
accumulation.  Gradients, bias gradients and ReLU masks are not rounded.
With rnd = None everything stays float64.

Loss of one snapshot with logged candidates (a_i, b_i, y_i), i = 1..n:
  L = 1/(2n) * sum_i (s1[a_i] + s0[b_i] - y_i)^2, or (listwise) the
  cross-entropy -sum_i q_i log p_i with q = softmax(y / beta) and
  p = softmax(s1[a] + s0[b]) over the snapshot's candidates.
"""
from __future__ import annotations

import numpy as np

CHANNELS = (2, 32, 64, 48, 32, 2)


def init_params(seed: int):
    """He-scaled normal weights (float64) and zero biases."""
    rng = np.random.default_rng(seed)
    params = []
    for cin, cout in zip(CHANNELS[:-1], CHANNELS[1:]):
        w = rng.normal(0.0, np.sqrt(2.0 / (9 * cin)), size=(9, cin, cout))
        b = np.zeros(cout)
        params.append((w, b))
    return params


def n_params() -> int:
    return sum(9 * a * b + b for a, b in zip(CHANNELS[:-1], CHANNELS[1:]))


def features(cell: np.ndarray) -> np.ndarray:
    """Input [H][W][2]: cell value and interfacial mask (4-neighbourhood, torus)."""
    c = np.asarray(cell, np.float64)
    inter = np.zeros(c.shape, bool)
    for ax, sh in ((0, 1), (0, -1), (1, 1), (1, -1)):
        inter |= np.roll(c, sh, axis=ax) != c
    return np.stack([c, inter.astype(np.float64)], axis=-1)


def _shift(x, dy, dx):
    """x[(y+dy)%H][(x+dx)%W] as an array indexed by (y, x)."""
    return np.roll(x, shift=(-dy, -dx), axis=(0, 1))


def conv(x, w, b):
    out = np.zeros(x.shape[:2] + (w.shape[2],))
    for tap in range(9):
        dy, dx = tap // 3 - 1, tap % 3 - 1
        out += _shift(x, dy, dx) @ w[tap]
    return out + b


def _id(a):
    return a


def forward(params, x, rnd=None):
    """Returns the output [H][W][2] and the list of layer inputs (for backward)."""
    r = rnd or _id
    acts = [x]
    h = x
    for li, (w, b) in enumerate(params):
        h = conv(r(h), w, b)
        if li < len(params) - 1:
            h = np.maximum(h, 0.0)
        acts.append(h)
    return h, acts


def loss(out, a_idx, b_idx, y):
    W = out.shape[1]
    s1 = out[a_idx // W, a_idx % W, 1]
    s0 = out[b_idx // W, b_idx % W, 0]
    r = s1 + s0 - y
    return 0.5 * np.mean(r * r)


def loss_grad_out(out, a_idx, b_idx, y):
    """dL/d out, [H][W][2]."""
    H, W = out.shape[:2]
    n = len(y)
    g = np.zeros_like(out)
    r = out[a_idx // W, a_idx % W, 1] + out[b_idx // W, b_idx % W, 0] - y
    for i in range(n):
        g[a_idx[i] // W, a_idx[i] % W, 1] += r[i] / n
        g[b_idx[i] // W, b_idx[i] % W, 0] += r[i] / n
    return g


def listwise_loss(out, a_idx, b_idx, y, beta: float):
    """Cross-entropy between the candidates' target distribution
    q = softmax(y / beta) and the model's p = softmax(s1[a] + s0[b])."""
    W = out.shape[1]
    s = out[a_idx // W, a_idx % W, 1] + out[b_idx // W, b_idx % W, 0]
    q = np.exp(y / beta - np.max(y / beta))
    q /= q.sum()
    ls = np.max(s) + np.log(np.sum(np.exp(s - np.max(s))))
    return float(ls - np.sum(q * s))


def listwise_grad_out(out, a_idx, b_idx, y, beta: float):
    """dL/d out of listwise_loss: p_i - q_i on both pixels of candidate i."""
    W = out.shape[1]
    s = out[a_idx // W, a_idx % W, 1] + out[b_idx // W, b_idx % W, 0]
    p = np.exp(s - np.max(s))
    p /= p.sum()
    q = np.exp(y / beta - np.max(y / beta))
    q /= q.sum()
    g = np.zeros_like(out)
    for i in range(len(y)):
        g[a_idx[i] // W, a_idx[i] % W, 1] += p[i] - q[i]
        g[b_idx[i] // W, b_idx[i] % W, 0] += p[i] - q[i]
    return g


def backward(params, acts, gout, rnd=None):
    """Gradients [(dW, db), ...] of the loss given dL/d out."""
    r = rnd or _id
    grads = [None] * len(params)
    g = gout
    for li in range(len(params) - 1, -1, -1):
        w, b = params[li]
        x = r(acts[li])
        if li < len(params) - 1:
            g = g * (acts[li + 1] > 0)       # ReLU: act > 0 exactly where its input was > 0
        gr = g
        dw = np.zeros_like(w)
        for tap in range(9):
            dy, dx = tap // 3 - 1, tap % 3 - 1
            xs = _shift(x, dy, dx)
            dw[tap] = xs.reshape(-1, xs.shape[2]).T @ gr.reshape(-1, gr.shape[2])
        db = g.sum(axis=(0, 1))
        grads[li] = (dw, db)
        if li > 0:
            gx = np.zeros_like(x)
            for tap in range(9):
                dy, dx = tap // 3 - 1, tap % 3 - 1
                gx += _shift(gr @ w[tap].T, -dy, -dx)
            g = gx
    return grads
