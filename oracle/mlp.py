"""Oracle: the surrogate MLP in FP64 on the CPU (forward, loss, backward, Adam).

TEST INFRASTRUCTURE (see oracle/__init__.py): never imported by the product.

Network (the paper has no counterpart; the form is the one the library
implements): h1 = tanh(x W1 + b1), h2 = tanh(h1 W2 + b2), y = h2 W3 + b3,
loss = mean over batch and outputs of (y - t)^2.

With bf16=True every matrix-product operand is rounded to bfloat16
(round-to-nearest-even from FP32) exactly where the GPU kernels round: the
input x, the weights, the activations h1 and h2 when they feed the next
product, and the back-propagated dy, dh2, dh1 when they feed a product; all
arithmetic is FP64.  With bf16=False this is the plain FP64 network (pinned
by finite differences in tests/test_oracle_mlp.py).

Parameter vector layout: W1 [d_in x w], b1 [w], W2 [w x w], b2 [w],
W3 [w x d_out], b3 [d_out] (row-major).
"""
from __future__ import annotations

import numpy as np


def bf16_round(a) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), via FP32, as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(params, d_in, w, d_out):
    p = np.asarray(params, dtype=np.float64)
    shapes = [(d_in, w), (w,), (w, w), (w,), (w, d_out), (d_out,)]
    out, o = [], 0
    for s in shapes:
        n = int(np.prod(s))
        out.append(p[o:o + n].reshape(s))
        o += n
    assert o == p.size
    return out


def pack(parts):
    return np.concatenate([np.asarray(x, dtype=np.float64).reshape(-1) for x in parts])


def init_params(rng, d_in, w, d_out, out_gain=0.1):
    """Glorot-style random weights, zero biases."""
    W1 = rng.normal(size=(d_in, w)) * np.sqrt(1.0 / d_in)
    W2 = rng.normal(size=(w, w)) * np.sqrt(1.0 / w)
    W3 = rng.normal(size=(w, d_out)) * np.sqrt(1.0 / w) * out_gain
    return pack([W1, np.zeros(w), W2, np.zeros(w), W3, np.zeros(d_out)])


def forward(params, x, d_in, w, d_out, bf16=True):
    W1, b1, W2, b2, W3, b3 = unpack(params, d_in, w, d_out)
    r = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    h1 = np.tanh(r(x) @ r(W1) + b1)
    h2 = np.tanh(r(h1) @ r(W2) + b2)
    y = r(h2) @ r(W3) + b3
    return y, (h1, h2)


def loss_and_grads(params, x, t, d_in, w, d_out, bf16=True):
    W1, b1, W2, b2, W3, b3 = unpack(params, d_in, w, d_out)
    r = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    y, (h1, h2) = forward(params, x, d_in, w, d_out, bf16)
    B = x.shape[0]
    e = y - t
    loss = float(np.mean(e * e))
    dy = 2.0 * e / (B * d_out)
    gW3 = r(h2).T @ r(dy)
    gb3 = dy.sum(axis=0)
    dh2 = (r(dy) @ r(W3).T) * (1.0 - h2 * h2)
    gW2 = r(h1).T @ r(dh2)
    gb2 = dh2.sum(axis=0)
    dh1 = (r(dh2) @ r(W2).T) * (1.0 - h1 * h1)
    gW1 = r(x).T @ r(dh1)
    gb1 = dh1.sum(axis=0)
    return loss, pack([gW1, gb1, gW2, gb2, gW3, gb3])


def adam_step(params, grads, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One bias-corrected Adam step (step counts from 1).  Returns new (p, m, v)."""
    m = b1 * m + (1 - b1) * grads
    v = b2 * v + (1 - b2) * grads * grads
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v
