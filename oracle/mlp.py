"""FP64 numpy reference of the surrogate network.  TEST INFRASTRUCTURE ONLY.

depth weight layers in -> hidden -> ... -> out, tanh after every layer but the last; loss
L = mean over samples and outputs of (y - t)^2; parameters one vector, per layer W (out x in,
row-major) then b (out).  Gradients by reverse-mode differentiation written out layer by
layer; Adam as in Kingma & Ba (2015), bias-corrected, beta1 0.9, beta2 0.999, eps 1e-8.
"""
from __future__ import annotations

import numpy as np


def layer_dims(in_dim, hidden, depth, out_dim):
    return [in_dim] + [hidden] * (depth - 1) + [out_dim]


def unpack(p, dims):
    Ws, bs, off = [], [], 0
    for a, b in zip(dims[:-1], dims[1:]):
        Ws.append(np.asarray(p[off: off + a * b], np.float64).reshape(b, a))
        off += a * b
        bs.append(np.asarray(p[off: off + b], np.float64))
        off += b
    return Ws, bs


def forward(p, dims, x):
    Ws, bs = unpack(p, dims)
    h = np.asarray(x, np.float64)
    acts = [h]
    for l, (W, b) in enumerate(zip(Ws, bs)):
        z = h @ W.T + b
        h = np.tanh(z) if l + 1 < len(Ws) else z
        acts.append(h)
    return acts


def loss_and_grad(p, dims, x, t):
    Ws, bs = unpack(p, dims)
    acts = forward(p, dims, x)
    y = acts[-1]
    t = np.asarray(t, np.float64)
    count = y.size
    loss = np.sum((y - t) ** 2) / count
    d = 2.0 * (y - t) / count
    grads = []
    for l in range(len(Ws) - 1, -1, -1):
        if l + 1 < len(Ws):
            d = d * (1.0 - acts[l + 1] ** 2)
        gW = d.T @ acts[l]
        gb = d.sum(0)
        grads.append((gW, gb))
        d = d @ Ws[l]
    flat = []
    for gW, gb in reversed(grads):
        flat.append(gW.reshape(-1))
        flat.append(gb)
    return loss, np.concatenate(flat)


def adam(p, g, m1, m2, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    m1 = b1 * m1 + (1 - b1) * g
    m2 = b2 * m2 + (1 - b2) * g * g
    p = p - lr * (m1 / (1 - b1 ** t)) / (np.sqrt(m2 / (1 - b2 ** t)) + eps)
    return p, m1, m2
