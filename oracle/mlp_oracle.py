"""Plain float64 reference of the schedule cost model's MLP.

TEST INFRASTRUCTURE ONLY (imported by tests, never by the product package).
Dense layers y = W x + b with ReLU between them and a linear output layer;
loss sum(mask * (y - t)^2) / sum(mask); gradients by backpropagation written
out layer by layer.  Parameter layout: per layer W [out][in] then b [out].
Pinned by central finite differences and by the one-layer case, which is a
plain affine map (numpy matmul).
"""
from __future__ import annotations

import numpy as np


def unpack(params, dims):
    """List of (W, b) from the flat parameter vector."""
    p = np.asarray(params, dtype=np.float64)
    out, off = [], 0
    for i in range(len(dims) - 1):
        n_in, n_out = dims[i], dims[i + 1]
        W = p[off:off + n_in * n_out].reshape(n_out, n_in)
        off += n_in * n_out
        b = p[off:off + n_out]
        off += n_out
        out.append((W, b))
    assert off == p.size
    return out


def forward(params, dims, X):
    """Activations of every layer (list, input first); the last is the output."""
    acts = [np.asarray(X, dtype=np.float64)]
    layers = unpack(params, dims)
    for i, (W, b) in enumerate(layers):
        z = acts[-1] @ W.T + b
        acts.append(np.maximum(z, 0.0) if i + 1 < len(layers) else z)
    return acts


def loss(params, dims, X, T, mask=None):
    Y = forward(params, dims, X)[-1]
    m = np.ones_like(Y) if mask is None else np.asarray(mask, dtype=np.float64)
    cnt = max(m.sum(), 1.0)
    return float((m * (Y - np.asarray(T, dtype=np.float64)) ** 2).sum() / cnt)


def gradients(params, dims, X, T, mask=None):
    """(loss, gradient in the flat layout)."""
    acts = forward(params, dims, X)
    layers = unpack(params, dims)
    Y = acts[-1]
    m = np.ones_like(Y) if mask is None else np.asarray(mask, dtype=np.float64)
    cnt = max(m.sum(), 1.0)
    diff = Y - np.asarray(T, dtype=np.float64)
    L = float((m * diff ** 2).sum() / cnt)
    delta = 2.0 * m * diff / cnt                      # dL/dy
    grads = [None] * len(layers)
    for i in range(len(layers) - 1, -1, -1):
        W, _ = layers[i]
        x = acts[i]
        grads[i] = (delta.T @ x, delta.sum(axis=0))   # dW [out][in], db [out]
        if i > 0:
            delta = (delta @ W) * (acts[i] > 0)       # through the ReLU of layer i-1
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return L, flat


def finite_difference(params, dims, X, T, mask=None, h=1e-6, idx=None):
    """Central differences of the loss for the parameter indices idx."""
    p = np.asarray(params, dtype=np.float64).copy()
    idx = range(p.size) if idx is None else idx
    out = []
    for k in idx:
        old = p[k]
        p[k] = old + h
        lp = loss(p, dims, X, T, mask)
        p[k] = old - h
        lm = loss(p, dims, X, T, mask)
        p[k] = old
        out.append((lp - lm) / (2 * h))
    return np.array(out)
