"""FP64 reference of the proposal network (test infrastructure only).

y1 = relu(x W1 + b1), y2 = relu(y1 W2 + b2), y3 = relu(y2 W3 + b3),
z = y3 W4 + b4; loss = mean over rows of -log softmax(z)[label].
Forward and analytic backward in numpy float64, parameters in the same flat
layout as the CUDA path: W1 [1536 x 256], b1, W2 [256 x 256], b2,
W3 [256 x 256], b3, W4 [256 x 4096], b4.
"""
from __future__ import annotations

import numpy as np

DIMS = [(1536, 256), (256, 256), (256, 256), (256, 4096)]


def num_params() -> int:
    return sum(i * o + o for i, o in DIMS)


def unpack(p):
    out, k = [], 0
    for i, o in DIMS:
        W = p[k:k + i * o].reshape(i, o)
        k += i * o
        b = p[k:k + o]
        k += o
        out.append((W, b))
    return out


def init_params(seed: int = 0) -> np.ndarray:
    """He-normal weights, zero biases (float32)."""
    rng = np.random.default_rng(seed)
    parts = []
    for i, o in DIMS:
        parts.append(rng.normal(0.0, np.sqrt(2.0 / i), size=i * o))
        parts.append(np.zeros(o))
    return np.concatenate(parts).astype(np.float32)


def _mm(A, B, rnd):
    return (rnd(A) @ rnd(B)) if rnd is not None else A @ B


def forward(p, X, rnd=None):
    """rnd, if given, is applied to both operands of every matrix product
    (used to emulate reduced-precision operands); biases stay exact."""
    layers = unpack(np.asarray(p, np.float64))
    h = np.asarray(X, np.float64)
    acts = [h]
    for li, (W, b) in enumerate(layers):
        h = _mm(h, W, rnd) + b
        if li < len(layers) - 1:
            h = np.maximum(h, 0.0)
        acts.append(h)
    return h, acts


def loss_and_grad(p, X, labels, rnd=None):
    p = np.asarray(p, np.float64)
    layers = unpack(p)
    z, acts = forward(p, X, rnd)
    B = z.shape[0]
    zm = z - z.max(axis=1, keepdims=True)
    e = np.exp(zm)
    P = e / e.sum(axis=1, keepdims=True)
    loss = float(np.mean(-np.log(P[np.arange(B), labels])))
    dz = P.copy()
    dz[np.arange(B), labels] -= 1.0
    dz /= B
    grads = []
    d = dz
    for li in range(len(layers) - 1, -1, -1):
        W, b = layers[li]
        a_in = acts[li]
        gW = _mm(a_in.T, d, rnd)
        gb = d.sum(axis=0)
        grads.append((gW, gb))
        if li > 0:
            d = _mm(d, W.T, rnd)
            d = d * (acts[li] > 0)
    grads.reverse()
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return loss, flat
