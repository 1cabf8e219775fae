"""FP64 oracle of the proposal MLP (forward and backward).

TEST INFRASTRUCTURE: imported only by the tests and the smoke check.

Network: d0 -> ... -> dL, ReLU after hidden layers, linear output.  The
library keeps weights and hidden activations in BF16 and accumulates in
FP32; this oracle computes every product in FP64 and applies BF16
round-to-nearest-even at exactly the points where the library stores BF16:
the input, the weights, each hidden activation (after bias + ReLU), and in
the backward pass the incoming dL/dy and each back-propagated signal (after
the ReLU mask).  With `bf16=False` no rounding is applied (used to pin the
backward pass against finite differences).
"""
from __future__ import annotations

import numpy as np


def bf16_round(x):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    x32 = np.asarray(x, dtype=np.float32)
    bits = x32.view(np.uint32).astype(np.uint64)
    bits = (bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000
    return bits.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(Ws, bs, x, bf16=True):
    """Returns (y, hs) with hs[0] = input and hs[l] the hidden activations."""
    r = bf16_round if bf16 else (lambda v: np.asarray(v, np.float64))
    h = r(x)
    hs = [h]
    L = len(Ws)
    for l in range(L):
        z = h @ r(Ws[l]).T + np.asarray(bs[l], np.float64)
        if l < L - 1:
            h = r(np.maximum(z, 0.0))
            hs.append(h)
        else:
            y = z
    return y, hs


def backward(Ws, bs, hs, dy, bf16=True):
    """Gradients of sum(dy * y): lists dW[l], db[l]."""
    r = bf16_round if bf16 else (lambda v: np.asarray(v, np.float64))
    L = len(Ws)
    dWs, dbs = [None] * L, [None] * L
    dz = r(dy)
    for l in range(L - 1, -1, -1):
        dWs[l] = dz.T @ hs[l]
        dbs[l] = dz.sum(0)
        if l > 0:
            dz = r((dz @ r(Ws[l])) * (hs[l] > 0))
    return dWs, dbs
