"""Plain fp64 reference of the proposal model (TEST INFRASTRUCTURE ONLY).

The model scores a feature row x (128 values):
    h = W1 x            (256 hidden units; no separate bias, feature 10 is 1)
    s = b2 + w2 . relu(h)
and is trained on the binary cross-entropy of s against a label y in {0, 1},
positives weighted by pos_weight, averaged over the rows:
    L = (1/n) sum_r wt_r (softplus(s_r) - y_r s_r).
This module writes that definition out with numpy in float64, together with
its gradient by the chain rule, and the rounding of float32 values to BF16
(round to nearest, ties to even) that the tensor-core path applies to its
inputs.  Parameters are one flat array: W1[256][128], then w2[256], then b2.
"""
from __future__ import annotations

import numpy as np

F, H = 128, 256
N_PARAMS = H * F + H + 1


def unpack(params):
    p = np.asarray(params, dtype=np.float64)
    return p[:H * F].reshape(H, F), p[H * F:H * F + H], p[H * F + H]


def bf16_round(a):
    """float32 -> nearest BF16 value (ties to even), returned as float32."""
    x = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (x >> 16) & 1
    r = ((x + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).reshape(np.shape(a))


def forward(params, X):
    """Scores s[n] and hidden pre-activations h[n][256] in float64."""
    W1, w2, b2 = unpack(params)
    X = np.asarray(X, dtype=np.float64)
    h = X @ W1.T
    return b2 + np.maximum(h, 0.0) @ w2, h


def loss_and_grad(params, X, y, pos_weight=1.0):
    """Mean weighted binary cross-entropy and its gradient (flat array)."""
    W1, w2, b2 = unpack(params)
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n = len(y)
    s, h = forward(params, X)
    wt = np.where(y > 0.5, pos_weight, 1.0)
    softplus = np.logaddexp(0.0, s)
    L = float(np.sum(wt * (softplus - y * s)) / n)
    ds = wt * (1.0 / (1.0 + np.exp(-s)) - y) / n          # dL/ds
    a = np.maximum(h, 0.0)
    g_w2 = a.T @ ds
    g_b2 = ds.sum()
    dh = np.outer(ds, w2) * (h > 0)                        # dL/dh
    g_W1 = dh.T @ X
    return L, np.concatenate([g_W1.ravel(), g_w2, [g_b2]]), dh
