"""Plain FP64 multilayer perceptron: forward pass, masked squared loss and its gradient by backpropagation.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Layers l = 0..L-1:  h_{l+1} = act_l(h_l W_l^T + b_l), act = ReLU for hidden layers, identity for the
last.  Loss = sum(mask * (out - target)^2) / max(sum(mask), 1).  Weights W_l have shape
(out_features, in_features).  The gradient is the textbook chain rule written out layer by layer.
"""
from __future__ import annotations

import numpy as np


def forward(x, Ws, bs):
    """Returns (output, activations list) with activations[0] = x."""
    acts = [np.asarray(x, dtype=np.float64)]
    pre = []
    h = acts[0]
    for l, (W, b) in enumerate(zip(Ws, bs)):
        z = h @ np.asarray(W, dtype=np.float64).T + np.asarray(b, dtype=np.float64)
        pre.append(z)
        h = np.maximum(z, 0.0) if l < len(Ws) - 1 else z
        acts.append(h)
    return h, acts, pre


def loss(out, target, mask):
    m = np.asarray(mask, dtype=np.float64)
    return float(np.sum(m * (out - target) ** 2) / max(np.sum(m), 1.0))


def backward(x, Ws, bs, target, mask):
    """Loss and gradients (dWs, dbs) of the masked mean squared error."""
    out, acts, pre = forward(x, Ws, bs)
    m = np.asarray(mask, dtype=np.float64)
    cnt = max(np.sum(m), 1.0)
    L = float(np.sum(m * (out - target) ** 2) / cnt)
    g = 2.0 * m * (out - target) / cnt                       # dL/d out
    dWs = [None] * len(Ws)
    dbs = [None] * len(Ws)
    for l in range(len(Ws) - 1, -1, -1):
        if l < len(Ws) - 1:
            g = g * (pre[l] > 0.0)                           # through ReLU
        dWs[l] = g.T @ acts[l]
        dbs[l] = g.sum(axis=0)
        g = g @ np.asarray(Ws[l], dtype=np.float64)           # to the layer input
    return L, dWs, dbs
