"""Plain MLP surrogate: forward, backward and Adam (oracle; test infrastructure only).

Not a method of the paper: a small fully connected network maps a circuit description
(chain length, noise rates, QAOA angles) to (energy per site, success probability).  The
oracle is the textbook network written out in float64 NumPy with no autograd:

  z_l = a_{l-1} W_l + b_l,  a_l = tanh(z_l) for hidden layers, a_L = z_L (linear output)
  loss = mean over batch and outputs of (a_L - t)^2
  backward: d a_L = 2 (a_L - t) / (B * n_out); d z_l = d a_l * (1 - a_l^2) (hidden);
            dW_l = a_{l-1}^T dz_l, db_l = sum_rows dz_l, d a_{l-1} = dz_l W_l^T
  Adam (Kingma & Ba 2015): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
            w -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps)
Weights W_l are stored [fan_in][fan_out] (row-major), matching x W.
"""
from __future__ import annotations

import numpy as np


def forward(params, x):
    acts = [x]
    a = x
    n = len(params)
    for l, (w, b) in enumerate(params):
        z = a @ w + b
        a = z if l == n - 1 else np.tanh(z)
        acts.append(a)
    return acts


def loss_and_grads(params, x, t):
    acts = forward(params, x)
    y = acts[-1]
    bsz, nout = y.shape
    loss = float(np.mean((y - t) ** 2))
    da = 2.0 * (y - t) / (bsz * nout)
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        w, _ = params[l]
        dz = da if l == len(params) - 1 else da * (1.0 - acts[l + 1] ** 2)
        grads[l] = (acts[l].T @ dz, dz.sum(axis=0))
        da = dz @ w.T
    return loss, grads, da          # da = d loss / d x


def input_grad(params, x, wout):
    """d (sum_j wout_j y_j) / d x for each row of x."""
    acts = forward(params, x)
    da = np.broadcast_to(np.asarray(wout, float), acts[-1].shape).copy()
    for l in range(len(params) - 1, -1, -1):
        w, _ = params[l]
        dz = da if l == len(params) - 1 else da * (1.0 - acts[l + 1] ** 2)
        da = dz @ w.T
    return da


def adam_step(params, grads, state, lr, b1=0.9, b2=0.999, eps=1e-8):
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    out = []
    for l, ((w, b), (gw, gb)) in enumerate(zip(params, grads)):
        new = []
        for name, p, g in (("w", w, gw), ("b", b, gb)):
            m = state.setdefault(f"m{name}{l}", np.zeros_like(p))
            v = state.setdefault(f"v{name}{l}", np.zeros_like(p))
            m[...] = b1 * m + (1 - b1) * g
            v[...] = b2 * v + (1 - b2) * g * g
            mh = m / (1 - b1 ** t)
            vh = v / (1 - b2 ** t)
            new.append(p - lr * mh / (np.sqrt(vh) + eps))
        out.append(tuple(new))
    return out
