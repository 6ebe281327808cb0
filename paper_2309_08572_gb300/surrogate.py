"""Learned surrogate for noisy QAOA circuits on top of the MPDO engine.

Not part of the paper: the workload's learned component.  The MPDO engine (batch
executor) produces samples (circuit description -> energy per site, success
probability); an MLP trained on the GPU by the library's own forward/backward/Adam kernels
learns that map; its input gradient proposes QAOA angles; every proposal is re-scored by
the MPDO engine, which stays the judge.  Argument marshalling and orchestration only; the
arithmetic runs in libmpdo.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence

import numpy as np

from . import Mlp, Mpdo, batch_run, circuit_layers

WIDTH = 256


def features(c, p: int) -> np.ndarray:
    """(N, decay, dephasing, crosstalk, alpha_1..p, beta_1..p) scaled to about [-1, 1]."""
    f = [c.n_sites / 50.0 - 1.0,
         (math.log10(max(c.gamma_diss, 1e-6)) + 3.0),
         (math.log10(max(c.gamma_deph, 1e-6)) + 3.0),
         c.xtalk_phase * 50.0]
    f += [2.0 * a / math.pi - 1.0 for a in c.alpha[:p]]
    f += [2.0 * b / math.pi - 1.0 for b in c.beta[:p]]
    return np.asarray(f, dtype=np.float32)


def angles_from_features(x: np.ndarray, p: int):
    a = (x[4:4 + p] + 1.0) * math.pi / 2.0
    b = (x[4 + p:4 + 2 * p] + 1.0) * math.pi / 2.0
    return [float(v) for v in a], [float(v) for v in b]


def simulate(circuits: Sequence, pool: List[Mpdo]) -> np.ndarray:
    """Run circuits on the engine; returns (n, 2): energy per site (success-conditioned)
    and success probability."""
    descs = []
    uploaded = []
    for c in circuits:
        dls = [pool[0].upload_layer(layer) for layer in circuit_layers(c)]
        uploaded.append(dls)
        descs.append(dict(n_sites=c.n_sites, chi_max=c.chi_max, k_max=c.k_max, layers=dls,
                          J=c.J, hx=c.hx, b=c.bz))
    out = batch_run(pool, descs)
    for dls in uploaded:
        for dl in dls:
            pool[0].free_uploaded(dl)
    n = np.array([c.n_sites for c in circuits], dtype=float)
    return np.stack([out[:, 1] / n, out[:, 2]], axis=1)


def make_net(n_in: int, max_batch: int, seed: int) -> Mlp:
    rng = np.random.default_rng(seed)
    widths = [n_in, WIDTH, WIDTH, WIDTH, 2]
    net = Mlp(widths, max_batch=max_batch)
    flat = []
    for a, b in zip(widths[:-1], widths[1:]):
        flat.append((rng.standard_normal((a, b)) / np.sqrt(a)).reshape(-1))
        flat.append(np.zeros(b))
    net.set_params(np.concatenate(flat).astype(np.float32))
    return net


def train(net: Mlp, x: np.ndarray, t: np.ndarray, steps: int, lr: float, batch: int,
          seed: int = 0):
    import torch
    rng = np.random.default_rng(seed)
    tx = torch.tensor(x, dtype=torch.float32, device="cuda")
    tt = torch.tensor(t, dtype=torch.float32, device="cuda")
    losses = []
    for s in range(steps):
        idx = torch.tensor(rng.integers(0, x.shape[0], size=batch), device="cuda")
        xb, tb = tx[idx].contiguous(), tt[idx].contiguous()
        loss, _ = net.loss_grad(xb, tb)
        net.adam_step(lr)
        losses.append(loss)
    return losses


def propose(net: Mlp, base_feat: np.ndarray, p: int, n_starts: int, steps: int, lr: float,
            seed: int, weight_success: float = 0.0) -> np.ndarray:
    """Gradient descent on the angle features of the surrogate's predicted energy (plus
    -weight_success * success probability) from n_starts random starts; fixed features (N,
    rates) are held.  Returns the final features, best predicted first."""
    import torch
    rng = np.random.default_rng(seed)
    x = np.repeat(base_feat[None, :], n_starts, axis=0).astype(np.float32)
    x[:, 4:4 + 2 * p] = rng.uniform(-1, 1, (n_starts, 2 * p))
    tx = torch.tensor(x, dtype=torch.float32, device="cuda")
    gx = torch.zeros_like(tx)
    wout = np.array([1.0, -weight_success], dtype=np.float32)
    for _ in range(steps):
        net.input_grad(tx, wout, gx)
        g = gx.cpu().numpy()
        x[:, 4:4 + 2 * p] = np.clip(x[:, 4:4 + 2 * p] - lr * g[:, 4:4 + 2 * p], -1.0, 1.0)
        tx.copy_(torch.from_numpy(x))
    y = torch.zeros((n_starts, 2), dtype=torch.float32, device="cuda")
    net.forward(tx, y)
    yh = y.cpu().numpy()
    order = np.argsort(yh[:, 0] - weight_success * yh[:, 1])
    return x[order]


def with_angles(c, a, b):
    d = dataclasses.replace(c)
    d.alpha, d.beta = list(a), list(b)
    return d
