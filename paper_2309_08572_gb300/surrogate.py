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


def _angle_block(theta: np.ndarray) -> np.ndarray:
    """Angle features of the rows of theta (n, 2p): the angle scaled to [-1, 1] and the
    first two harmonics sin/cos(2 theta), sin/cos(4 theta).  The energy is smooth and
    close to periodic in each angle, which the raw angle alone hides from the network."""
    return np.concatenate([2.0 * theta / math.pi - 1.0, np.sin(2 * theta), np.cos(2 * theta),
                           np.sin(4 * theta), np.cos(4 * theta)], axis=1)


def _angle_block_grad(theta: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Chain rule through _angle_block: d/dtheta from the gradient g on its 5 blocks."""
    q = theta.shape[1]
    gr, gs2, gc2, gs4, gc4 = (g[:, i * q:(i + 1) * q] for i in range(5))
    return (gr * (2.0 / math.pi) + 2.0 * (gs2 * np.cos(2 * theta) - gc2 * np.sin(2 * theta))
            + 4.0 * (gs4 * np.cos(4 * theta) - gc4 * np.sin(4 * theta)))


N_FIXED = 4


def fixed_features(c) -> np.ndarray:
    """(N, decay, dephasing, crosstalk) scaled to about [-1, 1]."""
    return np.asarray([c.n_sites / 50.0 - 1.0,
                       math.log10(max(c.gamma_diss, 1e-6)) + 3.0,
                       math.log10(max(c.gamma_deph, 1e-6)) + 3.0,
                       c.xtalk_phase * 50.0], dtype=np.float32)


def n_features(p: int) -> int:
    return N_FIXED + 10 * p


def features(c, p: int) -> np.ndarray:
    """Network input of one circuit: fixed_features, then _angle_block of
    (alpha_1..p, beta_1..p)."""
    theta = np.asarray([list(c.alpha[:p]) + list(c.beta[:p])], dtype=np.float64)
    return np.concatenate([fixed_features(c), _angle_block(theta)[0].astype(np.float32)])


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


def make_net(n_in: int, max_batch: int, seed: int, bf16: bool = True) -> Mlp:
    """The 4-layer, width-256 network; bf16: its products on the tensor cores with BF16
    operands (FP32 accumulation, FP32 master parameters and Adam moments)."""
    rng = np.random.default_rng(seed)
    widths = [n_in, WIDTH, WIDTH, WIDTH, 2]
    net = Mlp(widths, max_batch=max_batch, bf16=bf16)
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


def propose(net: Mlp, c, p: int, n_starts: int, steps: int, lr: float, seed: int,
            weight_success: float = 0.0) -> np.ndarray:
    """Gradient descent of the surrogate's predicted energy (plus -weight_success * success
    probability) over the 2p angles of circuit c, from n_starts random starts; N and the
    rates are held.  The input gradient comes from the network's backward kernels; the
    chain rule through the angle features is applied here.  Returns the angles (n_starts,
    2p) in [0, pi], best predicted first."""
    import torch
    rng = np.random.default_rng(seed)
    theta = rng.uniform(0.0, math.pi, (n_starts, 2 * p))
    fixed = np.repeat(fixed_features(c)[None, :], n_starts, axis=0)

    def feats(th):
        return np.concatenate([fixed, _angle_block(th).astype(np.float32)], axis=1)

    tx = torch.tensor(feats(theta), dtype=torch.float32, device="cuda")
    gx = torch.zeros_like(tx)
    wout = np.array([1.0, -weight_success], dtype=np.float32)
    for _ in range(steps):
        net.input_grad(tx, wout, gx)
        g = gx.cpu().numpy().astype(np.float64)[:, N_FIXED:]
        theta = np.clip(theta - lr * _angle_block_grad(theta, g), 0.0, math.pi)
        tx.copy_(torch.from_numpy(feats(theta)))
    y = torch.zeros((n_starts, 2), dtype=torch.float32, device="cuda")
    net.forward(tx, y)
    yh = y.cpu().numpy()
    order = np.argsort(yh[:, 0] - weight_success * yh[:, 1])
    return theta[order]


def with_angles(c, a, b):
    d = dataclasses.replace(c)
    d.alpha, d.beta = list(a), list(b)
    return d
