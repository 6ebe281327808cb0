"""Random-circuit layers on the three-level chain (oracle; test infrastructure only).

The paper's second workload (Sec. IV, Fig. 4 and Fig. 5 a-c): random circuits of Haar
one-qubit gates and CZs on a brickwork of bonds, with Rydberg dissipation.  Readings:
  * the Haar gates act on the qubit levels, |r> is left alone;
  * layer k: a Haar gate on every atom, then a noisy CZ on every bond (i, i+1) with
    i = k mod 2; the CZ in gate model G0: crosstalk phase, ideal CZ (|11> -> -|11>),
    post-promotion, one unit of decay and dephasing on both atoms (as the ZZ block of
    oracle.ops.g0_block_channel with the block replaced by one CZ);
  * the MPDO applies a layer as one sweep over all bonds (left to right in even layers,
    right to left in odd ones), bonds without a CZ carrying only the Haar gates (or the
    identity) so the orthogonality centre walks through; every atom's Haar gate is folded,
    exactly, into the first op of the sweep that touches it.
"""
from __future__ import annotations

from typing import List, Tuple

import numpy as np

from . import ops


def embed(u2: np.ndarray) -> np.ndarray:
    """2 x 2 unitary on the qubit levels as a 3 x 3 one (|r> -> |r>)."""
    u = np.eye(3, dtype=complex)
    u[:2, :2] = u2
    return u


def cz_channel(pre_left, pre_right, gamma_diss, gamma_deph, xtalk_phase, delta_pp, b0, b1, bd):
    """Kraus set of one noisy CZ on a bond, after the one-atom gates pre_left (x) pre_right."""
    u = ops.CZ
    if xtalk_phase != 0.0:
        u = u @ ops.expm_h(xtalk_phase, np.kron(ops.N_R, ops.N_R))
    u = u @ np.kron(pre_left, pre_right)
    if delta_pp != 0.0:
        pp = ops.expm_h(delta_pp, np.outer(ops.I3[1], ops.I3[2]) + np.outer(ops.I3[2], ops.I3[1]))
        u = np.kron(pp, pp) @ u
    n1 = ops.g0_noise_superop(gamma_diss, gamma_deph, b0, b1, bd)
    s = np.kron(n1, n1)
    s = s.reshape(3, 3, 3, 3, 3, 3, 3, 3).transpose(0, 2, 1, 3, 4, 6, 5, 7).reshape(81, 81)
    return ops.kraus_from_superop(s @ ops.superop([u]))


def layer_ops(c, k: int) -> List[Tuple[int, list]]:
    """Ordered two-site ops [(left site i, Kraus set)] of layer k (0-based)."""
    n = c.n_sites
    gates = [embed(c.haar[k, j]) for j in range(n)]
    ltr = (k % 2 == 0)
    order = range(n - 1) if ltr else range(n - 2, -1, -1)
    seen = [False] * n
    out = []
    for i in order:
        pre = []
        for j in (i, i + 1):
            pre.append(gates[j] if not seen[j] else ops.I3)
            seen[j] = True
        if i % 2 == k % 2:
            ch = cz_channel(pre[0], pre[1], c.gamma_diss, c.gamma_deph, c.xtalk_phase,
                            c.delta_pp, c.b0, c.b1, c.bd)
        else:
            ch = [np.kron(pre[0], pre[1])]
        out.append((i, ch))
    return out


def circuit_ops(c) -> List[Tuple[int, list]]:
    out = []
    for k in range(c.depth):
        out.extend(layer_ops(c, k))
    return out


def zero_state() -> np.ndarray:
    """|0> on every atom (the random circuits' initial state)."""
    return np.array([1.0, 0.0, 0.0], dtype=complex)
