"""Rydberg crosstalk on the pulse-level CZ (oracle; test infrastructure only).

Sec. III.B: residual Rydberg population on the non-active neighbours i-1 and i+2 of a gate
on (i, i+1) meets the pulse through the global blockade term B |rr><rr| of every bond.  The
blockade between an active atom and its non-active neighbour shifts that atom's detuning,
Delta -> Delta + B, when the neighbour is in |r>, so the gate with nearest-neighbour
crosstalk is the controlled combination

    C_x = sum_{a, b in {0, 1}} P_a(i-1) (x) C(Delta + a B, Delta + b B) (x) P_b(i+2),

P_1 = |r><r|, P_0 = 1 - |r><r|, C(Delta_i, Delta_{i+1}) the two-atom gate with those
detunings.  The paper evolves under the Hamiltonian alone for crosstalk (no dissipation).
Reading: the one-atom phase correction of the CZ (oracle.pulse.phase_correction) is that
of the unshifted pulse -- the hardware does not know the neighbours' states -- so
C(Delta_1, Delta_2) = (c (x) c) U(Delta_1, Delta_2), U the noiseless pulse with per-atom
detunings.
"""
from __future__ import annotations

import numpy as np

from . import ops, pulse

P_R = np.diag([0.0, 0.0, 1.0]).astype(complex)
P_NR = np.eye(3, dtype=complex) - P_R


def hamiltonian(om: float, delta1: float, delta2: float, blockade: float) -> np.ndarray:
    """H_p with a detuning per atom (9 x 9, index s_1 * 3 + s_2)."""
    e = lambda i, j: np.outer(ops.I3[i], ops.I3[j])
    drive = 0.5 * om * (e(2, 1) + e(1, 2))
    h1 = drive + delta1 * e(2, 2)
    h2 = drive + delta2 * e(2, 2)
    return np.kron(h1, ops.I3) + np.kron(ops.I3, h2) + blockade * np.kron(e(2, 2), e(2, 2))


def pulse_unitary(shift1: float, shift2: float, n_steps: int, p=pulse.GAUSSIAN) -> np.ndarray:
    """The noiseless Gaussian pulse with the atoms' detunings shifted by shift1, shift2
    (midpoint exponentials of H_p, as oracle.pulse.pulse_unitary)."""
    T = p["T"]
    tau = T / n_steps
    u = np.eye(9, dtype=complex)
    for k in range(n_steps):
        om = pulse.omega((k + 0.5) * tau, T, p["omega_max"], p["width"])
        h = hamiltonian(om, p["delta"] + shift1, p["delta"] + shift2, p["blockade"])
        u = ops.expm_h(tau, h) @ u
    return u


def crosstalk_cz(n_steps: int, p=pulse.GAUSSIAN, b_x: float | None = None) -> np.ndarray:
    """C_x on the four atoms (i-1, i, i+1, i+2) as an 81 x 81 unitary (index
    ((s_{i-1} * 3 + s_i) * 3 + s_{i+1}) * 3 + s_{i+2}); b_x the neighbour blockade (default
    the pulse's B)."""
    b = p["blockade"] if b_x is None else b_x
    _, c = pulse.phase_correction(pulse.pulse_unitary(n_steps, p))
    cc = np.kron(c, c)
    out = np.zeros((81, 81), dtype=complex)
    for a, pa in ((0, P_NR), (1, P_R)):
        for bb, pb in ((0, P_NR), (1, P_R)):
            g = cc @ pulse_unitary(a * b, bb * b, n_steps, p)
            out += np.kron(np.kron(pa, g), pb)
    return out


def gate_on_chain(n_sites: int, i: int, n_steps: int, p=pulse.GAUSSIAN,
                  b_x: float | None = None):
    """(sites, unitary) of the crosstalk CZ on (i, i+1) of an n-site chain: the neighbours
    that exist (i-1 >= 0, i+2 < n) control it; a missing one acts as a neighbour without
    Rydberg population."""
    u = crosstalk_cz(n_steps, p, b_x).reshape([3] * 8)   # (out_{i-1..i+2}, in_{i-1..i+2})
    keep_l, keep_r = i - 1 >= 0, i + 2 < n_sites
    # a missing neighbour is fixed in |0>, on which P_0 acts as 1 and P_1 as 0
    half = [slice(None) if k else 0 for k in (keep_l, True, True, keep_r)]
    u = u[tuple(half + half)]
    sites = [s for s, k in ((i - 1, keep_l), (i, True), (i + 1, True), (i + 2, keep_r)) if k]
    d = 3 ** len(sites)
    return sites, u.reshape(d, d)


def apply_dense(rho: np.ndarray, n_sites: int, sites, u: np.ndarray) -> np.ndarray:
    """U rho U^+ for a unitary on consecutive sites of a dense d^N x d^N density matrix."""
    k = len(sites)
    lo = sites[0]
    left, right = 3 ** lo, 3 ** (n_sites - lo - k)
    full = np.kron(np.kron(np.eye(left), u), np.eye(right))
    return full @ rho @ full.conj().T
