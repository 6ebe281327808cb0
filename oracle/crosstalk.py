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


def apply_mpdo(m, sites, u: np.ndarray, sv_cutoff: float = 1e-14) -> None:
    """U X on consecutive sites of an oracle MPDO m (oracle.mpdo.MPDO), U acting on the atom
    levels only (the inner indices are untouched, so rho -> U rho U^+).  The centre must lie
    in the block: the block's tensors are contracted into one, U applied, and the block
    split back left to right by SVDs keeping every value above sv_cutoff * s_max (exact up
    to that cut); the centre ends on the block's last site."""
    first, k = sites[0], len(sites)
    if not first <= m.centre < first + k:
        raise ValueError("the centre must lie in the block")
    th = m.A[first]                                   # [l, s, k, r]
    for j in range(1, k):
        th = np.tensordot(th, m.A[first + j], axes=([th.ndim - 1], [0]))
    # axes: l, (s_1, k_1), ..., (s_k, k_k), r
    inner = [th.shape[2 + 2 * j] for j in range(k)]
    perm = [0] + [1 + 2 * j for j in range(k)] + [2 + 2 * j for j in range(k)] + [th.ndim - 1]
    t = th.transpose(perm)                            # l, s_1..s_k, k_1..k_k, r
    dl, dr = t.shape[0], t.shape[-1]
    t = t.reshape(dl, 3 ** k, -1)
    t = np.einsum("st,ltr->lsr", u, t)
    t = t.reshape([dl] + [3] * k + inner + [dr])
    back = [0]
    for j in range(k):
        back += [1 + j, 1 + k + j]
    th = t.transpose(back + [2 * k + 1])              # l, (s_j, k_j)..., r
    for j in range(k - 1):
        rows = th.shape[0] * 3 * inner[j]
        mat = th.reshape(rows, -1)
        uu, s, vh = np.linalg.svd(mat, full_matrices=False)
        keep = max(1, int(np.count_nonzero(s > sv_cutoff * s[0])))
        m.A[first + j] = uu[:, :keep].reshape(th.shape[0], 3, inner[j], keep)
        th = (s[:keep, None] * vh[:keep]).reshape([keep] + list(th.shape[3:]))
    m.A[first + k - 1] = th.reshape(th.shape[0], 3, inner[k - 1], dr)
    m.centre = first + k - 1
