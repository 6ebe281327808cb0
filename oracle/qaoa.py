"""QAOA layers of the TFIM on the three-level chain (oracle; test infrastructure only).

Sec. IV, Eqs. tfim_hamiltonian, tfim_model, HZ_block_representation, HZ_representation.
Readings (the paper's signs disagree between Eq. tfim_model and Eq. HZ_block):
  * S^z, S^x are Pauli matrices on the qubit levels and zero on |r>.
  * Layer k applies every ZZ block exp(-i J alpha_k S^z S^z) (with the bias
    exp(-i b J alpha_k S^z) on each site), then exp(-i beta_k S^x) on every site;
    layers run k = 1..p.  The ZZ and X rotations carry the same sign; the noiseless
    statevector then reproduces Table II (pinned in tests).
  * Blocks run left->right in odd layers and right->left in even layers (snake); the
    single-site gates of a site are folded, exactly, into the last block that touches
    it in that layer (no later block in the layer acts on that site).
"""
from __future__ import annotations

from typing import List, Tuple

import numpy as np

from . import ops


def site_gate(alpha: float, beta: float, J: float, bz: float) -> np.ndarray:
    """exp(-i beta S^x) exp(-i b J alpha S^z) on one atom."""
    return ops.expm_h(beta, ops.X_Q) @ ops.expm_h(bz * J * alpha, ops.Z_Q)


def layer_ops(c, k: int) -> List[Tuple[int, list]]:
    """Ordered two-site ops [(left site i, Kraus set on (i, i+1))] of layer k (0-based)."""
    n = c.n_sites
    a, b = c.alpha[k], c.beta[k]
    v = site_gate(a, b, c.J, c.bz)
    common = dict(angle_zz=c.J * a, gamma_diss=c.gamma_diss, gamma_deph=c.gamma_deph,
                  xtalk_phase=c.xtalk_phase, delta_pp=c.delta_pp, b0=c.b0, b1=c.b1, bd=c.bd)
    both = ops.g0_block_channel(**common, post_left=v, post_right=v)
    if k % 2 == 0:                                   # left -> right
        mid = ops.g0_block_channel(**common, post_left=v)
        return [(i, both if i == n - 2 else mid) for i in range(n - 1)]
    mid = ops.g0_block_channel(**common, post_right=v)
    return [(i, both if i == 0 else mid) for i in range(n - 2, -1, -1)]


def layer_ops_appe(c, k: int, part: int) -> List[Tuple[int, list]]:
    """Layer k split by the coherent part of the dissipation (App. E): part 0 -- every
    block without dissipation, followed by the phases app_e_phases(gamma_diss) adds to the
    Ising phase gate (mimicking the dissipation's coherent part); part 1 -- the full block
    followed by the inverse of those phases (its incoherent part)."""
    n = c.n_sites
    a, b = c.alpha[k], c.beta[k]
    v = site_gate(a, b, c.J, c.bz)
    d1, d2 = ops.app_e_phases(c.gamma_diss)
    sh = ops.app_e_shift(c.J * a, d1, d2)
    common = dict(angle_zz=c.J * a, gamma_diss=c.gamma_diss if part == 1 else 0.0,
                  gamma_deph=c.gamma_deph, xtalk_phase=c.xtalk_phase, delta_pp=c.delta_pp,
                  b0=c.b0, b1=c.b1, bd=c.bd, shift=sh if part == 0 else sh.conj().T)
    both = ops.g0_block_channel(**common, post_left=v, post_right=v)
    if k % 2 == 0:                                   # left -> right
        mid = ops.g0_block_channel(**common, post_left=v)
        return [(i, both if i == n - 2 else mid) for i in range(n - 1)]
    mid = ops.g0_block_channel(**common, post_right=v)
    return [(i, both if i == 0 else mid) for i in range(n - 2, -1, -1)]


def layer_ops_cz(c, k: int, s_cz: np.ndarray) -> List[Tuple[int, list]]:
    """Layer k in gate model G1: every CZ of the ZZ blocks is the channel s_cz (81 x 81, e.g.
    the pulse CZ of oracle.pulse); crosstalk as in G0, no post-promotion and no separate
    noise unit (the pulse carries both)."""
    from . import pulse
    n = c.n_sites
    a, b = c.alpha[k], c.beta[k]
    v = site_gate(a, b, c.J, c.bz)
    blk = lambda **kw: pulse.g1_block_channel(c.J * a, s_cz, c.xtalk_phase, **kw)
    both = blk(post_left=v, post_right=v)
    if k % 2 == 0:                                   # left -> right
        mid = blk(post_left=v)
        return [(i, both if i == n - 2 else mid) for i in range(n - 1)]
    mid = blk(post_right=v)
    return [(i, both if i == 0 else mid) for i in range(n - 2, -1, -1)]


def circuit_ops(c, s_cz=None, appe_part=None) -> List[Tuple[int, list]]:
    """All ops of the circuit; gate model G0, or G1 with the CZ channel s_cz, or G0 split
    by App. E's coherent part (appe_part 0 / 1)."""
    out = []
    for k in range(c.p):
        if appe_part is not None:
            out.extend(layer_ops_appe(c, k, appe_part))
        else:
            out.extend(layer_ops(c, k) if s_cz is None else layer_ops_cz(c, k, s_cz))
    return out


def plus_state() -> np.ndarray:
    """|+_X> on the qubit levels (Sec. IV initial state)."""
    return np.array([1.0, 1.0, 0.0], dtype=complex) / np.sqrt(2.0)
