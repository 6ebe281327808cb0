"""Exact dense density-matrix simulation (oracle; test infrastructure only).

rho is kept as a tensor with N ket axes followed by N bra axes (local dim 3), the
direct representation whose exponential cost the tensor network avoids (Sec. III).
Channels act as rho -> sum_m E_m rho E_m^+ (Sec. III.A, Kraus form of the
integrated channel).
"""
from __future__ import annotations

import numpy as np

from . import ops

D = 3


class DenseRho:
    def __init__(self, n_sites: int, site_state: np.ndarray):
        self.n = n_sites
        psi = site_state
        for _ in range(n_sites - 1):
            psi = np.kron(psi, site_state)
        self.rho = np.outer(psi, psi.conj()).reshape((D,) * (2 * n_sites))

    def matrix(self) -> np.ndarray:
        m = D ** self.n
        return self.rho.reshape(m, m)

    def apply_two_site(self, i: int, kraus):
        n = self.n
        out = np.zeros_like(self.rho)
        for e in kraus:
            e4 = np.asarray(e).reshape(D, D, D, D)
            # ket side: axes i, i+1
            t = np.tensordot(e4, self.rho, axes=([2, 3], [i, i + 1]))
            t = np.moveaxis(t, [0, 1], [i, i + 1])
            # bra side: axes n+i, n+i+1 with conj(E)
            t = np.tensordot(e4.conj(), t, axes=([2, 3], [n + i, n + i + 1]))
            t = np.moveaxis(t, [0, 1], [n + i, n + i + 1])
            out += t
        self.rho = out

    # ---- observables (Sec. IV.A; S ops are Pauli on the qubit levels, 0 on |r>)
    def _local(self, opmap) -> np.ndarray:
        m = np.array([[1.0]], dtype=complex)
        for s in range(self.n):
            m = np.kron(m, opmap.get(s, ops.I3))
        return m

    def expect(self, J: float, hx: float, bz: float):
        rho = self.matrix()
        n = self.n
        tr = np.trace(rho).real
        pq = self._local({s: ops.P_Q for s in range(n)})
        psucc = np.trace(pq @ rho).real
        h = np.zeros_like(rho)
        for s in range(n - 1):
            h += -J * self._local({s: ops.Z_Q, s + 1: ops.Z_Q})
        for s in range(n):
            h += -hx * self._local({s: ops.X_Q}) - bz * J * self._local({s: ops.Z_Q})
        e_raw = np.trace(h @ rho).real / tr
        e_succ = np.trace(pq @ h @ pq @ rho).real / psucc
        return dict(e_raw=e_raw, e_succ=e_succ, p_succ=psucc, trace=tr)

    def probs_diag(self) -> np.ndarray:
        """<x|rho|x> for every x in {0,1,r}^N (row-major over sites)."""
        return np.real(np.diag(self.matrix()))
