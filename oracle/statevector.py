"""Noiseless qubit statevector QAOA and the TFIM ground state (oracle; tests only).

Used to pin the Hamiltonian and layer conventions to Table II (Sec. IV): with ideal
gates no population leaves the qubit levels, so the three-level model reduces to
2^N amplitudes.  Energy density = <H>/N with open boundary conditions.
"""
from __future__ import annotations

import numpy as np


def _zdiag(n: int, bz: float, J: float):
    idx = np.arange(2 ** n)
    z = 1 - 2 * ((idx[:, None] >> np.arange(n)[None, :]) & 1)
    zz = (z[:, :-1] * z[:, 1:]).sum(1).astype(float)
    return J * zz + bz * J * z.sum(1)       # H_z scaled by J (bias b J)


def _xrot_all(psi, n, ang):
    c, s = np.cos(ang), np.sin(ang)
    for q in range(n):
        p = psi.reshape(2 ** (n - q - 1), 2, 2 ** q)
        a0 = p[:, 0, :].copy()
        a1 = p[:, 1, :].copy()
        p[:, 0, :] = c * a0 - 1j * s * a1
        p[:, 1, :] = c * a1 - 1j * s * a0
    return psi


def _xsum(psi, n):
    out = np.zeros_like(psi)
    for q in range(n):
        p = psi.reshape(2 ** (n - q - 1), 2, 2 ** q)
        o = out.reshape(2 ** (n - q - 1), 2, 2 ** q)
        o[:, 0, :] += p[:, 1, :]
        o[:, 1, :] += p[:, 0, :]
    return out


def qaoa_energy_density(n: int, alpha, beta, J: float, g: float, bz: float) -> float:
    """Layers k = 1..p: exp(-i alpha_k J H_z) then exp(-i beta_k S^x) on every qubit,
    from |+>^N; returns <H>/N for H = -J H_z - g sum S^x."""
    hz = _zdiag(n, bz, J)
    psi = np.ones(2 ** n, dtype=complex) / 2 ** (n / 2)
    for a, b in zip(alpha, beta):
        psi = np.exp(-1j * a * hz) * psi
        psi = _xrot_all(psi, n, b)
    e = np.vdot(psi, -hz * psi).real - g * np.vdot(psi, _xsum(psi, n)).real
    return e / n


def ground_energy_density(n: int, J: float, g: float, bz: float) -> float:
    import scipy.sparse.linalg as sla
    hz = _zdiag(n, bz, J)

    def mv(v):
        v = np.asarray(v).reshape(-1)
        return -hz * v - g * _xsum(v.astype(float), n)

    op = sla.LinearOperator((2 ** n, 2 ** n), matvec=mv, dtype=float)
    w = sla.eigsh(op, k=1, which="SA", tol=1e-10)[0]
    return float(w[0]) / n
