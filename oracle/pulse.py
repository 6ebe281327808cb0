"""Pulse-level CZ channel, gate model G1 (oracle; test infrastructure only).

Sec. II: two atoms driven by identical pulses under
    H_p(t) = H_1(t) (x) I + I (x) H_2(t) + B |rr><rr|,
    H_i(t) = Omega(t)/2 (|r><1| + |1><r|) + Delta |r><r|         (Eqs. LME_Hamiltonian,
                                                                   LME_Single_Site)
with the Lindblad dissipators of Eq. LME on each atom (jump operators as in
ops.lindblad_generator).  Gaussian pulse (Fig. 1 caption):
    Omega(t) = Omega_max [exp(-(t - t0)^2 / u^2) - a] / (1 - a),  u = 0.1 T, t0 = T/2,
    a = exp(-(t0/u)^2),  Delta constant,
T = 2.165 us, Omega_max = 17 MHz, Delta = -14.7 MHz, B = 60 MHz.  Reading: every frequency
is an angular frequency 2 pi x (value) rad/us; times in us.  The rates gamma_diss and
gamma_deph are per pulse (the generator uses gamma / T), as in the paper's gamma_diss =
0.001 T^-1.

The channel of the whole pulse is the time-ordered exponential of the generator; Sec. III.A
integrates it into one channel before use, as a product of step channels built from exact
exponentials of the generator's parts (a Trotter split).  Here each step of length tau is
    exp(tau/2 D) exp(-i tau H_p(t_mid)) (x) conj(.) exp(tau/2 D),
with D the (time-independent) dissipators of both atoms and H_p exponentiated whole at the
step midpoint (reading: the paper also splits H_p into one-atom and blockade factors, a
first-order split whose error needs far smaller steps at B = 2 pi x 60 MHz; the symmetric
split and the whole H_p keep the per-step error at O(tau^3)).  pulse_superop_exact (the
midpoint exponential of the whole generator per step) pins the split.

Phase correction (reading of Sec. II, the Gaussian gate needs single-qubit rotations):
|00> is untouched by H_p, |01> and |10> pick up the single-atom phase phi_1; each atom gets
diag(1, e^{-i phi_1}, 1) after the pulse, which leaves |11> with phi_11 - 2 phi_1 (pi for
a CZ).  The correction is taken from the noiseless pulse.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import ops

TWO_PI = 2.0 * np.pi
# Gaussian CZ of Fig. 1 (d, e): times in us, angular frequencies in rad/us
GAUSSIAN = dict(T=2.165, omega_max=TWO_PI * 17.0, delta=TWO_PI * -14.7, blockade=TWO_PI * 60.0,
                width=0.1)


def omega(t: float, T: float, omega_max: float, width: float) -> float:
    """Gaussian Rabi profile of Fig. 1 (offset so that it starts and ends at 0)."""
    u = width * T
    t0 = T / 2.0
    a = np.exp(-(t0 / u) ** 2)
    return omega_max * (np.exp(-((t - t0) / u) ** 2) - a) / (1.0 - a)


def hamiltonian(om: float, delta: float, blockade: float) -> np.ndarray:
    """H_p on the two-atom space (9 x 9, index s_1 * 3 + s_2)."""
    e = lambda i, j: np.outer(ops.I3[i], ops.I3[j])
    h1 = 0.5 * om * (e(2, 1) + e(1, 2)) + delta * e(2, 2)
    return np.kron(h1, ops.I3) + np.kron(ops.I3, h1) + blockade * np.kron(e(2, 2), e(2, 2))


def _two_site(g1: np.ndarray, site: int) -> np.ndarray:
    """A one-atom superoperator (9 x 9 on (a, a')) acting on atom `site` of the two-atom
    row-major vec ((a, b), (a', b'))."""
    big = np.kron(g1, np.eye(9)) if site == 0 else np.kron(np.eye(9), g1)
    # big acts on (a, a', b, b'); reorder rows and columns to (a, b, a', b')
    return big.reshape(3, 3, 3, 3, 3, 3, 3, 3).transpose(0, 2, 1, 3, 4, 6, 5, 7).reshape(81, 81)


def generator(t: float, gamma_diss: float, gamma_deph: float, b0: float, b1: float, bd: float,
              p=GAUSSIAN) -> np.ndarray:
    """d vec(rho)/dt = G(t) vec(rho) (Eq. LME, row-major vec): -i (H (x) I - I (x) H^T) plus
    the dissipators of both atoms at rates gamma / T."""
    T = p["T"]
    h = hamiltonian(omega(t, T, p["omega_max"], p["width"]), p["delta"], p["blockade"])
    g = -1j * (np.kron(h, np.eye(9)) - np.kron(np.eye(9), h.T))
    d1 = ops.lindblad_generator(gamma_diss / T, gamma_deph / T, b0, b1, bd)
    return g + _two_site(d1, 0) + _two_site(d1, 1)


def pulse_superop(gamma_diss: float, gamma_deph: float, b0: float, b1: float, bd: float,
                  n_steps: int, p=GAUSSIAN) -> np.ndarray:
    """Channel of the whole pulse (81 x 81): n_steps symmetric split steps (module doc)."""
    T = p["T"]
    tau = T / n_steps
    d1 = ops.lindblad_generator(gamma_diss / T, gamma_deph / T, b0, b1, bd)
    d_half = sla.expm(0.5 * tau * (_two_site(d1, 0) + _two_site(d1, 1)))
    s = np.eye(81, dtype=complex)
    for k in range(n_steps):
        h = hamiltonian(omega((k + 0.5) * tau, T, p["omega_max"], p["width"]), p["delta"],
                        p["blockade"])
        s = d_half @ ops.superop([ops.expm_h(tau, h)]) @ d_half @ s
    return s


def pulse_superop_exact(gamma_diss: float, gamma_deph: float, b0: float, b1: float,
                        bd: float, n_steps: int, p=GAUSSIAN) -> np.ndarray:
    """The same channel with the whole generator exponentiated at each step midpoint (no
    split; slow, for pinning the split at few steps)."""
    T = p["T"]
    tau = T / n_steps
    s = np.eye(81, dtype=complex)
    for k in range(n_steps):
        s = sla.expm(tau * generator((k + 0.5) * tau, gamma_diss, gamma_deph, b0, b1, bd, p)) @ s
    return s


def pulse_unitary(n_steps: int, p=GAUSSIAN) -> np.ndarray:
    """The noiseless pulse as a 9 x 9 unitary (midpoint exponentials of H_p)."""
    T = p["T"]
    tau = T / n_steps
    u = np.eye(9, dtype=complex)
    for k in range(n_steps):
        h = hamiltonian(omega((k + 0.5) * tau, T, p["omega_max"], p["width"]), p["delta"],
                        p["blockade"])
        u = ops.expm_h(tau, h) @ u
    return u


def phase_correction(u: np.ndarray) -> tuple[float, np.ndarray]:
    """phi_1 = arg <01|U|01> - arg <00|U|00> and the one-atom correction diag(1, e^{-i phi_1}, 1)."""
    phi1 = float(np.angle(u[1, 1]) - np.angle(u[0, 0]))
    return phi1, np.diag([1.0, np.exp(-1j * phi1), 1.0])


def cz_superop(gamma_diss: float, gamma_deph: float, b0: float, b1: float, bd: float,
               n_steps: int, p=GAUSSIAN) -> tuple[np.ndarray, float]:
    """Phase-corrected pulse CZ channel (81 x 81 superoperator) and phi_1."""
    phi1, c = phase_correction(pulse_unitary(n_steps, p))
    s = ops.superop([np.kron(c, c)]) @ pulse_superop(gamma_diss, gamma_deph, b0, b1, bd,
                                                     n_steps, p)
    return s, phi1


def average_cz_infidelity(u: np.ndarray) -> float:
    """1 - average gate fidelity (|tr(CZ^+ U_q)|^2 + 4) / 20 of the corrected unitary on the
    qubit subspace {00, 01, 10, 11} (Nielsen's formula for d = 4)."""
    _, c = phase_correction(u)
    uq = (np.kron(c, c) @ u)[np.ix_([0, 1, 3, 4], [0, 1, 3, 4])]
    cz = np.diag([1.0, 1.0, 1.0, -1.0])
    return 1.0 - (abs(np.trace(cz.conj().T @ uq)) ** 2 + 4.0) / 20.0


def g1_block_channel(angle_zz: float, s_cz: np.ndarray, xtalk_phase: float = 0.0,
                     post_left=None, post_right=None, eta: float = 1e-15):
    """The ZZ block of Eq. HZ_block_representation with each CZ replaced by the pulse
    channel s_cz: CNOT (I (x) Rz) CNOT, CNOT = (I (x) Had) CZ (I (x) Had); crosstalk phase
    first (as in G0), optional one-site unitaries after.  Returns a Kraus set."""
    had2 = np.kron(ops.I3, ops.HAD_Q)
    rz = np.kron(ops.I3, ops.expm_h(angle_zz, ops.Z_Q))
    s = ops.superop([had2]) @ s_cz @ ops.superop([had2 @ rz @ had2]) @ s_cz @ ops.superop([had2])
    if xtalk_phase != 0.0:
        s = s @ ops.superop([ops.expm_h(xtalk_phase, np.kron(ops.N_R, ops.N_R))])
    if post_left is not None or post_right is not None:
        v = np.kron(post_left if post_left is not None else ops.I3,
                    post_right if post_right is not None else ops.I3)
        s = ops.superop([v]) @ s
    return ops.kraus_from_superop(s, eta)
