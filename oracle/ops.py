"""Local operators and noisy two-site channels (oracle; test infrastructure only).

Local basis of one atom: index 0 = |0>, 1 = |1>, 2 = |r> (Sec. II: two qubit levels
plus the Rydberg level; the dark states |d> lie outside the simulated space, so decay
into them removes trace, Sec. II and Sec. IV.A "qubit trace").

Two-site operators are 9x9 matrices on the index s_i*3 + s_j (left site first).
A channel is a list of Kraus operators E_m with rho -> sum_m E_m rho E_m^dagger.
The superoperator of a channel acts on row-major vec(rho): S = sum_m E_m (x) conj(E_m).
"""
from __future__ import annotations

import numpy as np

D = 3
I3 = np.eye(D, dtype=complex)
P_Q = np.diag([1.0, 1.0, 0.0]).astype(complex)          # projector on the qubit levels
N_R = np.diag([0.0, 0.0, 1.0]).astype(complex)          # Rydberg number operator
Z_Q = np.diag([1.0, -1.0, 0.0]).astype(complex)         # S^z as a Pauli on the qubit levels
X_Q = np.array([[0, 1, 0], [1, 0, 0], [0, 0, 0]], dtype=complex)
HAD_Q = np.array([[1, 1, 0], [1, -1, 0], [0, 0, np.sqrt(2.0)]], dtype=complex) / np.sqrt(2.0)
CZ = np.diag([1, 1, 1, 1, -1, 1, 1, 1, 1]).astype(complex)   # |11> -> -|11>


def expm_h(theta: float, h: np.ndarray) -> np.ndarray:
    """exp(-i theta h) for Hermitian h, by its eigendecomposition."""
    w, v = np.linalg.eigh(h)
    return (v * np.exp(-1j * theta * w)) @ v.conj().T


def kron(a, b):
    return np.kron(a, b)


# ---------------------------------------------------------------- channels

def superop(kraus) -> np.ndarray:
    """S = sum_m E_m (x) conj(E_m): vec(E rho E^+) = S vec(rho) for row-major vec."""
    kraus = np.asarray(kraus)
    return sum(np.kron(e, e.conj()) for e in kraus)


def unitary_channel(u):
    return [np.asarray(u, dtype=complex)]


def compose(second, first):
    """Kraus set of the channel 'second o first' (first acts first)."""
    return [b @ a for b in second for a in first]


def choi_from_kraus(kraus) -> np.ndarray:
    """Choi matrix C = sum_m vec(E_m) vec(E_m)^+ with row-major vec."""
    n = np.asarray(kraus[0]).shape[0]
    c = np.zeros((n * n, n * n), dtype=complex)
    for e in kraus:
        v = np.asarray(e).reshape(-1)
        c += np.outer(v, v.conj())
    return c


def kraus_from_choi(c: np.ndarray, eta: float = 1e-15):
    """Canonical Kraus set: eigenvectors of the Choi matrix scaled by sqrt(eigenvalue).

    Eigenvalues below eta * lambda_max are dropped (numerical zeros).  Returned in
    descending eigenvalue order.
    """
    n = int(round(np.sqrt(c.shape[0])))
    w, v = np.linalg.eigh(0.5 * (c + c.conj().T))
    order = np.argsort(w)[::-1]
    w, v = w[order], v[:, order]
    keep = w > eta * w[0]
    return [np.sqrt(w[m]) * v[:, m].reshape(n, n) for m in np.nonzero(keep)[0]]


def canonical_kraus(kraus, eta: float = 1e-15):
    return kraus_from_choi(choi_from_kraus(kraus), eta)


# ------------------------------------------------- single-atom noise (G0 form)

def lindblad_generator(gamma_diss: float, gamma_deph: float, b0: float, b1: float,
                       bd: float) -> np.ndarray:
    """Superoperator generator G of d rho/dt = sum_i L rho L^+ - 1/2 {L^+L, rho}
    (Eq. LME without the Hamiltonian) on one atom, acting on row-major vec(rho).

    Jump operators (Sec. II): L_j = sqrt(gamma_diss b_j)|j><r| for j in {0, 1, d} and
    L_deph = sqrt(gamma_deph/2) (|0><0| - |1><1|).  The printed L_deph has gamma/sqrt(2);
    the linear-rate reading sqrt(gamma/2) is used (its rate is linear in gamma).
    L_d maps out of the simulated space: only its anticommutator term is kept, which
    makes the channel trace-decreasing by the dark branch.
    """
    e = lambda i, j: np.outer(I3[i], I3[j])
    jumps_in = [np.sqrt(gamma_diss * b0) * e(0, 2), np.sqrt(gamma_diss * b1) * e(1, 2),
                np.sqrt(gamma_deph / 2.0) * Z_Q]
    loss = gamma_diss * bd * e(2, 2)                  # L_d^+ L_d
    g = np.zeros((9, 9), dtype=complex)
    for L in jumps_in:
        LdL = L.conj().T @ L
        g += np.kron(L, L.conj()) - 0.5 * (np.kron(LdL, I3) + np.kron(I3, LdL.T))
    g += -0.5 * (np.kron(loss, I3) + np.kron(I3, loss.T))
    return g


def g0_noise_superop(gamma_diss: float, gamma_deph: float, b0: float, b1: float,
                     bd: float) -> np.ndarray:
    """Closed form of one unit of the single-atom Lindblad evolution (Sec. II jump
    operators, linear-rate dephasing), written element by element:

      decay:     rho_rr -> e^{-g} rho_rr,   rho_qr -> e^{-g/2} rho_qr (q in {0,1}),
                 rho_jj -> rho_jj + b_j (1 - e^{-g}) rho_rr          (j in {0,1})
      dephasing: rho_01 -> e^{-gp} rho_01,  rho_qr -> e^{-gp/4} rho_qr
    The two generators commute, so the product is exact.
    """
    g, gp = gamma_diss, gamma_deph
    s = np.zeros((9, 9), dtype=complex)
    idx = lambda a, b: a * 3 + b
    for a in range(3):
        for b in range(3):
            f = 1.0
            if (a == 2) != (b == 2):                  # qubit-Rydberg coherence
                f = np.exp(-g / 2.0) * np.exp(-gp / 4.0)
            elif a == 2 and b == 2:
                f = np.exp(-g)
            elif a != b:                              # rho_01, rho_10
                f = np.exp(-gp)
            s[idx(a, b), idx(a, b)] = f
    s[idx(0, 0), idx(2, 2)] += b0 * (1.0 - np.exp(-g))
    s[idx(1, 1), idx(2, 2)] += b1 * (1.0 - np.exp(-g))
    return s


def kraus_from_superop(s: np.ndarray, eta: float = 1e-15):
    """Kraus set of a superoperator S (row-major vec) via its Choi reshuffle
    C[(a,b),(a',b')] = S[(a,a'),(b,b')]."""
    n = int(round(np.sqrt(s.shape[0])))
    c = s.reshape(n, n, n, n).transpose(0, 2, 1, 3).reshape(n * n, n * n)
    return kraus_from_choi(c, eta)


# ----------------------------------------------------------- QAOA block (G0)

def zz_block_unitary(angle_zz: float) -> np.ndarray:
    """Eq. HZ_block_representation: CNOT (I (x) exp(-i a S^z)) CNOT with
    CNOT = (I (x) Had) CZ (I (x) Had); Had and S^z act on the qubit levels only."""
    had2 = np.kron(I3, HAD_Q)
    cnot = had2 @ CZ @ had2
    rz = np.kron(I3, expm_h(angle_zz, Z_Q))
    return cnot @ rz @ cnot


def app_e_phases(gamma_diss: float):
    """App. E: coherence damping alpha = e^{-0.012291 gamma}, beta = e^{-0.0185454 gamma} of
    a dissipative pulse, and the phases it adds to the Ising phase gate:
    d1 = ((1 - alpha)/(1 + alpha))^2 on S^z_i + S^z_j, d2 = ((alpha - beta)/(alpha + beta))^2
    on S^z_i S^z_j."""
    alpha = np.exp(-0.012291 * gamma_diss)
    beta = np.exp(-0.0185454 * gamma_diss)
    return ((1 - alpha) / (1 + alpha)) ** 2, ((alpha - beta) / (alpha + beta)) ** 2


def app_e_shift(angle_zz: float, d1: float, d2: float) -> np.ndarray:
    """exp(-i a (d2 S^z (x) S^z + d1 (S^z (x) I + I (x) S^z))) on two atoms (S^z the Pauli
    matrix on the qubit levels, zero on |r>): the App. E phases of a block of angle a."""
    zz = np.kron(Z_Q, Z_Q)
    z1 = np.kron(Z_Q, I3) + np.kron(I3, Z_Q)
    return expm_h(angle_zz, d2 * zz + d1 * z1)


def g0_block_channel(angle_zz: float, gamma_diss: float, gamma_deph: float,
                     xtalk_phase: float, delta_pp: float, b0: float, b1: float, bd: float,
                     post_left=None, post_right=None, shift=None):
    """One noisy ZZ block on a bond in the G0 (gate-level) model, as a Kraus set.

    Order of action (reading): the crosstalk phase exp(-i phi n_r (x) n_r) on residual Rydberg population
    (Sec. III.B, simplified to the active pair), the ideal ZZ block, post-promotion
    exp(-i dPP (|1><r| + h.c.)) on both atoms (Sec. IV.A), one unit of decay +
    dephasing on both atoms (closed form above), then optional single-site unitaries
    after the block (post_*: the bias and transverse-field gates folded into the last
    block that touches a site).
    """
    u = zz_block_unitary(angle_zz)
    if xtalk_phase != 0.0:
        u = u @ expm_h(xtalk_phase, np.kron(N_R, N_R))
    if delta_pp != 0.0:
        pp = expm_h(delta_pp, np.outer(I3[1], I3[2]) + np.outer(I3[2], I3[1]))
        u = np.kron(pp, pp) @ u
    n1 = g0_noise_superop(gamma_diss, gamma_deph, b0, b1, bd)
    s = np.kron(n1, n1)
    # reorder the (a_i a_j, a_i' a_j') product superoperator to two-site row-major vec
    s = s.reshape(3, 3, 3, 3, 3, 3, 3, 3).transpose(0, 2, 1, 3, 4, 6, 5, 7).reshape(81, 81)
    s = s @ superop([u])
    if shift is not None:                              # a unitary after the noise unit
        s = superop([shift]) @ s
    if post_left is not None or post_right is not None:
        v = np.kron(post_left if post_left is not None else I3,
                    post_right if post_right is not None else I3)
        s = superop([v]) @ s
    return kraus_from_superop(s)
