"""Transfer-matrix observables and sampling on an MPDO (oracle; test infrastructure only).

For a product operator O = (x)_n O_n, tr(O rho) = sum_{s,s'} O[s',s] rho[s,s'] contracts
site by site with the transfer map (Sec. III.E, Fig. 6c uses the same environment
construction for second-order quantities):

    E'[r, r'] = sum_{l,l',s,s',k} E[l, l'] A[l,s,k,r] O[s',s] conj(A[l',s',k,r'])

Energies of H = -J sum S^z_i S^z_{i+1} - h sum S^x_i - b J sum S^z_i (Eq. tfim_hamiltonian,
S = Pauli on the qubit levels, zero on |r>):
  e_raw  = tr(H rho) / tr(rho)
  p_succ = tr(Pi_q rho), Pi_q = (x)(|0><0| + |1><1|)   (qubit trace, Sec. IV.A)
  e_succ = tr(Pi_q H Pi_q rho) / p_succ                (outcome given a successful
                                                         measurement, Sec. I and IV.A)
Sampling draws x in {0,1,r}^N with probability <x|rho|x>/tr(rho) site by site from the
conditional marginals; the probability reported for a sample is <x|rho|x>.
"""
from __future__ import annotations

import numpy as np

from . import ops, philox


def transfer(env: np.ndarray, a: np.ndarray, o: np.ndarray) -> np.ndarray:
    return np.einsum("ab,askr,ts,btkq->rq", env, a, o, a.conj(), optimize=True)


def _left_envs(m, o):
    envs = [np.ones((1, 1), dtype=complex)]
    for a in m.A:
        envs.append(transfer(envs[-1], a, o))
    return envs                                    # envs[n] = left of site n


def _right_envs(m, o):
    envs = [np.ones((1, 1), dtype=complex)]
    for a in reversed(m.A):
        envs.append(np.einsum("rq,askr,ts,btkq->ab", envs[-1], a, o, a.conj(), optimize=True))
    return envs[::-1]                              # envs[n] = right of site n-1


def _close(left, right):
    return complex(np.einsum("ab,ab->", left, right))


def expect_energy(m, J: float, hx: float, bz: float):
    n = m.n
    out = {}
    for tag, o in (("raw", ops.I3), ("succ", ops.P_Q)):
        le, re = _left_envs(m, o), _right_envs(m, o)
        norm = _close(le[n], re[n]).real
        tot = 0.0
        for s in range(n):
            t = transfer(le[s], m.A[s], -hx * ops.X_Q - bz * J * ops.Z_Q)
            tot += _close(t, re[s + 1]).real
        for s in range(n - 1):
            t = transfer(le[s], m.A[s], ops.Z_Q)
            t = transfer(t, m.A[s + 1], ops.Z_Q)
            tot += -J * _close(t, re[s + 2]).real
        out[tag] = (tot, norm)
    tr = out["raw"][1]
    ps = out["succ"][1]
    return dict(e_raw=out["raw"][0] / tr, e_succ=out["succ"][0] / ps, p_succ=ps, trace=tr)


def prob_of(m, x) -> float:
    """<x|rho|x> for one configuration x."""
    env = np.ones((1, 1), dtype=complex)
    for a, v in zip(m.A, x):
        proj = np.zeros((3, 3), dtype=complex)
        proj[v, v] = 1.0
        env = transfer(env, a, proj)
    return float(env[0, 0].real)


def sample(m, n_samples: int, seed: int):
    """Sequential conditional sampling with Philox uniforms u(seed, sample, site).

    At site n the three weights q_v = <x_<n, v| rho_{<=n} |x_<n, v> (rest traced) are
    formed in double precision; v = 0 if u < q_0/Q, v = 1 if u < (q_0+q_1)/Q, else 2.
    """
    re = _right_envs(m, ops.I3)
    n = m.n
    bits = np.zeros((n_samples, n), dtype=np.uint8)
    probs = np.zeros(n_samples)
    for smp in range(n_samples):
        env = np.ones((1, 1), dtype=complex)
        for s in range(n):
            cand = []
            q = np.zeros(3)
            for v in range(3):
                proj = np.zeros((3, 3), dtype=complex)
                proj[v, v] = 1.0
                t = transfer(env, m.A[s], proj)
                cand.append(t)
                q[v] = max(0.0, _close(t, re[s + 1]).real)
            tot = q.sum()
            u = philox.uniform(seed, smp, s)
            if u < q[0] / tot:
                v = 0
            elif u < (q[0] + q[1]) / tot:
                v = 1
            else:
                v = 2
            bits[smp, s] = v
            env = cand[v]
        probs[smp] = float(env[0, 0].real)
    return bits, probs
