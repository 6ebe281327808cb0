"""Vectorized MPO with purity-preserving truncation on the bond (oracle; test
infrastructure only).

The paper's main engine (Sec. III.A "vectorized MPO", Sec. III.D): rho is an MPS over the
doubled index eta = (s, s') (local dimension d^2 = 9),
    rho[(s_1..s_N), (s'_1..s'_N)] = sum_bonds prod_n A_n[b_{n-1}, (s_n, s'_n), b_n],
kept in mixed-canonical form for the Frobenius inner product <<X|Y>> = tr(X^+ Y).  A
two-site channel acts on the pair (eta_i, eta_j) as its superoperator; the pair is split by
an SVD and the bond truncated to at most chi values.  With the canonical gauge the purity is
tr rho^2 = sum_k Lambda_k^2 (P = identity) and the trace tr rho = sum_k T_k Lambda_k with the
trace environment
    T_k = (sum_{l,eta} L[l] tau[eta] U[(l,eta), k]) (sum_{eta,r} V^+[k, (eta,r)] tau[eta] R[r]),
tau[(s,s')] = delta_{s s'}, and L, R the contractions of the sites left / right of the bond
with tau.  "naive" keeps the largest values unchanged; "ppt" replaces them by PPT's values
(Eqs. xiformula and ppt with this T; oracle.ppt), which keep tr rho and
xi = tr rho^2 / tr rho^2 of the bond.
"""
from __future__ import annotations

import numpy as np

from . import ops, ppt as ppt_mod

D = 3
TAU = np.eye(D, dtype=complex).reshape(D * D)      # tau[(s, s')] = delta


def pair_superop(s: np.ndarray) -> np.ndarray:
    """The two-site superoperator (row-major vec over ((s_i,s_j),(s'_i,s'_j))) re-indexed to
    the MPO pair ((s_i,s'_i),(s_j,s'_j)) on rows and columns."""
    t = s.reshape(D, D, D, D, D, D, D, D)         # [si sj si' sj'] x [ti tj ti' tj']
    return t.transpose(0, 2, 1, 3, 4, 6, 5, 7).reshape(81, 81)


class VMPO:
    def __init__(self, n_sites: int, site_state: np.ndarray, chi_max: int, mode: str = "ppt",
                 sv_cutoff: float = 1e-14):
        v = np.asarray(site_state, dtype=complex)
        a = np.outer(v, v.conj()).reshape(1, D * D, 1)
        self.n = n_sites
        self.A = [a.copy() for _ in range(n_sites)]
        self.centre = 0
        self.chi_max = chi_max
        self.mode = mode
        self.sv_cutoff = sv_cutoff
        self.ppt_infeasible = 0
        self.t_imag_max = 0.0
        # smallest (Lambda_chi-1^2 - Lambda_chi^2) / Lambda_0^2 over the truncations at chi:
        # the conditioning of the kept subspace (a perturbation dH of the bond's Gram turns
        # it by ~|dH| / gap)
        self.cut_gap_min = np.inf

    # trace environments of the sites left of i and right of j (contractions with tau)
    def _left_trace(self, i: int) -> np.ndarray:
        e = np.ones(1, dtype=complex)
        for a in self.A[:i]:
            e = np.einsum("l,lhr,h->r", e, a, TAU)
        return e

    def _right_trace(self, j: int) -> np.ndarray:
        e = np.ones(1, dtype=complex)
        for a in reversed(self.A[j + 1:]):
            e = np.einsum("r,lhr,h->l", e, a, TAU)
        return e

    def apply_two_site(self, i: int, kraus):
        j = i + 1
        s = pair_superop(ops.superop(kraus))
        a, b = self.A[i], self.A[j]
        dl, dr = a.shape[0], b.shape[2]
        th = np.einsum("lhb,bgr->lhgr", a, b).reshape(dl, 81, dr)
        th = np.einsum("pq,lqr->lpr", s, th).reshape(dl * 9, 9 * dr)
        u, lam, vh = np.linalg.svd(th, full_matrices=False)
        # the Schmidt values of the state: numerical zeros (whose vectors are an arbitrary
        # basis of the null space) are not part of it, nor of PPT's Lambda and T
        nz = max(1, int(np.count_nonzero(lam > self.sv_cutoff * lam[0])))
        u, lam, vh = u[:, :nz], lam[:nz], vh[:nz]
        keep = max(1, min(nz, self.chi_max))
        if nz > keep:
            self.cut_gap_min = min(self.cut_gap_min,
                                   float((lam[keep - 1] ** 2 - lam[keep] ** 2) / lam[0] ** 2))
        if self.mode == "ppt":
            tl = np.einsum("l,h,lhk->k", self._left_trace(i), TAU, u.reshape(dl, 9, -1))
            tr = np.einsum("khr,h,r->k", vh.reshape(-1, 9, dr), TAU, self._right_trace(j))
            tc = tl * tr
            # real for a Hermitian rho (the vectorised rho is invariant under the site-wise
            # swap s <-> s' with conjugation, so each non-degenerate pair's phases cancel)
            self.t_imag_max = max(self.t_imag_max, float(np.abs(tc.imag).max() /
                                                         max(1e-300, np.abs(tc).max())))
            t = tc.real
            lk, info = ppt_mod.ppt(lam, keep, t)
            self.ppt_infeasible += int(info["infeasible"])
        else:
            lk = lam[:keep]
        if self.centre == i:
            self.A[i] = u[:, :keep].reshape(dl, 9, keep)
            self.A[j] = (lk[:, None] * vh[:keep]).reshape(keep, 9, dr)
            self.centre = j
        elif self.centre == j:
            self.A[i] = (u[:, :keep] * lk[None, :]).reshape(dl, 9, keep)
            self.A[j] = vh[:keep].reshape(keep, 9, dr)
            self.centre = i
        else:
            raise ValueError("two-site op must touch the orthogonality centre")

    # ---------------------------------------------------------------- observables
    def expect(self, op_map) -> complex:
        """tr(O rho) for O = (x)_n op_map.get(n, I): o[(s,s')] = O[s', s]."""
        e = np.ones(1, dtype=complex)
        for n, a in enumerate(self.A):
            o = op_map.get(n, ops.I3).T.reshape(9)
            e = np.einsum("l,lhr,h->r", e, a, o)
        return complex(e[0])

    def expect_energy(self, J: float, hx: float, bz: float):
        n = self.n
        out = {}
        for tag, proj in (("raw", ops.I3), ("succ", ops.P_Q)):
            base = {k: proj for k in range(n)}
            norm = self.expect(base).real
            tot = 0.0
            for s in range(n):
                m = dict(base)
                m[s] = proj @ (-hx * ops.X_Q - bz * J * ops.Z_Q) @ proj
                tot += self.expect(m).real
            for s in range(n - 1):
                m = dict(base)
                m[s] = proj @ ops.Z_Q @ proj
                m[s + 1] = proj @ ops.Z_Q @ proj
                tot += -J * self.expect(m).real
            out[tag] = (tot, norm)
        tr = out["raw"][1]
        ps = out["succ"][1]
        return dict(e_raw=out["raw"][0] / tr, e_succ=out["succ"][0] / ps, p_succ=ps, trace=tr)

    def purity(self) -> float:
        """tr rho^2 = <<rho|rho>> (Hermitian rho), contracted site by site."""
        e = np.ones((1, 1), dtype=complex)
        for a in self.A:
            e = np.einsum("ab,ahr,bhq->rq", e, a, a.conj())
        return float(e[0, 0].real)

    def collision(self) -> float:
        """Collision probability sum_x <x|rho|x>^2 / (tr rho)^2 (Sec. III.E, the
        anticoncentration of Fig. 7): the diagonal rho_xx = prod_n A_n[., (s_n, s_n), .]
        contracted with itself over x, and the trace sum_x rho_xx, site by site."""
        e2 = np.ones((1, 1), dtype=complex)
        e1 = np.ones(1, dtype=complex)
        for a in self.A:
            dg = a.reshape(a.shape[0], D, D, a.shape[2])[:, np.arange(D), np.arange(D), :]
            e2 = np.einsum("ab,asr,bsq->rq", e2, dg, dg)
            e1 = np.einsum("a,asr->r", e1, dg)
        return float(e2[0, 0].real / e1[0].real ** 2)

    def to_dense(self) -> np.ndarray:
        """rho as a d^N x d^N matrix (tiny N): x[(p,s),(q,s'),r] = sum_l x[p,q,l] A[l,(s,s'),r]."""
        x = np.ones((1, 1, 1), dtype=complex)
        for a in self.A:
            a4 = a.reshape(a.shape[0], D, D, a.shape[2])
            x = np.einsum("pql,lstr->psqtr", x, a4)
            p, s, q, t, r = x.shape
            x = x.reshape(p * s, q * t, r)
        return x[:, :, 0]
