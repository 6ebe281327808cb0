"""Plain MPDO with the two-site update (oracle; test infrastructure only).

State (Sec. III.C, Fig. 3a): rho = sum_{k_1..k_N} X_k X_k^+ with site tensors
A_n[l, s, k, r] (left bond, atom level, inner/Kraus index, right bond), i.e. an MPS
"purification" whose physical index at site n is (s_n, k_n).  tr(rho) = <X|X>.

Mixed-canonical gauge with a centre c (Sec. III.A "Canonization"): every site left of c
contracts to the identity on its right bond, every site right of c to the identity on
its left bond.

Two-site update of a channel {E_m} on (i, i+1) (Sec. III.A, Fig. 2c and Fig. 6a;
reading: the gate's Kraus index m is attached to the inner index of the site that
becomes the centre, X' = sum_m (E_m X) (x) |m>, exact before truncation):
  1. contract the two site tensors and the gate into theta
  2. SVD theta across the bond, keep at most chi values above sv_cutoff * s_max,
     rescale the kept values so sum s^2 (= tr rho) is unchanged
  3. the new centre's inner index (m, k) is truncated to at most K by the
     eigendecomposition of its Gram matrix W (the ancilla's reduced density matrix
     in this gauge), with the kept eigenvalues replaced by PPT's values
     (Sec. III.D, reading: Lambda = w, T = 1, P = identity).
The SVD of step 2 is taken either of theta itself (plain=True) or, by the exact QR
identity theta = Q_i Z Q_j, of the smaller Z; both give the same singular triplets.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import ppt as ppt_mod

D = 3


@dataclasses.dataclass
class TruncStats:
    disc_bond_w: float = 0.0
    disc_kraus_w: float = 0.0
    ppt_theta_min: float = float("inf")
    ppt_infeasible: int = 0
    ppt_clamped: int = 0
    chi_used_max: int = 0
    k_used_max: int = 0


class MPDO:
    def __init__(self, n_sites: int, site_state: np.ndarray, chi_max: int, k_max: int,
                 sv_cutoff: float = 1e-14, kraus_cutoff: float = 1e-14,
                 use_ppt: bool = True, plain: bool = False):
        self.n = n_sites
        self.A = [np.asarray(site_state, dtype=complex).reshape(1, D, 1, 1).copy()
                  for _ in range(n_sites)]
        self.centre = 0
        self.chi_max, self.k_max = chi_max, k_max
        self.sv_cutoff, self.kraus_cutoff = sv_cutoff, kraus_cutoff
        self.use_ppt, self.plain = use_ppt, plain
        self.stats = TruncStats()

    # ------------------------------------------------------------ helpers
    def _svd_bond(self, a, bt, e, left_to_right: bool):
        """theta' and its SVD for the pair (a = A_i, bt = A_{i+1}) under Kraus set e.

        Returns U, s, Vh with the row index of U ordered (l, s_i', [m,] k_i) and the
        column index of Vh ordered (s_j', [m,] k_j, r); m sits on the side of the new
        centre (right for left->right, left for right->left).
        """
        dl, _, ki, dm = a.shape
        _, _, kj, dr = bt.shape
        m = e.shape[0]
        e6 = e.reshape(m, D, D, D, D)              # [m, S, T, s, t]
        if self.plain:
            th = np.einsum("lskb,btqr->lsktqr", a, bt)
            thp = np.einsum("mSTst,lsktqr->lSkTmqr", e6, th)
            if left_to_right:
                mat = thp.reshape(dl * D * ki, D * m * kj * dr)
            else:
                mat = thp.transpose(0, 1, 4, 2, 3, 5, 6).reshape(dl * D * m * ki, D * kj * dr)
            return np.linalg.svd(mat, full_matrices=False)
        # QR identity: A_i as [(l,k),(s,b)] = Q_i R_i ; A_j as [(b,t),(q,r)] = L_j Q_j
        qi, ri = np.linalg.qr(a.transpose(0, 2, 1, 3).reshape(dl * ki, D * dm))
        qj_h, rj_h = np.linalg.qr(bt.reshape(dm * D, kj * dr).conj().T)
        lj, qj = rj_h.conj().T, qj_h.conj().T       # lj: (dm*D, rj), qj: (rj, kj*dr)
        ci, cj = ri.shape[0], lj.shape[1]
        r4 = ri.reshape(ci, D, dm)                  # [c, s, b]
        l3 = lj.reshape(dm, D, cj)                  # [b, t, e]
        core = np.einsum("csb,bte->cste", r4, l3)
        z = np.einsum("mSTst,cste->cSTme", e6, core)    # [c, S, T, m, e]
        if left_to_right:
            zm = z.reshape(ci * D, D * m * cj)
            u, s, vh = np.linalg.svd(zm, full_matrices=False)
            # U rows (l,k) x S from Q_i ; Vh columns (T, m, e) -> (T, m, q, r)
            u = np.einsum("xc,cSb->xSb", qi, u.reshape(ci, D, -1))       # x=(l,k)
            u = u.reshape(dl, ki, D, -1).transpose(0, 2, 1, 3).reshape(dl * D * ki, -1)
            vh = np.einsum("bTme,ey->bTmy", vh.reshape(-1, D, m, cj), qj)
            vh = vh.reshape(vh.shape[0], -1)
            return u, s, vh
        zm = z.transpose(0, 1, 3, 2, 4).reshape(ci * D * m, D * cj)     # rows (c,S,m)
        u, s, vh = np.linalg.svd(zm, full_matrices=False)
        u = np.einsum("xc,cSmb->xSmb", qi, u.reshape(ci, D, m, -1))
        u = u.reshape(dl, ki, D, m, -1).transpose(0, 2, 3, 1, 4).reshape(dl * D * m * ki, -1)
        vh = np.einsum("bTe,ey->bTy", vh.reshape(-1, D, cj), qj).reshape(vh.shape[0], -1)
        return u, s, vh

    def _cut(self, s: np.ndarray, chi: int):
        keep = int(np.count_nonzero(s > self.sv_cutoff * s[0]))
        keep = max(1, min(keep, chi))
        tot = float(s @ s)
        kept = s[:keep].copy()
        kw = float(kept @ kept)
        self.stats.disc_bond_w += (tot - kw) / tot
        kept *= np.sqrt(tot / kw)
        self.stats.chi_used_max = max(self.stats.chi_used_max, keep)
        return keep, kept

    def kraus_truncate(self, c: np.ndarray, k_max: int, use_ppt: bool) -> np.ndarray:
        """Truncate the inner index of the centre tensor c[l, s, kappa, r].

        W = C C^+ with C = c as a [kappa, (l,s,r)] matrix; its eigenpairs are taken from
        the SVD C = U S V^+ (w = S^2, eigenvectors U), the plain definition.  Values with
        sqrt(w) <= kraus_cutoff * sqrt(w_max) are numerical zeros.  The kept rows become
        sqrt(Lambda~_k) V^+_k, i.e. U_K^+ C rescaled so that its Gram is diag(Lambda~).
        """
        dl, _, kk, dr = c.shape
        cm = c.transpose(2, 0, 1, 3).reshape(kk, -1)         # rows kappa
        _, sv, vh = np.linalg.svd(cm, full_matrices=False)
        if sv[0] <= 0.0:
            raise FloatingPointError("zero state")
        w = sv * sv
        keep = int(np.count_nonzero(sv > self.kraus_cutoff * sv[0]))
        keep = max(1, min(keep, k_max))
        tot = float(w.sum())
        self.stats.disc_kraus_w += (tot - float(w[:keep].sum())) / tot
        if use_ppt:
            lt, info = ppt_mod.ppt(w, keep)
            self.stats.ppt_theta_min = min(self.stats.ppt_theta_min, info["theta"])
            self.stats.ppt_infeasible += int(info["infeasible"])
            self.stats.ppt_clamped += info["clamped"]
        else:
            lt = w[:keep] * (tot / float(w[:keep].sum()))
        new = np.sqrt(lt)[:, None] * vh[:keep]
        self.stats.k_used_max = max(self.stats.k_used_max, keep)
        return new.reshape(keep, dl, D, dr).transpose(1, 2, 0, 3)

    # ------------------------------------------------------------ the update
    def apply_two_site(self, i: int, kraus, chi_max: int = None, k_max: int = None,
                       use_ppt: bool = None):
        chi = self.chi_max if chi_max is None else chi_max
        kmax = self.k_max if k_max is None else k_max
        up = self.use_ppt if use_ppt is None else use_ppt
        e = np.asarray(kraus, dtype=complex).reshape(-1, D * D, D * D)
        a, bt = self.A[i], self.A[i + 1]
        dl, _, ki, _ = a.shape
        _, _, kj, dr = bt.shape
        m = e.shape[0]
        if self.centre == i:
            u, s, vh = self._svd_bond(a, bt, e, True)
            keep, sk = self._cut(s, chi)
            self.A[i] = u[:, :keep].reshape(dl, D, ki, keep)
            b = (sk[:, None] * vh[:keep]).reshape(keep, D, m * kj, dr)
            self.A[i + 1] = self.kraus_truncate(b, kmax, up)
            self.centre = i + 1
        elif self.centre == i + 1:
            u, s, vh = self._svd_bond(a, bt, e, False)
            keep, sk = self._cut(s, chi)
            self.A[i + 1] = vh[:keep].reshape(keep, D, kj, dr)
            b = (u[:, :keep] * sk[None, :]).reshape(dl, D, m * ki, keep)
            self.A[i] = self.kraus_truncate(b, kmax, up)
            self.centre = i
        else:
            raise ValueError("two-site op must touch the orthogonality centre")

    def truncate(self, chi_max: int, k_max: int, use_ppt: bool):
        """Re-truncate the whole chain to new limits: identity two-site updates swept
        from the centre to the far end and back (every bond and inner index visited
        once with the centre on it)."""
        ident = [np.eye(D * D, dtype=complex)]
        while self.centre < self.n - 1:
            self.apply_two_site(self.centre, ident, chi_max, k_max, use_ppt)
        while self.centre > 0:
            self.apply_two_site(self.centre - 1, ident, chi_max, k_max, use_ppt)

    # ------------------------------------------------------------ dense view
    def to_dense(self) -> np.ndarray:
        """rho as a d^N x d^N matrix (tiny N only); the inner index is summed site by
        site, rho_{<=n}[(p,s),(p',s'),r,r'] = sum rho_{<n}[p,p',l,l'] A[l,s,k,r] A*[l',s',k,r']."""
        x = np.ones((1, 1, 1, 1), dtype=complex)
        for a in self.A:
            x = np.einsum("pqab,askr,btkc->psqtrc", x, a, a.conj(), optimize=True)
            p, s, q, t, r, c = x.shape
            x = x.reshape(p * s, q * t, r, c)
        return x[:, :, 0, 0]

    def dims(self):
        return [a.shape for a in self.A]
