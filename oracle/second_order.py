"""Second-order observables of an MPDO (oracle; test infrastructure only).

Quantities quadratic in rho (Sec. III.E; their environments are the doubled transfer
matrices whose cost Fig. 6c-d discusses):

  purity      xi = tr(rho^2) / tr(rho)^2                           (Sec. III.D, Eq. xiformula)
  collision   Z  = sum_x <x|rho|x>^2 / tr(rho)^2   (anticoncentration of the outcome
                                                    distribution, Sec. III.E)
  Renyi-2     S2(A) = -log( tr(rho_A^2) / tr(rho)^2 ),  rho_A = tr_B rho
  mutual info I2(L:R) = S2(L) + S2(R) - S2(LR) for the cut between sites cut-1 and cut.

With rho = sum_k X_k X_k^+ and the site tensors A[l, s, k, r], one site of rho is the
operator R[(l,l'), s, s', (r,r')] = sum_k A[l,s,k,r] conj(A[l',s',k,r']).  Two copies of rho
are contracted site by site with a four-index environment E[(a,b),(c,d)]:
  crossed (tr rho^2 on the site): E' = sum_{s,s'} E . R[.., s, s', ..] (x) R[.., s', s, ..]
  diagonal (collision):           E' = sum_s     E . R[.., s, s, ..]  (x) R[.., s, s, ..]
  separate (the site traced out in each copy): E' = sum_{s,s2} E . R[.., s, s, ..] (x)
                                                R[.., s2, s2, ..]
Plain einsum, no reordering beyond the definitions.
"""
from __future__ import annotations

import numpy as np


def _R(a: np.ndarray) -> np.ndarray:
    """R[l, l', s, s', r, r'] = sum_k A[l,s,k,r] conj(A[l',s',k,r'])."""
    return np.einsum("askr,btkq->abstrq", a, a.conj(), optimize=True)


def _step(env: np.ndarray, r: np.ndarray, kind: str) -> np.ndarray:
    """One site of the four-index environment env[a, b, c, d] (first copy a, b; second
    copy c, d)."""
    if kind == "cross":
        return np.einsum("abcd,abstrq,cdtsxy->rqxy", env, r, r, optimize=True)
    if kind == "diag":
        return np.einsum("abcd,abssrq,cdssxy->rqxy", env, r, r, optimize=True)
    if kind == "sep":
        return np.einsum("abcd,abssrq,cdttxy->rqxy", env, r, r, optimize=True)
    raise ValueError(kind)


def _sweep(A, kinds) -> complex:
    env = np.ones((1, 1, 1, 1), dtype=complex)
    for a, kind in zip(A, kinds):
        env = _step(env, _R(a), kind)
    return complex(env.reshape(-1)[0])


def second_order(m, cut: int):
    """xi, collision, S2(L), S2(R), I2(L:R) of the MPDO m for the cut before site `cut`."""
    n = m.n
    if not 1 <= cut <= n - 1:
        raise ValueError("cut must be within 1..n-1")
    tr2 = _sweep(m.A, ["sep"] * n).real            # tr(rho)^2
    p2 = _sweep(m.A, ["cross"] * n).real           # tr(rho^2)
    col = _sweep(m.A, ["diag"] * n).real           # sum_x <x|rho|x>^2
    pl = _sweep(m.A, ["cross"] * cut + ["sep"] * (n - cut)).real    # tr(rho_L^2)
    pr = _sweep(m.A, ["sep"] * cut + ["cross"] * (n - cut)).real    # tr(rho_R^2)
    s2 = -np.log(p2 / tr2)
    s2l = -np.log(pl / tr2)
    s2r = -np.log(pr / tr2)
    return dict(xi=p2 / tr2, collision=col / tr2, s2_left=s2l, s2_right=s2r,
                i2=s2l + s2r - s2)


def second_order_dense(rho: np.ndarray, n: int, cut: int, d: int = 3):
    """The same quantities from a dense d^n x d^n density matrix (definitions written out)."""
    tr = np.trace(rho).real
    p2 = np.sum(np.abs(rho) ** 2)                  # tr(rho^2) for Hermitian rho
    col = np.sum(np.real(np.diag(rho)) ** 2)
    t = rho.reshape(d ** cut, d ** (n - cut), d ** cut, d ** (n - cut))
    rl = np.einsum("ajbj->ab", t)                  # tr_R
    rr = np.einsum("iaib->ab", t)                  # tr_L
    pl = np.sum(np.abs(rl) ** 2)
    pr = np.sum(np.abs(rr) ** 2)
    s2, s2l, s2r = -np.log(p2 / tr ** 2), -np.log(pl / tr ** 2), -np.log(pr / tr ** 2)
    return dict(xi=p2 / tr ** 2, collision=col / tr ** 2, s2_left=s2l, s2_right=s2r,
                i2=s2l + s2r - s2)
