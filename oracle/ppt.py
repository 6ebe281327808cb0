"""Purity-preserving truncation (oracle; test infrastructure only).

Sec. III.D and App. B.  A diagonal truncation keeps tr(rho) = sum_i T_i Lambda_i and,
with P = identity, tr(rho^2) = |Lambda|^2, so xi = |Lambda|^2 / (T.Lambda)^2.
After projecting Lambda to Lambda' = P_T Lambda (and T' = P_T T), the new values are
the point on the cone of half-angle theta about T' reached from Lambda' inside the
plane span(Lambda', T'), with

    theta = arccos(|T| cos(phi) / |T'|)                           (Eq. xiformula)
    Lambda~ = Lambda' + (tan theta / tan sigma - 1)
                        (Lambda' - |Lambda'| cos(sigma) T' / |T'|)   (Eq. ppt)

phi = angle(Lambda, T), sigma = angle(Lambda', T').

Readings where the paper is silent:
  * infeasible (|T'| < |T| cos phi): theta = 0, so Lambda~ is along T' (Sec. III.D end);
  * sigma = 0 (Lambda' parallel to T'): Lambda~ = Lambda';
  * negative entries of Lambda~ are clamped to 0 (keeps the MPDO positive) and counted;
  * overall scale ("up to some normalization constant", App. B): Lambda~ is rescaled
    so that T'.Lambda~ = T.Lambda, i.e. the truncation keeps tr(rho).
"""
from __future__ import annotations

import numpy as np


def ppt(lam: np.ndarray, keep: int, t: np.ndarray = None):
    """Return (Lambda~ restricted to the first `keep` entries, info dict).

    lam: all values (any order; entries [0, keep) are the ones kept).
    t:   trace environment T (default: all ones, the MPDO Kraus case).
    """
    lam = np.asarray(lam, dtype=float)
    t = np.ones_like(lam) if t is None else np.asarray(t, dtype=float)
    lam_p = lam[:keep].copy()
    t_p = t[:keep].copy()
    nl, nt = np.linalg.norm(lam), np.linalg.norm(t)
    nlp, ntp = np.linalg.norm(lam_p), np.linalg.norm(t_p)
    info = dict(theta=None, infeasible=False, clamped=0)
    if nlp == 0.0:
        raise ValueError("all kept values are zero")
    cos_phi = float(lam @ t) / (nl * nt)
    cos_sig = min(1.0, float(lam_p @ t_p) / (nlp * ntp))
    ratio = nt * cos_phi / ntp
    if ratio > 1.0:
        info["infeasible"] = True
        theta = 0.0
    else:
        theta = float(np.arccos(ratio))
    info["theta"] = theta
    sigma = float(np.arccos(cos_sig))
    if sigma == 0.0:
        out = lam_p.copy()
    else:
        x = np.tan(theta) / np.tan(sigma) - 1.0
        out = lam_p + x * (lam_p - nlp * cos_sig * t_p / ntp)
    neg = out < 0.0
    info["clamped"] = int(np.count_nonzero(neg))
    out[neg] = 0.0
    out *= float(lam @ t) / float(out @ t_p)
    return out, info


def xi(lam: np.ndarray, t: np.ndarray = None) -> float:
    """xi = tr(rho^2) / tr(rho)^2 with P = identity (Sec. III.D)."""
    lam = np.asarray(lam, dtype=float)
    t = np.ones_like(lam) if t is None else np.asarray(t, dtype=float)
    return float(lam @ lam) / float(lam @ t) ** 2
