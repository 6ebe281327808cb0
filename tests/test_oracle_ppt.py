"""Pins for purity-preserving truncation (Sec. III.D, Eqs. xiformula / ppt, App. B)."""
import numpy as np
import pytest
import scipy.optimize

from oracle import ppt


def _spectrum(rng, n):
    return np.sort(rng.exponential(size=n) ** 3)[::-1]


@pytest.mark.parametrize("seed", range(6))
def test_purity_ratio_preserved_when_feasible(seed):
    rng = np.random.default_rng(seed)
    lam = _spectrum(rng, 24)
    keep = 10
    out, info = ppt.ppt(lam, keep)
    if info["infeasible"] or info["clamped"]:
        pytest.skip("case is infeasible or clamped")
    assert abs(ppt.xi(out) - ppt.xi(lam)) < 1e-13 * ppt.xi(lam)
    # trace kept (normalisation reading)
    assert abs(out.sum() - lam.sum()) < 1e-13 * lam.sum()


@pytest.mark.parametrize("seed", range(6))
def test_result_lies_in_span_of_truncated_values_and_trace_env(seed):
    rng = np.random.default_rng(seed)
    lam = _spectrum(rng, 16)
    keep = 6
    out, info = ppt.ppt(lam, keep)
    basis = np.stack([lam[:keep], np.ones(keep)], axis=1)
    coef, res, *_ = np.linalg.lstsq(basis, out, rcond=None)
    if info["clamped"] == 0:
        assert np.linalg.norm(basis @ coef - out) < 1e-12 * np.linalg.norm(out)


def test_infeasible_gives_vector_along_trace_env():
    # one dominant value and a long flat tail: |T'| small compared with |T| cos(phi)
    lam = np.array([1.0] + [0.9] * 40)
    out, info = ppt.ppt(lam, 2)
    assert info["infeasible"]
    assert info["theta"] == 0.0
    assert np.allclose(out / out[0], np.ones(2), atol=1e-14)


def test_no_truncation_is_identity():
    lam = np.array([3.0, 2.0, 0.5, 0.1])
    out, info = ppt.ppt(lam, 4)
    assert np.allclose(out, lam, rtol=1e-13)


def test_matches_brute_force_nearest_point_on_cone():
    """App. B: Lambda~ points along the nearest point of the cone {angle(x, T') = theta}
    to Lambda'.  Brute force: minimise |x - Lambda'| over unit directions on that cone."""
    rng = np.random.default_rng(7)
    lam = _spectrum(rng, 12)
    keep = 5
    out, info = ppt.ppt(lam, keep)
    assert not info["infeasible"]
    theta = info["theta"]
    lp = lam[:keep]
    tp = np.ones(keep) / np.sqrt(keep)

    def on_cone(y):
        # direction = cos(theta) tp + sin(theta) * unit component of y orthogonal to tp
        o = y - (y @ tp) * tp
        o /= np.linalg.norm(o)
        return np.cos(theta) * tp + np.sin(theta) * o

    def dist(y):
        d = on_cone(y)
        return np.linalg.norm(lp - (lp @ d) * d)

    best = None
    for trial in range(20):
        y0 = rng.standard_normal(keep)
        r = scipy.optimize.minimize(dist, y0, method="Nelder-Mead",
                                    options=dict(xatol=1e-12, fatol=1e-14, maxiter=20000))
        if best is None or r.fun < best.fun:
            best = r
    d = on_cone(best.x)
    got = out / np.linalg.norm(out)
    assert abs(abs(got @ d) - 1.0) < 1e-8
