"""Pins of the second-order observables of the oracle (oracle/second_order.py): the MPDO
environments against the definitions on the dense rho (N <= 6), and closed forms: a pure
product state has purity 1, collision prod_n sum_s |v_s|^4, zero Renyi-2 entropies and
mutual information; a state mixed by dephasing only has tr(rho^2) < 1 and symmetric halves."""
import numpy as np

import synth
from oracle import dense as odense
from oracle import mpdo as ompdo
from oracle import qaoa as oqaoa
from oracle import second_order as so


def _run(c):
    m = ompdo.MPDO(c.n_sites, oqaoa.plus_state(), c.chi_max, c.k_max)
    d = odense.DenseRho(c.n_sites, oqaoa.plus_state())
    for i, k in oqaoa.circuit_ops(c):
        m.apply_two_site(i, k)
        d.apply_two_site(i, k)
    return m, d


def test_mpdo_environments_match_dense_definitions():
    c = synth.tiny()
    m, d = _run(c)
    for cut in (1, 3, 5):
        got = so.second_order(m, cut)
        want = so.second_order_dense(d.matrix(), c.n_sites, cut)
        for key in want:
            assert abs(got[key] - want[key]) < 1e-11 * max(1.0, abs(want[key])), (cut, key)
    # the noisy circuit is mixed, and entangled across the middle
    assert 0.0 < got["xi"] < 1.0
    assert so.second_order(m, 3)["i2"] > 1e-3


def test_product_state_closed_forms():
    v = np.array([0.6, 0.8j, 0.0])
    m = ompdo.MPDO(5, v, 4, 4)
    r = so.second_order(m, 2)
    assert abs(r["xi"] - 1.0) < 1e-14
    assert abs(r["collision"] - (0.6 ** 4 + 0.8 ** 4) ** 5) < 1e-14
    assert abs(r["s2_left"]) < 1e-14 and abs(r["s2_right"]) < 1e-14 and abs(r["i2"]) < 1e-14


def test_truncated_chain_matches_dense_within_truncation():
    """A truncated MPDO (chi = 6, K = 3 on 6 sites): its own rho, reassembled densely,
    gives the same second-order values as its environments."""
    c = synth.scaled(synth.chain40(), n_sites=6, chi_max=6, k_max=3)
    m = ompdo.MPDO(c.n_sites, oqaoa.plus_state(), c.chi_max, c.k_max)
    for i, k in oqaoa.circuit_ops(c):
        m.apply_two_site(i, k)
    got = so.second_order(m, 3)
    want = so.second_order_dense(m.to_dense(), c.n_sites, 3)
    for key in want:
        assert abs(got[key] - want[key]) < 1e-11 * max(1.0, abs(want[key])), key
