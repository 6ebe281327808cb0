"""Pins of the random-circuit workload in the oracle (oracle/rcs.py): the swept MPDO layers
reproduce the dense density matrix (untruncated), a noiseless circuit keeps tr rho = 1 and
no Rydberg population, and a deep noiseless brickwork on 6 qubits approaches the
Porter-Thomas collision probability 2/(2^N + 1) (Sec. III.E, Fig. 5b's anticoncentration);
decay lowers the trace and the purity."""
import dataclasses

import numpy as np

import synth
from oracle import dense as odense
from oracle import mpdo as ompdo
from oracle import observables as oobs
from oracle import rcs as orcs
from oracle import second_order as so


def _run(c, dense=True):
    m = ompdo.MPDO(c.n_sites, orcs.zero_state(), c.chi_max, c.k_max)
    d = odense.DenseRho(c.n_sites, orcs.zero_state()) if dense else None
    for i, k in orcs.circuit_ops(c):
        m.apply_two_site(i, k)
        if dense:
            d.apply_two_site(i, k)
    return m, d


def test_haar_inputs_are_unitary():
    c = synth.rcs(4, 3, 8, 4)
    for u in c.haar.reshape(-1, 2, 2):
        assert np.abs(u.conj().T @ u - np.eye(2)).max() < 1e-14


def test_untruncated_rcs_mpdo_equals_dense():
    c = dataclasses.replace(synth.rcs(4, 5, 81, 729, gamma_diss=0.05, delta_pp=0.1),
                            gamma_deph=0.02)
    m, d = _run(c)
    assert np.abs(m.to_dense() - d.matrix()).max() < 1e-12


def test_noiseless_rcs_stays_in_the_qubit_space_and_anticoncentrates():
    c = synth.rcs(6, 24, 729, 4, gamma_diss=0.0)
    m, _ = _run(c, dense=False)
    r = oobs.expect_energy(m, 1.0, 0.0, 0.0)
    assert abs(r["trace"] - 1.0) < 1e-12 and abs(r["p_succ"] - 1.0) < 1e-12
    z = so.second_order(m, 3)["collision"]
    pt = 2.0 / (2 ** 6 + 1)
    assert abs(z - pt) < 0.25 * pt, (z, pt)
    assert abs(so.second_order(m, 3)["xi"] - 1.0) < 1e-10


def test_decay_lowers_trace_and_purity():
    c = synth.rcs(4, 4, 81, 729, gamma_diss=0.2, delta_pp=0.3)
    m, d = _run(c)
    r = oobs.expect_energy(m, 1.0, 0.0, 0.0)
    assert r["trace"] < 1.0 - 1e-4
    assert abs(r["trace"] - np.trace(d.matrix()).real) < 1e-12
    assert so.second_order(m, 2)["xi"] < 1.0 - 1e-4
