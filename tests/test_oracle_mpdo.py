"""Pins for the oracle MPDO: exact dense equality without truncation, trace /
Hermiticity / positivity invariants with truncation, the QR identity of the bond
split, the canonical-gauge meaning of the Kraus Gram, observables and sampling."""
import dataclasses

import numpy as np
import pytest

import synth
from oracle import dense, mpdo, observables, ops, qaoa


def _run(c, plain=False, use_ppt=True, n_ops=None):
    m = mpdo.MPDO(c.n_sites, qaoa.plus_state(), c.chi_max, c.k_max, plain=plain,
                  use_ppt=use_ppt)
    d = dense.DenseRho(c.n_sites, qaoa.plus_state())
    opl = qaoa.circuit_ops(c)[:n_ops]
    for i, k in opl:
        m.apply_two_site(i, k)
        d.apply_two_site(i, k)
    return m, d


@pytest.mark.parametrize("plain", [True, False])
def test_untruncated_mpdo_equals_dense(plain):
    c = synth.tiny()
    m, d = _run(c, plain=plain)
    assert np.abs(m.to_dense() - d.matrix()).max() < 1e-12
    e1 = observables.expect_energy(m, c.J, c.hx, c.bz)
    e2 = d.expect(c.J, c.hx, c.bz)
    for k in e1:
        assert abs(e1[k] - e2[k]) < 1e-12 * max(1.0, abs(e2[k]))


def test_two_layers_snake_untruncated_equals_dense():
    c = dataclasses.replace(synth.tiny(), n_sites=3, p=2, alpha=[0.3, 1.1], beta=[0.7, 0.2],
                            xtalk_phase=0.05, delta_pp=0.05, gamma_diss=0.0, gamma_deph=0.05)
    m, d = _run(c)
    assert np.abs(m.to_dense() - d.matrix()).max() < 1e-12


def test_trace_one_without_dark_branch_and_monotone_with_it():
    base = dataclasses.replace(synth.tiny(), n_sites=5, delta_pp=0.2, gamma_diss=0.1,
                               chi_max=6, k_max=3)
    tp = dataclasses.replace(base, b0=0.5, b1=0.5, bd=0.0)
    m, _ = _run(tp)
    assert abs(observables.expect_energy(m, 1, 1, 0)["trace"] - 1.0) < 1e-12
    m = mpdo.MPDO(base.n_sites, qaoa.plus_state(), 729, 729)
    d = dense.DenseRho(base.n_sites, qaoa.plus_state())
    last = 1.0
    for i, k in qaoa.circuit_ops(base):
        m.apply_two_site(i, k)
        d.apply_two_site(i, k)
        tr = np.trace(m.to_dense()).real
        assert tr <= last + 1e-14
        assert abs(tr - np.trace(d.matrix()).real) < 1e-13
        last = tr
    assert last < 1.0 - 1e-6


@pytest.mark.parametrize("use_ppt", [True, False])
def test_truncated_state_is_hermitian_and_positive(use_ppt):
    c = dataclasses.replace(synth.tiny(), n_sites=5, p=2, alpha=[0.9, 0.4], beta=[0.3, 1.3],
                            gamma_diss=0.2, gamma_deph=0.2, delta_pp=0.3, chi_max=4, k_max=2)
    m, _ = _run(c, use_ppt=use_ppt)
    rho = m.to_dense()
    assert np.abs(rho - rho.conj().T).max() < 1e-14
    assert np.linalg.eigvalsh(rho).min() > -1e-12
    assert m.stats.disc_bond_w > 0 and m.stats.disc_kraus_w > 0


def test_plain_and_qr_reduced_split_agree_under_truncation():
    c = dataclasses.replace(synth.tiny(), n_sites=5, p=2, alpha=[0.9, 0.4], beta=[0.3, 1.3],
                            gamma_diss=0.05, gamma_deph=0.05, delta_pp=0.2, chi_max=5, k_max=3)
    m1, _ = _run(c, plain=True)
    m2, _ = _run(c, plain=False)
    assert np.abs(m1.to_dense() - m2.to_dense()).max() < 1e-11


def test_kraus_gram_is_reduced_density_of_the_ancilla():
    """In the mixed-canonical gauge the local Gram W of the centre's inner index equals
    the reduced density matrix of that ancilla computed from the full purification."""
    c = dataclasses.replace(synth.tiny(), n_sites=4, alpha=[0.8], beta=[0.5],
                            gamma_diss=0.1, gamma_deph=0.1, delta_pp=0.3, chi_max=64, k_max=64)
    m, _ = _run(c, n_ops=2)
    ctr = m.centre
    # full purification X[phys..., anc...]
    x = np.ones((1, 1, 1), dtype=complex)            # (phys, anc, r)
    anc_dims = []
    for a in m.A:
        x = np.einsum("pqb,bskr->psqkr", x, a)
        p, s, q, k, r = x.shape
        anc_dims.append(k)
        x = x.reshape(p * s, q * k, r)
    x = x[:, :, 0].reshape([3 ** m.n] + anc_dims)
    xc = np.moveaxis(x, 1 + ctr, 0).reshape(anc_dims[ctr], -1)
    red = xc @ xc.conj().T
    cm = m.A[ctr].transpose(2, 0, 1, 3).reshape(anc_dims[ctr], -1)
    assert np.abs(red - cm @ cm.conj().T).max() < 1e-13


def test_transfer_energies_match_dense_formula_on_truncated_state():
    c = dataclasses.replace(synth.tiny(), n_sites=5, p=2, alpha=[0.9, 0.4], beta=[0.3, 1.3],
                            gamma_diss=0.1, gamma_deph=0.1, delta_pp=0.2, chi_max=4, k_max=2)
    m, _ = _run(c)
    d = dense.DenseRho(c.n_sites, qaoa.plus_state())
    d.rho = m.to_dense().reshape((3,) * (2 * c.n_sites))
    e1 = observables.expect_energy(m, 1.0, 0.7, 0.3)
    e2 = d.expect(1.0, 0.7, 0.3)
    for k in e1:
        assert abs(e1[k] - e2[k]) < 1e-12 * max(1.0, abs(e2[k]))


def test_sampling_probabilities_and_frequencies():
    c = dataclasses.replace(synth.tiny(), n_sites=3, alpha=[0.8], beta=[0.5], delta_pp=0.4,
                            gamma_diss=0.3, gamma_deph=0.1)
    m, d = _run(c)
    diag = d.probs_diag()
    bits, probs = observables.sample(m, 4000, seed=99)
    idx = (bits.astype(int) * np.array([9, 3, 1])).sum(1)
    assert np.allclose(probs, diag[idx], rtol=1e-12, atol=1e-15)
    freq = np.bincount(idx, minlength=27) / len(idx)
    want = diag / diag.sum()
    # 4000 draws: every cell within 5 standard errors
    se = np.sqrt(want * (1 - want) / len(idx)) + 1e-12
    assert np.all(np.abs(freq - want) < 5 * se + 1e-3)
