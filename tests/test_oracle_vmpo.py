"""Pins of the vectorized-MPO oracle (oracle/vmpo.py, Sec. III.A and III.D): untruncated it
equals the dense density matrix and the MPDO; a PPT truncation keeps tr rho and
xi = tr rho^2 / tr rho^2 of the whole state (the quantities Eqs. xiformula and ppt fix in the
canonical gauge), where the naive truncation changes both; the trace environment T is real
up to rounding and near-degeneracies."""
import dataclasses

import numpy as np

import synth
from oracle import dense as odense
from oracle import mpdo as ompdo
from oracle import observables as oobs
from oracle import qaoa as oqaoa
from oracle import vmpo as ovmpo


def test_untruncated_vmpo_equals_dense_and_mpdo():
    c = synth.tiny()
    v = ovmpo.VMPO(c.n_sites, oqaoa.plus_state(), 729)
    d = odense.DenseRho(c.n_sites, oqaoa.plus_state())
    m = ompdo.MPDO(c.n_sites, oqaoa.plus_state(), 729, 729)
    for i, k in oqaoa.circuit_ops(c):
        v.apply_two_site(i, k)
        d.apply_two_site(i, k)
        m.apply_two_site(i, k)
    assert np.abs(v.to_dense() - d.matrix()).max() < 1e-12
    ev, em = v.expect_energy(c.J, c.hx, c.bz), oobs.expect_energy(m, c.J, c.hx, c.bz)
    for key in em:
        assert abs(ev[key] - em[key]) < 1e-11 * max(1.0, abs(em[key])), key


def _trace_and_xi(v):
    tr = v.expect({}).real
    return tr, v.purity() / tr ** 2


def test_ppt_truncation_keeps_trace_and_purity_naive_does_not():
    c = synth.scaled(synth.chain40(), n_sites=8, chi_max=4, k_max=4)
    ops_ = oqaoa.circuit_ops(c)
    for mode in ("ppt", "naive"):
        big = ovmpo.VMPO(c.n_sites, oqaoa.plus_state(), 6561)
        small = ovmpo.VMPO(c.n_sites, oqaoa.plus_state(), 3, mode=mode)
        changed = 0.0
        for step, (i, k) in enumerate(ops_[:14]):
            # the untruncated update of the same state, then the truncated one
            ref = ovmpo.VMPO(c.n_sites, oqaoa.plus_state(), 6561)
            ref.A = [a.copy() for a in small.A]
            ref.centre = small.centre
            ref.apply_two_site(i, k)
            small.apply_two_site(i, k)
            t0, x0 = _trace_and_xi(ref)
            t1, x1 = _trace_and_xi(small)
            if mode == "ppt":
                assert abs(t1 - t0) < 1e-12 * abs(t0), (step, t0, t1)
                assert abs(x1 - x0) < 1e-10 * abs(x0), (step, x0, x1)
            else:
                changed = max(changed, abs(t1 - t0) / abs(t0))
        if mode == "naive":
            assert changed > 1e-6
        assert small.ppt_infeasible == 0 or mode == "naive"


def test_trace_environment_is_real():
    c = synth.scaled(synth.chain40(), n_sites=6, chi_max=5, k_max=4)
    v = ovmpo.VMPO(c.n_sites, oqaoa.plus_state(), 5)
    for i, k in oqaoa.circuit_ops(c):
        v.apply_two_site(i, k)
    # zero for non-degenerate Schmidt values (rho = rho^+ makes the vectorised state invariant
    # under the site-wise swap s <-> s' with conjugation); near-degenerate pairs at the cut
    # leave a small imaginary part, which the reading drops
    assert v.t_imag_max < 1e-5


def test_collision_probability_pins():
    """sum_x <x|rho|x>^2 / (tr rho)^2 of the vectorized MPO: the dense definition on the tiny
    circuit, the MPDO's two-copy diagonal contraction on the same circuit, and the product
    state |+>^N, whose diagonal is uniform over the 2^N qubit strings (collision 2^-N)."""
    c = synth.tiny()
    v = ovmpo.VMPO(c.n_sites, oqaoa.plus_state(), 729)
    d = odense.DenseRho(c.n_sites, oqaoa.plus_state())
    m = ompdo.MPDO(c.n_sites, oqaoa.plus_state(), 729, 729)
    assert abs(v.collision() - 0.5 ** c.n_sites) < 1e-15
    for i, k in oqaoa.circuit_ops(c):
        v.apply_two_site(i, k)
        d.apply_two_site(i, k)
        m.apply_two_site(i, k)
    rho = d.matrix()
    want = np.sum(np.real(np.diag(rho)) ** 2) / np.trace(rho).real ** 2
    assert abs(v.collision() - want) < 1e-13 * want
    from oracle import second_order as oso
    assert abs(oso.second_order(m, 3)["collision"] - v.collision()) < 1e-12 * want
