"""Pins of the App. E split of Rydberg dissipation into a coherent and an incoherent part
(oracle.ops.app_e_phases / app_e_shift, oracle.qaoa.layer_ops_appe), and the library's
builder of the split layers against them.

App. E: a dissipative pulse damps the two-atom coherences by alpha = e^{-a gamma} and
beta = e^{-b gamma} (a = 0.012291, b = 0.0185454, tests/golden/gaussian_cz.txt), which act
on the Ising phase gate as the phases d1 = ((1 - alpha)/(1 + alpha))^2 on S^z_i + S^z_j and
d2 = ((alpha - beta)/(alpha + beta))^2 on S^z_i S^z_j."""
import dataclasses

import numpy as np
import pytest
import scipy.linalg

import synth
from golden_io import gaussian_cz
from oracle import ops, pulse, qaoa

GOLD = gaussian_cz()
B0, B1, BD = 1 / 16, 1 / 16, 7 / 8


@pytest.mark.parametrize("gamma", [0.0, 1e-3, 0.05, 1.0, 30.0])
def test_phases_are_half_angle_tangents_of_the_damping_rates(gamma):
    """(1 - e^-x)/(1 + e^-x) = tanh(x/2): d1 = tanh^2(a gamma / 2) and
    d2 = tanh^2((b - a) gamma / 2), with the rates read from the golden file.  Tolerance:
    1e-12 plus the FP64 cancellation in 1 - e^-x (relative 4 u / x, u = 2.2e-16, doubled by
    the square)."""
    a, b = GOLD["app_e_alpha_rate"], GOLD["app_e_beta_rate"]
    d1, d2 = ops.app_e_phases(gamma)
    for d, x in ((d1, a * gamma), (d2, (b - a) * gamma)):
        tol = 1e-12 + (8 * 2.2e-16 / x if x > 0 else 0.0)
        assert d == pytest.approx(np.tanh(x / 2) ** 2, rel=tol, abs=1e-300)


def test_phases_follow_from_the_pulse_oracles_own_damping():
    """The damping rates the pulse oracle measures on its Gaussian CZ (within 6% and 2% of
    App. E's printed ones) give phases within 20% of App. E's (d scales as a rate squared)."""
    g = 0.01
    s, _ = pulse.cz_superop(g, 0.0, B0, B1, BD, 2000)
    a_rate = -np.log(abs(s[1, 1])) / g                  # <00|rho|01>
    b_rate = -np.log(abs(s[4 * 9 + 4, 4 * 9 + 4])) / (2 * g)   # <11|rho|11> = |beta|^2
    gamma = 1.0
    d1, d2 = ops.app_e_phases(gamma)
    assert np.tanh(a_rate * gamma / 2) ** 2 == pytest.approx(d1, rel=0.2)
    assert np.tanh((b_rate - a_rate) * gamma / 2) ** 2 == pytest.approx(d2, rel=0.2)


def test_shift_is_the_exponential_of_its_generator():
    """app_e_shift against scipy's expm of the Pauli-Z generator (qubit levels, zero on
    |r>), and its diagonal phases on |00>, |01>, |11>, |0r>, |rr>."""
    a, d1, d2 = 0.7, 0.013, 0.004
    z = np.diag([1.0, -1.0, 0.0])
    gen = d2 * np.kron(z, z) + d1 * (np.kron(z, np.eye(3)) + np.kron(np.eye(3), z))
    u = ops.app_e_shift(a, d1, d2)
    assert np.abs(u - scipy.linalg.expm(-1j * a * gen)).max() < 1e-14
    ph = lambda x: np.exp(-1j * a * x)
    for (s, t), x in {(0, 0): d2 + 2 * d1, (0, 1): -d2, (1, 1): d2 - 2 * d1, (0, 2): d1,
                      (2, 2): 0.0}.items():
        assert u[3 * s + t, 3 * s + t] == pytest.approx(ph(x), abs=1e-15)


def test_coherent_part_is_unitary_and_the_parts_compose_to_the_block():
    """Part 0 without other noise is one unitary Kraus operator (trace kept); the
    incoherent part followed by the coherent shift is the full dissipative block."""
    a, gamma = 0.9, 0.2
    v = qaoa.site_gate(0.4, 0.9, 1.0, 0.2)
    d1, d2 = ops.app_e_phases(gamma)
    sh = ops.app_e_shift(a, d1, d2)
    k0 = ops.g0_block_channel(a, 0.0, 0.0, 0.0, 0.0, B0, B1, BD, shift=sh)
    assert len(k0) == 1
    assert np.abs(k0[0].conj().T @ k0[0] - np.eye(9)).max() < 1e-13
    k1 = ops.g0_block_channel(a, gamma, 0.0, 0.0, 0.0, B0, B1, BD, shift=sh.conj().T)
    full = ops.g0_block_channel(a, gamma, 0.0, 0.0, 0.0, B0, B1, BD)
    assert np.abs(ops.superop([sh]) @ ops.superop(k1) - ops.superop(full)).max() < 1e-13
    # with the folded single-site gates the shift sits between the block and them
    k1v = ops.g0_block_channel(a, gamma, 0.0, 0.0, 0.0, B0, B1, BD, post_left=v,
                               shift=sh.conj().T)
    fullv = ops.g0_block_channel(a, gamma, 0.0, 0.0, 0.0, B0, B1, BD, post_left=v)
    vv = ops.superop([np.kron(v, np.eye(3))])
    lhs = vv @ ops.superop([sh]) @ np.linalg.inv(vv) @ ops.superop(k1v)
    assert np.abs(lhs - ops.superop(fullv)).max() < 1e-12


def test_zero_dissipation_leaves_the_g0_layers():
    c = dataclasses.replace(synth.tiny(), gamma_diss=0.0)
    for part in (0, 1):
        for k in range(c.p):
            for (i, a), (j, b) in zip(qaoa.layer_ops_appe(c, k, part), qaoa.layer_ops(c, k)):
                assert i == j
                assert np.abs(ops.superop(a) - ops.superop(b)).max() < 1e-13


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_2309_08572_gb300 as lib
    return lib


@pytest.mark.parametrize("part", [0, 1])
def test_library_builder_matches_oracle(pkg, part):
    c = dataclasses.replace(synth.scaled(synth.chain40(), n_sites=6), gamma_diss=0.3)
    for k in range(c.p):
        lib = pkg.build_qaoa_layer(c.n_sites, k, c.alpha[k], c.beta[k], c.J, c.bz, c.gamma_diss,
                                   c.gamma_deph, c.xtalk_phase, c.delta_pp, appe_part=part)
        orc = qaoa.layer_ops_appe(c, k, part)
        assert [s for s, _ in lib] == [s for s, _ in orc]
        for (_, a), (_, b) in zip(lib, orc):
            assert np.abs(ops.superop(a) - ops.superop(b)).max() < 1e-13


def test_library_builder_rejects_bad_parts(pkg):
    with pytest.raises(pkg.MpdoError):
        pkg.build_qaoa_layer(4, 0, 0.1, 0.2, gamma_diss=0.1, appe_part=2)
    with pytest.raises(pkg.MpdoError):
        pkg.build_qaoa_layer(4, 0, 0.1, 0.2, gamma_diss=-0.1, appe_part=0)
