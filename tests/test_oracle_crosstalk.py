"""Pins of the crosstalk CZ oracle (oracle/crosstalk.py, Sec. III.B): the controlled
combination of pulse gates with shifted detunings that a Rydberg neighbour produces."""
import numpy as np
import pytest

from oracle import crosstalk as xt
from oracle import pulse

STEPS = 400
Q = [0, 1, 3, 4]                      # |00>, |01>, |10>, |11> of two atoms


def test_unshifted_pulse_is_the_g1_pulse():
    """Per-atom detunings with zero shifts reproduce the G1 oracle's pulse unitary."""
    assert np.abs(xt.pulse_unitary(0.0, 0.0, STEPS) - pulse.pulse_unitary(STEPS)).max() < 1e-13


def test_crosstalk_gate_is_unitary_and_reduces_without_neighbour_blockade():
    u = xt.crosstalk_cz(STEPS)
    assert np.abs(u.conj().T @ u - np.eye(81)).max() < 1e-12
    _, c = pulse.phase_correction(pulse.pulse_unitary(STEPS))
    g = np.kron(c, c) @ pulse.pulse_unitary(STEPS)
    want = np.kron(np.kron(np.eye(3), g), np.eye(3))
    assert np.abs(xt.crosstalk_cz(STEPS, b_x=0.0) - want).max() < 1e-13


def test_neighbours_without_rydberg_population_see_the_plain_gate():
    """|q> (x) psi (x) |q'> with q, q' qubit states: the neighbours are untouched and the
    active pair gets the corrected pulse gate."""
    u = xt.crosstalk_cz(STEPS)
    _, c = pulse.phase_correction(pulse.pulse_unitary(STEPS))
    g = np.kron(c, c) @ pulse.pulse_unitary(STEPS)
    rng = np.random.default_rng(3)
    psi = rng.standard_normal(9) + 1j * rng.standard_normal(9)
    for q in (0, 1):
        for q2 in (0, 1):
            e, e2 = np.eye(3)[q], np.eye(3)[q2]
            out = u @ np.kron(np.kron(e, psi), e2)
            assert np.abs(out - np.kron(np.kron(e, g @ psi), e2)).max() < 1e-12


def test_far_detuned_atom_is_the_one_next_to_the_rydberg_neighbour():
    """With the left neighbour in |r> and a neighbour blockade far above the drive, atom i is
    far detuned: it is not driven, keeps only its phase correction e^{-i phi_1} on |1>, and
    atom i+1's pulse phase is cancelled by its own correction.  The qubit block is then
    diag(1, 1, e^{-i phi_1}, e^{-i phi_1}) up to atom i's ac Stark phase
    int Omega^2 / (4 (Delta + B)) dt (adiabatic elimination), which bounds the difference;
    the mirror assignment (atom i+1 detuned) would give diag(1, e^{-i phi_1}, 1, ...)."""
    b = 2 * np.pi * 1e4
    p = pulse.GAUSSIAN
    phi1, _ = pulse.phase_correction(pulse.pulse_unitary(STEPS))
    u = xt.crosstalk_cz(STEPS, b_x=b).reshape([3] * 8)
    g = u[2, :, :, 0, 2, :, :, 0].reshape(9, 9)       # left neighbour |r>, right |0>
    blk = g[np.ix_(Q, Q)]
    want = np.diag([1, 1, np.exp(-1j * phi1), np.exp(-1j * phi1)])
    t = np.linspace(0.0, p["T"], 20001)
    om = np.array([pulse.omega(s, p["T"], p["omega_max"], p["width"]) for s in t])
    w2 = om ** 2
    stark = float(np.sum(0.5 * (w2[1:] + w2[:-1]) * np.diff(t))) / (4 * abs(p["delta"] + b))
    assert np.abs(blk - want).max() < 1.2 * stark
    wrong = np.diag([1, np.exp(-1j * phi1), 1, np.exp(-1j * phi1)])
    assert np.abs(blk - wrong).max() > 0.5


@pytest.mark.parametrize("n,i,sites", [(4, 0, [0, 1, 2]), (4, 1, [0, 1, 2, 3]),
                                       (4, 2, [1, 2, 3]), (2, 0, [0, 1])])
def test_chain_ends_drop_the_missing_neighbours(n, i, sites):
    s, u = xt.gate_on_chain(n, i, STEPS)
    assert s == sites
    assert np.abs(u.conj().T @ u - np.eye(u.shape[0])).max() < 1e-12
    if n == 2:
        _, c = pulse.phase_correction(pulse.pulse_unitary(STEPS))
        assert np.abs(u - np.kron(c, c) @ pulse.pulse_unitary(STEPS)).max() < 1e-13


def _sweep(n, v, b_x=None):
    from oracle import mpdo
    m = mpdo.MPDO(n, v, 3 ** n, 3 ** n)
    rho = np.ones((1, 1), dtype=complex)
    for _ in range(n):
        rho = np.kron(rho, np.outer(v, v.conj()))
    for i in range(n - 1):
        sites, u = xt.gate_on_chain(n, i, STEPS, b_x=b_x)
        xt.apply_mpdo(m, sites, u)
        rho = xt.apply_dense(rho, n, sites, u)
    return m, rho


def test_mpdo_sweep_of_crosstalk_gates_equals_the_dense_rho():
    """A left-to-right sweep of crosstalk CZs over a 5-site chain with Rydberg population on
    every atom: the oracle MPDO's multi-site update, untruncated, equals the dense rho; the
    neighbours' Rydberg populations enter (B = 0 gives a different state) and the gates
    leave the population of a non-active neighbour unchanged."""
    n = 5
    v = np.array([1.0, 1.0, 0.4], dtype=complex)
    v /= np.linalg.norm(v)
    m, rho = _sweep(n, v)
    assert np.abs(m.to_dense() - rho).max() < 1e-13
    _, rho0 = _sweep(n, v, b_x=0.0)
    assert np.abs(rho - rho0).max() > 1e-3
    # one gate on (1, 2): site 0 and site 3 are controls, their |r> population is kept
    sites, u = xt.gate_on_chain(n, 1, STEPS)
    nr = lambda s: np.kron(np.kron(np.eye(3 ** s), np.diag([0.0, 0.0, 1.0])),
                           np.eye(3 ** (n - s - 1)))
    after = xt.apply_dense(rho, n, sites, u)
    for s in (0, 3):
        assert abs(np.trace(nr(s) @ after) - np.trace(nr(s) @ rho)) < 1e-13


@pytest.mark.parametrize("b_x", [None, 0.0, 2 * np.pi * 1e3])
def test_library_builder_matches_oracle(b_x):
    """mpdo_build_crosstalk_cz (host C++) against the oracle, gate by gate.  Bound: the two
    sides exponentiate each of the n steps independently, so their phases differ by rounding
    of order n eps tau |H| (tau |H| up to ~37 rad at the largest shift): 10 n eps max(1, tau |H|)."""
    import __graft_entry__ as g
    g.build()
    import paper_2309_08572_gb300 as lib
    p = pulse.GAUSSIAN
    a = lib.build_crosstalk_cz(b_x=b_x, n_steps=STEPS)
    b = xt.crosstalk_cz(STEPS, b_x=b_x)
    bx = p["blockade"] if b_x is None else b_x
    th = p["T"] / STEPS * (abs(p["delta"]) + abs(bx) + p["blockade"] + p["omega_max"])
    assert np.abs(a - b).max() < 10 * STEPS * 2.2e-16 * max(1.0, th)
