"""Pins for the oracle's channels (G0 model): closed forms vs the Lindblad generator,
CPTP / trace-loss structure, and the ideal ZZ block (Eq. HZ_block_representation)."""
import numpy as np
import pytest
import scipy.linalg

from oracle import ops


@pytest.mark.parametrize("g,gp", [(0.01, 0.0), (0.0, 0.02), (0.3, 0.7), (1e-4, 1e-2)])
@pytest.mark.parametrize("bd", [7.0 / 8, 0.0])
def test_closed_form_noise_equals_lindblad_exponential(g, gp, bd):
    b0 = b1 = (1.0 - bd) / 2.0
    gen = ops.lindblad_generator(g, gp, b0, b1, bd)
    s_exact = scipy.linalg.expm(gen)
    s_closed = ops.g0_noise_superop(g, gp, b0, b1, bd)
    assert np.abs(s_exact - s_closed).max() < 1e-13


def test_noise_trace_structure():
    g, gp = 0.05, 0.02
    # no dark branch: trace preserving
    k = ops.kraus_from_superop(ops.g0_noise_superop(g, gp, 0.5, 0.5, 0.0))
    assert np.abs(sum(e.conj().T @ e for e in k) - np.eye(3)).max() < 1e-13
    # dark branch b_d: sum E^+E = I - b_d (1 - e^-g) |r><r|
    k = ops.kraus_from_superop(ops.g0_noise_superop(g, gp, 1 / 16, 1 / 16, 7 / 8))
    want = np.eye(3) - np.diag([0, 0, 7 / 8 * (1 - np.exp(-g))])
    assert np.abs(sum(e.conj().T @ e for e in k) - want).max() < 1e-13


def test_kraus_choi_roundtrip():
    rng = np.random.default_rng(0)
    ks = [rng.standard_normal((9, 9)) + 1j * rng.standard_normal((9, 9)) for _ in range(3)]
    k2 = ops.canonical_kraus(ks)
    assert len(k2) == 3
    assert np.abs(ops.superop(ks) - ops.superop(k2)).max() < 1e-12


def test_noiseless_block_is_zz_rotation_on_qubits():
    """On qubit pairs the block is exp(-i a Z Z).  A Rydberg atom is no CZ control
    (only |1> is), so with the left atom in |r> the two CNOTs cancel and the block is
    the bare exp(-i a Z) on the right atom; with the right atom in |r> it is identity."""
    a = 0.37
    u = ops.zz_block_unitary(a)
    want = np.ones(9, dtype=complex)
    for si in range(3):
        for sj in range(2):
            zj = 1 - 2 * sj
            zi = 1 - 2 * si if si < 2 else 1
            want[si * 3 + sj] = np.exp(-1j * a * zi * zj)
    assert np.abs(u - np.diag(want)).max() < 1e-14
    ks = ops.g0_block_channel(a, 0.0, 0.0, 0.0, 0.0, 1 / 16, 1 / 16, 7 / 8)
    assert len(ks) == 1
    assert np.abs(ops.superop(ks) - ops.superop([u])).max() < 1e-13


def test_post_promotion_closed_form():
    d = 0.2
    pp = ops.expm_h(d, np.outer(ops.I3[1], ops.I3[2]) + np.outer(ops.I3[2], ops.I3[1]))
    assert np.allclose(pp @ ops.I3[1], [0, np.cos(d), -1j * np.sin(d)], atol=1e-15)
    assert np.allclose(pp @ ops.I3[0], [1, 0, 0], atol=1e-15)


def test_block_channel_kraus_rank_and_trace_loss():
    g, gp = 0.01, 0.01
    ks = ops.g0_block_channel(0.3, g, gp, 0.01, 0.01, 1 / 16, 1 / 16, 7 / 8)
    s = sum(e.conj().T @ e for e in ks)
    # trace loss only from Rydberg population, bounded by the dark branch of both atoms
    loss_r = 7 / 8 * (1 - np.exp(-g))
    ev = np.linalg.eigvalsh(np.eye(9) - s)
    assert ev.min() > -1e-13 and ev.max() < 2 * loss_r + 1e-12
    # single-atom noise has Choi rank 5 (decay: no-jump + 2 jumps; dephasing adds 2
    # independent phase operators on the 3-level no-jump part), the block its square
    n1 = ops.kraus_from_superop(ops.g0_noise_superop(g, gp, 1 / 16, 1 / 16, 7 / 8))
    assert len(ks) == len(n1) ** 2
