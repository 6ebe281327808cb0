"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module holds workload *descriptions* and random draws only -- circuit sizes,
QAOA angles, noise rates, bond/Kraus limits -- and none of the method's arithmetic
(no channels, no tensors, no truncation).  Both sides build everything else from
these numbers with their own code.

The paper's workloads are synthetic (QAOA on a transverse-field Ising chain, Sec. IV;
Table I gives the only printed angles).  The shapes here follow the five workloads the
build is measured on:

  tiny      N=6,   p=1, exact MPDO (no truncation), decay 0.01, dephasing 0.01
  chain40   N=40,  p=2, chi=64,  K=8,  decay 0.005, dephasing 0.005, crosstalk 0.01 rad
  chain100  N=100, p=3, chi=256, K=16, same noise as chain40 (precision form)
  chain100deep  the same chain with p=8 layers (bond dimension reaches chi=256)
  rcs8 / rcs12  random circuits: a Haar-random one-qubit gate on every atom, then noisy CZs on
            alternating bonds (brickwork), per layer; 8 sites, depth 40, chi=32 (Fig. 5 a-c) and
            12 sites, depth 20, chi=64, K=4 (Fig. 4), Rydberg decay 0.001 per CZ, post-promotion
            0.01 rad
  batch512  512 circuits, N~U{20..100}, chi in {32,64,128}, K=8, p in {1,2},
            decay/dephasing log-uniform in [1e-4, 1e-2]
  surrogate MLP 4x256 trained on batch512-style samples

Angles alpha_k, beta_k are drawn uniform in [0, pi) from numpy's Philox generator
seeded with the workload seed.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

# Table I of the paper (Sec. IV): classically pre-optimised angles for a 10-site,
# 8-layer TFIM QAOA.  Kept here as plain inputs; tests/golden holds the cited copy.
TABLE_I_ALPHA = (0.11076513, 0.2771272, 0.36282021, 0.40618171,
                 0.43256044, 0.44492256, 0.42887337, 0.3225842)
TABLE_I_BETA = (0.75428624, 0.73016842, 0.7096901, 0.68739375,
                0.65733871, 0.60978220, 0.51570246, 0.19145101)


@dataclasses.dataclass
class Circuit:
    """One noisy QAOA circuit on a 1D chain of three-level atoms (|0>,|1>,|r>)."""
    n_sites: int
    p: int
    alpha: List[float]
    beta: List[float]
    gamma_diss: float = 0.0      # Rydberg decay rate per two-site block (units 1/T)
    gamma_deph: float = 0.0      # qubit dephasing rate per two-site block
    xtalk_phase: float = 0.0     # nearest-neighbour Rydberg crosstalk phase (rad)
    delta_pp: float = 0.0        # post-promotion angle (rad)
    b0: float = 1.0 / 16         # decay branching ratios (Fig. 1 caption)
    b1: float = 1.0 / 16
    bd: float = 7.0 / 8
    J: float = 1.0               # TFIM couplings for the energy and the layer angles
    hx: float = 1.0
    bz: float = 0.0
    chi_max: int = 64
    k_max: int = 8
    seed: int = 0


def _angles(rng: np.random.Generator, p: int):
    a = rng.uniform(0.0, math.pi, size=p)
    b = rng.uniform(0.0, math.pi, size=p)
    return [float(x) for x in a], [float(x) for x in b]


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(seed))


def tiny(seed: int = 1) -> Circuit:
    a, b = _angles(rng_for(seed), 1)
    return Circuit(n_sites=6, p=1, alpha=a, beta=b, gamma_diss=0.01, gamma_deph=0.01,
                   delta_pp=0.01, chi_max=729, k_max=729, seed=seed)


def chain40(seed: int = 2) -> Circuit:
    a, b = _angles(rng_for(seed), 2)
    return Circuit(n_sites=40, p=2, alpha=a, beta=b, gamma_diss=0.005, gamma_deph=0.005,
                   xtalk_phase=0.01, delta_pp=0.01, chi_max=64, k_max=8, seed=seed)


def chain100(seed: int = 3) -> Circuit:
    a, b = _angles(rng_for(seed), 3)
    return Circuit(n_sites=100, p=3, alpha=a, beta=b, gamma_diss=0.005, gamma_deph=0.005,
                   xtalk_phase=0.01, delta_pp=0.01, chi_max=256, k_max=16, seed=seed)


def chain100deep(seed: int = 3, p: int = 8) -> Circuit:
    """chain100 with more QAOA layers (angles drawn from the same seed): at the numerical
    floor of the cuts its bond dimension reaches the cap chi = 256, which three layers do not."""
    a, b = _angles(rng_for(seed), p)
    return Circuit(n_sites=100, p=p, alpha=a, beta=b, gamma_diss=0.005, gamma_deph=0.005,
                   xtalk_phase=0.01, delta_pp=0.01, chi_max=256, k_max=16, seed=seed)


def scaled(c: Circuit, n_sites: Optional[int] = None, chi_max: Optional[int] = None,
           k_max: Optional[int] = None, p: Optional[int] = None) -> Circuit:
    """Same noise model and angle draw, smaller sizes (for oracle-sized parity cases)."""
    d = dataclasses.replace(c)
    if n_sites is not None:
        d.n_sites = n_sites
    if chi_max is not None:
        d.chi_max = chi_max
    if k_max is not None:
        d.k_max = k_max
    if p is not None:
        d.p = p
        d.alpha = list(c.alpha[:p]) + list(c.alpha[:max(0, p - len(c.alpha))])
        d.beta = list(c.beta[:p]) + list(c.beta[:max(0, p - len(c.beta))])
    return d


def batch512(seed: int = 4, count: int = 512) -> List[Circuit]:
    rng = rng_for(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(20, 101))
        chi = int(rng.choice([32, 64, 128]))
        p = int(rng.integers(1, 3))
        gd = float(10.0 ** rng.uniform(-4.0, -2.0))
        gp = float(10.0 ** rng.uniform(-4.0, -2.0))
        a, b = _angles(rng, p)
        out.append(Circuit(n_sites=n, p=p, alpha=a, beta=b, gamma_diss=gd, gamma_deph=gp,
                           delta_pp=0.01, chi_max=chi, k_max=8, seed=seed * 100000 + i))
    return out


def random_site_tensors(seed: int, dims_left, d: int, kdims, dims_right):
    """Seeded complex Gaussian site tensors A[l][s][k][r] (no normalisation, no gauge)."""
    rng = rng_for(seed)
    out = []
    for dl, k, dr in zip(dims_left, kdims, dims_right):
        re = rng.standard_normal((dl, d, k, dr))
        im = rng.standard_normal((dl, d, k, dr))
        out.append(re + 1j * im)
    return out


def philox_key(seed: int):
    """The 64-bit sampling seed split into the two 32-bit Philox key words."""
    return (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)


def haar_u2(rng: np.random.Generator) -> np.ndarray:
    """A Haar-random 2 x 2 unitary: QR of a complex Gaussian matrix with the phases of R's
    diagonal moved into Q (Mezzadri, Notices AMS 54, 2007).  An input draw, like the angles."""
    z = (rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    return q * (d / np.abs(d))[None, :]


@dataclasses.dataclass
class RcsCircuit:
    """Random circuit on a chain of three-level atoms: per layer a Haar one-qubit gate on
    every atom (acting on the qubit levels, |r> untouched), then CZ channels on the bonds
    (i, i+1) with i = layer mod 2 (brickwork)."""
    n_sites: int
    depth: int
    haar: np.ndarray             # (depth, n_sites, 2, 2) complex
    gamma_diss: float = 0.001
    gamma_deph: float = 0.0
    xtalk_phase: float = 0.0
    delta_pp: float = 0.0
    b0: float = 1.0 / 16
    b1: float = 1.0 / 16
    bd: float = 7.0 / 8
    chi_max: int = 32
    k_max: int = 4
    seed: int = 0


def rcs(n_sites: int, depth: int, chi_max: int, k_max: int, gamma_diss: float = 0.001,
        seed: int = 5, delta_pp: float = 0.0) -> RcsCircuit:
    rng = rng_for(seed)
    haar = np.stack([np.stack([haar_u2(rng) for _ in range(n_sites)]) for _ in range(depth)])
    return RcsCircuit(n_sites=n_sites, depth=depth, haar=haar, gamma_diss=gamma_diss,
                      delta_pp=delta_pp, chi_max=chi_max, k_max=k_max, seed=seed)


def rcs8(seed: int = 5) -> RcsCircuit:
    # post-promotion 0.01 rad, as in the chain workloads: in the gate-level model decay acts
    # only on Rydberg population, which the ideal CZ alone never leaves behind
    return rcs(8, 40, 32, 4, seed=seed, delta_pp=0.01)


def rcs12(seed: int = 6) -> RcsCircuit:
    return rcs(12, 20, 64, 4, seed=seed, delta_pp=0.01)
