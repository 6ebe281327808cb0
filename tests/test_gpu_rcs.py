"""The random-circuit workload (Sec. IV, Figs. 4 and 5 a-c) on the GPU through the C ABI,
against the oracle on the same seeded Haar gates: 8 sites, depth 40, chi = 32, K = 4,
Rydberg decay 0.001 per CZ (Fig. 5 a-c's truncated run) -- nearest-neighbour S^z
correlations (from the TFIM energy with J = 1, h = 0), success probability, trace and the
collision probability (anticoncentration, Fig. 5b).  FP64: 1e-9 relative (the GPU's Gram
floor drops weights below 1e-15 that the oracle's SVD keeps); the mixed-tc form (FP32 sites,
tensor-core products, FP64-accurate Grams): 1e-5 relative (FP32 site rounding over 280
updates, with the chi = 32 cap binding).  An untruncated 5-site circuit is compared with the
dense density matrix (1e-9, the same floor argument)."""
import numpy as np
import pytest

import synth
from oracle import dense as odense
from oracle import mpdo as ompdo
from oracle import observables as oobs
from oracle import rcs as orcs
from oracle import second_order as so

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()
    import paper_2309_08572_gb300 as pkg
    return pkg


def _gpu(lib, c, prec, m_max, gram=False):
    g = lib.Mpdo(c.n_sites, c.chi_max, c.k_max, m_max=m_max, prec=prec, gram_fp64=gram,
                 init_vec=orcs.zero_state())
    for layer in lib.circuit_layers(c):
        g.apply_layer(layer)
    return g


@pytest.mark.parametrize("prec,gram,tol", [("fp64", False, 1e-9), ("tf32x3", True, 1e-5)])
def test_rcs8_matches_oracle(lib, prec, gram, tol):
    c = synth.rcs8()
    m = ompdo.MPDO(c.n_sites, orcs.zero_state(), c.chi_max, c.k_max)
    for i, k in orcs.circuit_ops(c):
        m.apply_two_site(i, k)
    r = oobs.expect_energy(m, 1.0, 0.0, 0.0)
    g = _gpu(lib, c, prec, m_max=25, gram=gram)
    e = g.expect_energy(1.0, 0.0, 0.0)
    print(prec, "rcs8 errors", {key: abs(e[key] - r[key]) / max(1e-2, abs(r[key])) for key in r})
    for key in r:
        assert abs(e[key] - r[key]) < tol * max(1e-2, abs(r[key])), (key, e[key], r[key])
    z = so.second_order(m, 4)["collision"]
    zg = g.second_order(4)["collision"]
    print(prec, "rcs8 ZZ per bond", -e["e_raw"] / (c.n_sites - 1), "collision", zg, z,
          "dims", g.dims()[0])
    assert abs(zg - z) < (1e-8 if prec == "fp64" else 1e-4) * z
    g.close()


def test_untruncated_rcs_matches_dense(lib):
    # 5 sites, 2 brickwork layers: the inner index needs at most 54 (oracle, exact), within
    # the handle's m_max * k_max <= 1024 with the CZ channel's 9 Kraus operators
    c = synth.rcs(5, 2, 243, 113, gamma_diss=0.05, delta_pp=0.1)
    d = odense.DenseRho(c.n_sites, orcs.zero_state())
    for i, k in orcs.circuit_ops(c):
        d.apply_two_site(i, k)
    g = _gpu(lib, c, "fp64", m_max=9)
    e = g.expect_energy(1.0, 0.0, 0.0)
    r = d.expect(1.0, 0.0, 0.0)
    for key in r:
        assert abs(e[key] - r[key]) < 1e-9 * max(1.0, abs(r[key])), key
    g.close()
