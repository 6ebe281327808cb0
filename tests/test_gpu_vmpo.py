"""The vectorized-MPO engine (Sec. III.A, with PPT on the bond, Sec. III.D) through the C ABI
against the oracle (oracle/vmpo.py, pinned to the dense rho and to PPT's kept trace and
purity): untruncated on 4 sites (= dense rho), and truncated chains in both truncation modes
(naive and PPT) -- energies, success probability, trace, purity and the bond dimensions.
FP64 throughout: 1e-9 relative (the GPU's Gram floor, Schmidt values below sqrt(1e-15) of the
largest, drops what the oracle's SVD keeps above its 1e-7 cut only at the 1e-15 level)."""
import numpy as np
import pytest

import synth
from oracle import dense as odense
from oracle import qaoa as oqaoa
from oracle import vmpo as ovmpo

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


def _run(lib, c, chi, ppt, sv=1e-7):
    ref = ovmpo.VMPO(c.n_sites, oqaoa.plus_state(), chi, mode="ppt" if ppt else "naive",
                     sv_cutoff=sv)
    for i, k in oqaoa.circuit_ops(c):
        ref.apply_two_site(i, k)
    g = lib.Vmpo(c.n_sites, chi, ppt=ppt, sv_cutoff=sv)
    stats = [g.apply_layer(layer) for layer in lib.circuit_layers(c)]
    return ref, g, stats


def test_untruncated_vmpo_matches_dense(lib):
    c = synth.scaled(synth.tiny(), n_sites=4)
    d = odense.DenseRho(c.n_sites, oqaoa.plus_state())
    for i, k in oqaoa.circuit_ops(c):
        d.apply_two_site(i, k)
    _, g, _ = _run(lib, c, 81, True)
    e = g.expect_energy(c.J, c.hx, c.bz)
    r = d.expect(c.J, c.hx, c.bz)
    for key in r:
        assert abs(e[key] - r[key]) < 1e-10 * max(1.0, abs(r[key])), key
    assert abs(g.purity() - np.sum(np.abs(d.matrix()) ** 2)) < 1e-10
    g.close()


@pytest.mark.parametrize("ppt", [True, False])
@pytest.mark.parametrize("n,chi", [(8, 6), (10, 12)])
def test_truncated_vmpo_matches_oracle(lib, ppt, n, chi):
    c = synth.scaled(synth.chain40(), n_sites=n, chi_max=chi, k_max=4)
    ref, g, stats = _run(lib, c, chi, ppt)
    e = g.expect_energy(c.J, c.hx, c.bz)
    r = ref.expect_energy(c.J, c.hx, c.bz)
    print("vmpo", "ppt" if ppt else "naive", n, chi, {k: (e[k], r[k]) for k in r},
          "purity", g.purity(), ref.purity())
    for key in r:
        assert abs(e[key] - r[key]) < 1e-9 * max(1.0, abs(r[key])), (key, e[key], r[key])
    assert abs(g.purity() - ref.purity()) < 1e-9 * ref.purity()
    b, centre = g.dims()
    assert list(b) == [a.shape[2] for a in ref.A[:-1]] and centre == ref.centre
    assert max(s["chi_used_max"] for s in stats) <= chi
    g.close()


@pytest.mark.parametrize("ppt", [True, False])
def test_vmpo_collision_matches_oracle(lib, ppt):
    """The collision probability sum_x <x|rho|x>^2 / (tr rho)^2 through the C ABI: the dense
    definition on the untruncated 4-site chain, the oracle's vectorized MPO on a truncated
    8-site chain (1e-9 relative, FP64)."""
    c = synth.scaled(synth.tiny(), n_sites=4)
    d = odense.DenseRho(c.n_sites, oqaoa.plus_state())
    for i, k in oqaoa.circuit_ops(c):
        d.apply_two_site(i, k)
    rho = d.matrix()
    want = np.sum(np.real(np.diag(rho)) ** 2) / np.trace(rho).real ** 2
    _, g, _ = _run(lib, c, 81, ppt)
    assert abs(g.collision() - want) < 1e-10 * want
    g.close()
    c = synth.scaled(synth.chain40(), n_sites=8, chi_max=6, k_max=4)
    ref, g, _ = _run(lib, c, 6, ppt)
    assert abs(g.collision() - ref.collision()) < 1e-9 * ref.collision()
    g.close()


@pytest.mark.parametrize("ppt", [True, False])
def test_vmpo_tensor_core_form_matches_oracle(lib, ppt):
    """The tensor-core form of the vMPO (exact-slice FP64-accurate products, mixed-precision
    eigensolver) on the random-circuit workload with gamma_diss = 0.1 (8 sites, depth 12,
    chi = 24, bond cut s > 1e-5 s_max), against the oracle: energies, trace, purity and
    collision probability.

    Bound from the conditioning of the truncations: the form's products perturb the bond
    Gram by ~eps |H| with eps = 2^-48 sqrt(9 chi), which turns the kept Schmidt subspace by
    eps / gap, gap the smallest (Lambda_chi-1^2 - Lambda_chi^2) / Lambda_0^2 the oracle met
    at its cuts (1.9e-7 here); outputs move by at most 10 eps / gap (floor 1e-9)."""
    from oracle import rcs as orcs
    cut = 1e-5
    c = synth.rcs(8, 12, 24, 1, gamma_diss=0.1, seed=5, delta_pp=0.01)
    ref = ovmpo.VMPO(c.n_sites, orcs.zero_state(), c.chi_max, mode="ppt" if ppt else "naive",
                     sv_cutoff=cut)
    for i, k in orcs.circuit_ops(c):
        ref.apply_two_site(i, k)
    eps = 2.0 ** -48 * np.sqrt(9 * c.chi_max)
    tol = max(1e-9, 10 * eps / ref.cut_gap_min)
    g = lib.Vmpo(c.n_sites, c.chi_max, ppt=ppt, sv_cutoff=cut, init_vec=[1, 0, 0], tc=True)
    stats = [g.apply_layer(layer) for layer in lib.circuit_layers(c)]
    e = g.expect_energy(1.0, 1.0, 0.0)
    r = ref.expect_energy(1.0, 1.0, 0.0)
    print("vmpo tc", "ppt" if ppt else "naive", "gap", ref.cut_gap_min, "tol", tol,
          {k: abs(e[k] - r[k]) for k in r})
    for key in r:
        assert abs(e[key] - r[key]) < tol * max(1.0, abs(r[key])), (key, e[key], r[key])
    assert abs(g.purity() - ref.purity()) < tol * ref.purity()
    assert abs(g.collision() - ref.collision()) < tol * ref.collision()
    b, _ = g.dims()
    assert list(b) == [a.shape[2] for a in ref.A[:-1]]
    assert max(s["chi_used_max"] for s in stats) == c.chi_max
    g.close()
