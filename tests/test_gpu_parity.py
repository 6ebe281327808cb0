"""GPU parity through the C ABI against the CPU oracle, on the same seeded workloads.

Gauge-invariant outputs are compared (the split is unique only up to unitaries on the
bond and inner indices): energies, success probability, trace, sampled configurations
and their probabilities, and the dense rho on tiny chains.  FP64 mode: 1e-10 relative on
energies.  C64 mode (FP32 arithmetic, FP64 scalars): 5e-5 relative -- the FP32 Gram
eigenvalues resolve weights only down to ~10 eps_32 = 6e-7 of the largest, so each update
drops that much weight at most per mode (measured 2e-6 .. 4e-5 on these cases).

Cases whose truncation cuts through a near-degenerate part of the spectrum are
ill-conditioned (the kept subspace is then not unique); the truncated cases here keep
the relative gap at the inner-index cut above ~1e-6.

The GPU path forms Gram matrices, whose eigenvalues resolve only down to ~eps * max; it
therefore drops bond/inner values with lambda = s^2 below 1e-15 lambda_max (FP64) or
6e-7 lambda_max (FP32), where the oracle's SVD keeps s > 1e-14 s_max.  Kept dimensions
can thus be smaller on the GPU when the spectrum has values between the two floors;
what is dropped carries a weight below the floor, i.e. amplitude below 3.2e-8 of the
largest (FP64), which bounds the probability of a configuration with p >= 1e-3 to a
relative change below 2 * 3.2e-8 / sqrt(1e-3) ~ 2e-6.
"""
import dataclasses

import numpy as np
import pytest

import synth
from oracle import dense as odense
from oracle import mpdo as ompdo
from oracle import observables as oobs
from oracle import qaoa as oqaoa

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = {"fp64": 1e-10, "c64": 5e-5}


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()
    import paper_2309_08572_gb300 as pkg
    return pkg


def _oracle(c, sv_cutoff=1e-14):
    m = ompdo.MPDO(c.n_sites, oqaoa.plus_state(), c.chi_max, c.k_max, sv_cutoff=sv_cutoff)
    for i, k in oqaoa.circuit_ops(c):
        m.apply_two_site(i, k)
    return m, oobs.expect_energy(m, c.J, c.hx, c.bz)


def _gpu(lib, c, prec, m_max=25, **kw):
    g = lib.Mpdo(c.n_sites, c.chi_max, c.k_max, m_max=m_max, prec=prec, **kw)
    stats = [g.apply_layer(layer) for layer in lib.circuit_layers(c)]
    return g, g.expect_energy(c.J, c.hx, c.bz), stats


def _rel(a, b):
    return abs(a - b) / max(1.0, abs(b))


def _dense(g):
    """rho of a GPU handle as a d^N x d^N matrix, reassembled on the host from the site
    tensors the library returns (tiny chains only; test helper)."""
    x = np.ones((1, 1, 1, 1), dtype=complex)
    for n in range(g.n):
        a = g.site(n)
        x = np.einsum("pqab,askr,btkc->psqtrc", x, a, a.conj(), optimize=True)
        p, s, q, t, r, c = x.shape
        x = x.reshape(p * s, q * t, r, c)
    return x[:, :, 0, 0]


@pytest.mark.parametrize("prec", ["fp64", "c64"])
def test_tiny_exact_matches_dense(lib, prec):
    c = dataclasses.replace(synth.tiny(), k_max=40)
    g, e, _ = _gpu(lib, c, prec)
    d = odense.DenseRho(c.n_sites, oqaoa.plus_state())
    for i, k in oqaoa.circuit_ops(c):
        d.apply_two_site(i, k)
    r = d.expect(c.J, c.hx, c.bz)
    for key in r:
        assert _rel(e[key], r[key]) < TOL[prec], (key, e[key], r[key])
    rho = _dense(g)
    assert np.abs(rho - d.matrix()).max() < (1e-11 if prec == "fp64" else 5e-5)


@pytest.mark.parametrize("part", [0, 1])
def test_appe_parts_match_dense(lib, part):
    """The tiny circuit with the App. E split of its dissipation (part 0: coherent phases
    only; part 1: dissipation with those phases reversed), library-built layers through the
    engine in FP64, against the dense rho of the oracle's split layers: energies and
    probabilities at the FP64 tolerance, rho to 1e-11 (as the unsplit tiny circuit)."""
    c = dataclasses.replace(synth.tiny(), k_max=40, gamma_diss=0.2)
    g = lib.Mpdo(c.n_sites, c.chi_max, c.k_max, m_max=25, prec="fp64")
    for layer in lib.circuit_layers(c, appe_part=part):
        g.apply_layer(layer)
    e = g.expect_energy(c.J, c.hx, c.bz)
    d = odense.DenseRho(c.n_sites, oqaoa.plus_state())
    for i, k in oqaoa.circuit_ops(c, appe_part=part):
        d.apply_two_site(i, k)
    r = d.expect(c.J, c.hx, c.bz)
    for key in r:
        assert _rel(e[key], r[key]) < TOL["fp64"], (key, e[key], r[key])
    assert np.abs(_dense(g) - d.matrix()).max() < 1e-11
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "c64"])
@pytest.mark.parametrize("n,chi,k", [(8, 6, 3), (12, 16, 4), (9, 64, 8)])
def test_truncated_snake_circuit_matches_oracle(lib, prec, n, chi, k):
    c = synth.scaled(synth.chain40(), n_sites=n, chi_max=chi, k_max=k)
    ref, r = _oracle(c)
    g, e, stats = _gpu(lib, c, prec)
    for key in r:
        assert _rel(e[key], r[key]) < TOL[prec], (key, e[key], r[key])
    b, kd, centre = g.dims()
    assert centre == ref.centre
    # the GPU's numerical floor is higher than the oracle's: never more kept, caps hold
    assert all(x <= a.shape[2] for x, a in zip(kd, ref.A)) and max(kd) <= c.k_max
    assert all(x <= a.shape[3] for x, a in zip(b, ref.A[:-1])) and max(b) <= c.chi_max
    print(prec, n, chi, k, {key: _rel(e[key], r[key]) for key in r})


# Mixed precision (FP32 site tensors, FP64 Grams, eigenpairs, factors and observables) at
# the bond cut s > 1e-4 s_max, against the oracle at the same cut: energies within 1e-6;
# trace and success probability within 1e-5 (the isometric sites are stored in FP32, so
# the norm carries ~1e-8 of rounding per update; measured 2e-6 on chain40).
MIXED_TOL = {"e_succ": 1e-6, "e_raw": 1e-6, "p_succ": 1e-5, "trace": 1e-5}


@pytest.mark.parametrize("case", ["n12c16k4", "n9c64k8", "chain40"])
def test_mixed_precision_matches_oracle(lib, case):
    if case == "chain40":
        c = synth.chain40()
    else:
        n, chi, k = {"n12c16k4": (12, 16, 4), "n9c64k8": (9, 64, 8)}[case]
        c = synth.scaled(synth.chain40(), n_sites=n, chi_max=chi, k_max=k)
    _, r = _oracle(c, sv_cutoff=1e-4)
    g, e, _ = _gpu(lib, c, "c64", gram_fp64=True, sv_cutoff=1e-4)
    errs = {key: _rel(e[key], r[key]) for key in r}
    print("mixed", case, errs)
    for key in r:
        assert errs[key] < MIXED_TOL[key], (key, e[key], r[key])


def test_chain40_full_fp64(lib):
    c = synth.chain40()
    ref, r = _oracle(c)
    g, e, _ = _gpu(lib, c, "fp64")
    for key in r:
        assert _rel(e[key], r[key]) < TOL["fp64"], (key, e[key], r[key])


def test_sampling_matches_oracle_fp64(lib):
    c = synth.scaled(synth.chain40(), n_sites=7, chi_max=12, k_max=4)
    ref, _ = _oracle(c)
    g, _, _ = _gpu(lib, c, "fp64")
    bits, probs = g.sample_probs(200, seed=1234)
    rbits, rprobs = oobs.sample(ref, 200, seed=1234)
    same = np.all(bits == rbits, axis=1)
    assert same.mean() > 0.99
    rel = np.abs(probs[same] - rprobs[same]) / rprobs[same]
    print("sampling: identical configurations", same.mean(), "max rel prob error", rel.max())
    assert rel.max() < 2e-6


def test_truncate_entry_point(lib):
    c = synth.scaled(synth.chain40(), n_sites=8, chi_max=16, k_max=6)
    g, e0, _ = _gpu(lib, c, "fp64")
    ref, _ = _oracle(c)
    st = g.truncate(4, 2, True)
    ref.truncate(4, 2, True)
    e = g.expect_energy(c.J, c.hx, c.bz)
    r = oobs.expect_energy(ref, c.J, c.hx, c.bz)
    for key in r:
        assert _rel(e[key], r[key]) < 1e-9, (key, e[key], r[key])
    b, kd, centre = g.dims()
    assert max(b) <= 4 and max(kd) <= 2 and centre == 0


def test_errors_are_reported(lib):
    g = lib.Mpdo(4, 8, 4, m_max=25)
    k = lib.build_block_channel(0.3, 0.01, 0.01)
    with pytest.raises(lib.MpdoError) as ex:
        g.apply_layer([(2, k)])            # centre is at 0
    assert ex.value.code == -6
    bad = k.copy()
    bad[0, 0, 0] = np.nan
    with pytest.raises(lib.MpdoError) as ex:
        g.apply_layer([(0, bad)])
    assert ex.value.code == -4
    with pytest.raises(lib.MpdoError):
        lib.Mpdo(1, 8, 4)


def test_batch_executor_matches_oracle_fp64(lib):
    """Batched form: circuits of different sizes and angles run concurrently on a pool of
    handles (own streams); each must equal its own oracle run."""
    base = synth.chain40()
    circs = []
    for j, n in enumerate([6, 9, 7, 10, 8]):
        a, b = synth._angles(synth.rng_for(500 + j), 2)
        c = synth.scaled(base, n_sites=n, chi_max=64, k_max=4)
        c.alpha, c.beta = a, b
        circs.append(c)
    pool = [lib.Mpdo(10, 64, 4, m_max=25, prec="fp64", own_stream=True) for _ in range(3)]
    descs = []
    for c in circs:
        dls = [pool[0].upload_layer(layer) for layer in lib.circuit_layers(c)]
        descs.append(dict(n_sites=c.n_sites, chi_max=c.chi_max, k_max=c.k_max, layers=dls,
                          J=c.J, hx=c.hx, b=c.bz))
    out = lib.batch_run(pool, descs)
    out2 = lib.batch_run(pool[:1], descs)            # same circuits, one at a time
    assert np.array_equal(out, out2)
    # The left factor comes from the eigenvectors of the Gram G_i, whose small-sigma
    # directions carry errors ~ eps sigma_max / sigma; through sigma^-1/2 they reach the new
    # tensors as ~ eps / sqrt(sigma_min / sigma_max) ~ 1e-16 / 3e-7 for the 1e-13 modes
    # these short chains keep: 3e-10 (measured 4.8e-10 on the 6-site circuit, 1e-11 on the
    # others), hence 1e-9 here.
    for c, row in zip(circs, out):
        _, r = _oracle(c)
        for j, key in enumerate(("e_raw", "e_succ", "p_succ", "trace")):
            assert _rel(row[j], r[key]) < 1e-9, (c.n_sites, key, row[j], r[key])
    for m in pool:
        m.close()


def test_batch_executor_mixed_repeatable(lib):
    """Mixed precision through the executor: a pool reused for a second batch, and the
    same circuits one at a time, give identical results (no state carried between
    circuits on a handle), within the mixed tolerances of the oracle."""
    base = synth.chain40()
    circs = []
    for j, n in enumerate([8, 11, 9, 12, 10, 7]):
        a, b = synth._angles(synth.rng_for(700 + j), 2)
        c = synth.scaled(base, n_sites=n, chi_max=32, k_max=6)
        c.alpha, c.beta = a, b
        circs.append(c)
    pool = [lib.Mpdo(12, 32, 6, m_max=25, prec="c64", gram_fp64=True, sv_cutoff=1e-4,
                     own_stream=True) for _ in range(3)]
    descs = []
    for c in circs:
        dls = [pool[0].upload_layer(layer) for layer in lib.circuit_layers(c)]
        descs.append(dict(n_sites=c.n_sites, chi_max=c.chi_max, k_max=c.k_max, layers=dls,
                          J=c.J, hx=c.hx, b=c.bz))
    out = lib.batch_run(pool, descs)
    out2 = lib.batch_run(pool, descs[::-1])[::-1]
    out3 = lib.batch_run(pool[:1], descs)
    assert np.array_equal(out, out2) and np.array_equal(out, out3)
    # the host-layer executor uploads the same ops on each worker's stream: same results
    hosts = [lib.HostCircuit(c.n_sites, c.chi_max, c.k_max, lib.circuit_layers(c), J=c.J,
                             hx=c.hx, b=c.bz) for c in circs]
    assert np.array_equal(out, lib.batch_run_host(pool, hosts))
    for c, row in zip(circs[:2], out[:2]):
        _, r = _oracle(c, sv_cutoff=1e-4)
        for j, key in enumerate(("e_raw", "e_succ", "p_succ", "trace")):
            assert _rel(row[j], r[key]) < MIXED_TOL[key], (c.n_sites, key, row[j], r[key])
    for m in pool:
        m.close()


def test_batch512_sample_through_executor(lib):
    """The batched workload (512 circuits, N ~ U{20..100}, chi in {32,64,128}, K=8,
    p in {1,2}, log-uniform rates): 24 of its circuits run concurrently in complex64 on a
    pool sized for the largest; the two shortest single-layer ones are checked against the
    oracle, the rest for finite physical outputs (0 < p_succ <= trace <= 1)."""
    circs = synth.batch512()[:24]
    m_max = 25
    pool = [lib.Mpdo(100, 128, 8, m_max=m_max, prec="c64", own_stream=True) for _ in range(8)]
    descs = []
    for c in circs:
        dls = [pool[0].upload_layer(layer) for layer in lib.circuit_layers(c)]
        descs.append(dict(n_sites=c.n_sites, chi_max=c.chi_max, k_max=c.k_max, layers=dls,
                          J=c.J, hx=c.hx, b=c.bz))
    out = lib.batch_run(pool, descs)
    assert np.all(np.isfinite(out))
    # complex64: tr(rho) carries the FP32 rounding of ~1e2 renormalisations (~1e-4)
    assert np.all(out[:, 2] > 0) and np.all(out[:, 2] <= out[:, 3] + 1e-6)
    assert np.all(out[:, 3] <= 1 + 2e-4)
    order = sorted(range(len(circs)), key=lambda i: (circs[i].p, circs[i].n_sites))[:2]
    for i in order:
        _, r = _oracle(circs[i])
        for j, key in enumerate(("e_raw", "e_succ", "p_succ", "trace")):
            assert _rel(out[i][j], r[key]) < TOL["c64"], (i, key, out[i][j], r[key])
    for m in pool:
        m.close()


def _g1_run(lib, c, s_lib, s_or, prec, sv_cutoff=0.0, **kw):
    g = lib.Mpdo(c.n_sites, c.chi_max, c.k_max, m_max=63, prec=prec, sv_cutoff=sv_cutoff, **kw)
    for k in range(c.p):
        g.apply_layer(lib.build_qaoa_layer_cz(c.n_sites, k, c.alpha[k], c.beta[k], s_lib, c.J,
                                              c.bz, c.xtalk_phase))
    e = g.expect_energy(c.J, c.hx, c.bz)
    g.close()
    m = ompdo.MPDO(c.n_sites, oqaoa.plus_state(), c.chi_max, c.k_max,
                   sv_cutoff=sv_cutoff if sv_cutoff > 0 else 1e-14)
    for i, kr in oqaoa.circuit_ops(c, s_or):
        m.apply_two_site(i, kr)
    return e, oobs.expect_energy(m, c.J, c.hx, c.bz)


def test_g1_pulse_circuit_mixed_precision(lib):
    """Gate model G1 in the mixed precision form (FP32 site tensors, FP64 Grams) at the bond
    cut 1e-4, against the FP64 oracle at the same cut: within the mixed form's bounds."""
    from oracle import pulse as opulse
    c = synth.scaled(synth.chain40(), n_sites=7, chi_max=64, k_max=16)
    s_lib, _, _ = lib.build_cz_pulse(c.gamma_diss, c.gamma_deph, c.b0, c.b1, n_steps=300)
    s_or, _ = opulse.cz_superop(c.gamma_diss, c.gamma_deph, c.b0, c.b1, c.bd, 300)
    e, r = _g1_run(lib, c, s_lib, s_or, "c64", sv_cutoff=1e-4, gram_fp64=True)
    for key in r:
        assert _rel(e[key], r[key]) < MIXED_TOL[key], (key, e[key], r[key])


def test_g1_pulse_circuit_matches_oracle(lib):
    """Gate model G1: blocks built from the pulse-level CZ (63 Kraus operators each) by the
    library's host builder, run through the CUDA path in FP64, against the oracle MPDO on the
    oracle's own G1 ops (its pulse integration and block composition); the inner index is
    cut at K = 16 with PPT on both sides (swapping the two op sets moves the oracle's
    energies by 4e-13, so the cut is well conditioned)."""
    from oracle import pulse as opulse
    c = synth.scaled(synth.chain40(), n_sites=7, chi_max=64, k_max=16)
    s_lib, _, _ = lib.build_cz_pulse(c.gamma_diss, c.gamma_deph, c.b0, c.b1, n_steps=300)
    s_or, _ = opulse.cz_superop(c.gamma_diss, c.gamma_deph, c.b0, c.b1, c.bd, 300)
    g = lib.Mpdo(c.n_sites, c.chi_max, c.k_max, m_max=63, prec="fp64")
    for k in range(c.p):
        g.apply_layer(lib.build_qaoa_layer_cz(c.n_sites, k, c.alpha[k], c.beta[k], s_lib, c.J,
                                              c.bz, c.xtalk_phase))
    e = g.expect_energy(c.J, c.hx, c.bz)
    g.close()
    m = ompdo.MPDO(c.n_sites, oqaoa.plus_state(), c.chi_max, c.k_max)
    for i, kr in oqaoa.circuit_ops(c, s_or):
        m.apply_two_site(i, kr)
    r = oobs.expect_energy(m, c.J, c.hx, c.bz)
    for key in r:
        assert _rel(e[key], r[key]) < 1e-9, (key, e[key], r[key])


# Tensor-core modes.  Every complex64 product of the update (and of sampling) runs on the
# tcgen05 path here (MPDO_TC_MIN_MACS=0 routes even the smallest), checked against the
# oracle at the same bond cut, chosen above each mode's numerical floor (10 x the relative
# error of one split product: 2.4e-6 for TF32x3, 1.5e-4 for BF16x3, in lambda = s^2) so the
# cut, not the floor, decides what is kept.  Bounds: one product of relative error e per
# update and output, accumulated over the ~100 updates of these circuits: ~100 e for the
# FP32-Gram forms (TF32x3: 2.4e-7 -> 1e-4 with headroom for the FP32 site rounding; BF16x3:
# 1.5e-5 -> 2e-3); with FP64 Grams (gram_fp64) only the centre tensor and the inner
# isometry carry the split products, as FP32 products do in the mixed form (MIXED_TOL x 4).
TC_CASES = {
    ("tf32x3", False): (3e-3, {"e_succ": 1e-4, "e_raw": 1e-4, "p_succ": 1e-4, "trace": 1e-4}),
    ("bf16x3", False): (2e-2, {"e_succ": 2e-3, "e_raw": 2e-3, "p_succ": 2e-3, "trace": 2e-3}),
    ("tf32x3", True): (1e-4, {k: 4 * v for k, v in MIXED_TOL.items()}),
    ("bf16x3", True): (1e-4, {"e_succ": 1e-4, "e_raw": 1e-4, "p_succ": 1e-4, "trace": 1e-4}),
}


@pytest.mark.parametrize("prec,gram", list(TC_CASES))
@pytest.mark.parametrize("case", ["n12c16k4", "chain40"])
def test_tensor_core_modes_match_oracle(lib, monkeypatch, prec, gram, case):
    monkeypatch.setenv("MPDO_TC_MIN_MACS", "0")
    sv, tol = TC_CASES[(prec, gram)]
    if case == "chain40":
        c = synth.chain40()
    else:
        c = synth.scaled(synth.chain40(), n_sites=12, chi_max=16, k_max=4)
    _, r = _oracle(c, sv_cutoff=sv)
    n0 = lib.tc_gemm_launches()
    g, e, _ = _gpu(lib, c, prec, gram_fp64=gram, sv_cutoff=sv)
    used = lib.tc_gemm_launches() - n0
    errs = {key: _rel(e[key], r[key]) for key in r}
    print(prec, "gram_fp64" if gram else "", case, used, errs)
    assert used > 0
    for key in r:
        assert errs[key] < tol[key], (key, e[key], r[key])
    g.close()


# The headline workload, chain100 (N = 100, p = 3, chi = 256, K = 16), in the mixed form at
# reading A4's bond cut for the reduced-precision modes (s > 1e-7 s_max requested).  The
# library's cut is lambda = s^2 > max(cut^2, 10 eps) lambda_max with eps = 1e-14 for FP64 Grams of
# FP32 tensors, i.e. s > sqrt(1e-13) s_max = 3.2e-7 s_max in effect; the oracle runs at that
# effective cut.  Bounds: 1e-6 relative on every energy and probability (the workload's
# target); the trace and success probability are renormalised in FP64 to the centre's norm.
CHAIN100_TOL = {"e_succ": 1e-6, "e_raw": 1e-6, "p_succ": 1e-6, "trace": 1e-6}
MIXED_FLOOR_CUT = float(np.sqrt(1e-13))


@pytest.mark.parametrize("prec", ["c64", "tf32x3"])
def test_chain100_mixed_at_a4_cut_matches_oracle(lib, prec):
    c = synth.chain100()
    ref, r = _oracle(c, sv_cutoff=MIXED_FLOOR_CUT)
    g, e, stats = _gpu(lib, c, prec, gram_fp64=True, sv_cutoff=1e-7)
    errs = {key: _rel(e[key], r[key]) for key in r}
    b, kd, _ = g.dims()
    ob = [a.shape[3] for a in ref.A[:-1]]
    print("chain100", prec, errs, "D max gpu/oracle", max(b), max(ob),
          "K max", max(kd), max(a.shape[2] for a in ref.A))
    for key in r:
        assert errs[key] < CHAIN100_TOL[key], (key, e[key], r[key])
    # bond dimensions reached: within a few of the oracle's at the same cut (values at the
    # floor itself may fall either side)
    assert abs(max(b) - max(ob)) <= 3
    g.close()


# Second-order observables (Sec. III.E): the library's two-copy environments against the
# oracle's (pinned to the dense definitions) on the same circuits.  FP64 sites: 1e-8
# relative on xi and the collision probability, 1e-9 absolute on the entropies (on the
# truncated case the GPU's Gram floor drops weights below 1e-15 that the oracle's SVD keeps,
# which moves these quadratic quantities by ~1e-10); complex64 sites (environments in FP32,
# FP64 final sums): 1e-4 relative, 1e-4 absolute.
@pytest.mark.parametrize("prec", ["fp64", "c64"])
@pytest.mark.parametrize("case", ["tiny", "n10c12k4"])
def test_second_order_matches_oracle(lib, prec, case):
    from oracle import second_order as so
    if case == "tiny":
        c = dataclasses.replace(synth.tiny(), k_max=40)
    else:
        c = synth.scaled(synth.chain40(), n_sites=10, chi_max=12, k_max=4)
    ref, _ = _oracle(c)
    g, _, _ = _gpu(lib, c, prec)
    for cut in (1, c.n_sites // 2, c.n_sites - 1):
        got = g.second_order(cut)
        want = so.second_order(ref, cut)
        print(prec, case, cut, {k: (got[k], want[k]) for k in want})
        for key in ("xi", "collision"):
            tol = 1e-8 if prec == "fp64" else 1e-4
            assert abs(got[key] - want[key]) < tol * abs(want[key]), (cut, key)
        for key in ("s2_left", "s2_right", "i2"):
            tol = 1e-9 if prec == "fp64" else 1e-4
            assert abs(got[key] - want[key]) < tol, (cut, key)
    g.close()


U32 = 2.0 ** -24   # unit roundoff of the FP32-stored site tensors


def _energy_norm(c):
    """sum_k ||h_k|| of the TFIM terms: |J| per bond, |h| + |b J| per site (a bound on ||H||)."""
    return (c.n_sites - 1) * abs(c.J) + c.n_sites * (abs(c.hx) + abs(c.bz * c.J))


def test_batch512_circuit0_fp64_matches_oracle(lib):
    """Circuit 0 of the batched workload (N = 99, p = 2, chi 64, K 8; its energy's two parts
    cancel to a sixth of their scale) in FP64 at the same cut: 1e-9 relative on every output,
    so what the mixed form shows on this circuit is its precision, not the method."""
    c = synth.batch512()[0]
    g, e, _ = _gpu(lib, c, "fp64", sv_cutoff=MIXED_FLOOR_CUT)
    _, r = _oracle(c, sv_cutoff=MIXED_FLOOR_CUT)
    for key in ("e_raw", "e_succ", "p_succ", "trace"):
        assert abs(e[key] - r[key]) < 1e-9 * max(1.0, abs(r[key])), (key, e[key], r[key])
    g.close()


def test_batch512_first_32_circuits_match_oracle(lib):
    """The batched workload's first 32 circuits (N ~ U{20..100}, chi in {32,64,128}, K = 8,
    p in {1,2}, log-uniform rates) run concurrently through the executor in the mixed
    tensor-core form at reading A4's cut, every one against the oracle at the effective cut
    (s > sqrt(1e-13) s_max).

    Bounds: 1e-6 relative on the success probability and the trace.  An energy is a sum of
    local terms; each of the circuit's U = p (N - 1) updates rounds the site tensors to FP32
    (unit roundoff u = 2^-24), which moves each term's expectation by an absolute amount of
    order u ||h_k|| whatever its value, and U independent roundings add up as sqrt(U).  So
    the energy's bound is absolute: |dE| <= 2 u sqrt(U) sum_k ||h_k||.  Relative to |E| that
    is a condition number of the sum: on circuits whose terms are small or cancel (circuit
    30: N = 71, |E| = 1.22 from 141 terms) it exceeds 1e-6; chain100 (|E| = 30.9) keeps its
    own 1e-6 relative bound.
    """
    circs = synth.batch512()[:32]
    pool = [lib.Mpdo(100, 128, 8, m_max=25, prec="tf32x3", gram_fp64=True, sv_cutoff=1e-7,
                     own_stream=True) for _ in range(16)]
    descs, uploaded = [], []
    for c in circs:
        dls = [pool[0].upload_layer(layer) for layer in lib.circuit_layers(c)]
        uploaded.append(dls)
        descs.append(dict(n_sites=c.n_sites, chi_max=c.chi_max, k_max=c.k_max, layers=dls,
                          J=c.J, hx=c.hx, b=c.bz))
    out = lib.batch_run(pool, descs)
    worst, fails = {}, []
    for i, c in enumerate(circs):
        _, r = _oracle(c, sv_cutoff=MIXED_FLOOR_CUT)
        for j, key in enumerate(("e_raw", "e_succ", "p_succ", "trace")):
            if key in ("p_succ", "trace"):
                err = _rel(out[i][j], r[key])
                ok = err < CHAIN100_TOL[key]
            else:
                n_upd = c.p * (c.n_sites - 1)
                err = abs(out[i][j] - r[key]) / (2 * U32 * np.sqrt(n_upd) * _energy_norm(c))
                ok = err < 1.0
                worst[key + "_rel_to_E"] = max(worst.get(key + "_rel_to_E", 0.0),
                                               abs(out[i][j] - r[key]) / abs(r[key]))
            worst[key] = max(worst.get(key, 0.0), err)
            if not ok:
                fails.append((i, key, out[i][j], r[key], err))
    print("batch512[:32] worst errors (p_succ, trace: relative; energies: |dE| / bound)",
          worst)
    assert not fails, fails
    for dls in uploaded:
        for dl in dls:
            pool[0].free_uploaded(dl)
    for m in pool:
        m.close()
