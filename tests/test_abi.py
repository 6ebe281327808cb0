"""CPU checks of the C ABI: the library loads, exports every symbol include/mpdo.h
declares, and its host channel builder matches the oracle's channels (superoperators
are unique, Kraus sets are not)."""
import os
import re
import subprocess

import numpy as np
import pytest

import synth
from oracle import ops as oops
from oracle import qaoa as oqaoa

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    import paper_2309_08572_gb300 as pkg
    return pkg


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    return _lib()


def test_exports_every_declared_symbol(pkg):
    hdr = open(os.path.join(ROOT, "include", "mpdo.h")).read()
    declared = set(re.findall(r"^(?:int|long long|const char\*)\s+(mpdo_\w+)\s*\(", hdr, re.M))
    out = subprocess.run(["nm", "-D", "--defined-only", pkg.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (mpdo_\w+)$", out, re.M))
    assert declared and declared <= exported, declared - exported


@pytest.mark.parametrize("args", [
    dict(angle_zz=0.3, gamma_diss=0.01, gamma_deph=0.01, xtalk_phase=0.0, delta_pp=0.01),
    dict(angle_zz=1.7, gamma_diss=0.2, gamma_deph=0.05, xtalk_phase=0.3, delta_pp=0.2),
    dict(angle_zz=0.0, gamma_diss=0.0, gamma_deph=0.0, xtalk_phase=0.0, delta_pp=0.0),
])
def test_block_channel_superoperator_matches_oracle(pkg, args):
    v = oqaoa.site_gate(0.4, 0.9, 1.0, 0.2)
    k_lib = pkg.build_block_channel(**args, post_left=v)
    k_or = oops.g0_block_channel(**args, b0=1 / 16, b1=1 / 16, bd=7 / 8, post_left=v)
    assert len(k_lib) == len(k_or)
    assert np.abs(oops.superop(k_lib) - oops.superop(k_or)).max() < 1e-13


def test_qaoa_layer_ops_match_oracle(pkg):
    c = synth.scaled(synth.chain40(), n_sites=7)
    for k in range(c.p):
        lib = pkg.build_qaoa_layer(c.n_sites, k, c.alpha[k], c.beta[k], c.J, c.bz, c.gamma_diss,
                                   c.gamma_deph, c.xtalk_phase, c.delta_pp)
        orc = oqaoa.layer_ops(c, k)
        assert [s for s, _ in lib] == [s for s, _ in orc]
        for (_, a), (_, b) in zip(lib, orc):
            assert np.abs(oops.superop(a) - oops.superop(b)).max() < 1e-13


def test_invalid_arguments_are_rejected_without_gpu(pkg):
    with pytest.raises(pkg.MpdoError):
        pkg.build_block_channel(0.1, -1.0, 0.0)
    with pytest.raises(pkg.MpdoError):
        pkg.build_block_channel(float("nan"), 0.0, 0.0)


def test_create_argument_checks_without_gpu(pkg):
    """mpdo_create validates sizes before any CUDA call: oversized m_max*k_max is
    ERR_ARG; the smoke circuit's sizes pass validation and fail only on the missing GPU."""
    import ctypes as C
    import __graft_entry__ as g

    def create(k_max, m_max):
        cfg = pkg.Config(6, 3, 729, k_max, m_max, pkg.PREC["fp64"], 0.0, 0.0, 1, None, 0)
        h = C.c_void_p(None)
        rc = pkg.LIB.mpdo_create(C.byref(cfg), None, C.byref(h))
        if rc == 0:
            pkg.LIB.mpdo_destroy(h)
        return rc

    assert create(64, 25) == -1
    assert create(g.SMOKE_K_MAX, g.SMOKE_M_MAX) != -1


@pytest.mark.parametrize("args", [
    dict(gamma_diss=0.0, gamma_deph=0.0, b0=1 / 16, b1=1 / 16, n_steps=200),
    dict(gamma_diss=0.05, gamma_deph=0.02, b0=1 / 16, b1=1 / 16, n_steps=300),
    dict(gamma_diss=0.3, gamma_deph=0.1, b0=0.4, b1=0.6, n_steps=150),
])
def test_cz_pulse_matches_oracle(pkg, args):
    """Gate model G1: the library's pulse CZ (closed-form dissipators, structured products)
    against the oracle's (matrix exponentials of the dissipator generator, dense products)."""
    from oracle import pulse as opulse
    s_lib, phi_lib, inf_lib = pkg.build_cz_pulse(**args)
    bd = 1.0 - args["b0"] - args["b1"]
    s_or, phi_or = opulse.cz_superop(args["gamma_diss"], args["gamma_deph"], args["b0"],
                                     args["b1"], bd, args["n_steps"])
    assert np.abs(s_lib - s_or).max() < 1e-11
    assert abs(phi_lib - phi_or) < 1e-12
    u = opulse.pulse_unitary(args["n_steps"])
    assert abs(inf_lib - opulse.average_cz_infidelity(u)) < 1e-12


def test_qaoa_layer_cz_ops_match_oracle(pkg):
    from oracle import pulse as opulse
    s_cz, _ = opulse.cz_superop(0.02, 0.01, 1 / 16, 1 / 16, 7 / 8, 200)
    c = synth.scaled(synth.chain40(), n_sites=6)
    for k in range(c.p):
        lib = pkg.build_qaoa_layer_cz(c.n_sites, k, c.alpha[k], c.beta[k], s_cz, c.J, c.bz,
                                      c.xtalk_phase)
        orc = oqaoa.layer_ops_cz(c, k, s_cz)
        assert [s for s, _ in lib] == [s for s, _ in orc]
        for (_, a), (_, b) in zip(lib, orc):
            assert np.abs(oops.superop(a) - oops.superop(b)).max() < 1e-12


def test_cz_pulse_rejects_bad_arguments(pkg):
    with pytest.raises(pkg.MpdoError):
        pkg.build_cz_pulse(n_steps=0)
    with pytest.raises(pkg.MpdoError):
        pkg.build_cz_pulse(gamma_diss=-1.0, n_steps=10)
    with pytest.raises(pkg.MpdoError):
        pkg.build_cz_pulse(n_steps=10, pulse=dict(pkg.GAUSSIAN_CZ, T=float("nan")))


def test_qaoa_layer_cz_rejects_bad_channels(pkg):
    """The G1 layer builder validates its CZ channel: non-finite entries are
    MPDO_ERR_NUMERIC, not a silent layer."""
    s = np.eye(81, dtype=complex)
    s[3, 5] = np.nan
    with pytest.raises(pkg.MpdoError) as err:
        pkg.build_qaoa_layer_cz(5, 0, 0.3, 0.2, s)
    assert err.value.code == -4
    with pytest.raises(pkg.MpdoError):
        pkg.build_qaoa_layer_cz(1, 0, 0.3, 0.2, np.eye(81))


def test_g1_layer_of_the_ideal_cz_is_the_noiseless_g0_layer(pkg):
    """With the ideal CZ channel, the G1 layer builder returns the noiseless G0 layer (same
    ZZ block, same folded one-site gates)."""
    c = synth.scaled(synth.chain40(), n_sites=5)
    cz = oops.superop([oops.CZ])
    for k in range(c.p):
        g1 = pkg.build_qaoa_layer_cz(c.n_sites, k, c.alpha[k], c.beta[k], cz, c.J, c.bz, 0.0)
        g0 = pkg.build_qaoa_layer(c.n_sites, k, c.alpha[k], c.beta[k], c.J, c.bz)
        assert [s for s, _ in g1] == [s for s, _ in g0]
        for (_, a), (_, b) in zip(g1, g0):
            assert np.abs(oops.superop(a) - oops.superop(b)).max() < 1e-13


def test_negative_eta_is_rejected(pkg):
    """A negative Choi cut would keep negative eigenvalues (NaN Kraus operators): every
    channel builder refuses it."""
    import ctypes as C
    out = np.zeros(81 * 81 * 2)
    m = C.c_int(0)
    rc = pkg.LIB.mpdo_build_block_channel(0.3, 0.01, 0.01, 0.0, 0.0, 1 / 16, 1 / 16, 7 / 8, None,
                                          None, -1e-9, pkg._dptr(out), 81, C.byref(m))
    assert rc == -1
    sites = (C.c_int * 8)()
    ms = (C.c_int * 8)()
    big = np.zeros(8 * 81 * 81 * 2)
    rc = pkg.LIB.mpdo_build_qaoa_layer(4, 0, 0.3, 0.2, 1.0, 0.0, 0.01, 0.01, 0.0, 0.0, 1 / 16,
                                       1 / 16, 7 / 8, -1.0, sites, ms, pkg._dptr(big), big.size // 2)
    assert rc == -1
    sup = np.eye(81, dtype=complex).view(float).reshape(-1).copy()
    rc = pkg.LIB.mpdo_build_qaoa_layer_cz(4, 0, 0.3, 0.2, 1.0, 0.0, pkg._dptr(sup), 0.0, -1.0,
                                          sites, ms, pkg._dptr(big), big.size // 2)
    assert rc == -1


def test_create_rejects_bad_order_and_hooks(pkg):
    import ctypes as C
    cfg = pkg.Config(6, 3, 8, 4, 4, pkg.PREC["fp64"], 0.0, 0.0, 1, None, 0, 2)
    h = C.c_void_p(None)
    assert pkg.LIB.mpdo_create(C.byref(cfg), None, C.byref(h)) == -1
    cfg = pkg.Config(6, 3, 8, 4, 4, pkg.PREC["fp64"], 0.0, 0.0, 1, None, 0, 1)
    cfg.alloc = pkg.ALLOC_FN(lambda n, ctx: None)   # alloc without free
    assert pkg.LIB.mpdo_create(C.byref(cfg), None, C.byref(h)) == -1


def test_forced_oom_through_the_alloc_hook(pkg):
    """The handle's device memory comes from the config's hooks: an allocator that refuses
    makes mpdo_create fail with MPDO_ERR_OOM (no GPU needed: the stream is given, so the
    first device request is the hook's), and nothing it handed out is left behind."""
    import ctypes as C
    calls = {"alloc": 0, "free": 0}

    def alloc(n, ctx):
        calls["alloc"] += 1
        return None

    def free(p, ctx):
        calls["free"] += 1

    fa, ff = pkg.ALLOC_FN(alloc), pkg.FREE_FN(free)
    cfg = pkg.Config(6, 3, 8, 4, 4, pkg.PREC["fp64"], 0.0, 0.0, 1, C.c_void_p(1), 0, 1)
    cfg.alloc, cfg.free = fa, ff
    h = C.c_void_p(None)
    rc = pkg.LIB.mpdo_create(C.byref(cfg), None, C.byref(h))
    assert rc == -2 and not h.value
    assert calls["alloc"] == 1 and calls["free"] == 0
    assert b"allocation" in pkg.LIB.mpdo_last_error(None)


def test_rcs_layer_ops_match_oracle(pkg):
    """The library's random-circuit layers equal the oracle's op by op (same bonds, same
    channel superoperators), in both sweep directions."""
    from oracle import rcs as orcs
    c = synth.rcs(6, 2, 16, 4, gamma_diss=0.01, delta_pp=0.05)
    c.xtalk_phase = 0.02
    for k in range(c.depth):
        lib_ops = pkg.build_rcs_layer(c.n_sites, k, c.haar[k], c.gamma_diss, c.gamma_deph,
                                      c.xtalk_phase, c.delta_pp)
        or_ops = orcs.layer_ops(c, k)
        assert [i for i, _ in lib_ops] == [i for i, _ in or_ops]
        for (_, a), (_, b) in zip(lib_ops, or_ops):
            assert np.abs(oops.superop(a) - oops.superop(b)).max() < 1e-13
