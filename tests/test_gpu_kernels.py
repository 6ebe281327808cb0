"""Kernel-level GPU tests through the C ABI: the complex GEMM against numpy for every op
combination and ragged shapes (including the cluster split-K form), the Jacobi
eigensolver against numpy's eigh."""
import numpy as np
import pytest

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


def _rand(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _op(x, op):
    return {0: x, 1: x.T, 2: x.conj().T, 3: x.conj()}[op]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("opa", [0, 1, 2, 3])
@pytest.mark.parametrize("opb", [0, 1, 2, 3])
def test_cgemm_ops(lib, prec, opa, opb):
    rng = np.random.default_rng(opa * 4 + opb)
    m, n, k, batch = 67, 45, 130, 3
    ash = (m, k) if opa in (0, 3) else (k, m)
    bsh = (k, n) if opb in (0, 3) else (n, k)
    a = _rand(rng, (batch,) + ash)
    b = _rand(rng, (batch,) + bsh)
    ct = torch.complex128 if prec == 0 else torch.complex64
    ta = torch.tensor(a, dtype=ct, device="cuda")
    tb = torch.tensor(b, dtype=ct, device="cuda")
    tc = torch.zeros((batch, m, n), dtype=ct, device="cuda")
    lib.kernel_cgemm(prec, opa, opb, m, n, k, ta, ash[1], ash[0] * ash[1], tb, bsh[1],
                     bsh[0] * bsh[1], tc, n, m * n, batch)
    torch.cuda.synchronize()
    want = np.stack([_op(a[i], opa) @ _op(b[i], opb) for i in range(batch)])
    err = np.abs(tc.cpu().numpy() - want).max() / np.abs(want).max()
    assert err < (1e-14 if prec == 0 else 2e-6)


@pytest.mark.parametrize("m,n,k,batch", [(16, 16, 257, 1), (20, 33, 70, 1), (5, 7, 33, 2),
                                         (3, 40, 17, 1), (67, 45, 130, 3)])
def test_cgemm_fp64_split_k(lib, m, n, k, batch):
    """FP64 products with few output tiles split K over a thread-block cluster (2-8 CTAs,
    slices of whole 16-steps, ragged last slice): same result as numpy to rounding, and
    bitwise the same on a second run (partials are added in rank order)."""
    rng = np.random.default_rng(m * 1000 + k)
    a = _rand(rng, (batch, m, k))
    b = _rand(rng, (batch, k, n))
    ta = torch.tensor(a, dtype=torch.complex128, device="cuda")
    tb = torch.tensor(b, dtype=torch.complex128, device="cuda")
    outs = []
    for _ in range(2):
        tc = torch.zeros((batch, m, n), dtype=torch.complex128, device="cuda")
        lib.kernel_cgemm(0, 0, 0, m, n, k, ta, k, m * k, tb, n, k * n, tc, n, m * n, batch)
        torch.cuda.synchronize()
        outs.append(tc.cpu().numpy())
    want = np.einsum("bik,bkj->bij", a, b)
    err = np.abs(outs[0] - want).max() / np.abs(want).max()
    assert err < 1e-14
    assert np.array_equal(outs[0], outs[1])


def test_autotuned_gemm_tiles_stay_correct(lib):
    """The tile-shape autotuner picks, per (output-tile count, K) bucket, the fastest of the
    64x64, 16x16 and cluster split-K kernels; products afterwards still match numpy, and
    reps <= 0 returns to the size rules."""
    try:
        for prec in (0, 1):
            assert lib.autotune_gemm(prec, reps=2) == 11 * 9
        for m, n, k, batch in [(16, 16, 257, 1), (67, 45, 130, 3), (200, 150, 40, 1),
                               (5, 7, 33, 2), (300, 260, 500, 1)]:
            rng = np.random.default_rng(m + n + k)
            a = _rand(rng, (batch, m, k))
            b = _rand(rng, (batch, k, n))
            want = np.einsum("bik,bkj->bij", a, b)
            for prec, ct, tol in ((0, torch.complex128, 1e-14), (1, torch.complex64, 2e-6)):
                ta = torch.tensor(a, dtype=ct, device="cuda")
                tb = torch.tensor(b, dtype=ct, device="cuda")
                tc = torch.zeros((batch, m, n), dtype=ct, device="cuda")
                lib.kernel_cgemm(prec, 0, 0, m, n, k, ta, k, m * k, tb, n, k * n, tc, n, m * n,
                                 batch)
                torch.cuda.synchronize()
                err = np.abs(tc.cpu().numpy() - want).max() / np.abs(want).max()
                assert err < tol, (prec, m, n, k, err)
    finally:
        for prec in (0, 1):
            assert lib.autotune_gemm(prec, reps=0) == 0


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n", [1, 5, 16, 37, 130, 300])
def test_heig_matches_numpy(lib, prec, n):
    rng = np.random.default_rng(n)
    x = _rand(rng, (n, n + 3))
    h = x @ x.conj().T                               # Hermitian PSD
    ct = torch.complex128 if prec == 0 else torch.complex64
    ta = torch.tensor(h, dtype=ct, device="cuda")
    tv = torch.zeros((n, n), dtype=ct, device="cuda")
    tw = torch.zeros(n, dtype=torch.float64, device="cuda")
    sweeps = lib.kernel_heig(prec, n, ta, tv, tw)
    torch.cuda.synchronize()
    w = tw.cpu().numpy()
    v = tv.cpu().numpy().astype(complex)
    wref = np.sort(np.linalg.eigvalsh(h))[::-1]
    # backward-stable bound ~ n eps |H| (eps = 6e-8 in FP32; the rounding of H itself to
    # FP32 adds up to ~n eps |H| more)
    tol = (4e-16 if prec == 0 else 2e-7) * max(n, 25)
    assert np.abs(w - wref).max() < tol * wref[0]
    # eigen-equation residual and orthonormality
    res = np.abs(h @ v - v * w[None, :]).max() / wref[0]
    assert res < tol * 10
    assert np.abs(v.conj().T @ v - np.eye(n)).max() < tol * 10
    assert 0 < sweeps < 30


@pytest.mark.parametrize("n", [30, 90])
def test_mixed_heig_graded_spectrum(lib, n):
    """The mixed-precision eigensolver (FP32 sweeps, FP64 refinement levels) on an FP64
    Hermitian matrix whose spectrum spans 14 decades, like the Gram matrices of the update:
    eigenvalues above 1e-10 of the largest to 1e-6 relative, FP64-level residuals."""
    rng = np.random.default_rng(n)
    q, _ = np.linalg.qr(_rand(rng, (n, n)))
    lam = 10.0 ** (-np.linspace(0, 14, n))
    h = (q * lam) @ q.conj().T
    h = 0.5 * (h + h.conj().T)
    ta = torch.tensor(h, dtype=torch.complex128, device="cuda")
    tv = torch.zeros_like(ta)
    tw = torch.zeros(n, dtype=torch.float64, device="cuda")
    levels = lib.kernel_heig(2, n, ta, tv, tw)
    torch.cuda.synchronize()
    w = tw.cpu().numpy()
    v = tv.cpu().numpy()
    order = np.argsort(w)[::-1]
    w, v = w[order], v[:, order]
    big = lam > 1e-10
    assert (np.abs(w[big] - lam[big]) / lam[big]).max() < 1e-6
    res = np.linalg.norm(h @ v - v * w[None, :], axis=0).max()
    assert res < 1e-8
    assert np.abs(v.conj().T @ v - np.eye(n)).max() < 1e-4
    assert 1 <= levels <= 24


@pytest.mark.parametrize("prec,n", [(2, 300), (3, 300), (3, 1350), (3, 2304)])
def test_mixed_heig_bond_sizes(lib, prec, n):
    """The mixed solver at bond-Gram sizes n = 9 D (D = 150 and 256): FP32 Jacobi levels and
    FP64 refinement, with the refinement's products on the CUDA cores (prec 2) or as exact
    BF16 slice products on the tensor cores (prec 3).  Spectrum over 14 decades, dense
    (neighbours 1.4-10 % apart).

    Bounds, with eps = 2^-48 sqrt(n) (the slice products carry ~2^-48 of each row's largest
    entry; FP64's rounding is below it): eigenvalues to 10 eps of the largest; for the pairs
    above 1e-10 of the largest, residuals to 1e-8 and orthonormality to the perturbation
    bound of the products (Davis-Kahan): |<v_i, v_j>| |l_i - l_j| <= 10 eps l_0, norms to
    1e-8 -- a pair is corrected once its mixing angle is below the pass's bound and the last
    pass leaves angles and norms off by at most ~1e-8; pairs the FP32 sweeps leave mixed are
    settled by Rayleigh-Ritz."""
    rng = np.random.default_rng(n + prec)
    q, _ = np.linalg.qr(_rand(rng, (n, n)))
    lam = 10.0 ** (-np.linspace(0, 14, n))
    h = (q * lam) @ q.conj().T
    h = 0.5 * (h + h.conj().T)
    ta = torch.tensor(h, dtype=torch.complex128, device="cuda")
    tv = torch.zeros_like(ta)
    tw = torch.zeros(n, dtype=torch.float64, device="cuda")
    levels = lib.kernel_heig(prec, n, ta, tv, tw)
    torch.cuda.synchronize()
    w = tw.cpu().numpy()
    v = tv.cpu().numpy()
    order = np.argsort(w)[::-1]
    w, v = w[order], v[:, order]
    eps = 2.0 ** -48 * np.sqrt(n)
    big = lam > 1e-10
    vb, wb = v[:, big], w[big]
    eig_err = np.abs(w - lam).max()
    res = np.linalg.norm(h @ vb - vb * wb[None, :], axis=0).max()
    ov = np.abs(vb.conj().T @ vb)
    norm_err = np.abs(np.diag(ov) - 1.0).max()
    np.fill_diagonal(ov, 0.0)
    dk = (ov * np.abs(wb[:, None] - wb[None, :])).max()
    print(f"n={n} prec={prec}: levels {levels}, eigenvalues {eig_err:.2e}, residual {res:.2e}, "
          f"norms {norm_err:.2e}, overlap x gap {dk:.2e} (bound {10 * eps:.1e})")
    assert eig_err < 10 * eps
    assert res < 1e-8
    assert norm_err < 1e-8
    assert dk < 10 * eps
    assert 1 <= levels <= 24
