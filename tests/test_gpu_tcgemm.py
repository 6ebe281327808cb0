"""Tensor-core GEMM (tcgen05 + TMA) through the C ABI.

The real core is checked bit-exactly on small-integer inputs (every product and partial
sum is exact in FP32, so any layout, swizzle or descriptor slip shows as a wrong entry),
over ragged shapes that span several 128 x BN tiles, k-blocks and pipeline stages.  The
complex split-precision products are checked against numpy complex128 within the bound of
their arithmetic, relative to sum |a||b|: the operand rounding (TF32x3 keeps ~22
significand bits per operand, 3 x 2^-22 ~ 7e-7 per product plus headroom -> 3e-6; BF16x3
~16 bits -> 6e-5; plain TF32 2^-11 -> 2e-3; plain BF16 2^-8 -> 1.6e-2) plus the FP32
accumulation in tensor memory over the real K extent kr = parts * 2k, which behaves as a
random walk of roundings: 2 sqrt(kr) 2^-24.
"""
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


def _ld(k, elt):
    q = 16 // elt
    return (k + q - 1) // q * q


@pytest.mark.parametrize("elt", [4, 2])
@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (128, 64, 32), (129, 65, 33), (300, 200, 97),
                                   (256, 256, 512), (77, 513, 1000), (640, 130, 70)])
def test_real_core_exact_on_integers(lib, elt, m, n, k):
    rng = np.random.default_rng(m * 7 + n * 13 + k + elt)
    a = rng.integers(-4, 5, size=(m, k)).astype(np.float32)
    b = rng.integers(-4, 5, size=(n, k)).astype(np.float32)
    lda = ldb = _ld(k, elt)
    dt = torch.float32 if elt == 4 else torch.bfloat16
    ta = torch.zeros((m, lda), dtype=dt, device="cuda")
    tb = torch.zeros((n, ldb), dtype=dt, device="cuda")
    ta[:, :k] = torch.tensor(a, device="cuda").to(dt)
    tb[:, :k] = torch.tensor(b, device="cuda").to(dt)
    td = torch.full((m, n), float("nan"), dtype=torch.float32, device="cuda")
    lib.kernel_tcgemm_real(elt, m, n, k, ta, lda, tb, ldb, td, n)
    torch.cuda.synchronize()
    want = a.astype(np.float64) @ b.astype(np.float64).T
    got = td.cpu().numpy().astype(np.float64)
    assert np.array_equal(got, want), np.argwhere(got != want)[:5]


def _rand(rng, shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)


def _op(x, op):
    return {0: x, 1: x.T, 2: x.conj().T, 3: x.conj()}[op]


BOUND = {"tf32x3": 3e-6, "bf16x3": 6e-5, "tf32": 2e-3, "bf16": 1.6e-2}
PARTS = {"tf32x3": 3, "bf16x3": 3, "tf32": 1, "bf16": 1}


def _bound(mode, k):
    return BOUND[mode] + 2.0 * np.sqrt(PARTS[mode] * 2 * k) * 2.0 ** -24


@pytest.mark.parametrize("mode", ["tf32x3", "bf16x3", "tf32", "bf16"])
@pytest.mark.parametrize("opa,opb", [(0, 0), (1, 0), (2, 0), (0, 1), (0, 2), (3, 3), (2, 2)])
def test_complex_modes_vs_numpy(lib, mode, opa, opb):
    rng = np.random.default_rng(opa * 4 + opb)
    m, n, k, batch = 150, 70, 133, 2
    ash = (m, k) if opa in (0, 3) else (k, m)
    bsh = (k, n) if opb in (0, 3) else (n, k)
    a = _rand(rng, (batch,) + ash)
    b = _rand(rng, (batch,) + bsh)
    ta = torch.tensor(a, device="cuda")
    tb = torch.tensor(b, device="cuda")
    tc = torch.zeros((batch, m, n), dtype=torch.complex64, device="cuda")
    lib.kernel_tcgemm(mode, opa, opb, m, n, k, ta, ash[1], ash[0] * ash[1], tb, bsh[1],
                      bsh[0] * bsh[1], tc, n, m * n, batch)
    torch.cuda.synchronize()
    a64, b64 = a.astype(np.complex128), b.astype(np.complex128)
    want = np.stack([_op(a64[i], opa) @ _op(b64[i], opb) for i in range(batch)])
    scale = np.stack([np.abs(_op(a64[i], opa)) @ np.abs(_op(b64[i], opb)) for i in range(batch)])
    err = (np.abs(tc.cpu().numpy() - want) / scale).max()
    assert err < _bound(mode, k), err


@pytest.mark.parametrize("m,n,k", [(2304, 2304, 768), (400, 400, 5292), (3150, 672, 126)])
def test_tf32x3_update_shapes(lib, m, n, k):
    """Shapes of the update's contractions at chi = 256 (bond Gram), and at D = 42 with 25
    gate Kraus operators and K = 16 (inner Gram, centre tensor)."""
    rng = np.random.default_rng(m + n + k)
    a = _rand(rng, (m, k))
    b = _rand(rng, (k, n))
    tc = torch.zeros((m, n), dtype=torch.complex64, device="cuda")
    lib.kernel_tcgemm("tf32x3", 0, 0, m, n, k, torch.tensor(a, device="cuda"), k, 0,
                      torch.tensor(b, device="cuda"), n, 0, tc, n, 0, 1)
    torch.cuda.synchronize()
    rows = rng.choice(m, 24, replace=False)
    want = a[rows].astype(np.complex128) @ b.astype(np.complex128)
    scale = np.abs(a[rows]).astype(np.float64) @ np.abs(b).astype(np.float64)
    err = (np.abs(tc.cpu().numpy()[rows] - want) / scale).max()
    assert err < _bound("tf32x3", k), err


@pytest.mark.parametrize("elt", [2, 4])
def test_real_core_throughput(lib, elt):
    """Large square product (8192^3, the real core alone): correct on sampled entries, and
    its rate (CUDA events, best of 5) printed against cuBLAS on the same GPU; the rate is
    asserted only loosely (a tenth of cuBLAS), the measured fraction goes to the profiles."""
    n = 8192
    dt = torch.bfloat16 if elt == 2 else torch.float32
    g = torch.Generator(device="cuda").manual_seed(7)
    a = torch.randn((n, n), device="cuda", generator=g).to(dt)
    b = torch.randn((n, n), device="cuda", generator=g).to(dt)
    d = torch.empty((n, n), dtype=torch.float32, device="cuda")
    for _ in range(2):
        lib.kernel_tcgemm_real(elt, n, n, n, a, n, b, n, d, n)
    best = float("inf")
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        lib.kernel_tcgemm_real(elt, n, n, n, a, n, b, n, d, n)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    ours = 2 * n ** 3 / (best / 1e3) / 1e12
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        bt = b.t()
        for _ in range(2):
            torch.matmul(a, bt)
        ref_best = float("inf")
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, bt)
            e1.record()
            torch.cuda.synchronize()
            ref_best = min(ref_best, e0.elapsed_time(e1))
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    cublas = 2 * n ** 3 / (ref_best / 1e3) / 1e12
    print(f"tc_gemm_kernel {'bf16' if elt == 2 else 'tf32'} {n}^3: {ours:.0f} TFLOP/s, "
          f"cuBLAS {cublas:.0f} TFLOP/s, ratio {ours / cublas:.2f}")
    rows = torch.randint(0, n, (8,), device="cuda", generator=g)
    want = a[rows].double() @ b.double().t()
    err = (d[rows].double() - want).abs().max().item() / (a[rows].double().abs() @ b.double().abs().t()).max().item()
    assert err < (2e-3 if elt == 4 else 1e-2)
    assert ours > 0.1 * cublas


@pytest.mark.parametrize("opa,opb", [(0, 0), (2, 0), (0, 2), (1, 3), (3, 1)])
@pytest.mark.parametrize("m,n,k", [(70, 45, 130), (129, 200, 1100), (5, 300, 3000)])
def test_exact_slices_match_fp64_product(lib, opa, opb, m, n, k):
    """The exact-slice product of FP32 operands equals their product in FP64 (numpy
    complex128) up to the 2^-48 row slicing: |err| <= 2^-40 sum |a||b| per entry; chunks of
    1024 real terms (k > 512) and ragged tiles included."""
    rng = np.random.default_rng(m + n + k + opa * 5 + opb)
    ash = (m, k) if opa in (0, 3) else (k, m)
    bsh = (k, n) if opb in (0, 3) else (n, k)
    a = _rand(rng, (2,) + ash)
    b = _rand(rng, (2,) + bsh)
    tc = torch.zeros((2, m, n), dtype=torch.complex128, device="cuda")
    lib.kernel_tcgemm_exact(opa, opb, m, n, k, torch.tensor(a, device="cuda"), ash[1],
                            ash[0] * ash[1], torch.tensor(b, device="cuda"), bsh[1],
                            bsh[0] * bsh[1], tc, n, m * n, 2)
    torch.cuda.synchronize()
    a64, b64 = a.astype(np.complex128), b.astype(np.complex128)
    want = np.stack([_op(a64[i], opa) @ _op(b64[i], opb) for i in range(2)])
    scale = np.stack([np.abs(_op(a64[i], opa)) @ np.abs(_op(b64[i], opb)) for i in range(2)])
    err = (np.abs(tc.cpu().numpy() - want) / scale).max()
    assert err < 2.0 ** -40, err


def test_exact_gram_keeps_the_small_eigenvalues(lib):
    """Gram G = X^+ X of an FP32 matrix whose singular values fall from 1 to 1e-7: the
    eigenvalues of the exact-slice Gram agree with those of the FP64 Gram of the same FP32
    data to 1e-14 of the largest, absolute -- the FP64 rounding floor, below the 1e-13 cut
    of the mixed form -- while an FP32-accumulated (TF32x3) Gram misses the small ones by
    more than 1e-9 of the largest."""
    rng = np.random.default_rng(11)
    rows, cols = 600, 96
    u, _ = np.linalg.qr(_rand(rng, (rows, cols)).astype(np.complex128))
    v, _ = np.linalg.qr(_rand(rng, (cols, cols)).astype(np.complex128))
    s = np.logspace(0, -7, cols)
    x = ((u * s) @ v.conj().T).astype(np.complex64)
    tx = torch.tensor(x, device="cuda")
    g = torch.zeros((cols, cols), dtype=torch.complex128, device="cuda")
    lib.kernel_tcgemm_exact(2, 0, cols, cols, rows, tx, cols, 0, tx, cols, 0, g, cols, 0, 1)
    torch.cuda.synchronize()
    x64 = x.astype(np.complex128)
    want = np.linalg.eigvalsh(x64.conj().T @ x64)[::-1]
    got = np.linalg.eigvalsh(g.cpu().numpy())[::-1]
    err = np.abs(got - want).max() / want[0]
    assert err < 1e-14, err
    g32 = torch.zeros((cols, cols), dtype=torch.complex64, device="cuda")
    lib.kernel_tcgemm("tf32x3", 2, 0, cols, cols, rows, tx, cols, 0, tx, cols, 0, g32, cols, 0, 1)
    torch.cuda.synchronize()
    got32 = np.linalg.eigvalsh(g32.cpu().numpy().astype(np.complex128))[::-1]
    assert np.abs(got32 - want).max() / want[0] > 1e-9
