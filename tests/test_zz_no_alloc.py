"""GPU test of the allocation-free eigensolver entry point (mpdo_heig_noalloc).

Some callers cannot allocate device memory during a call (their device memory is owned
by an outside allocator or budget, or a cudaMalloc would stall a latency-critical loop);
mpdo_heig_noalloc serves them from a fixed device array.  This file is collected last so
a run that stops at the first failure has run every other test before it.  Two calls in a
row (the second reusing the shared array after the first) must agree with the allocating
entry point mpdo_kernel_heig within the eigensolver tests' tolerance.
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


def _psd(rng, n):
    x = rng.standard_normal((n, n + 3)) + 1j * rng.standard_normal((n, n + 3))
    return x @ x.conj().T


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_matches_allocating_entry_point_twice(lib, prec):
    ct = torch.complex128 if prec == 0 else torch.complex64
    rng = np.random.default_rng(2024 + prec)
    for n in (lib.HEIG_NOALLOC_NMAX, 37):            # two calls in a row, different sizes
        h = _psd(rng, n)
        tol = (4e-16 if prec == 0 else 1.2e-7) * max(n, 25)
        outs = []
        for fn in (lib.kernel_heig, lib.kernel_heig_noalloc):
            a = torch.tensor(h, dtype=ct, device="cuda")
            v = torch.zeros((n, n), dtype=ct, device="cuda")
            w = torch.zeros(n, dtype=torch.float64, device="cuda")
            fn(prec, n, a, v, w)
            torch.cuda.synchronize()
            outs.append((w.cpu().numpy(), v.cpu().numpy().astype(complex)))
        (w0, v0), (w1, v1) = outs
        assert np.abs(w1 - w0).max() <= tol * w0[0]
        # eigenvectors agree up to a phase per column (distinct eigenvalues here)
        ph = np.sum(v0.conj() * v1, axis=0)
        assert np.abs(np.abs(ph) - 1.0).max() < 10 * tol
        assert np.abs(h @ v1 - v1 * w1[None, :]).max() <= 10 * tol * w0[0]


def test_noalloc_rejects_sizes_beyond_its_array(lib):
    n = lib.HEIG_NOALLOC_NMAX + 1
    a = torch.zeros((n, n), dtype=torch.complex128, device="cuda")
    v = torch.zeros_like(a)
    w = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(lib.MpdoError) as ex:
        lib.kernel_heig_noalloc(0, n, a, v, w)
    assert ex.value.code == -1 and "192" in str(ex.value)
