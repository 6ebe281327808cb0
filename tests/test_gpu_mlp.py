"""GPU MLP surrogate kernels against the float64 CPU oracle (oracle/mlp.py): loss,
parameter gradients, input gradients and one Adam step, for the 4-layer width-256 network
of the surrogate workload.  FP32 on the GPU: relative tolerance 2e-4 on gradients
(FP32 accumulation over the 256-wide layers)."""
import numpy as np
import pytest

from oracle import mlp as omlp

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

WIDTHS = [8, 256, 256, 256, 2]


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()
    import paper_2309_08572_gb300 as pkg
    return pkg


def _setup(lib, seed=0, batch=64):
    rng = np.random.default_rng(seed)
    params = [(rng.standard_normal((a, b)) / np.sqrt(a), 0.1 * rng.standard_normal(b))
              for a, b in zip(WIDTHS[:-1], WIDTHS[1:])]
    flat = lib.mlp_flat(params).astype(np.float32)
    params32 = lib.mlp_unflat(flat.astype(np.float64), WIDTHS)
    x = rng.uniform(-1, 1, (batch, WIDTHS[0]))
    t = rng.standard_normal((batch, WIDTHS[-1]))
    net = lib.Mlp(WIDTHS, max_batch=256)
    net.set_params(flat)
    tx = torch.tensor(x, dtype=torch.float32, device="cuda")
    tt = torch.tensor(t, dtype=torch.float32, device="cuda")
    x32 = tx.cpu().numpy().astype(np.float64)
    t32 = tt.cpu().numpy().astype(np.float64)
    return net, params32, tx, tt, x32, t32


def test_forward_loss_and_parameter_gradients(lib):
    net, params, tx, tt, x, t = _setup(lib)
    y = torch.zeros((tx.shape[0], WIDTHS[-1]), dtype=torch.float32, device="cuda")
    net.forward(tx, y)
    torch.cuda.synchronize()
    ref_y = omlp.forward(params, x)[-1]
    assert np.abs(y.cpu().numpy() - ref_y).max() < 1e-4 * max(1.0, np.abs(ref_y).max())
    loss, g = net.loss_grad(tx, tt, want_grad=True)
    ref_loss, ref_g, _ = omlp.loss_and_grads(params, x, t)
    assert abs(loss - ref_loss) < 1e-5 * max(1.0, ref_loss)
    ref_flat = lib.mlp_flat(ref_g)
    err = np.abs(g - ref_flat).max() / np.abs(ref_flat).max()
    assert err < 2e-4, err
    net.close()


def test_input_gradient(lib):
    net, params, tx, tt, x, t = _setup(lib, seed=1)
    gx = torch.zeros_like(tx)
    wout = np.array([1.0, -0.5])
    net.input_grad(tx, wout, gx)
    torch.cuda.synchronize()
    ref = omlp.input_grad(params, x, wout)
    err = np.abs(gx.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err < 2e-4, err
    net.close()


def test_adam_step_matches_oracle(lib):
    net, params, tx, tt, x, t = _setup(lib, seed=2)
    _, g = net.loss_grad(tx, tt, want_grad=True)
    net.adam_step(1e-3)
    new = net.get_params()
    grads = lib.mlp_unflat(g.astype(np.float64), WIDTHS)
    ref = omlp.adam_step(params, grads, {}, lr=1e-3)
    ref_flat = lib.mlp_flat(ref)
    assert np.abs(new - ref_flat).max() < 1e-6 + 1e-5 * np.abs(ref_flat).max()
    net.close()


def test_training_reduces_loss(lib):
    rng = np.random.default_rng(3)
    x = rng.uniform(-1, 1, (256, WIDTHS[0]))
    t = np.stack([np.sin(2 * x[:, 0]) * x[:, 1], np.cos(x[:, 2] + x[:, 3])], axis=1)
    net = lib.Mlp(WIDTHS, max_batch=256)
    params = [(rng.standard_normal((a, b)) / np.sqrt(a), np.zeros(b))
              for a, b in zip(WIDTHS[:-1], WIDTHS[1:])]
    net.set_params(lib.mlp_flat(params).astype(np.float32))
    tx = torch.tensor(x, dtype=torch.float32, device="cuda")
    tt = torch.tensor(t, dtype=torch.float32, device="cuda")
    first = None
    for step in range(300):
        loss, _ = net.loss_grad(tx, tt)
        first = loss if first is None else first
        net.adam_step(1e-3)
    assert loss < 0.05 * first, (first, loss)
    net.close()


# BF16 tensor-core products (tcgen05) with FP32 accumulation and FP32 parameters.  Each
# product rounds its operands to BF16 (unit roundoff 2^-9 = 2e-3); outputs and gradients
# then carry a few of those roundings relative to their largest entry: bounds 1e-2 on the
# forward output and 3e-2 on gradients (max-normalised), against the same float64 oracle.
def test_bf16_tensor_core_gradients_match_oracle(lib):
    net, params, tx, tt, x, t = _setup(lib, seed=5)
    from paper_2309_08572_gb300 import LIB
    assert LIB.mpdo_mlp_set_precision(net._h, 1) == 0
    n0 = lib.tc_gemm_launches()
    y = torch.zeros((tx.shape[0], WIDTHS[-1]), dtype=torch.float32, device="cuda")
    net.forward(tx, y)
    torch.cuda.synchronize()
    ref_y = omlp.forward(params, x)[-1]
    assert np.abs(y.cpu().numpy() - ref_y).max() < 1e-2 * max(1.0, np.abs(ref_y).max())
    loss, g = net.loss_grad(tx, tt, want_grad=True)
    ref_loss, ref_g, _ = omlp.loss_and_grads(params, x, t)
    assert abs(loss - ref_loss) < 1e-2 * max(1.0, ref_loss)
    ref_flat = lib.mlp_flat(ref_g)
    err = np.abs(g - ref_flat).max() / np.abs(ref_flat).max()
    assert err < 3e-2, err
    gx = torch.zeros_like(tx)
    net.input_grad(tx, np.array([1.0, -0.5]), gx)
    torch.cuda.synchronize()
    ref = omlp.input_grad(params, x, np.array([1.0, -0.5]))
    assert np.abs(gx.cpu().numpy() - ref).max() / np.abs(ref).max() < 3e-2
    assert lib.tc_gemm_launches() - n0 >= 3 * (len(WIDTHS) - 1)
    net.close()


def test_bf16_training_reduces_loss(lib):
    rng = np.random.default_rng(6)
    x = rng.uniform(-1, 1, (256, WIDTHS[0]))
    t = np.stack([np.sin(2 * x[:, 0]) * x[:, 1], np.cos(x[:, 2] + x[:, 3])], axis=1)
    net = lib.Mlp(WIDTHS, max_batch=256, bf16=True)
    params = [(rng.standard_normal((a, b)) / np.sqrt(a), np.zeros(b))
              for a, b in zip(WIDTHS[:-1], WIDTHS[1:])]
    net.set_params(lib.mlp_flat(params).astype(np.float32))
    tx = torch.tensor(x, dtype=torch.float32, device="cuda")
    tt = torch.tensor(t, dtype=torch.float32, device="cuda")
    first = None
    for step in range(300):
        loss, _ = net.loss_grad(tx, tt)
        first = loss if first is None else first
        net.adam_step(1e-3)
    assert loss < 0.05 * first, (first, loss)
    net.close()
