"""Pins for the oracle MLP: gradients equal central finite differences (float64), the
input gradient likewise, and Adam's first step moves each weight by lr * sign(g)."""
import numpy as np

from oracle import mlp


def _params(rng, widths):
    return [(rng.standard_normal((a, b)) / np.sqrt(a), 0.1 * rng.standard_normal(b))
            for a, b in zip(widths[:-1], widths[1:])]


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    widths = [6, 16, 16, 2]
    params = _params(rng, widths)
    x = rng.standard_normal((5, 6))
    t = rng.standard_normal((5, 2))
    loss, grads, gx = mlp.loss_and_grads(params, x, t)
    h = 1e-6
    for l, (w, b) in enumerate(params):
        for arr, g in ((w, grads[l][0]), (b, grads[l][1])):
            for idx in [tuple(rng.integers(0, s) for s in arr.shape) for _ in range(6)]:
                old = arr[idx]
                arr[idx] = old + h
                lp = mlp.loss_and_grads(params, x, t)[0]
                arr[idx] = old - h
                lm = mlp.loss_and_grads(params, x, t)[0]
                arr[idx] = old
                assert abs((lp - lm) / (2 * h) - g[idx]) < 1e-7 * max(1.0, abs(g[idx]))
    for idx in [(0, 0), (3, 5), (4, 2)]:
        xp = x.copy(); xp[idx] += h
        xm = x.copy(); xm[idx] -= h
        fd = (mlp.loss_and_grads(params, xp, t)[0] - mlp.loss_and_grads(params, xm, t)[0]) / (2 * h)
        assert abs(fd - gx[idx]) < 1e-7


def test_input_grad_matches_finite_differences():
    rng = np.random.default_rng(1)
    params = _params(rng, [4, 8, 2])
    x = rng.standard_normal((3, 4))
    wout = np.array([0.7, -1.3])
    g = mlp.input_grad(params, x, wout)
    h = 1e-6
    for i in range(3):
        for j in range(4):
            xp = x.copy(); xp[i, j] += h
            xm = x.copy(); xm[i, j] -= h
            fp = mlp.forward(params, xp)[-1][i] @ wout
            fm = mlp.forward(params, xm)[-1][i] @ wout
            assert abs((fp - fm) / (2 * h) - g[i, j]) < 1e-8


def test_adam_first_step_is_lr_times_sign():
    rng = np.random.default_rng(2)
    params = _params(rng, [3, 4, 2])
    grads = [(rng.standard_normal(w.shape), rng.standard_normal(b.shape)) for w, b in params]
    new = mlp.adam_step(params, grads, {}, lr=1e-3)
    for (w, b), (nw, nb), (gw, gb) in zip(params, new, grads):
        assert np.allclose(w - nw, 1e-3 * np.sign(gw), rtol=1e-4)
        assert np.allclose(b - nb, 1e-3 * np.sign(gb), rtol=1e-4)
