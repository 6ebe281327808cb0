"""Learned surrogate end to end on the GPU: samples from the MPDO engine (batch executor),
training by the library's MLP kernels (BF16 products on the tensor cores, FP32 master
parameters), angle proposals from its input gradient, and re-scoring of every proposal by
the engine.  The gain over the method without the network: with the same number of engine
evaluations, the proposals reach a lower energy than random angle draws, on 12-atom chains
and on the workload's target (N = 100, p = 2, re-scored by the mixed-precision MPDO at
chi = 128).  A bounded version of the 100k-sample workload: N_SAMPLES samples of 8-12-atom
chains (the sample count is printed with its generation time)."""
import dataclasses
import math

import numpy as np
import pytest

import synth

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


def _circuit(rng, n, p, gd, gp, xt, a=None, b=None):
    if a is None:
        a = list(rng.uniform(0, math.pi, p))
        b = list(rng.uniform(0, math.pi, p))
    return synth.Circuit(n_sites=n, p=p, alpha=a, beta=b, gamma_diss=gd, gamma_deph=gp,
                         xtalk_phase=xt, delta_pp=0.01, chi_max=16, k_max=4)


N_SAMPLES = 12000


def test_surrogate_proposals_beat_random_draws(lib):
    from paper_2309_08572_gb300 import surrogate as sg
    p = 2
    rng = synth.rng_for(55)
    pool = [lib.Mpdo(12, 16, 4, m_max=25, prec="c64", own_stream=True) for _ in range(16)]
    data = []
    for _ in range(N_SAMPLES):
        n = int(rng.integers(8, 13))
        data.append(_circuit(rng, n, p, float(10 ** rng.uniform(-4, -2)),
                             float(10 ** rng.uniform(-4, -2)), float(rng.choice([0.0, 0.01]))))
    import time
    t0 = time.perf_counter()
    y = sg.simulate(data, pool)
    print("engine samples", len(data), "in %.1f s" % (time.perf_counter() - t0))
    x = np.stack([sg.features(c, p) for c in data])
    assert np.all(np.isfinite(y))
    mu, sd = y.mean(axis=0), y.std(axis=0) + 1e-12
    yn = (y - mu) / sd                      # standardised targets
    net = sg.make_net(x.shape[1], max_batch=512, seed=1, bf16=True)
    ntr = N_SAMPLES - 400
    losses = sg.train(net, x[:ntr], yn[:ntr], steps=2000, lr=1e-3, batch=256, seed=2)
    assert losses[-1] < 0.2 * losses[0], (losses[0], losses[-1])
    # held-out error well below the spread of the targets
    tx = torch.tensor(x[ntr:], dtype=torch.float32, device="cuda")
    ty = torch.zeros((len(x) - ntr, 2), dtype=torch.float32, device="cuda")
    net.forward(tx, ty)
    pred = ty.cpu().numpy() * sd + mu
    rmse = np.sqrt(np.mean((pred[:, 0] - y[ntr:, 0]) ** 2))
    print("held-out rmse", rmse, "target std", np.std(y[:, 0]))
    assert rmse < 0.5 * np.std(y[:, 0]), (rmse, np.std(y[:, 0]))
    # proposals for a 12-atom chain at fixed noise, re-scored by the engine
    target = _circuit(rng, 12, p, 0.005, 0.005, 0.01, a=[0.0] * p, b=[0.0] * p)
    theta = sg.propose(net, target, p, n_starts=64, steps=200, lr=0.05, seed=3)
    props = [sg.with_angles(target, t[:p], t[p:]) for t in theta[:8]]
    e_prop = sg.simulate(props, pool)[:, 0]
    rand = [_circuit(rng, 12, p, 0.005, 0.005, 0.01) for _ in range(8)]
    e_rand = sg.simulate(rand, pool)[:, 0]
    print("surrogate best E/N", e_prop.min(), "random best E/N", e_rand.min(),
          "final train loss", losses[-1])
    assert e_prop.min() < e_rand.min()
    # the workload's target: proposals for N = 100, p = 2, re-scored by the MPDO at chi = 128
    # (mixed precision, bond cut of reading A4); the network saw only 8-12-atom chains, so
    # this is transfer.  Equal engine budget: the best of 8 proposals against the best of 8
    # random draws.
    big = dataclasses.replace(target, n_sites=100, chi_max=128, k_max=8)
    pool100 = [lib.Mpdo(100, 128, 8, m_max=25, prec="c64", gram_fp64=True, sv_cutoff=1e-7,
                        own_stream=True) for _ in range(8)]
    theta100 = sg.propose(net, big, p, n_starts=64, steps=200, lr=0.05, seed=4)
    e100 = sg.simulate([sg.with_angles(big, t[:p], t[p:]) for t in theta100[:8]], pool100)[:, 0]
    r100 = sg.simulate([dataclasses.replace(big, alpha=list(rng.uniform(0, math.pi, p)),
                                            beta=list(rng.uniform(0, math.pi, p)))
                        for _ in range(8)], pool100)[:, 0]
    print("N=100 chi=128: surrogate best E/N", e100.min(), "random best E/N", r100.min(),
          "random mean E/N", r100.mean())
    assert np.all(np.isfinite(e100)) and e100.min() < r100.min()
    for m in pool100:
        m.close()
    net.close()
    for m in pool:
        m.close()
