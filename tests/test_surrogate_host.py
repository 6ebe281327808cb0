"""Host-side logic of the learned surrogate (no GPU): the angle feature map and the
chain rule that turns the network's input gradient into an angle gradient."""
import math

import numpy as np

import synth
from paper_2309_08572_gb300 import surrogate as sg


def test_feature_layout():
    c = synth.tiny()
    p = c.p
    f = sg.features(c, p)
    assert f.shape == (sg.n_features(p),)
    theta = np.array(list(c.alpha[:p]) + list(c.beta[:p]))
    q = 2 * p
    blocks = f[sg.N_FIXED:].reshape(5, q)
    np.testing.assert_allclose(blocks[0], 2 * theta / math.pi - 1, atol=1e-6)
    np.testing.assert_allclose(blocks[1] ** 2 + blocks[2] ** 2, 1.0, atol=1e-6)
    np.testing.assert_allclose(blocks[3] ** 2 + blocks[4] ** 2, 1.0, atol=1e-6)


def test_angle_chain_rule_matches_finite_differences():
    # a fixed linear-plus-quadratic function of the features; its angle gradient through
    # the feature map against central differences
    rng = np.random.default_rng(4)
    q = 4
    theta = rng.uniform(0, math.pi, (3, q))
    w = rng.standard_normal(5 * q)
    qm = rng.standard_normal((5 * q, 5 * q)) * 0.1

    def fun(th):
        f = sg._angle_block(th)
        return f @ w + 0.5 * np.einsum("ni,ij,nj->n", f, qm, f)

    f = sg._angle_block(theta)
    g_feat = w[None, :] + 0.5 * f @ (qm + qm.T)
    g = sg._angle_block_grad(theta, g_feat)
    h = 1e-6
    fd = np.zeros_like(theta)
    for j in range(q):
        e = np.zeros(q)
        e[j] = h
        fd[:, j] = (fun(theta + e) - fun(theta - e)) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-8)
