"""Pins of the oracle's learned-eps network: central finite differences of
the loss against the analytic backward pass, Adam's first step, GELU values,
and the invariances of the stencil features."""
import math

import numpy as np

from oracle import mlp as om
from oracle import stencils as ost
from paper_1404_0812_gb300 import workloads as W


def _params(D, seed=0):
    return W.mlp_init(D, seed)


def test_gelu_values():
    z = np.array([0.0, 1.0, -1.0, 6.0, -6.0])
    # GELU(1) = Phi(1) with Phi the standard normal CDF
    np.testing.assert_allclose(om.gelu(z), [0.0, 0.8413447460685429, -0.15865525393145707,
                                            6.0, 0.0], atol=1e-8)
    h = 1e-6
    np.testing.assert_allclose(om.gelu_grad(z), (om.gelu(z + h) - om.gelu(z - h)) / (2 * h), atol=1e-8)
    assert om.gelu_grad(np.array([0.0]))[0] == 0.5


def test_backward_matches_finite_differences():
    D = 12
    p = _params(D, 1)
    rng = np.random.default_rng(5)
    x = rng.standard_normal((9, D))
    t = rng.standard_normal(9)
    _, g = om.loss_and_grads(p, x, t)
    h = 1e-6
    for k in p:
        flat = p[k].reshape(-1)
        for i in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[i]
            flat[i] = old + h
            lp, _ = om.loss_and_grads(p, x, t)
            flat[i] = old - h
            lm, _ = om.loss_and_grads(p, x, t)
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[k].reshape(-1)[i]) <= 1e-7 * max(1.0, abs(fd)), k


def test_adam_first_step_is_lr_sign():
    D = 6
    p = _params(D, 2)
    p0 = {k: v.copy() for k, v in p.items()}
    g = {k: np.random.default_rng(3).standard_normal(v.shape) for k, v in p.items()}
    st = {}
    om.adam_step(p, g, st, lr=1e-3)
    # m_hat = g and v_hat = g^2 after one step, so the update is
    # lr g / (|g| + 1e-8), i.e. lr sign(g) away from tiny gradients
    for k in p:
        np.testing.assert_allclose(p[k], p0[k] - 1e-3 * g[k] / (np.abs(g[k]) + 1e-8), atol=1e-15)
        big = np.abs(g[k]) > 1e-3
        np.testing.assert_allclose(p[k][big], p0[k][big] - 1e-3 * np.sign(g[k][big]), atol=1e-8)


def test_features_invariant_and_shaped():
    ns = W.fibonacci_sphere(2000)
    idx = ost.stencil(ns.X, 123, 50)
    P, nh = ns.X[idx], ns.normals[idx[0]]
    f, rs = om.features(P, nh)
    assert f.shape == (150,)
    np.testing.assert_array_equal(f[:3], 0.0)               # the centre itself
    assert abs(f[3 + 1]) < 1e-15                             # nearest neighbour on t1
    assert math.isclose(np.max(np.linalg.norm(f.reshape(50, 3), axis=1)), 1.0, rel_tol=1e-14)
    q, _ = np.linalg.qr(np.random.default_rng(1).standard_normal((3, 3)))
    f2, rs2 = om.features(P @ q.T + 5.0, nh @ q.T)
    np.testing.assert_allclose(f2, f, atol=1e-12)
    f3, _ = om.features(P, -nh)
    np.testing.assert_allclose(f3, f, atol=1e-15)
