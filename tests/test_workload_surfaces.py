"""Pins of the synthetic input generators (test data, not the method): the
bumpy sphere's nodes satisfy r = 1 + 0.1 sin(3 theta) cos(4 phi) and its
analytic normals are orthogonal to the surface's tangent vectors, computed
here independently by central differences of the parametrisation; PCA
normals recover the sphere's radial direction and the bumpy surface's
analytic normal away from the poles; the MLP parameter layout round-trips."""
import numpy as np

from paper_1404_0812_gb300 import workloads as W


def _surface(theta, phi):
    r = 1.0 + 0.1 * np.sin(3.0 * theta) * np.cos(4.0 * phi)
    return np.stack([r * np.sin(theta) * np.cos(phi), r * np.sin(theta) * np.sin(phi), r * np.cos(theta)], -1)


def test_bumpy_sphere_nodes_and_analytic_normals():
    ns = W.bumpy_sphere(5000)
    X, nrm = ns.X, ns.normals
    rho = np.linalg.norm(X, axis=1)
    theta = np.arccos(X[:, 2] / rho)
    phi = np.arctan2(X[:, 1], X[:, 0])
    assert np.allclose(rho, 1.0 + 0.1 * np.sin(3 * theta) * np.cos(4 * phi), atol=1e-13)
    assert np.allclose(np.linalg.norm(nrm, axis=1), 1.0, atol=1e-13)
    h = 1e-6
    t_theta = (_surface(theta + h, phi) - _surface(theta - h, phi)) / (2 * h)
    t_phi = (_surface(theta, phi + h) - _surface(theta, phi - h)) / (2 * h)
    ok = np.sin(theta) > 1e-3          # away from the poles, where the parametrisation degenerates
    assert np.max(np.abs(np.sum(nrm * t_theta, axis=1)[ok])) < 1e-8
    assert np.max(np.abs(np.sum(nrm * t_phi, axis=1)[ok])) < 1e-8
    assert np.all(np.sum(nrm * X, axis=1) > 0.0)   # outward


def test_jittered_bumpy_sphere_stays_on_the_surface():
    ns = W.bumpy_sphere(4000, jitter=0.25)
    X = ns.X
    rho = np.linalg.norm(X, axis=1)
    theta = np.arccos(X[:, 2] / rho)
    phi = np.arctan2(X[:, 1], X[:, 0])
    assert np.allclose(rho, 1.0 + 0.1 * np.sin(3 * theta) * np.cos(4 * phi), atol=1e-13)
    plain = W.bumpy_sphere(4000)
    assert np.max(np.linalg.norm(X - plain.X, axis=1)) > 0.01   # the jitter moved the nodes


def test_pca_normals():
    s = W.fibonacci_sphere(20000)
    n = W.pca_normals(s.X, 20)
    cosang = np.abs(np.sum(n * s.X, axis=1))         # sign is arbitrary
    assert np.min(cosang) > 1.0 - 1e-3
    b = W.bumpy_sphere(20000)
    nb = W.pca_normals(b.X, 20)
    rho = np.linalg.norm(b.X, axis=1)
    away = np.abs(b.X[:, 2] / rho) < 0.9
    assert np.median(np.abs(np.sum(nb * b.normals, axis=1))[away]) > 0.999


def test_mlp_layout_round_trip():
    D = 3 * 50
    p = W.mlp_init(D, seed=3)
    flat = W.mlp_pack(p)
    assert flat.size == sum(int(np.prod(s)) for s in W.mlp_shapes(D).values())
    q = W.mlp_unpack(flat, D)
    assert set(q) == set(p)
    for k in p:
        assert np.array_equal(q[k], p[k])
