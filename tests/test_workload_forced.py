"""Pins of the manufactured forced-diffusion problems of Section 6 (sphere
and torus): the Laplace-Beltrami operator of each g is recomputed here from
the surface's parametrisation alone -- metric tensor by finite differences of
the embedding, Delta f = |g|^{-1/2} d_i(|g|^{1/2} g^{ij} d_j f) by nested
central differences -- and compared with the closed forms behind the sources
h = -5 g - Delta g."""
import math

import numpy as np

from paper_1404_0812_gb300 import workloads as W


def _lb_numeric(embed, f_of_X, p, q, h=1e-3):
    """Laplace-Beltrami of f on the surface embed(p, q) at (p, q)."""
    def metric(p, q):
        xp = (embed(p + h, q) - embed(p - h, q)) / (2 * h)
        xq = (embed(p, q + h) - embed(p, q - h)) / (2 * h)
        G = np.array([[xp @ xp, xp @ xq], [xq @ xp, xq @ xq]])
        return G

    def F(p, q):
        return f_of_X(embed(p, q)[None, :])[0]

    def flux(p, q):
        # sqrt|g| g^{ij} d_j f at (p, q)
        G = metric(p, q)
        sg = math.sqrt(np.linalg.det(G))
        df = np.array([(F(p + h, q) - F(p - h, q)) / (2 * h), (F(p, q + h) - F(p, q - h)) / (2 * h)])
        return sg * np.linalg.solve(G, df)

    G = metric(p, q)
    sg = math.sqrt(np.linalg.det(G))
    div = ((flux(p + h, q)[0] - flux(p - h, q)[0]) + (flux(p, q + h)[1] - flux(p, q - h)[1])) / (2 * h)
    return div / sg


def test_sphere_forced_laplacian():
    centers = W.sphere_forced_centers()
    embed = lambda th, ph: np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
    rng = np.random.default_rng(0)
    for th, ph in zip(rng.uniform(0.3, math.pi - 0.3, 12), rng.uniform(0, 2 * math.pi, 12)):
        x = embed(th, ph)[None, :]
        g, h = W.sphere_forced(x, centers)
        lap = _lb_numeric(embed, lambda X: W.sphere_forced(X, centers)[0], th, ph)
        assert abs((-5 * g[0] - h[0]) - lap) <= 2e-4 * max(1.0, abs(lap))
    # at a centre the zonal closed form takes its limit -40 G
    g, h = W.sphere_forced(centers[:1], centers[:1])
    assert abs(h[0] - (-5.0 + 40.0)) < 1e-12


def test_torus_forced_laplacian():
    centers = W.torus_forced_centers()
    embed = lambda p, l: np.array([(1 + math.cos(p) / 3) * math.cos(l), (1 + math.cos(p) / 3) * math.sin(l),
                                   math.sin(p) / 3])
    rng = np.random.default_rng(1)
    for p, l in zip(rng.uniform(-math.pi, math.pi, 12), rng.uniform(-math.pi, math.pi, 12)):
        x = embed(p, l)[None, :]
        ph, la = W.torus_angles(x)
        assert abs(math.remainder(ph[0] - p, 2 * math.pi)) < 1e-12
        assert abs(math.remainder(la[0] - l, 2 * math.pi)) < 1e-12
        g, h = W.torus_forced(x, centers)
        # a = 9 makes g sharp (width ~ 1/9): a smaller step keeps the
        # differencing error below the bound
        lap = _lb_numeric(embed, lambda X: W.torus_forced(X, centers)[0], p, l, h=2e-4)
        assert abs((-5 * g[0] - h[0]) - lap) <= 2e-4 * max(1.0, abs(lap))
