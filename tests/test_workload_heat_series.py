"""Pins of the exact solution used by the sphere heat-equation study
(Section 6, diffusion on the sphere): the sectoral harmonics Y_ll against
scipy's spherical harmonics, their harmonic-polynomial form (so that
Delta_S2 Y_ll = -l(l+1) Y_ll), orthonormality by quadrature, and the series
solving u_t = Delta_S2 u term by term."""
import math

import numpy as np
import pytest
import scipy.special as sp

from paper_1404_0812_gb300 import workloads as W


def _points(k=40, seed=0):
    rng = np.random.default_rng(seed)
    theta = rng.uniform(0.05, math.pi - 0.05, k)     # colatitude
    phi = rng.uniform(0, 2 * math.pi, k)             # azimuth
    X = np.stack([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)], axis=1)
    return X, theta, phi


@pytest.mark.parametrize("l", [1, 2, 5, 12, 30])
def test_sectoral_harmonic_matches_scipy(l):
    X, theta, phi = _points()
    ref = math.sqrt(2.0) * (-1) ** l * sp.sph_harm_y(l, l, theta, phi).real   # no Condon-Shortley sign
    np.testing.assert_allclose(W.sectoral_harmonic(X, l), ref, rtol=1e-10, atol=1e-13)


def test_sectoral_harmonic_is_harmonic_polynomial():
    """Re((x + i y)^l) is harmonic in R^3 and homogeneous of degree l, so on
    the unit sphere Delta_S2 = Delta_R3 - l(l+1) (radial part) gives the
    eigenvalue -l(l+1): check Delta_R3 = 0 and homogeneity numerically."""
    X, _, _ = _points(10, seed=1)
    h = 1e-3
    for l in (2, 5, 9):
        f = lambda P: W.sectoral_harmonic(P, l)
        lap = sum((f(X + h * e) - 2 * f(X) + f(X - h * e)) / h ** 2 for e in np.eye(3))
        assert np.abs(lap).max() < 1e-4 * max(1.0, np.abs(f(X)).max() * l * l)
        assert np.allclose(f(1.7 * X), 1.7 ** l * f(X), rtol=1e-12)


def test_orthonormal_by_quadrature():
    ns = W.fibonacci_sphere(400_000)
    Y = np.stack([W.sectoral_harmonic(ns.X, l) for l in range(1, 7)])
    G = 4 * math.pi * (Y @ Y.T) / ns.N
    assert np.abs(G - np.eye(6)).max() < 2e-3


def test_series_solves_heat_equation_termwise():
    X, _, _ = _points(20, seed=2)
    t, dt = 0.05, 1e-5
    ut = (W.sphere_heat_series(X, t + dt) - W.sphere_heat_series(X, t - dt)) / (2 * dt)
    lap = sum(-l * (l + 1) * (20 / (3 * math.pi)) * math.exp(-l * l / 9 - t * l * (l + 1))
              * W.sectoral_harmonic(X, l) for l in range(1, 31))
    assert np.abs(ut - lap).max() < 1e-6 * np.abs(lap).max()
    u0 = W.sphere_heat_series(X, 0.0)
    direct = (20 / (3 * math.pi)) * sum(math.exp(-l * l / 9) * W.sectoral_harmonic(X, l) for l in range(1, 31))
    np.testing.assert_allclose(u0, direct, rtol=1e-13, atol=1e-15)
