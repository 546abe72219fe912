"""Pins of the high-precision oracle (oracle/weights_hp.py) that checks the
double-double build: its Jacobi eigenvalues against LAPACK, the two-node
closed forms of kappa and of its root at kappa_T = 1e20 / 1e24 (far beyond
float64), agreement with the float64 oracle where float64 suffices, and
invariants of the weights at kappa_T = 1e20."""
import decimal
import math
from decimal import Decimal

import numpy as np
import pytest

from oracle import stencils as ost
from oracle import weights as ow
from oracle import weights_hp as hp
from paper_1404_0812_gb300 import workloads as W


def test_jacobi_matches_lapack():
    rng = np.random.default_rng(0)
    B = rng.normal(size=(12, 12))
    B = B + B.T
    with hp._ctx():
        lam = sorted(float(x) for x in hp.jacobi_eigenvalues([[Decimal(float(v)) for v in r] for r in B]))
    assert np.abs(np.array(lam) - np.linalg.eigvalsh(B)).max() <= 1e-13 * np.abs(B).max()


def _two_node_root(kT: int, kernel: int, r: Decimal):
    """Exact root of lambda_+(a) = kT (1 - a) for the two-node stencil (a
    quadratic in s = 1 + a, solved in 60-digit decimal), as eps."""
    with decimal.localcontext(decimal.Context(prec=60)):
        k = Decimal(kT)
        A2, B2, C2 = k * k + k, -2 * k * (2 * k + 1), 4 * k * k - 2
        disc = (B2 * B2 - 4 * A2 * C2).sqrt()
        s = [c for c in ((-B2 - disc) / (2 * A2), (-B2 + disc) / (2 * A2)) if 1 < c < 2][0]
        a = s - 1
        e = (-a.ln()).sqrt() / r if kernel == ow.GAUSSIAN else (1 / (a * a) - 1).sqrt() / r
        # kappa at that eps from the closed-form eigenvalues 1 - a, (s +- sqrt(s^2 + 8)) / 2
        lp = (s + (s * s + 8).sqrt()) / 2
        lm = abs((s - (s * s + 8).sqrt()) / 2)
        kap = max(lp, lm, 1 - a) / min(lp, lm, 1 - a)
        return float(e), float(kap)


@pytest.mark.parametrize("kernel", [ow.GAUSSIAN, ow.IMQ])
@pytest.mark.parametrize("kT", [10 ** 20, 10 ** 24])
def test_two_node_closed_form_beyond_float64(kernel, kT):
    r = Decimal("0.5")
    e_true, k_true = _two_node_root(kT, kernel, r)
    assert k_true == pytest.approx(kT, rel=1e-12)
    P = np.array([[0.0, 0.0, 1.0], [0.5, 0.0, 1.0]])
    assert hp.cond2_hp(P, e_true, kernel) == pytest.approx(kT, rel=1e-6)
    e, kap, ev = hp.search_eps_hp(P, kernel, float(kT), xtol=1e-15 * e_true)
    assert e == pytest.approx(e_true, rel=1e-6)
    # float64 cannot even represent the matrix's small eigenvalue here
    assert ow.cond2(ow.interp_matrix(P, e_true, kernel)) < 1e-3 * kT


def test_agrees_with_float64_oracle_at_moderate_kappa():
    ns = W.fibonacci_sphere(400)
    idx = ost.stencil(ns.X, 7, 11)
    P, Nr = ns.X[idx], ns.normals[idx]
    e8, _, _ = ow.search_eps(P, ow.IMQ, 1e8)
    assert hp.cond2_hp(P, e8, ow.IMQ) == pytest.approx(ow.cond2(ow.interp_matrix(P, e8, ow.IMQ)), rel=1e-7)
    w = ow.stencil_weights(P, Nr, e8, ow.IMQ)
    assert np.abs(hp.stencil_weights_hp(P, Nr, e8, ow.IMQ) - w).max() <= 1e-8 * np.abs(w).max()
    eh, _, _ = hp.search_eps_hp(P, ow.IMQ, 1e8)
    assert abs(eh - e8) <= 2e-4


def test_weights_invariants_at_kappa_1e20():
    ns = W.fibonacci_sphere(400)
    idx = ost.stencil(ns.X, 7, 17)
    P, Nr = ns.X[idx], ns.normals[idx]
    e, kap, _ = hp.search_eps_hp(P, ow.IMQ, 1e20)
    assert abs(math.log(kap / 1e20)) < 0.1
    w = hp.stencil_weights_hp(P, Nr, e, ow.IMQ)
    assert abs(w.sum()) <= 1e-14 * np.abs(w).sum()                 # constants are reproduced
    assert np.array_equal(hp.stencil_weights_hp(P, -Nr, e, ow.IMQ), w)   # P = I - n n^T
    u = W.sph_harm_y32(P)
    assert abs(w @ u + 12 * u[0]) <= 1e-2 * 12 * np.abs(u).max()   # Delta Y_3^2 = -12 Y_3^2
