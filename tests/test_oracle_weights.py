"""Pins of the oracle's weights, condition number and shape-parameter search
against facts the paper and the mathematics fix (not against the oracle's own
formulas): closed forms, the paper's singular-value definition of kappa,
finite differences, exact reproduction properties, invariances, and the
accuracy / convergence behaviour Section 6 reports."""
import math

import numpy as np
import pytest

from oracle import weights as ow
from oracle import stencils as ost
from oracle import operator as oop
from paper_1404_0812_gb300 import workloads as W


def _rot(seed):
    q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((3, 3)))
    return q * np.sign(np.linalg.det(q))


@pytest.fixture(scope="module")
def sphere642():
    return W.icosahedral_sphere(3)


def _stencil(ns, k, n):
    idx = ost.stencil(ns.X, k, n)
    return ns.X[idx], ns.normals[idx]


# --------------------------------------------------------------------------
# kappa and the eps search: n = 2 closed form (Section 5, Eq. target_cond)
# --------------------------------------------------------------------------

def _kappa_n2(a):
    """Eigenvalues of [[1,a,1],[a,1,1],[1,1,0]]: 1-a and ((1+a) +- sqrt((1+a)^2+8))/2."""
    s = 1.0 + a
    lp = 0.5 * (s + math.sqrt(s * s + 8.0))
    lm = 0.5 * (s - math.sqrt(s * s + 8.0))
    return max(abs(lp), abs(lm), abs(1 - a)) / min(abs(lp), abs(lm), abs(1 - a))


@pytest.mark.parametrize("kernel", [ow.GAUSSIAN, ow.IMQ])
@pytest.mark.parametrize("eps", [0.05, 0.3, 1.0, 4.0])
def test_cond2_two_node_closed_form(kernel, eps):
    r = 0.7
    P = np.array([[0.1, 0.2, 0.3], [0.1 + r, 0.2, 0.3]])
    a = math.exp(-(eps * r) ** 2) if kernel == ow.GAUSSIAN else 1 / math.sqrt(1 + (eps * r) ** 2)
    got = ow.cond2(ow.interp_matrix(P, eps, kernel))
    assert got == pytest.approx(_kappa_n2(a), rel=1e-9)


@pytest.mark.parametrize("kernel", [ow.GAUSSIAN, ow.IMQ])
@pytest.mark.parametrize("kT", [1e3, 1e5])
def test_eps_root_two_node_closed_form(kernel, kT):
    """Solve lambda_+(a) = kT (1 - a) exactly (quadratic in s = 1 + a) and
    compare with the oracle's search to its 1e-4 tolerance (Section 5)."""
    r = 0.5
    A2, B2, C2 = kT * kT + kT, -2 * kT * (2 * kT + 1), 4 * kT * kT - 2
    disc = math.sqrt(B2 * B2 - 4 * A2 * C2)
    cands = [(-B2 - disc) / (2 * A2), (-B2 + disc) / (2 * A2)]
    s = [c for c in cands if 1 < c < 2 and 2 * kT * (2 - c) - c >= 0][0]
    a = s - 1.0
    lm = abs(0.5 * (s - math.sqrt(s * s + 8)))
    assert 1 - a < lm  # the small eigenvalue is 1 - a in this regime
    eps_true = math.sqrt(-math.log(a)) / r if kernel == ow.GAUSSIAN else math.sqrt(1 / a ** 2 - 1) / r
    P = np.array([[0.0, 0.0, 1.0], [r, 0.0, 1.0]])
    eps, kap, ev = ow.search_eps(P, kernel, kT, xtol=1e-4)
    assert abs(eps - eps_true) <= 1e-4
    assert ev >= 2


def test_cond2_equals_singular_value_ratio(sphere642):
    """Section 5 defines kappa as sigma_max / sigma_min; the oracle uses
    |eigenvalues| of the symmetric A.  Check with an SVD."""
    P, _ = _stencil(sphere642, 5, 31)
    for eps, rel in ((8.0, 1e-10), (3.0, 1e-8), (1.0, 1e-4)):
        A = ow.interp_matrix(P, eps, ow.GAUSSIAN)
        sv = np.linalg.svd(A, compute_uv=False)
        assert ow.cond2(A) == pytest.approx(sv.max() / sv.min(), rel=rel)


def test_kappa_monotone_in_eps(sphere642):
    """Section 5: kappa grows monotonically as eps decreases."""
    P, _ = _stencil(sphere642, 11, 31)
    ks = [ow.cond2(ow.interp_matrix(P, e, ow.IMQ)) for e in np.geomspace(20, 0.6, 25)]
    assert all(b > a for a, b in zip(ks, ks[1:]))


def test_brent_on_known_roots():
    r, ev = ow.brent_root(lambda x: x ** 3 - 2.0, 0.0, 3.0, -2.0, 25.0, 1e-10)
    assert abs(r - 2.0 ** (1 / 3)) < 1e-10
    f = lambda x: math.log(x) + 5.0
    r, _ = ow.brent_root(f, 1e-4, 1.0, f(1e-4), f(1.0), 1e-9)
    assert abs(r - math.exp(-5.0)) < 1e-9
    with pytest.raises(ValueError):
        ow.brent_root(f, 1.0, 2.0, f(1.0), f(2.0), 1e-6)


def test_search_hits_target_condition(sphere642):
    P, _ = _stencil(sphere642, 200, 31)
    eps, kap, ev = ow.search_eps(P, ow.GAUSSIAN, 1e12, xtol=1e-4)
    # F(eps +- 1e-4) brackets zero: kappa is on target to the eps tolerance
    f = lambda e: math.log(ow.cond2(ow.interp_matrix(P, e, ow.GAUSSIAN)) / 1e12)
    assert f(eps - 2e-4) > 0 > f(eps + 2e-4)
    assert abs(math.log(kap / 1e12)) < 0.05


# --------------------------------------------------------------------------
# the gradient matrices (Eq. grad_x_f_interp) against finite differences
# --------------------------------------------------------------------------

@pytest.mark.parametrize("kernel", [ow.GAUSSIAN, ow.IMQ])
def test_B_is_projected_gradient(sphere642, kernel):
    P, nr = _stencil(sphere642, 7, 10)
    eps = 2.5
    B = ow.grad_matrices(P, nr, eps, kernel)
    h = 1e-6

    def phi_at(x, xj):
        r = np.linalg.norm(x - xj)
        return math.exp(-(eps * r) ** 2) if kernel == ow.GAUSSIAN else 1 / math.sqrt(1 + (eps * r) ** 2)

    for i in range(4):
        Pi = np.eye(3) - np.outer(nr[i], nr[i])
        for j in range(10):
            g = np.array([(phi_at(P[i] + h * e, P[j]) - phi_at(P[i] - h * e, P[j])) / (2 * h)
                          for e in np.eye(3)])
            np.testing.assert_allclose(B[:, i, j], Pi @ g, atol=1e-8)
    assert np.all(B[:, :, 10] == 0.0)
    # projector: P n = 0 and P^2 = P (Eq. proj_mat)
    Pr = ow.projectors(nr)
    np.testing.assert_allclose(np.einsum("kij,kj->ki", Pr, nr), 0, atol=1e-15)
    np.testing.assert_allclose(Pr @ Pr, Pr, atol=1e-15)


# --------------------------------------------------------------------------
# exact reproduction properties of the local operators (Section 4)
# --------------------------------------------------------------------------

def test_constants_and_kernel_differences_reproduced(sphere642):
    """G^d 1 = 0 (constants have zero gradient) and, for f = phi_k - phi_l
    (coefficients summing to zero, so the interpolant is f itself),
    G^d f = B^d[:, k] - B^d[:, l]."""
    P, nr = _stencil(sphere642, 42, 31)
    eps = 6.0  # kappa ~ 1e6: rounding far below the checked tolerance
    G = ow.diff_matrices(P, nr, eps, ow.GAUSSIAN)
    B = ow.grad_matrices(P, nr, eps, ow.GAUSSIAN)
    Phi = ow.interp_matrix(P, eps, ow.GAUSSIAN)[:31, :31]
    scale = np.abs(B).max()
    np.testing.assert_allclose(G @ np.ones(31), 0.0, atol=1e-9 * scale)
    for k, l in ((0, 5), (3, 30), (17, 2)):
        np.testing.assert_allclose(G @ (Phi[:, k] - Phi[:, l]), B[:, :, k] - B[:, :, l],
                                   atol=1e-8 * scale)


@pytest.mark.parametrize("kernel", [ow.GAUSSIAN, ow.IMQ])
def test_row_sums_vanish(sphere642, kernel):
    P, nr = _stencil(sphere642, 99, 31)
    eps, _, _ = ow.search_eps(P, kernel, 1e12)
    w = ow.stencil_weights(P, nr, eps, kernel)
    assert abs(w.sum()) <= 1e-9 * np.abs(w).sum()


def test_invariances(sphere642):
    """Rigid motion of (X, normals), normal sign, and order of the non-centre
    neighbours leave the weights unchanged (up to rounding); scaling X by s
    and eps by 1/s scales the weights by 1/s^2."""
    P, nr = _stencil(sphere642, 300, 31)
    eps = 5.0
    w = ow.stencil_weights(P, nr, eps, ow.IMQ)
    Q = _rot(3)
    w_rot = ow.stencil_weights(P @ Q.T + np.array([0.3, -2.0, 1.0]), nr @ Q.T, eps, ow.IMQ)
    np.testing.assert_allclose(w_rot, w, rtol=0, atol=1e-8 * np.abs(w).max())
    w_flip = ow.stencil_weights(P, -nr, eps, ow.IMQ)
    np.testing.assert_allclose(w_flip, w, rtol=0, atol=1e-10 * np.abs(w).max())
    perm = np.concatenate([[0], 1 + np.random.default_rng(0).permutation(30)])
    w_perm = ow.stencil_weights(P[perm], nr[perm], eps, ow.IMQ)
    np.testing.assert_allclose(w_perm, w[perm], rtol=0, atol=1e-8 * np.abs(w).max())
    s = 3.0
    w_s = ow.stencil_weights(s * P, nr, eps / s, ow.IMQ)
    np.testing.assert_allclose(w_s, w / s ** 2, rtol=0, atol=1e-8 * np.abs(w).max() / s ** 2)


# --------------------------------------------------------------------------
# accuracy: Laplace-Beltrami eigenfunctions (Section 6) and the torus
# --------------------------------------------------------------------------

def _y44(X):
    x, y, _ = X.T
    return x ** 4 - 6 * x * x * y * y + y ** 4      # degree 4, eigenvalue -20


def test_sphere_harmonic_at_target_condition(sphere642):
    """Delta_M Y_3^2 = -12 Y_3^2 on the unit sphere (N = 642, n = 31,
    kappa_T = 1e12, Gaussian and IMQ)."""
    u = W.sph_harm_y32(sphere642.X)
    for kernel, bound in ((ow.GAUSSIAN, 5e-4), (ow.IMQ, 1e-3)):
        op = oop.build_operator(sphere642.X, sphere642.normals, 31, kernel, kappa_T=1e12)
        y = oop.apply(op, u)
        assert np.abs(y + 12 * u).max() / np.abs(12 * u).max() < bound
        assert np.all(op.evals >= 2)


def test_convergence_rate_fixed_eps():
    """Section 6: n = 17 converges at close to order 4 in h ~ N^(-1/2).  With
    eps fixed (the paper's growing-kappa_T regime), the error of
    Delta_M of a degree-4 harmonic falls at an order in [3, 5] from N = 642
    to 2562 (h halves)."""
    errs = []
    for lev in (3, 4):
        ns = W.icosahedral_sphere(lev)
        op = oop.build_operator(ns.X, ns.normals, 17, ow.GAUSSIAN, eps=1.0)
        u = _y44(ns.X)
        errs.append(np.abs(oop.apply(op, u) + 20 * u).max() / np.abs(20 * u).max())
    order = math.log2(errs[0] / errs[1])
    assert 3.0 <= order <= 5.0


def _torus_u_and_lap(vp, la, centres, a=9.0, b=3.0):
    """The manufactured torus function of Eq. torus_forced at t = 0 and its
    Laplacian from the intrinsic formula of Section 6 (derivatives by hand)."""
    u = np.zeros_like(vp)
    lap = np.zeros_like(vp)
    rho = 1.0 + np.cos(vp) / 3.0
    for vk, lk in centres:
        g = np.exp(-a * a * (1 - np.cos(la - lk)) - b * b * (1 - np.cos(vp - vk)))
        g_ll = g * (a ** 4 * np.sin(la - lk) ** 2 - a * a * np.cos(la - lk))
        g_v = g * (-b * b * np.sin(vp - vk))
        g_vv = g * (b ** 4 * np.sin(vp - vk) ** 2 - b * b * np.cos(vp - vk))
        u += g
        lap += g_ll / rho ** 2 + 9.0 / rho * (-np.sin(vp) / 3.0 * g_v + rho * g_vv)
    return u, lap


def test_torus_manufactured_laplacian():
    ns = W.torus_staggered(20)   # N = 2400 (a Section 6 size)
    assert ns.N == 2400
    cen = np.random.default_rng(7).uniform(-np.pi, np.pi, (3, 2))
    u, lap = _torus_u_and_lap(ns.extra["varphi"], ns.extra["lam"], cen)
    rows = np.arange(0, ns.N, 7)
    op = oop.build_operator(ns.X, ns.normals, 31, ow.IMQ, kappa_T=1e12, rows=rows)
    y = oop.apply(op, u)
    err = np.abs(y - lap[rows]).max() / np.abs(lap).max()
    assert err < 2e-2
