"""Pins of the oracle's method-of-lines stepping (Section 4.2, Section 6,
Section 7): BiCGSTAB against a dense direct solve, SBDF2 against the
closed-form recurrence of a scalar linear test problem, fixed points of the
kinetics, exact heat-equation decay of a spherical harmonic, and the
iteration counts Section 6 reports."""
import json
import cmath
import math
import os

import numpy as np
import pytest

from oracle import operator as oop
from oracle import stepping as ostp
from oracle import weights as ow
from paper_1404_0812_gb300 import workloads as W

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


@pytest.fixture(scope="module")
def op642():
    ns = W.icosahedral_sphere(3)
    return ns, oop.build_operator(ns.X, ns.normals, 31, ow.GAUSSIAN, kappa_T=1e12)


def test_bicgstab_matches_dense_solve(op642):
    ns, op = op642
    L = oop.dense(op, ns.N)
    A = 3.0 * np.eye(ns.N) - 2 * 0.05 * L
    b = W.uniform_field(ns.N, seed=11)
    x, it, rel, ok = ostp.bicgstab(lambda v: A @ v, b, np.zeros(ns.N), 1e-13, 500)
    assert ok and rel <= 1e-13
    xd = np.linalg.solve(A, b)
    assert np.abs(x - xd).max() <= 1e-11 * np.abs(xd).max()


def _sbdf2_closed_form(lam, mu, dt, u0, n):
    """Scalar problem u' = -lam u + mu u (L = -I, diffusion lam): step 1 is
    IMEX Euler, then (3 + 2 lam dt) u+ = (4 + 4 mu dt) u - (1 + 2 mu dt) u-,
    whose solution is A r1^n + B r2^n with r the roots of the characteristic
    quadratic."""
    u1 = (1.0 + dt * mu) * u0 / (1.0 + dt * lam)
    a, b, cc = 3.0 + 2.0 * lam * dt, -(4.0 + 4.0 * mu * dt), 1.0 + 2.0 * mu * dt
    disc = cmath.sqrt(b * b - 4 * a * cc)
    r1, r2 = (-b + disc) / (2 * a), (-b - disc) / (2 * a)
    B = (u1 - r1 * u0) / (r2 - r1)
    A = u0 - B
    return (A * r1 ** n + B * r2 ** n).real


def test_sbdf2_recurrence_closed_form():
    lam, mu, dt = 7.0, 0.6, 0.05
    p = dict(model="linear", lu=mu, lv=-mu, dt=dt, delta_u=1.0, delta_v=2.0)
    u0 = np.array([1.0, -0.5, 2.0])
    v0 = np.array([0.3, 0.1, -1.0])
    out = ostp.imex_run(lambda x: -lam * x, u0, v0, p, 40, tol=1e-14)
    ref_u = _sbdf2_closed_form(lam * 1.0, mu, dt, 1.0, 40)
    ref_v = _sbdf2_closed_form(lam * 2.0, -mu, dt, 1.0, 40)
    np.testing.assert_allclose(out["u"], u0 * ref_u, rtol=1e-12)
    np.testing.assert_allclose(out["v"], v0 * ref_v, rtol=1e-12)


def test_kinetics_fixed_points():
    # Section 7: with alpha = -gamma, (0, 0) is an equilibrium; the linear part
    # of Eqs. turing1/turing2 at the origin is [[alpha, 1], [gamma, beta]].
    row = GOLDEN["turing_table"]["rows"][0]
    p = dict(model="barrio", **{k: row[k] for k in ("alpha", "beta", "gamma", "tau1", "tau2")})
    assert p["alpha"] == -p["gamma"]
    z = np.zeros(1)
    f, g = ostp.reaction(p, z, z)
    assert f[0] == 0.0 and g[0] == 0.0
    h = 1e-7
    fu, gu = ostp.reaction(p, z + h, z)
    fv, gv = ostp.reaction(p, z, z + h)
    J = np.array([[fu[0], fv[0]], [gu[0], gv[0]]]) / h
    np.testing.assert_allclose(J, [[p["alpha"], 1.0], [p["gamma"], p["beta"]]], atol=1e-6)
    assert W.BARRIO_SPOTS["delta_u"] == pytest.approx(
        GOLDEN["turing_table"]["delta_u_over_delta_v"] * W.BARRIO_SPOTS["delta_v"])
    s = W.SCHNAKENBERG
    us, vs = s["a"] + s["b"], s["b"] / (s["a"] + s["b"]) ** 2
    f, g = ostp.reaction(s, np.array([us]), np.array([vs]))
    assert abs(f[0]) < 1e-15 and abs(g[0]) < 1e-15
    f, g = ostp.reaction(W.GRAY_SCOTT, np.ones(1), np.zeros(1))
    assert f[0] == 0.0 and g[0] == 0.0


def test_steady_state_stays_constant(op642):
    ns, op = op642
    s = W.SCHNAKENBERG
    u = np.full(ns.N, s["a"] + s["b"])
    v = np.full(ns.N, s["b"] / (s["a"] + s["b"]) ** 2)
    out = ostp.imex_run(lambda x: oop.apply(op, x), u, v, s, 5)
    assert np.abs(out["u"] - u).max() < 1e-10 and np.abs(out["v"] - v).max() < 1e-10


def test_heat_equation_decay_and_iteration_count(op642):
    """u0 = Y_3^2 decays as exp(-12 t) (Section 6 series with l = 3); at
    dt = 1e-4 BiCGSTAB needs at most three iterations per step to a relative
    tolerance of 1e-12 (Section 6)."""
    ns, op = op642
    g = GOLDEN["bicgstab_bdf"]
    u0 = W.sph_harm_y32(ns.X)
    p = dict(model="none", dt=g["dt"], delta_u=1.0)
    out = ostp.imex_run(lambda x: oop.apply(op, x), u0, None, p, 100, tol=g["tol"])
    err = np.abs(out["u"] - math.exp(-12 * 0.01) * u0).max() / np.abs(u0).max()
    assert err < 2e-5
    assert max(i for i, _ in out["iters"]) <= g["max_iters"]


def _scalar_run(order, lam, mu, dt, T):
    """u' = -lam u + mu u (L = -I with delta = lam; f = mu u), u(0) = 1, the
    order-1 past levels taken from the exact solution exp((mu - lam) t)."""
    r = mu - lam
    hist = [(np.array([math.exp(-r * dt * j)]), None, np.array([mu * math.exp(-r * dt * j)]), None)
            for j in range(1, order)]
    p = dict(model="linear", lu=mu, lv=0.0, dt=dt, delta_u=lam)
    n = int(round(T / dt))
    out = ostp.imex_run(lambda x: -x, np.array([1.0]), None, p, n, tol=1e-15, history=hist or None,
                        order=order)
    return abs(out["u"][0] - math.exp(r * n * dt))


@pytest.mark.parametrize("order", [1, 2, 3, 4])
def test_sbdf_order_of_accuracy(order):
    """SBDFk is k-th order: with exact past levels, halving dt divides the
    error at t = 1 by about 2^k -- separately for the implicit (diffusion)
    and the explicit (kinetics) part, so every coefficient of both halves of
    the scheme is pinned (a wrong one lowers the order)."""
    for lam, mu in ((3.0, 0.0), (0.0, 1.5)):
        e1 = _scalar_run(order, lam, mu, 0.02, 1.0)
        e2 = _scalar_run(order, lam, mu, 0.01, 1.0)
        rate = math.log2(e1 / e2)
        assert abs(rate - order) < 0.25, (order, lam, mu, rate)


def test_sbdf4_recurrence_closed_form():
    """Scalar problem with L = -I: SBDF4 is the linear recurrence
    u^{n+1} = sum_j c_j u^{n-j}; its solution is sum_i C_i z_i^n with z_i the
    roots of the characteristic quartic (C from the four starting values)."""
    lam, mu, dt = 4.0, 0.7, 0.03
    alpha, a, b = 25.0 / 12.0, (4.0, -3.0, 4.0 / 3.0, -0.25), (4.0, -6.0, 4.0, -1.0)
    c = [(a[j] + dt * mu * b[j]) / (alpha + dt * lam) for j in range(4)]
    z = np.roots([1.0, -c[0], -c[1], -c[2], -c[3]])
    start = np.array([1.0, 0.9, 0.83, 0.71])          # u^0, u^-1, u^-2, u^-3
    V = np.array([[zi ** (-m) for zi in z] for m in range(4)])
    C = np.linalg.solve(V, start.astype(complex))
    n = 30
    ref = float(np.real(np.sum(C * z ** n)))
    hist = [(np.array([start[j]]), None, np.array([mu * start[j]]), None) for j in range(1, 4)]
    p = dict(model="linear", lu=mu, lv=0.0, dt=dt, delta_u=lam)
    out = ostp.imex_run(lambda x: -x, np.array([start[0]]), None, p, n, tol=1e-15, history=hist, order=4)
    assert abs(out["u"][0] - ref) <= 1e-12 * abs(ref)


def test_heat_equation_bdf4_exact_bootstrap(op642):
    """Section 6's setting: BDF4 for the heat equation on the sphere started
    from the exact solution (three past levels of exp(-12 t) Y_3^2); the
    error at t = 0.01 is the spatial error of L_X (as for SBDF2) and BiCGSTAB
    needs at most three iterations per step at dt = 1e-4."""
    ns, op = op642
    g = GOLDEN["bicgstab_bdf"]
    dt = g["dt"]
    y = W.sph_harm_y32(ns.X)
    hist = [(math.exp(12 * dt * j) * y, None, np.zeros(ns.N), None) for j in range(1, 4)]
    p = dict(model="none", dt=dt, delta_u=1.0)
    out = ostp.imex_run(lambda x: oop.apply(op, x), y, None, p, 100, tol=g["tol"], history=hist, order=4)
    err = np.abs(out["u"] - math.exp(-12 * 0.01) * y).max() / np.abs(y).max()
    assert err < 2e-5
    assert max(i for i, _ in out["iters"]) <= g["max_iters"]
    assert len(out["levels"]) == 3


@pytest.mark.parametrize("order", [1, 2, 3, 4])
def test_implicit_source_keeps_order(order):
    """u' = -lam u + exp(c t) h has the exact solution
    u = (u0 - h/(c+lam)) exp(-lam t) + h exp(c t)/(c+lam); with exact past
    levels SBDF-k keeps order k only if the source is taken at t^{n+1} (a
    source at t^n would cost the scheme its order)."""
    lam, c, h, T = 2.0, -1.0, 2.0, 1.0
    exact = lambda t: (1.0 - h / (c + lam)) * math.exp(-lam * t) + h * math.exp(c * t) / (c + lam)
    errs = []
    for dt in (0.02, 0.01):
        hist = [(np.array([exact(-dt * j)]), None, np.zeros(1), None) for j in range(1, order)]
        p = dict(model="none", dt=dt, delta_u=lam)
        n = int(round(T / dt))
        out = ostp.imex_run(lambda x: -x, np.array([exact(0.0)]), None, p, n, tol=1e-15,
                            history=hist or None, order=order, source=(c, np.array([h]), None))
        assert out["t"] == pytest.approx(T)
        errs.append(abs(out["u"][0] - exact(T)))
    assert abs(math.log2(errs[0] / errs[1]) - order) < 0.3


def _monomials(fn, deg=3):
    """Coefficients c[a, b] of u^a v^b (a, b <= deg) of the polynomial fn(u, v),
    recovered exactly (to rounding) by interpolation on a (deg+1)^2 grid: a
    polynomial of that bidegree is determined by its values there."""
    pts = np.arange(deg + 1, dtype=np.float64) - 1.0      # -1, 0, 1, 2
    U, V = np.meshgrid(pts, pts, indexing="ij")
    Vd = np.polynomial.polynomial.polyvander2d(U.ravel(), V.ravel(), [deg, deg])
    return np.linalg.solve(Vd, fn(U.ravel(), V.ravel())).reshape(deg + 1, deg + 1)


def _expect(terms, deg=3):
    c = np.zeros((deg + 1, deg + 1))
    for (a, b), val in terms.items():
        c[a, b] = val
    return c


def test_barrio_kinetics_every_term():
    """Eqs. turing1/turing2 with Table tur_param's constants: every monomial of
    f = alpha u - alpha tau1 u v^2 + v - tau2 u v and of
    g = beta v + alpha tau1 u v^2 + gamma u + tau2 u v has the coefficient the
    equations give, and no other monomial appears (a dropped term, a wrong
    sign or u^2 v for u v^2 changes one of them)."""
    for row in GOLDEN["turing_table"]["rows"]:
        p = dict(model="barrio", **{k: row[k] for k in ("alpha", "beta", "gamma", "tau1", "tau2")})
        a, b, g, t1, t2 = p["alpha"], p["beta"], p["gamma"], p["tau1"], p["tau2"]
        cf = _monomials(lambda u, v: ostp.reaction(p, u, v)[0])
        cg = _monomials(lambda u, v: ostp.reaction(p, u, v)[1])
        np.testing.assert_allclose(cf, _expect({(1, 0): a, (1, 2): -a * t1, (0, 1): 1.0, (1, 1): -t2}),
                                   atol=1e-12)
        np.testing.assert_allclose(cg, _expect({(0, 1): b, (1, 2): a * t1, (1, 0): g, (1, 1): t2}),
                                   atol=1e-12)
        # the mixed derivatives at the origin that the terms above fix
        assert cf[1, 1] == pytest.approx(-t2, abs=1e-12) and 2 * cf[1, 2] == pytest.approx(-2 * a * t1)
        assert cg[1, 1] == pytest.approx(t2, abs=1e-12) and 2 * cg[1, 2] == pytest.approx(2 * a * t1)


def test_gray_scott_kinetics_every_term_and_double_root():
    """Gray-Scott f = -u v^2 + F (1 - u), g = u v^2 - (F + k) v: every monomial,
    the Jacobian diag(-F, -(F + k)) at the trivial state (1, 0), and for
    F = 0.04, k = 0.06 -- where F^2 = 4 F (F + k)^2, so the two nontrivial
    equilibria merge -- the double root (u, v) = (1/2, 1/5) with f = g = 0
    there and a singular Jacobian (a saddle-node)."""
    p = W.GRAY_SCOTT
    F, k = p["F"], p["k"]
    cf = _monomials(lambda u, v: ostp.reaction(p, u, v)[0])
    cg = _monomials(lambda u, v: ostp.reaction(p, u, v)[1])
    np.testing.assert_allclose(cf, _expect({(0, 0): F, (1, 0): -F, (1, 2): -1.0}), atol=1e-13)
    np.testing.assert_allclose(cg, _expect({(1, 2): 1.0, (0, 1): -(F + k)}), atol=1e-13)
    assert F * F == pytest.approx(4 * F * (F + k) ** 2, rel=1e-12)
    us, vs = (F + k) / (F / (2 * (F + k))), F / (2 * (F + k))
    assert (us, vs) == (pytest.approx(0.5), pytest.approx(0.2))
    f, g = ostp.reaction(p, np.array([us]), np.array([vs]))
    assert abs(f[0]) < 1e-16 and abs(g[0]) < 1e-16

    def jac(u0, v0, h=1e-6):
        fu = (np.array(ostp.reaction(p, np.array([u0 + h]), np.array([v0])))
              - np.array(ostp.reaction(p, np.array([u0 - h]), np.array([v0])))) / (2 * h)
        fv = (np.array(ostp.reaction(p, np.array([u0]), np.array([v0 + h])))
              - np.array(ostp.reaction(p, np.array([u0]), np.array([v0 - h])))) / (2 * h)
        return np.array([[fu[0, 0], fv[0, 0]], [fu[1, 0], fv[1, 0]]])

    np.testing.assert_allclose(jac(1.0, 0.0), [[-F, 0.0], [0.0, -(F + k)]], atol=1e-9)
    J = jac(us, vs)
    np.testing.assert_allclose(J, [[-vs * vs - F, -2 * us * vs], [vs * vs, 2 * us * vs - (F + k)]], atol=1e-9)
    assert abs(np.linalg.det(J)) < 1e-9


def test_schnakenberg_kinetics_every_term():
    """Schnakenberg f = gamma (a - u + u^2 v), g = gamma (b - u^2 v)."""
    p = W.SCHNAKENBERG
    a, b, g = p["a"], p["b"], p["gamma"]
    cf = _monomials(lambda u, v: ostp.reaction(p, u, v)[0])
    cg = _monomials(lambda u, v: ostp.reaction(p, u, v)[1])
    np.testing.assert_allclose(cf, _expect({(0, 0): g * a, (1, 0): -g, (2, 1): g}), atol=1e-13)
    np.testing.assert_allclose(cg, _expect({(0, 0): g * b, (2, 1): -g}), atol=1e-13)


def test_sparse_lu_solver_matches_dense_and_bicgstab(op642):
    """Section 7's direct solves: the oracle's sparse-LU SBDF2 steps equal the
    same steps with each implicit system solved densely (numpy), and the
    BiCGSTAB steps to their tolerance; the sparse matrix is the operator's."""
    ns, op = op642
    L = oop.sparse_matrix(op, ns.N)
    Ld = oop.dense(op, ns.N)
    assert np.array_equal(L.toarray(), Ld)
    s = W.SCHNAKENBERG
    u0, v0 = W.schnakenberg_initial(ns.N, seed=2)
    lu = ostp.imex_run(lambda x: oop.apply(op, x), u0, v0, s, 20, solver="lu", L_matrix=L)
    bi = ostp.imex_run(lambda x: oop.apply(op, x), u0, v0, s, 20, tol=1e-14)
    assert all(i == (0, 0) for i in lu["iters"])
    for k in ("u", "v"):
        assert np.abs(lu[k] - bi[k]).max() <= 1e-11 * np.abs(bi[k]).max()
    # one SBDF1 step by hand with a dense solve
    f, g = ostp.reaction(s, u0, v0)
    M = np.eye(ns.N) - s["dt"] * s["delta_u"] * Ld
    one = ostp.imex_run(lambda x: oop.apply(op, x), u0, v0, s, 1, solver="lu", L_matrix=L)
    ref = np.linalg.solve(M, u0 + s["dt"] * f)
    assert np.abs(one["u"] - ref).max() <= 1e-13 * np.abs(ref).max()
