"""GPU parity of the IMEX stepper (reaction + SBDF2 right-hand side +
BiCGSTAB: one cooperative launch per step for small operators, phase kernels
under a device-side loop for large ones) against the oracle's stepper on the
same operator.

Tolerances: float64 stepping at BiCGSTAB tolerance 1e-12 matches the oracle
to 1e-9 relative (both solve the same systems to 1e-12; the difference is
the solver's residual times the system's conditioning).  float32 stepping is
held to the 1e-5 relative L_inf bar against the float64 oracle on the
horizons the parity plan names (heat equation to t = 0.1; reaction-diffusion
over the first 100 steps)."""
import math

import numpy as np
import pytest
import torch

from oracle import operator as oop
from oracle import stepping as ostp
from oracle import weights as ow
from paper_1404_0812_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def T(a, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def rel_inf(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.fixture(scope="module")
def R():
    import paper_1404_0812_gb300 as R
    R._lib.load()
    return R


def _pair(R, ns, n, kernel, kT=1e12):
    """GPU operator (searched eps) and the oracle operator at the GPU's eps."""
    op = R.build_operator(T(ns.X), T(ns.normals), n, kernel=kernel, kappa_target=kT)
    eps = R.get_stencil_info(op)["eps"].cpu().numpy()
    ref = oop.build_operator(ns.X, ns.normals, n, ow.KERNELS[kernel], eps=eps)
    return op, ref


def _pair_fixed(R, ns, n, kernel, eps):
    """Both operators at one fixed eps with kappa ~ 1e6, where the two float64
    weight computations agree to ~1e-13 even on rough fields: float64
    stepper parity is then limited by the stepper alone.  (At kappa_T = 1e12
    the weights of two float64 orderings differ by ~3.5e-6, which a random
    initial state carries straight into the solution.)"""
    e = np.full(ns.N, eps)
    op = R.build_operator(T(ns.X), T(ns.normals), n, kernel=kernel, eps_override=T(e))
    ref = oop.build_operator(ns.X, ns.normals, n, ow.KERNELS[kernel], eps=e)
    return op, ref


@pytest.fixture(scope="module")
def sphere2562(R):
    ns = W.icosahedral_sphere(4)
    return (ns,) + _pair(R, ns, 31, "gaussian")


def test_heat_equation_fp64_parity(R, sphere2562):
    ns, op, ref = sphere2562
    u0 = W.sph_harm_y32(ns.X)
    p = R.StepParams(model="none", nspecies=1, dtype=torch.float64, dt=1e-4, delta_u=1.0, tol=1e-12)
    st = R.StepState.create(T(u0))
    rep = R.step_imex(op, st, p, 50)
    o = ostp.imex_run(lambda x: oop.apply(ref, x), u0, None, dict(model="none", dt=1e-4, delta_u=1.0), 50)
    assert rel_inf(st.u.cpu().numpy(), o["u"]) <= 1e-9
    assert rep["max_iters_u"] <= 3          # Section 6: at most three iterations
    assert st.has_history == 1 and st.step == 50


def test_heat_equation_fp32_to_t01(R, sphere2562):
    """Unit sphere N = 2562, n = 31, Gaussian: u0 = Y_3^2 to t = 0.1 (1000
    steps of 1e-4) in float32 against the float64 oracle stepper, and both
    against the exact exp(-12 t) decay."""
    ns, op, ref = sphere2562
    u0 = W.sph_harm_y32(ns.X)
    p = R.StepParams(model="none", nspecies=1, dtype=torch.float32, dt=1e-4, delta_u=1.0, tol=1e-6)
    st = R.StepState.create(T(u0, torch.float32))
    R.step_imex(op, st, p, 1000)
    o = ostp.imex_run(lambda x: oop.apply(ref, x), u0, None, dict(model="none", dt=1e-4, delta_u=1.0), 1000)
    u = st.u.cpu().numpy().astype(np.float64)
    assert rel_inf(u, o["u"]) <= 1e-5
    exact = math.exp(-1.2) * u0
    assert rel_inf(o["u"], exact) < 1e-3
    assert rel_inf(u, exact) < 1e-3


# float32: BiCGSTAB runs until the recursive residual reaches 1e-8, i.e. to the
# float32 floor; a looser tolerance leaves tol * |b| of error per step, which
# accumulates linearly over the 100 steps.
@pytest.mark.parametrize("dtype,tol,bound", [(torch.float64, 1e-12, 1e-9), (torch.float32, 1e-8, 1e-5)])
def test_schnakenberg_torus_100_steps(R, dtype, tol, bound):
    """Two-species Schnakenberg on the staggered torus (m = 20, N = 2400),
    n = 31, IMQ, 100 steps of dt = 0.01 from the seeded +-1% perturbation of
    the steady state.  float64: fixed eps (kappa ~ 1e6); float32: the
    searched kappa_T = 1e12 operator."""
    ns = W.torus_staggered(20)
    op, ref = _pair_fixed(R, ns, 31, "imq", 5.0) if dtype == torch.float64 else _pair(R, ns, 31, "imq")
    s = W.SCHNAKENBERG
    u0, v0 = W.schnakenberg_initial(ns.N, seed=2)
    name, coef = R.model_coefs(s)
    p = R.StepParams(model=name, nspecies=2, dtype=dtype, dt=s["dt"], delta_u=s["delta_u"],
                     delta_v=s["delta_v"], coef=coef, tol=tol)
    st = R.StepState.create(T(u0, dtype), T(v0, dtype))
    R.step_imex(op, st, p, 100)
    o = ostp.imex_run(lambda x: oop.apply(ref, x), u0, v0, s, 100)
    assert rel_inf(st.u.cpu().numpy().astype(np.float64), o["u"]) <= bound
    assert rel_inf(st.v.cpu().numpy().astype(np.float64), o["v"]) <= bound


@pytest.mark.parametrize("which", ["gray_scott", "barrio"])
def test_other_kinetics_fp64(R, which):
    ns = W.icosahedral_sphere(3)
    op, ref = _pair_fixed(R, ns, 31, "imq", 2.5)
    if which == "gray_scott":
        prm = dict(W.GRAY_SCOTT)
        prm["delta_u"], prm["delta_v"] = 2e-4, 1e-4
        u0, v0 = W.gray_scott_initial(ns.X, seed=5, spots=5, radius=0.3)
    else:
        prm = dict(W.BARRIO_SPOTS)
        rng = np.random.default_rng(9)
        u0, v0 = 0.01 * rng.uniform(-1, 1, ns.N), 0.01 * rng.uniform(-1, 1, ns.N)
    name, coef = R.model_coefs(prm)
    p = R.StepParams(model=name, nspecies=2, dtype=torch.float64, dt=prm["dt"], delta_u=prm["delta_u"],
                     delta_v=prm["delta_v"], coef=coef, tol=1e-12)
    st = R.StepState.create(T(u0), T(v0))
    R.step_imex(op, st, p, 30)
    o = ostp.imex_run(lambda x: oop.apply(ref, x), u0, v0, prm, 30)
    assert rel_inf(st.u.cpu().numpy(), o["u"]) <= 1e-9
    assert rel_inf(st.v.cpu().numpy(), o["v"]) <= 1e-9


def test_split_runs_equal_one_run(R, sphere2562):
    """History carried across calls: 10 + 15 steps equal 25 steps."""
    ns, op, _ = sphere2562
    u0 = W.sph_harm_y32(ns.X)
    p = R.StepParams(model="none", nspecies=1, dtype=torch.float64, dt=1e-3, delta_u=1.0, tol=1e-12)
    a = R.StepState.create(T(u0))
    R.step_imex(op, a, p, 25)
    b = R.StepState.create(T(u0))
    R.step_imex(op, b, p, 10)
    R.step_imex(op, b, p, 15)
    assert torch.equal(a.u, b.u)


def test_steady_state_and_solver_failure(R):
    ns = W.icosahedral_sphere(3)
    op = R.build_operator(T(ns.X), T(ns.normals), 31, kernel="imq", kappa_target=1e12)
    s = W.SCHNAKENBERG
    us, vs = s["a"] + s["b"], s["b"] / (s["a"] + s["b"]) ** 2
    name, coef = R.model_coefs(s)
    p = R.StepParams(model=name, nspecies=2, dtype=torch.float64, dt=0.01, delta_u=s["delta_u"],
                     delta_v=s["delta_v"], coef=coef, tol=1e-12)
    st = R.StepState.create(T(np.full(ns.N, us)), T(np.full(ns.N, vs)))
    R.step_imex(op, st, p, 5)
    assert (st.u - us).abs().max().item() < 1e-10 and (st.v - vs).abs().max().item() < 1e-10
    # an iteration cap of 1 at a tolerance it cannot meet is reported, not hidden
    p2 = R.StepParams(model="none", nspecies=1, dtype=torch.float64, dt=0.5, delta_u=1.0, tol=1e-14,
                      maxit=1)
    st2 = R.StepState.create(T(W.uniform_field(ns.N, 3)))
    rep = R.step_imex(op, st2, p2, 2, allow_failure=True)
    assert rep["status"] == 5 and rep["failed_step"] == 0


def test_bounded_barrier_wait_times_out(R):
    """A barrier wait that nothing satisfies gives up after about a second
    and reports RBFFD_TIMEOUT; the context stays usable afterwards."""
    assert R.selftest_barrier_timeout() == 6
    x = torch.ones(10, device="cuda")
    assert float((x * 2).sum().item()) == 20.0


def test_graph_replay_matches_direct_launches(R):
    """A step captured once into a CUDA graph and replayed gives the same
    bits as direct cooperative launches (two species, float32)."""
    ns = W.torus_staggered(20)
    op = R.build_operator(T(ns.X), T(ns.normals), 31, kernel="imq", kappa_target=1e12)
    s = W.SCHNAKENBERG
    u0, v0 = W.schnakenberg_initial(ns.N, seed=2)
    name, coef = R.model_coefs(s)
    out = []
    for g in (False, True):
        p = R.StepParams(model=name, nspecies=2, dtype=torch.float32, dt=s["dt"], delta_u=s["delta_u"],
                         delta_v=s["delta_v"], coef=coef, tol=1e-6, use_graph=g)
        st = R.StepState.create(T(u0, torch.float32), T(v0, torch.float32))
        R.step_imex(op, st, p, 20)
        R.step_imex(op, st, p, 20)
        out.append((st.u.clone(), st.v.clone()))
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])


def test_bdf4_heat_exact_bootstrap_parity(R, sphere2562):
    """Section 6's time stepping: BDF4 for the heat equation, the three past
    levels taken from the exact solution exp(-12 t) Y_3^2; 100 steps of 1e-4
    in float64 against the oracle's SBDF4 (<= 1e-9), at most three BiCGSTAB
    iterations per step, and the same run in float32 (<= 1e-5)."""
    ns, op, ref = sphere2562
    dt = 1e-4
    y = W.sph_harm_y32(ns.X)
    levels = [math.exp(12 * dt * j) * y for j in (1, 2, 3)]
    o = ostp.imex_run(lambda x: oop.apply(ref, x), y, None, dict(model="none", dt=dt, delta_u=1.0), 100,
                      history=[(lv, None, np.zeros(ns.N), None) for lv in levels], order=4)
    for dtype, tol, bound in ((torch.float64, 1e-12, 1e-9), (torch.float32, 1e-8, 1e-5)):
        p = R.StepParams(model="none", nspecies=1, dtype=dtype, dt=dt, delta_u=1.0, tol=tol, order=4)
        st = R.StepState.create(T(y, dtype), order=4)
        st.u_prev.copy_(T(levels[0], dtype))
        st.u_prev2.copy_(T(levels[1], dtype))
        st.u_prev3.copy_(T(levels[2], dtype))
        st.has_history = 3
        rep = R.step_imex(op, st, p, 100)
        assert rel_inf(st.u.cpu().numpy().astype(np.float64), o["u"]) <= bound
        assert rep["max_iters_u"] <= 3 and st.has_history == 3
    assert rel_inf(o["u"], math.exp(-12 * 0.01) * y) < 2e-5


@pytest.mark.parametrize("order", [3, 4])
def test_sbdf_high_order_two_species_ramp(R, order):
    """Two-species Schnakenberg (fixed-eps torus operator) from no history:
    the first steps climb SBDF1, SBDF2, ... to the requested order, as the
    oracle does; 30 steps in one call and as 7 + 23 (the state carries the
    three past levels across calls); float64 parity <= 1e-9."""
    ns = W.torus_staggered(20)
    op, ref = _pair_fixed(R, ns, 31, "imq", 5.0)
    s = W.SCHNAKENBERG
    u0, v0 = W.schnakenberg_initial(ns.N, seed=2)
    name, coef = R.model_coefs(s)
    o = ostp.imex_run(lambda x: oop.apply(ref, x), u0, v0, s, 30, order=order)
    for split in ((30,), (7, 23)):
        p = R.StepParams(model=name, nspecies=2, dtype=torch.float64, dt=s["dt"], delta_u=s["delta_u"],
                         delta_v=s["delta_v"], coef=coef, tol=1e-12, order=order, use_graph=True)
        st = R.StepState.create(T(u0), T(v0), order=order)
        for k in split:
            R.step_imex(op, st, p, k)
        assert st.has_history == order - 1 and st.step == 30
        assert rel_inf(st.u.cpu().numpy(), o["u"]) <= 1e-9
        assert rel_inf(st.v.cpu().numpy(), o["v"]) <= 1e-9


def test_sbdf4_needs_its_history_buffers(R):
    ns = W.icosahedral_sphere(1)
    op = R.build_operator(T(ns.X), T(ns.normals), 10, kernel="imq", eps_override=T(np.full(ns.N, 2.0)))
    st = R.StepState.create(T(W.sph_harm_y32(ns.X)), order=3)   # no level n-3
    p = R.StepParams(model="none", nspecies=1, dtype=torch.float64, dt=1e-3, order=4)
    with pytest.raises(R.RbffdError) as e:
        R.step_imex(op, st, p, 1)
    assert e.value.status == 1
    with pytest.raises(R.RbffdError):
        R.step_imex(op, st, R.StepParams(model="none", nspecies=1, dtype=torch.float64, dt=1e-3, order=5), 1)


def test_sphere_heat_convergence_bdf4(R):
    """Section 6, diffusion on the sphere: the 30-term series to t = 0.5 with
    BDF4 from the exact solution, kappa_T = 1e5 at N = 642 and grown with N
    so that the mean eps stays fixed; the observed orders in sqrt(N) are
    those the section reports: between two and three for n = 11, close to
    four for n = 17 (relative l2 error against the exact solution)."""
    import bench
    res = bench.sphere_heat_study(R, W, T, torch, stencil_sizes=(11, 17), levels=(3, 4, 5))
    for rows in res.values():
        assert all(r["stencils_ok"] and r["solver_status"] == 0 for r in rows)
        e0 = rows[0]["eps_mean"]
        assert all(abs(r["eps_mean"] / e0 - 1) < 1e-3 for r in rows)
        assert rows[0]["kappa_T"] == 1e5 and rows[1]["kappa_T"] < rows[2]["kappa_T"]
    assert 1.8 <= res["n11"][2]["order_l2"] <= 3.2
    assert 3.3 <= res["n17"][2]["order_l2"] <= 4.7
    assert res["n17"][2]["l2"] < 1e-3


def test_forced_sphere_bdf4_source_parity(R, sphere2562):
    """Section 6's forced diffusion on the sphere (manufactured solution
    exp(-5 t) g with its source exp(-5 t) h taken at t^{n+1}): BDF4 from the
    exact solution, 40 steps of 1e-4 from t = 3e-4, float64 against the
    oracle (<= 1e-9) and float32 (<= 1e-5); the state's time advances."""
    ns, op, ref = sphere2562
    dt = 1e-4
    g, h = W.sphere_forced(ns.X, W.sphere_forced_centers())
    ex = lambda t: math.exp(-5 * t) * g
    o = ostp.imex_run(lambda x: oop.apply(ref, x), ex(3 * dt), None, dict(model="none", dt=dt, delta_u=1.0), 40,
                      history=[(ex(2 * dt), None, np.zeros(ns.N), None), (ex(dt), None, np.zeros(ns.N), None),
                               (ex(0.0), None, np.zeros(ns.N), None)],
                      order=4, source=(-5.0, h, None), t0=3 * dt)
    assert rel_inf(o["u"], ex(o["t"])) < 1e-3
    for dtype, tol, bound in ((torch.float64, 1e-12, 1e-9), (torch.float32, 1e-8, 1e-5)):
        p = R.StepParams(model="none", nspecies=1, dtype=dtype, dt=dt, delta_u=1.0, tol=tol, order=4,
                         source_u=T(h, dtype), source_rate=-5.0, use_graph=True)
        st = R.StepState.create(T(ex(3 * dt), dtype), order=4)
        st.u_prev.copy_(T(ex(2 * dt), dtype))
        st.u_prev2.copy_(T(ex(dt), dtype))
        st.u_prev3.copy_(T(ex(0.0), dtype))
        st.has_history, st.t = 3, 3 * dt
        R.step_imex(op, st, p, 15)
        R.step_imex(op, st, p, 25)        # the device time continues across calls
        assert st.t == pytest.approx(3 * dt + 40 * dt)
        assert rel_inf(st.u.cpu().numpy().astype(np.float64), o["u"]) <= bound


def test_invalid_step_parameters_are_rejected(R):
    ns = W.icosahedral_sphere(1)
    op = R.build_operator(T(ns.X), T(ns.normals), 10, kernel="imq", eps_override=T(np.full(ns.N, 2.0)))
    st = R.StepState.create(T(W.sph_harm_y32(ns.X)))
    for kw in (dict(dt=0.0), dict(tol=0.0), dict(maxit=0), dict(nspecies=3), dict(model="barrio", nspecies=1)):
        base = dict(model="none", nspecies=1, dtype=torch.float64, dt=1e-3)
        base.update(kw)
        with pytest.raises(R.RbffdError) as e:
            R.step_imex(op, st, R.StepParams(**base), 1)
        assert e.value.status == 1, kw
    with pytest.raises(R.RbffdError):     # two species without the v state
        R.step_imex(op, st, R.StepParams(model="none", nspecies=2, dtype=torch.float64, dt=1e-3), 1)


def _csr_rows(R, op, N):
    import scipy.sparse as sps
    idx, w = (t.cpu().numpy() for t in R.get_rows(op))
    n = idx.shape[1]
    return sps.csr_matrix((w.ravel(), (np.repeat(np.arange(N), n), idx.ravel())), shape=(N, N))


@pytest.fixture(scope="module")
def sphere200k(R):
    """200k-node Fibonacci sphere, n = 31, IMQ at a fixed eps: above the
    size (1024 rows per SM) where the stepper switches to the phase-kernel
    path.  The oracle steps with the same operator (its rows as a sparse
    matrix): the parity checked is the stepper's."""
    ns = W.fibonacci_sphere(200_000)
    op = R.build_operator(T(ns.X), T(ns.normals), 31, kernel="imq",
                          eps_override=T(np.full(ns.N, 2.5 * math.sqrt(ns.N / 2562.0))))
    return ns, op, _csr_rows(R, op, ns.N)


@pytest.mark.parametrize("dtype,tol,bound", [(torch.float64, 1e-12, 1e-9), (torch.float32, 1e-8, 1e-5)])
def test_phase_kernel_path_large_operator(R, sphere200k, dtype, tol, bound):
    """Schnakenberg, 20 SBDF2 steps on the phase-kernel path: against the
    oracle's BiCGSTAB steps on the same operator (float64 1e-9, float32
    1e-5: the bars of the cooperative path); the WHILE-graph replay and the
    host-driven loop of the same kernels give the same bits; the loop
    launches five kernels per iteration (the launch counter)."""
    ns, op, L = sphere200k
    s = W.SCHNAKENBERG
    u0, v0 = W.schnakenberg_initial(ns.N, seed=4)
    name, coef = R.model_coefs(s)
    out = []
    for graph in (True, False):
        p = R.StepParams(model=name, nspecies=2, dtype=dtype, dt=s["dt"], delta_u=s["delta_u"],
                         delta_v=s["delta_v"], coef=coef, tol=tol, use_graph=graph)
        st = R.StepState.create(T(u0, dtype), T(v0, dtype))
        n0 = R.launch_count()
        rep = R.step_imex(op, st, p, 20)
        launches = R.launch_count() - n0
        assert rep["status"] == 0
        assert rep["max_iters_u"] >= 1 and launches >= 20 * (2 + 5)
        out.append((st.u.clone(), st.v.clone()))
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])
    o = ostp.imex_run(lambda x: L @ x, u0, v0, s, 20)
    assert rel_inf(out[0][0].cpu().numpy().astype(np.float64), o["u"]) <= bound
    assert rel_inf(out[0][1].cpu().numpy().astype(np.float64), o["v"]) <= bound


def test_phase_kernel_path_one_species_heat(R, sphere200k):
    """One species (the second species' branches off): float64 heat
    equation, 30 SBDF2 steps of Y_3^2 on the phase-kernel path against the
    oracle's steps on the same operator, 1e-9."""
    ns, op, L = sphere200k
    u0 = W.sph_harm_y32(ns.X)
    p = R.StepParams(model="none", nspecies=1, dtype=torch.float64, dt=1e-4, delta_u=1.0, tol=1e-12)
    st = R.StepState.create(T(u0))
    rep = R.step_imex(op, st, p, 30)
    assert rep["status"] == 0 and rep["max_iters_v"] == 0
    o = ostp.imex_run(lambda x: L @ x, u0, None, dict(model="none", dt=1e-4, delta_u=1.0), 30)
    assert rel_inf(st.u.cpu().numpy(), o["u"]) <= 1e-9


def test_phase_kernel_path_ragged_and_unaligned(R):
    """The phase kernels' vector phases move 16-byte groups when the state
    is 16-byte aligned and take the last N mod 4 elements one by one; with
    an unaligned state (a view one element into a buffer) they run element
    by element.  N = 200,003 (N mod 4 = 3), float32 Schnakenberg, 10 SBDF2
    steps: both layouts against the oracle's steps on the same operator
    (1e-5), and against each other (1e-6: the same steps, dot products
    summed in another order)."""
    ns = W.fibonacci_sphere(200_003)
    op = R.build_operator(T(ns.X), T(ns.normals), 31, kernel="imq",
                          eps_override=T(np.full(ns.N, 2.5 * math.sqrt(ns.N / 2562.0))))
    L = _csr_rows(R, op, ns.N)
    s = W.SCHNAKENBERG
    u0, v0 = W.schnakenberg_initial(ns.N, seed=6)
    name, coef = R.model_coefs(s)
    p = R.StepParams(model=name, nspecies=2, dtype=torch.float32, dt=s["dt"], delta_u=s["delta_u"],
                     delta_v=s["delta_v"], coef=coef, tol=1e-8, use_graph=True)
    o = ostp.imex_run(lambda x: L @ x, u0, v0, s, 10)
    out = []
    for offset in (0, 1):
        bu = torch.zeros(ns.N + 1, dtype=torch.float32, device="cuda")
        bv = torch.zeros(ns.N + 1, dtype=torch.float32, device="cuda")
        u, v = bu[offset:offset + ns.N], bv[offset:offset + ns.N]
        u.copy_(T(u0, torch.float32))
        v.copy_(T(v0, torch.float32))
        assert (u.data_ptr() % 16 == 0) == (offset == 0)
        st = R.StepState.create(u, v)
        rep = R.step_imex(op, st, p, 10)
        assert rep["status"] == 0
        uu, vv = st.u.cpu().numpy().astype(np.float64), st.v.cpu().numpy().astype(np.float64)
        assert rel_inf(uu, o["u"]) <= 1e-5 and rel_inf(vv, o["v"]) <= 1e-5
        out.append((uu, vv))
    assert rel_inf(out[0][0], out[1][0]) <= 1e-6 and rel_inf(out[0][1], out[1][1]) <= 1e-6
