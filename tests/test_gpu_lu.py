"""GPU banded LU (Section 7: the SBDF2 matrix factorised once, a forward and
a back substitution per step) against dense solves and the oracle's
sparse-LU stepping.

Tolerances: float64 factor and solve of a matrix with condition number
~10-100 against numpy's dense solve of the same matrix: 1e-12 relative
(two backward-stable solves); float32: 1e-5.  Stepping: float64 against
the oracle's sparse-LU steps driven by the same operator: 1e-9 (the
stepping tolerance of the float64 path); float32: 1e-5.
"""
import numpy as np
import pytest
import scipy.sparse as sps
import torch

from oracle import stepping as ostp
from paper_1404_0812_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def T(a, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


@pytest.fixture(scope="module")
def R():
    import paper_1404_0812_gb300 as R
    R._lib.load()
    return R


def _rcm_built(R, ns, n, kernel="imq", kappa=1e10):
    """Build, renumber by the library's reverse Cuthill-McKee, rebuild."""
    op = R.build_operator(T(ns.X), T(ns.normals), n, kernel=kernel, kappa_target=kappa)
    perm = R.rcm_order(op).cpu().numpy()
    X, Nr = ns.X[perm].copy(), ns.normals[perm].copy()
    return R.build_operator(T(X), T(Nr), n, kernel=kernel, kappa_target=kappa), X, Nr, perm


def _matrix(R, op, N):
    idx, w = (t.cpu().numpy() for t in R.get_rows(op))
    n = idx.shape[1]
    return sps.csr_matrix((w.ravel(), (np.repeat(np.arange(N), n), idx.ravel())), shape=(N, N))


@pytest.mark.parametrize("order", ["rcm", "natural"])
def test_lu_solve_matches_dense(R, order):
    ns = W.icosahedral_sphere(4 if order == "rcm" else 3)
    if order == "rcm":
        op, X, Nr, _ = _rcm_built(R, ns, 31)
    else:
        op = R.build_operator(T(ns.X), T(ns.normals), 31, kernel="imq", kappa_target=1e10)
    N = ns.N
    kl, ku = R.op_bandwidth(op)
    L = _matrix(R, op, N)
    coo = L.tocoo()
    assert kl == int((coo.row - coo.col).max()) and ku == int((coo.col - coo.row).max())
    if order == "rcm":
        assert kl + ku < N / 4     # the renumbering made it banded
    alpha, beta = 3.0, 2 * 1e-3
    M = alpha * np.eye(N) - beta * L.toarray()
    b = W.uniform_field(N, seed=3)
    xr = np.linalg.solve(M, b)
    lu = R.lu_factor(op, alpha, beta, torch.float64)
    x = R.lu_solve(lu, T(b)).cpu().numpy()
    assert np.abs(x - xr).max() <= 1e-12 * np.abs(xr).max()
    # in place (x aliases b), and a second solve with the same factor
    bb = T(2 * b)
    R.lu_solve(lu, bb, bb)
    assert np.abs(bb.cpu().numpy() - 2 * xr).max() <= 1e-12 * np.abs(xr).max()
    lu32 = R.lu_factor(op, alpha, beta, torch.float32)
    x32 = R.lu_solve(lu32, T(b, torch.float32)).cpu().numpy().astype(np.float64)
    assert np.abs(x32 - xr).max() <= 1e-5 * np.abs(xr).max()
    assert lu.bytes > 0


def test_lu_pivoting_on_a_matrix_that_needs_it(R):
    """alpha = 0: M = -beta L_X has a small diagonal relative to its rows
    (row sums of L_X vanish), so row interchanges occur; the solve still
    matches the dense solve (the constant null vector of L_X is removed by
    a small alpha = 1e-3)."""
    ns = W.icosahedral_sphere(3)
    op, X, Nr, _ = _rcm_built(R, ns, 17)
    N = ns.N
    L = _matrix(R, op, N).toarray()
    alpha, beta = 1e-3, 1.0
    M = alpha * np.eye(N) - beta * L
    b = W.uniform_field(N, seed=4)
    xr = np.linalg.solve(M, b)
    x = R.lu_solve(R.lu_factor(op, alpha, beta), T(b)).cpu().numpy()
    cond = np.linalg.cond(M)
    assert np.abs(x - xr).max() <= 1e-15 * cond * np.abs(xr).max() * 50


def test_lu_singular_and_too_wide(R):
    ns = W.icosahedral_sphere(2)
    op = R.build_operator(T(ns.X), T(ns.normals), 11, kernel="imq", kappa_target=1e8)
    with pytest.raises(R.RbffdError) as e:
        R.lu_factor(op, 0.0, 0.0)           # M = 0
    assert e.value.status == 8
    big = W.fibonacci_sphere(40_000)
    sh = np.random.default_rng(1).permutation(big.N)    # a numbering with no locality
    opb = R.build_operator(T(big.X[sh]), T(big.normals[sh]), 11, kernel="imq", kappa_target=1e8)
    kl, ku = R.op_bandwidth(opb)
    assert kl + ku > 10_000
    with pytest.raises(R.RbffdError) as e:
        R.lu_factor(opb, 3.0, 1e-3)
    assert e.value.status == 1


def _oracle_run(L, u0, v0, p, nsteps, order=2):
    return ostp.imex_run(lambda x: L @ x, u0, v0, p, nsteps, solver="lu", L_matrix=L, order=order)


@pytest.mark.parametrize("dtype,bound", [(torch.float64, 1e-9), (torch.float32, 1e-5)])
def test_step_imex_lu_schnakenberg_against_oracle(R, dtype, bound):
    """Two-species Schnakenberg, SBDF2 (IMEX Euler first) with the LU solver
    on an RCM-ordered staggered torus (N = 2400, n = 50), 50 steps, against
    the oracle's sparse-LU steps on the same operator; the CUDA graph replay
    gives the same bits as direct launches."""
    ns = W.torus_staggered(20)
    op, X, Nr, perm = _rcm_built(R, ns, 50, kappa=1e12)
    L = _matrix(R, op, ns.N)
    s = W.SCHNAKENBERG
    u0, v0 = W.schnakenberg_initial(ns.N, seed=2)
    ref = _oracle_run(L, u0, v0, s, 50)
    name, coef = R.model_coefs(s)
    out = []
    for graph in (True, False):
        p = R.StepParams(model=name, nspecies=2, dtype=dtype, dt=s["dt"], delta_u=s["delta_u"],
                         delta_v=s["delta_v"], coef=coef, use_graph=graph, solver="lu")
        st = R.StepState.create(T(u0, dtype), T(v0, dtype))
        rep = R.step_imex(op, st, p, 50)
        assert rep["status"] == 0 and rep["total_iters"] == 0
        out.append((st.u.clone(), st.v.clone()))
        for x, r in ((st.u, ref["u"]), (st.v, ref["v"])):
            got = x.cpu().numpy().astype(np.float64)
            assert np.abs(got - r).max() <= bound * np.abs(r).max()
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])


def test_step_imex_lu_equals_bicgstab_and_bdf4(R):
    """Heat equation on the RCM-ordered 2562-node sphere: SBDF2 with the LU
    solver equals SBDF2 with BiCGSTAB at tolerance 1e-14 (to 1e-11), and the
    BDF4 run (orders 1..4 while the history builds up, four factors) matches
    the oracle's sparse-LU BDF4 run."""
    ns = W.icosahedral_sphere(4)
    op, X, Nr, _ = _rcm_built(R, ns, 31, kernel="gaussian", kappa=1e12)
    u0 = W.sph_harm_y32(X)
    res = {}
    for solver, tol in (("lu", 1e-12), ("bicgstab", 1e-14)):
        p = R.StepParams(model="none", nspecies=1, dtype=torch.float64, dt=1e-4, delta_u=1.0, tol=tol,
                         use_graph=True, solver=solver)
        st = R.StepState.create(T(u0))
        R.step_imex(op, st, p, 100)
        res[solver] = st.u.cpu().numpy()
    assert np.abs(res["lu"] - res["bicgstab"]).max() <= 1e-11 * np.abs(res["bicgstab"]).max()
    L = _matrix(R, op, ns.N)
    ref = ostp.imex_run(lambda x: L @ x, u0, None, dict(model="none", dt=1e-4, delta_u=1.0), 30, order=4,
                        solver="lu", L_matrix=L)
    p = R.StepParams(model="none", nspecies=1, dtype=torch.float64, dt=1e-4, delta_u=1.0, order=4,
                     use_graph=True, solver="lu")
    st = R.StepState.create(T(u0), order=4)
    R.step_imex(op, st, p, 30)
    assert np.abs(st.u.cpu().numpy() - ref["u"]).max() <= 1e-12 * np.abs(ref["u"]).max()
