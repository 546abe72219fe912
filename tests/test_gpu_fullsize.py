"""Parity at the benchmark's full size, in the configuration bench.py times:
the 1,000,000-node Fibonacci sphere in four stencil-size bands (n = 31 / 50 /
70 / 101), IMQ, kappa_T = 1e12, learned first guess (networks trained as the
bench trains them), the bench's launch shape; then one float32 SBDF2 step of
Schnakenberg on the built operator.  Sampled rows are checked against the
oracle one by one; the step, a global solve, is checked by a property that
holds at any size (its implicit equations are satisfied)."""
import numpy as np
import pytest
import torch

import hp_arbiter as H
from oracle import stencils as ost
from oracle import weights as ow
from paper_1404_0812_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SIZES = (31, 50, 70, 101)


def T(a, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


@pytest.fixture(scope="module")
def R():
    import paper_1404_0812_gb300 as R
    R._lib.load()
    return R


@pytest.fixture(scope="module")
def nets(R):
    import bench
    return bench.train_networks(R, W, T, torch)


@pytest.fixture(scope="module")
def built(R, nets):
    ns = W.fibonacci_sphere(1_000_000)
    nper = W.stencil_size_groups(ns.N, SIZES)
    op = R.build_operator(T(ns.X), T(ns.normals), T(nper, torch.int32), kernel="imq", kappa_target=1e12,
                          mlps=nets, block_threads=128, blocks_per_sm=4)
    return ns, nper, op


def test_learned_full_size_sampled_rows(R, built):
    ns, nper, op = built
    info = {k: v.cpu().numpy() for k, v in R.get_stencil_info(op).items()}
    assert np.all((info["status"] == 0) | (info["status"] == 4))
    assert (info["status"] == 4).mean() > 0.9          # the learned start carries the build
    acc = info["status"] == 4
    assert np.all((info["kappa"][acc] >= 0.5e12) & (info["kappa"][acc] <= 2e12))
    assert np.all(np.abs(np.log(info["kappa"][~acc] / 1e12)) < 0.05)
    idx, w = R.get_rows(op)
    u = W.sph_harm_y32(ns.X)
    y = R.apply(op, T(u)).cpu().numpy()
    rng = np.random.default_rng(1)
    rows = np.concatenate([rng.choice(np.where(nper == n)[0], 5, replace=False) for n in SIZES])
    rows = np.concatenate([rows, [0, ns.N - 1]])
    sel = torch.as_tensor(rows, device="cuda")
    idx_r, w_r = idx[sel].cpu().numpy(), w[sel].cpu().numpy()
    st, wg = [], []
    for r, k in enumerate(rows):
        n = int(nper[k])
        sref = ost.stencil(ns.X, int(k), n)
        assert np.array_equal(idx_r[r, :n], sref.astype(np.int32))
        P = ns.X[sref]
        kc = ow.cond2(ow.interp_matrix(P, info["eps"][k], ow.IMQ))
        if info["status"][k] == 4:    # accepted prediction: inside the band by the oracle's kappa,
            assert 0.5e12 * 0.999 <= kc <= 2e12 * 1.001     # its reported kappa a lower estimate
            assert info["kappa"][k] <= kc * 1.001
        else:
            assert abs(np.log(kc / info["kappa"][k])) < 1e-3
        # the apply reproduces the stored weights' row exactly (same float64 sum)
        assert abs(y[k] - w_r[r, :n] @ u[sref]) <= 1e-12 * np.abs(w_r[r, :n]).sum() * np.abs(u).max()
        st.append(sref)
        wg.append(w_r[r, :n])
    # weights and applied rows (relative L-infinity over the sampled rows)
    # against the 45-digit oracle: no worse than the float64 oracle's
    res = H.arbitrate(ns.X, ns.normals, rows, st, info["eps"][rows], ow.IMQ, wg,
                      {"y32": u, "random": W.uniform_field(ns.N, seed=1)})
    print(res)
    H.assert_no_worse_than_f64(res)
    assert res["y32"]["gpu"] <= 1e-8


def test_accepted_predictions_inside_the_band_by_the_oracle(R, built):
    """Every accepted learned guess of the 1M-node build -- many of them
    accepted before the A^{-1} Lanczos run reached its full length, on a
    lower estimate of kappa -- has the oracle's kappa_2 (LAPACK eigenvalues
    of A_P at the GPU's eps) inside [0.5, 2] kappa_T: 100,000 accepted
    stencils, 25,000 per stencil size."""
    ns, nper, op = built
    info = {k: v.cpu().numpy() for k, v in R.get_stencil_info(op).items()}
    idx, _ = R.get_rows(op)
    rng = np.random.default_rng(5)
    rows = np.concatenate([rng.choice(np.flatnonzero((nper == n) & (info["status"] == 4)), 25_000, replace=False)
                           for n in SIZES])
    idx_r = idx[torch.as_tensor(rows, device="cuda")].cpu().numpy()
    Ps = [ns.X[idx_r[i, :int(nper[k])]] for i, k in enumerate(rows)]
    kc = H.cond2_many(Ps, info["eps"][rows], ow.IMQ)
    lo, hi = kc.min() / 1e12, kc.max() / 1e12
    print(f"oracle kappa / kappa_T over {len(rows)} accepted stencils: [{lo:.4f}, {hi:.4f}]")
    assert np.all((kc >= 0.5e12 * 0.999) & (kc <= 2e12 * 1.001)), (lo, hi)
    # the reported kappa of an accepted stencil is a lower estimate of it
    assert np.all(info["kappa"][rows] <= kc * 1.001)


@pytest.mark.parametrize("dtype,tol,bound", [(torch.float64, 1e-10, 1e-9), (torch.float32, 1e-6, 2e-5)])
def test_full_size_step_satisfies_its_equations(R, built, dtype, tol, bound):
    """One Schnakenberg step (IMEX Euler from no history) on the 1M operator:
    the new state solves (I - dt delta L) u1 = u0 + dt f(u0), checked with the
    apply of the same precision.  float64: to the solver's tolerance; float32
    (the bench's stepping precision): to 2e-5, the solver's 1e-6 plus the
    float32 rounding of a 101-term apply scaled by dt delta |L| ~ 10."""
    ns, nper, op = built
    s = W.SCHNAKENBERG
    name, coef = R.model_coefs(s)
    u0, v0 = W.schnakenberg_initial(ns.N, seed=2)
    p = R.StepParams(model=name, nspecies=2, dtype=dtype, dt=s["dt"], delta_u=s["delta_u"],
                     delta_v=s["delta_v"], coef=coef, tol=tol, use_graph=True)
    st = R.StepState.create(T(u0, dtype), T(v0, dtype))
    rep = R.step_imex(op, st, p, 1)
    assert rep["status"] == 0
    a, b, gam = s["a"], s["b"], s["gamma"]
    f = gam * (a - u0 + u0 * u0 * v0)
    g = gam * (b - u0 * u0 * v0)
    for x1, x0, r0, d in ((st.u, u0, f, s["delta_u"]), (st.v, v0, g, s["delta_v"])):
        Lx = R.apply(op, x1).double().cpu().numpy()
        x = x1.double().cpu().numpy()
        rhs = x0 + s["dt"] * r0
        res = np.linalg.norm(x - s["dt"] * d * Lx - rhs) / np.linalg.norm(rhs)
        assert res < bound, res


def test_pointcloud_2m_build_sampled_rows(R, nets):
    """The 2M-node bumpy point cloud (Gaussian tangent jitter 0.25 h, 20-NN
    PCA normals), n = 70, kappa_T = 1e12, learned start as the bench builds
    it: sampled rows against the oracle."""
    ns = W.workload("bumpy2m")
    n = 70
    op = R.build_operator(T(ns.X), T(ns.normals), n, kernel="imq", kappa_target=1e12,
                          mlps=[nets[SIZES.index(n)]], allow_failures=True)
    info = {k: v.cpu().numpy() for k, v in R.get_stencil_info(op).items()}
    assert np.all((info["status"] == 0) | (info["status"] == 4))
    acc = info["status"] == 4
    assert np.all((info["kappa"][acc] >= 0.5e12) & (info["kappa"][acc] <= 2e12))
    idx, w = R.get_rows(op)
    rows = np.random.default_rng(2).choice(ns.N, 8, replace=False)
    sel = torch.as_tensor(rows, device="cuda")
    idx_r, w_r = idx[sel].cpu().numpy(), w[sel].cpu().numpy()
    st, wg = [], []
    for r, k in enumerate(rows):
        sref = ost.stencil(ns.X, int(k), n)
        assert np.array_equal(idx_r[r, :n], sref.astype(np.int32))
        P = ns.X[sref]
        kc = ow.cond2(ow.interp_matrix(P, info["eps"][k], ow.IMQ))
        if info["status"][k] == 4:
            assert 0.5e12 * 0.999 <= kc <= 2e12 * 1.001 and info["kappa"][k] <= kc * 1.001
        else:
            assert abs(np.log(kc / info["kappa"][k])) < 1e-3
        st.append(sref)
        wg.append(w_r[r, :n])
    res = H.arbitrate(ns.X, ns.normals, rows, st, info["eps"][rows], ow.IMQ, wg,
                      {"random": W.uniform_field(ns.N, seed=1)})
    print(res)
    H.assert_no_worse_than_f64(res)


def test_torus_40k_schnakenberg_float32_against_float64_oracle(R):
    """The staggered torus m = 82 (N = 40,344), n = 50, kappa_T = 1e12:
    100 float32 Schnakenberg steps on the GPU against the oracle's float64
    stepper driven by the same operator's weights (<= 1e-5)."""
    import scipy.sparse as sps
    from oracle import stepping as ostp
    ns = W.workload("torus40344")
    n = 50
    op = R.build_operator(T(ns.X), T(ns.normals), n, kernel="imq", kappa_target=1e12)
    idx, w = (t.cpu().numpy() for t in R.get_rows(op))
    Lx = sps.csr_matrix((w[:, :n].ravel(), idx[:, :n].ravel(), np.arange(0, ns.N * n + 1, n)), shape=(ns.N, ns.N))
    s = W.SCHNAKENBERG
    u0, v0 = W.schnakenberg_initial(ns.N, seed=2)
    o = ostp.imex_run(lambda x: Lx @ x, u0, v0, s, 100)
    name, coef = R.model_coefs(s)
    p = R.StepParams(model=name, nspecies=2, dtype=torch.float32, dt=s["dt"], delta_u=s["delta_u"],
                     delta_v=s["delta_v"], coef=coef, tol=1e-8, use_graph=True)
    st = R.StepState.create(T(u0, torch.float32), T(v0, torch.float32))
    R.step_imex(op, st, p, 100)
    for x, ref in ((st.u, o["u"]), (st.v, o["v"])):
        got = x.cpu().numpy().astype(np.float64)
        assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()
