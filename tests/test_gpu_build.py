"""GPU parity of the operator build (stencils, shape parameters, weights) and
of the apply, through the C ABI, against the CPU oracle.

Tolerances (floating point; derived from the arithmetic):
* applied operator, smooth u: ||L_gpu u - L_cpu u||_inf / ||L_cpu u||_inf
  <= 1e-8 (also at kappa_T = 1e12);
* applied operator, random u at kappa_T = 1e12: the float64 oracle is itself
  ~1.2e-6 (relative L-infinity) from the 45-digit truth there, so GPU against
  oracle is held to 5e-6 (the two errors, each at most ~2x that spread); the
  arbitration by the 45-digit oracle is in test_gpu_parity_hp.py and in the
  full-size test below; at kappa <= 1e8 random u is held to 1e-8;
* stencil indices: bit-exact (the (d^2, index) key is bit-reproducible);
* eps: |eps_gpu - eps_cpu| <= 2 * tol + 1e-5 * eps (both searches stop
  within tol of the root; the root itself moves with kappa's float64 noise).
"""
import math

import numpy as np
import pytest
import torch

import hp_arbiter as H
from oracle import operator as oop
from oracle import stencils as ost
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


@pytest.fixture(scope="module")
def sphere():
    ns = W.icosahedral_sphere(4)
    ref = oop.build_operator(ns.X, ns.normals, 31, ow.GAUSSIAN, kappa_T=1e12)
    return ns, ref


def test_stencils_bit_exact(R, sphere):
    ns, ref = sphere
    op = R.build_operator(T(ns.X), T(ns.normals), 31, kernel="gaussian", eps_override=T(ref.eps))
    idx, _ = R.get_rows(op)
    assert np.array_equal(idx.cpu().numpy(), ref.idx.astype(np.int32))
    assert op.nnz == 31 * ns.N


def test_weights_at_oracle_eps(R, sphere):
    ns, ref = sphere
    op = R.build_operator(T(ns.X), T(ns.normals), 31, kernel="gaussian", eps_override=T(ref.eps))
    u_s = W.sph_harm_y32(ns.X)
    u_r = W.uniform_field(ns.N, seed=1)
    y_s = R.apply(op, T(u_s)).cpu().numpy()
    y_r = R.apply(op, T(u_r)).cpu().numpy()
    assert rel_inf(y_s, oop.apply(ref, u_s)) <= 1e-8
    # random u at kappa_T = 1e12: the float64 oracle is itself ~1e-6 from the
    # 45-digit weights (test_gpu_parity_hp); GPU and oracle differ by their two
    # errors, held to three times the oracle's measured spread there
    assert rel_inf(y_r, oop.apply(ref, u_r)) <= 5e-6
    # float32 apply of the float32 weights against the float64 oracle
    y32 = R.apply(op, T(u_s, torch.float32)).cpu().numpy().astype(np.float64)
    assert rel_inf(y32, oop.apply(ref, u_s)) <= 1e-3
    _, w = R.get_rows(op)
    w = w.cpu().numpy()
    assert np.abs(w.sum(axis=1)).max() <= 1e-9 * np.abs(w).sum(axis=1).max()


def test_eps_search_matches_oracle(R, sphere):
    ns, ref = sphere
    op = R.build_operator(T(ns.X), T(ns.normals), 31, kernel="gaussian", kappa_target=1e12)
    info = {k: v.cpu().numpy() for k, v in R.get_stencil_info(op).items()}
    assert np.all(info["status"] == 0)
    d = np.abs(info["eps"] - ref.eps)
    assert np.all(d <= 2e-4 + 1e-5 * ref.eps), d.max()
    assert np.all(np.abs(np.log(info["kappa"] / 1e12)) < 0.05)
    assert np.all((info["evals"] >= 2) & (info["evals"] <= 20))
    # spot-check the GPU's kappa at its eps with the oracle's definition
    for k in range(0, ns.N, 257):
        P = ns.X[ref.idx[k]]
        kc = ow.cond2(ow.interp_matrix(P, info["eps"][k], ow.GAUSSIAN))
        assert abs(math.log(kc / info["kappa"][k])) < 1e-3
    # accuracy of Delta_M Y_3^2 with the GPU-searched operator
    u = W.sph_harm_y32(ns.X)
    y = R.apply(op, T(u)).cpu().numpy()
    assert np.abs(y + 12 * u).max() / np.abs(12 * u).max() < 2e-4


@pytest.mark.parametrize("kernel", ["imq", "gaussian"])
def test_moderate_kappa_random_field(R, kernel):
    ns = W.icosahedral_sphere(3)
    kid = ow.KERNELS[kernel]
    ref = oop.build_operator(ns.X, ns.normals, 31, kid, eps=5.0)
    op = R.build_operator(T(ns.X), T(ns.normals), 31, kernel=kernel, eps_override=T(ref.eps))
    for u in (W.uniform_field(ns.N, seed=2), W.sph_harm_y32(ns.X)):
        y = R.apply(op, T(u)).cpu().numpy()
        assert rel_inf(y, oop.apply(ref, u)) <= 1e-8


def test_mixed_sizes_ragged_rows(R):
    """N = 3001 (not a multiple of 32), three stencil sizes that are not
    multiples of 4, all rows checked."""
    ns = W.fibonacci_sphere(3001)
    nper = np.array([11, 17, 31])[np.arange(ns.N) % 3].astype(np.int32)
    ref = oop.build_operator(ns.X, ns.normals, nper, ow.IMQ, eps=np.full(ns.N, 6.0))
    op = R.build_operator(T(ns.X), T(ns.normals), T(nper, torch.int32), kernel="imq",
                          eps_override=T(ref.eps))
    idx, w = R.get_rows(op)
    assert np.array_equal(idx.cpu().numpy(), ref.idx.astype(np.int32))
    assert op.nnz == int(nper.sum())
    u = W.uniform_field(ns.N, seed=3)
    assert rel_inf(R.apply(op, T(u)).cpu().numpy(), oop.apply(ref, u)) <= 1e-8


def test_stencil_equals_all_nodes_and_minimum_size(R):
    ns = W.icosahedral_sphere(1)       # N = 42
    for n in (2, 42):
        ref = oop.build_operator(ns.X, ns.normals, n, ow.IMQ, eps=2.0)
        op = R.build_operator(T(ns.X), T(ns.normals), n, kernel="imq", eps_override=T(ref.eps))
        idx, _ = R.get_rows(op)
        assert np.array_equal(idx.cpu().numpy(), ref.idx.astype(np.int32))
        u = W.uniform_field(ns.N, seed=4)
        assert rel_inf(R.apply(op, T(u)).cpu().numpy(), oop.apply(ref, u)) <= 1e-8


def test_invalid_inputs_are_reported(R):
    ns = W.icosahedral_sphere(1)
    with pytest.raises(R.RbffdError) as e:
        R.build_operator(T(ns.X), T(ns.normals), 43)
    assert e.value.status == 1
    X = ns.X.copy()
    X[5, 1] = np.nan
    with pytest.raises(R.RbffdError) as e:
        R.build_operator(T(X), T(ns.normals), 10)
    assert e.value.status == 1
    # a duplicated node makes the local matrices singular (Section 2 needs
    # distinct nodes): the search reports failure per stencil
    X = np.vstack([ns.X, ns.X[:1]])
    Nr = np.vstack([ns.normals, ns.normals[:1]])
    op = R.build_operator(T(X), T(Nr), 10, allow_failures=True)
    st = R.get_stencil_info(op)["status"].cpu().numpy()
    assert op.status in (4, 8)
    assert st[0] != 0 and st[42] != 0
    assert np.sum(st == 0) >= 30


def test_full_size_mixed_build_sampled(R):
    """Fibonacci sphere N = 1,000,000 in four latitude bands with n = 31, 50,
    70, 101 (the batched-build workload), searched to kappa_T = 1e12 with the
    IMQ kernel in one launch; sampled rows checked against the oracle."""
    ns = W.fibonacci_sphere(1_000_000)
    nper = W.stencil_size_groups(ns.N)
    op = R.build_operator(T(ns.X), T(ns.normals), T(nper, torch.int32), kernel="imq",
                          kappa_target=1e12)
    info = {k: v.cpu().numpy() for k, v in R.get_stencil_info(op).items()}
    assert np.all(info["status"] == 0)
    assert np.all(np.abs(np.log(info["kappa"] / 1e12)) < 0.05)
    idx, w = R.get_rows(op)
    rng = np.random.default_rng(0)
    rows = np.concatenate([rng.choice(np.where(nper == n)[0], 3, replace=False) for n in (31, 50, 70, 101)])
    rows = np.concatenate([rows, [0, ns.N - 1]])
    idx_r = idx[torch.as_tensor(rows, device="cuda")].cpu().numpy()
    w_r = w[torch.as_tensor(rows, device="cuda")].cpu().numpy()
    st, wg = [], []
    for r, k in enumerate(rows):
        n = int(nper[k])
        sref = ost.stencil(ns.X, int(k), n)
        assert np.array_equal(idx_r[r, :n], sref.astype(np.int32))
        st.append(sref)
        wg.append(w_r[r, :n])
    # weights and applied rows (relative L-infinity over the sampled rows)
    # against the 45-digit oracle, no worse than the float64 oracle's
    res = H.arbitrate(ns.X, ns.normals, rows, st, info["eps"][rows], ow.IMQ, wg,
                      {"y32": W.sph_harm_y32(ns.X), "random": W.uniform_field(ns.N, seed=1)})
    print(res)
    H.assert_no_worse_than_f64(res)
    assert res["y32"]["gpu"] <= 1e-8
    for k in rows[::4]:
        n = int(nper[k])
        sref = ost.stencil(ns.X, int(k), n)
        e_ref, _, _ = ow.search_eps(ns.X[sref], ow.IMQ, 1e12)
        assert abs(info["eps"][k] - e_ref) <= 2e-4 + 1e-5 * e_ref


def test_autotune_picks_a_shape_and_caches_it(R, tmp_path):
    ns = W.fibonacci_sphere(40_000)
    nper = W.stencil_size_groups(ns.N, (31, 50))
    X, Nr, P = T(ns.X), T(ns.normals), T(nper, torch.int32)
    cache = tmp_path / "tune.txt"
    r = R.autotune_build(X, Nr, P, kernel="imq", sample=8000, cache_path=cache)
    assert r["block_threads"] in (64, 128) and 3 <= r["blocks_per_sm"] <= 8 and r["ms"] > 0
    r2 = R.autotune_build(X, Nr, P, kernel="imq", sample=8000, cache_path=cache)
    assert (r2["block_threads"], r2["blocks_per_sm"]) == (r["block_threads"], r["blocks_per_sm"])
    assert r2["ms"] == -1.0
    # the chosen shape builds the same operator as the default one
    a = R.build_operator(X, Nr, P, kernel="imq", kappa_target=1e12)
    b = R.build_operator(X, Nr, P, kernel="imq", kappa_target=1e12,
                         block_threads=r["block_threads"], blocks_per_sm=r["blocks_per_sm"])
    ia, ib = R.get_stencil_info(a), R.get_stencil_info(b)
    assert torch.equal(ia["eps"], ib["eps"])
    assert torch.equal(R.get_rows(a)[1], R.get_rows(b)[1])


def test_get_eps_and_ell_views(R):
    """rbffd_get_eps equals the first three arrays of rbffd_get_stencil_info;
    the borrowed sliced-ELL views, decoded with the documented element
    formula, give exactly the rows of rbffd_get_rows."""
    ns = W.fibonacci_sphere(2001)
    nper = np.array([13, 31, 7])[np.arange(ns.N) % 3].astype(np.int32)
    op = R.build_operator(T(ns.X), T(ns.normals), T(nper, torch.int32), kernel="imq", kappa_target=1e10)
    eps, kappa, evals = R.get_eps(op)
    info = R.get_stencil_info(op)
    assert torch.equal(eps, info["eps"]) and torch.equal(kappa, info["kappa"])
    assert torch.equal(evals, info["evals"])
    v = R.get_ell(op)
    assert v["ngroups"] == 3 and v["n"] == [31, 13, 7] and v["npad"] == [32, 16, 8]
    idx = v["idx"].cpu().numpy()
    w64 = v["w64"].cpu().numpy()
    w32 = v["w32"].cpu().numpy()
    row_node = v["row_node"].cpu().numpy()
    assert sorted(row_node.tolist()) == list(range(ns.N))
    ridx, rw = (t.cpu().numpy() for t in R.get_rows(op))
    for g in range(v["ngroups"]):
        n, npad, off = v["n"][g], v["npad"][g], v["elem_begin"][g]
        for r in range(v["row_begin"][g], v["row_begin"][g + 1]):
            q = r - v["row_begin"][g]
            j = np.arange(npad)
            e = off + (q // 32) * 32 * npad + (j // 4) * 128 + (q % 32) * 4 + j % 4
            node = row_node[r]
            assert nper[node] == n
            assert np.array_equal(idx[e[:n]], ridx[node, :n])
            assert np.array_equal(w64[e[:n]], rw[node, :n])
            assert np.array_equal(w32[e[:n]], rw[node, :n].astype(np.float32))
            assert np.all(w64[e[n:]] == 0.0) and np.all(idx[e[n:]] == node)
    assert v["elems"] == v["elem_begin"][-1]


def test_eps_search_range(R):
    """A range that contains every root changes nothing beyond the search
    tolerance; a range on the wrong side of the roots reports
    RBFFD_STENCIL_NO_BRACKET for every stencil (build status
    RBFFD_EPS_SEARCH_FAILED) instead of a wrong eps."""
    ns = W.icosahedral_sphere(3)
    X, Nr = T(ns.X), T(ns.normals)
    free = R.build_operator(X, Nr, 31, kernel="imq", kappa_target=1e12)
    e0 = R.get_stencil_info(free)["eps"].cpu().numpy()
    inside = R.build_operator(X, Nr, 31, kernel="imq", kappa_target=1e12, eps_range=(1e-3, 1e3))
    i1 = {k: t.cpu().numpy() for k, t in R.get_stencil_info(inside).items()}
    assert np.all(i1["status"] == 0)
    assert np.all(np.abs(i1["eps"] - e0) <= 2e-4 + 1e-5 * e0)
    # kappa far above kappa_T (at eps * r_s = 1e-3 Phi does not even factor
    # in float64: such a stencil reports SINGULAR) / far below it
    for rng, allowed in (((1e-4, 1e-3), (1, 3)), ((1e3, 1e4), (1,))):
        op = R.build_operator(X, Nr, 31, kernel="imq", kappa_target=1e12, eps_range=rng,
                              allow_failures=True)
        st = R.get_stencil_info(op)["status"].cpu().numpy()
        assert op.status == 4 and np.all(np.isin(st, allowed))
    with pytest.raises(R.RbffdError) as e:
        R.build_operator(X, Nr, 31, eps_range=(2.0, 1.0))
    assert e.value.status == 1


def test_largest_stencil_size(R):
    """n = 128 (the largest the ABI accepts, m = 129): stencils bit-exact,
    apply parity at fixed eps, and sampled searched eps against the oracle."""
    ns = W.fibonacci_sphere(700)
    n = 128
    ref = oop.build_operator(ns.X, ns.normals, n, ow.IMQ, eps=np.full(ns.N, 1.5))
    op = R.build_operator(T(ns.X), T(ns.normals), n, kernel="imq", eps_override=T(ref.eps))
    idx, _ = R.get_rows(op)
    assert np.array_equal(idx.cpu().numpy(), ref.idx.astype(np.int32))
    u = W.sph_harm_y32(ns.X)
    assert rel_inf(R.apply(op, T(u)).cpu().numpy(), oop.apply(ref, u)) <= 1e-8
    op = R.build_operator(T(ns.X), T(ns.normals), n, kernel="imq", kappa_target=1e10)
    info = {k: v.cpu().numpy() for k, v in R.get_stencil_info(op).items()}
    assert np.all(info["status"] == 0)
    for k in range(0, ns.N, 173):
        e_ref, _, _ = ow.search_eps(ns.X[ref.idx[k]], ow.IMQ, 1e10)
        assert abs(info["eps"][k] - e_ref) <= 2e-4 + 1e-5 * e_ref


def test_degenerate_sizes_rejected(R):
    ns = W.icosahedral_sphere(1)
    X, Nr = T(ns.X), T(ns.normals)
    for bad in (dict(n=129), dict(n=1)):
        with pytest.raises(R.RbffdError) as e:
            R.build_operator(X, Nr, bad["n"])
        assert e.value.status == 1
    with pytest.raises(R.RbffdError) as e:      # a single node has no stencil
        R.build_operator(X[:1].contiguous(), Nr[:1].contiguous(), 2)
    assert e.value.status == 1
    nper = (np.arange(ns.N) % 9 + 2).astype(np.int32)   # nine distinct sizes > 8 groups
    with pytest.raises(R.RbffdError) as e:
        R.build_operator(X, Nr, T(nper, torch.int32))
    assert e.value.status == 1


def test_invalid_options_are_rejected(R):
    ns = W.icosahedral_sphere(1)
    X, Nr = T(ns.X), T(ns.normals)
    for kw in (dict(kappa_target=1.0), dict(kappa_target=float("inf")), dict(eps_tol=0.0), dict(max_evals=1),
               dict(kernel=7), dict(block_threads=48), dict(precision="quad")):
        with pytest.raises((R.RbffdError, KeyError)) as e:
            R.build_operator(X, Nr, 10, **kw)
        if isinstance(e.value, R.RbffdError):
            assert e.value.status == 1, kw
    net = R.EpsNet(10)
    with pytest.raises(R.RbffdError) as e:
        R.build_operator(X, Nr, 10, mlps=[net], accept=(2.0, 0.5))
    assert e.value.status == 1


def test_memory_pool_keeps_and_releases_scratch(R):
    """The build's transient scratch comes from the library's pool: all of it
    is returned when the build is done, stays mapped for the next build
    (which reuses it, dirty, with bit-identical results) and goes back to the
    device on rbffd_release_memory."""
    ns = W.fibonacci_sphere(20_000)
    X, Nr = T(ns.X), T(ns.normals)
    try:
        R.memory_pool_config(32 << 30)
        a = R.build_operator(X, Nr, 50, kernel="imq", kappa_target=1e12)
        torch.cuda.synchronize()
        st = R.memory_stats()
        assert st["used"] == 0 and st["reserved"] > 0
        b = R.build_operator(X, Nr, 50, kernel="imq", kappa_target=1e12)
        torch.cuda.synchronize()
        assert R.memory_stats()["reserved"] == st["reserved"]   # reused, not grown
        ia, ib = R.get_stencil_info(a), R.get_stencil_info(b)
        assert torch.equal(ia["eps"], ib["eps"]) and torch.equal(ia["kappa"], ib["kappa"])
        ea, eb = R.get_ell(a), R.get_ell(b)
        assert torch.equal(ea["w64"], eb["w64"])
        R.release_memory()
        assert R.memory_stats()["reserved"] == 0
        with pytest.raises(R.RbffdError) as e:
            R.memory_pool_config(-1)
        assert e.value.status == 1
    finally:
        R.memory_pool_config(32 << 30)


def test_fp64_throughput_microbenchmarks(R):
    """Both FP64 paths report a plausible rate for a GPU (GFLOP/s)."""
    v, t = R.fp64_peak(), R.fp64_mma_peak()
    assert 100.0 < v < 1e5 and 100.0 < t < 1e5, (v, t)


def test_rows_grouped_by_size_in_node_order(R):
    """Rows are grouped by stencil size (largest first) and keep the nodes'
    order inside a group, across many blocks of the device-side grouping
    (60,000 nodes, sizes drawn at random per node)."""
    ns = W.fibonacci_sphere(60_000)
    rng = np.random.default_rng(7)
    sizes = np.array([9, 21, 40, 64, 101])
    nper = sizes[rng.integers(0, len(sizes), ns.N)].astype(np.int32)
    eps = torch.full((ns.N,), 30.0, dtype=torch.float64, device="cuda")
    op = R.build_operator(T(ns.X), T(ns.normals), T(nper, torch.int32), kernel="imq", eps_override=eps,
                          allow_failures=True)
    v = R.get_ell(op)
    assert v["n"] == sorted(sizes.tolist(), reverse=True)
    row_node = v["row_node"].cpu().numpy()
    for g, n in enumerate(v["n"]):
        rows = row_node[v["row_begin"][g]:v["row_begin"][g + 1]]
        assert np.array_equal(rows, np.flatnonzero(nper == n))
