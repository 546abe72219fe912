"""Locality orderings on the GPU (Section 4.1 reorders L_X by reverse
Cuthill-McKee): the Morton order equals a numpy restatement of its key, the
RCM order of a shuffled node set's stencil graph shrinks its bandwidth, and
the operator built on reordered nodes is the same operator, permuted."""
import numpy as np
import pytest
import torch

from paper_1404_0812_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def T(a, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


@pytest.fixture(scope="module")
def R():
    import paper_1404_0812_gb300 as R
    R._lib.load()
    return R


def _morton_ref(X):
    lo = X.min(axis=0)
    ext = (X.max(axis=0) - lo).max()
    q = np.clip(np.floor((X - lo) * (2097151.0 / ext)), 0, 2097151).astype(np.uint64)
    key = np.zeros(X.shape[0], dtype=np.uint64)
    for b in range(21):
        for a in range(3):
            key |= ((q[:, a] >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b + a)
    return np.lexsort((np.arange(X.shape[0]), key)).astype(np.int32)


@pytest.fixture(scope="module")
def shuffled():
    ns = W.fibonacci_sphere(20_000)
    p = np.random.default_rng(9).permutation(ns.N)
    return ns.X[p].copy(), ns.normals[p].copy()


def _bandwidth_stats(idx):
    k = np.repeat(np.arange(idx.shape[0]), idx.shape[1])
    d = np.abs(idx.ravel() - k)
    return int(d.max()), float(d.mean())


def test_morton_order_matches_its_definition(R, shuffled):
    X, _ = shuffled
    perm = R.morton_order(T(X)).cpu().numpy()
    assert np.array_equal(perm, _morton_ref(X))


def test_rcm_shrinks_bandwidth_and_reordered_operator_is_the_same(R, shuffled):
    X, Nr = shuffled
    n = 31
    op = R.build_operator(T(X), T(Nr), n, kernel="imq", kappa_target=1e12)
    perm = R.rcm_order(op).cpu().numpy()
    assert sorted(perm.tolist()) == list(range(len(perm)))
    idx0, _ = R.get_rows(op)
    b0 = _bandwidth_stats(idx0.cpu().numpy())
    Xr, Nrr = X[perm], Nr[perm]
    op2 = R.build_operator(T(Xr), T(Nrr), n, kernel="imq", kappa_target=1e12)
    idx2, _ = R.get_rows(op2)
    b2 = _bandwidth_stats(idx2.cpu().numpy())
    assert b2[0] < 0.1 * b0[0] and b2[1] < 0.05 * b0[1]
    # same stencils, permuted
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    assert np.array_equal(np.sort(perm[idx2.cpu().numpy()], axis=1), np.sort(idx0.cpu().numpy()[perm], axis=1))
    # same operator: at the same eps per node, L_X u in the new numbering is
    # the old result permuted, bit for bit (the searched eps themselves differ
    # within the search tolerance: the Lanczos start vectors are seeded by the
    # node number)
    eps = R.get_stencil_info(op)["eps"].cpu().numpy()
    a = R.build_operator(T(X), T(Nr), n, kernel="imq", eps_override=T(eps))
    b = R.build_operator(T(Xr), T(Nrr), n, kernel="imq", eps_override=T(eps[perm]))
    u = W.uniform_field(len(perm), seed=4)
    ya = R.apply(a, T(u)).cpu().numpy()
    yb = R.apply(b, T(u[perm])).cpu().numpy()
    assert np.array_equal(yb, ya[perm])
    e2 = R.get_stencil_info(op2)["eps"].cpu().numpy()
    assert np.all(np.abs(e2 - eps[perm]) <= 2e-4 + 1e-5 * e2)
    # Morton renumbering also localises the stencils
    pm = R.morton_order(T(X)).cpu().numpy()
    op3 = R.build_operator(T(X[pm]), T(Nr[pm]), n, kernel="imq", kappa_target=1e12)
    b3 = _bandwidth_stats(R.get_rows(op3)[0].cpu().numpy())
    assert b3[1] < 0.1 * b0[1]
