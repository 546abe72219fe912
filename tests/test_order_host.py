"""Host-side reverse Cuthill-McKee (Section 4.1's reordering) through the
C ABI, no GPU needed: a shuffled path comes back with bandwidth 1, grid
graphs get a bandwidth no worse than scipy's RCM allows (a library check of
the same algorithm), components and invalid input are handled."""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import reverse_cuthill_mckee

from paper_1404_0812_gb300 import _lib


@pytest.fixture(scope="module")
def R():
    import paper_1404_0812_gb300 as R
    _lib.load()
    return R


def _csr(n, edges):
    A = sp.coo_matrix((np.ones(len(edges)), (edges[:, 0], edges[:, 1])), shape=(n, n)).tocsr()
    A.sum_duplicates()
    return A


def _bandwidth(A, perm):
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    C = A.tocoo()
    return int(np.abs(inv[C.row] - inv[C.col]).max())


def _shuffle(A, seed):
    p = np.random.default_rng(seed).permutation(A.shape[0])
    return A[p][:, p].tocsr()


def test_path_graph(R):
    n = 200
    e = np.array([[i, i + 1] for i in range(n - 1)])
    A = _shuffle(_csr(n, e), 1)
    perm = R.rcm_order_host(A.indptr, A.indices)
    assert sorted(perm.tolist()) == list(range(n))
    assert _bandwidth(A + A.T, perm) == 1


@pytest.mark.parametrize("w,h", [(30, 40), (7, 90)])
def test_grid_graph_bandwidth(R, w, h):
    idx = np.arange(w * h).reshape(h, w)
    e = np.concatenate([np.stack([idx[:, :-1].ravel(), idx[:, 1:].ravel()], 1),
                        np.stack([idx[:-1, :].ravel(), idx[1:, :].ravel()], 1)])
    A = _shuffle(_csr(w * h, e), 2)
    S = (A + A.T).tocsr()
    perm = R.rcm_order_host(A.indptr, A.indices)
    assert sorted(perm.tolist()) == list(range(w * h))
    ours = _bandwidth(S, perm)
    ref = _bandwidth(S, reverse_cuthill_mckee(S, symmetric_mode=True).astype(np.int32))
    assert ours <= min(w, h) + 2 and ours <= 1.5 * ref + 1
    assert _bandwidth(S, np.arange(w * h, dtype=np.int32)) > 5 * ours   # the shuffle was bad


def test_components_and_invalid(R):
    e = np.array([[0, 1], [1, 2], [3, 4], [5, 5]])          # two paths, an isolated node with a loop
    A = _csr(7, e)
    perm = R.rcm_order_host(A.indptr, A.indices)
    assert sorted(perm.tolist()) == list(range(7))
    with pytest.raises(R.RbffdError) as exc:
        R.rcm_order_host(np.array([0, 1]), np.array([5]))    # column out of range
    assert exc.value.status == 1
