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


def _rcm_reference(S):
    """The same reverse Cuthill-McKee, written plainly and sequentially:
    George-Liu pseudo-peripheral start (from the component's node of least
    (degree, index), up to 8 moves to the least-(degree, index) node of the
    deepest BFS level while the depth grows), then a BFS visiting neighbours
    by (degree, index), components in order of their first node, reversed."""
    n = S.shape[0]
    S = S.tolil()
    S.setdiag(0)
    S = S.tocsr()
    S.eliminate_zeros()
    deg = np.diff(S.indptr)
    adj = [sorted(S.indices[S.indptr[i]:S.indptr[i + 1]].tolist(), key=lambda j: (deg[j], j)) for i in range(n)]

    def levels(s):
        lev = {s: 0}
        q = [s]
        for v in q:
            for w in adj[v]:
                if w not in lev:
                    lev[w] = lev[v] + 1
                    q.append(w)
        return lev

    done = np.zeros(n, bool)
    order = []
    for seed in range(n):
        if done[seed]:
            continue
        comp = levels(seed)
        start = min(comp, key=lambda v: (deg[v], v))
        d0 = -1
        for _ in range(8):
            lev = levels(start)
            depth = max(lev.values())
            best = min((v for v, l in lev.items() if l == depth), key=lambda v: (deg[v], v))
            if depth <= d0:
                break
            d0 = depth
            if best == start:
                break
            start = best
        q = [start]
        done[start] = True
        for v in q:
            order.append(v)
            for w in adj[v]:
                if not done[w]:
                    done[w] = True
                    q.append(w)
    return np.array(order[::-1], dtype=np.int32)


def test_large_graph_matches_sequential_definition(R):
    """70,000-node graph (a 200 x 160 grid with diagonals; a 30,000-node
    random graph of degree ~8, whose BFS levels grow to thousands of nodes;
    more small components, isolated nodes; asymmetric and repeated edges;
    shuffled): large enough for the threaded adjacency build and the threaded
    level-synchronous BFS, whose permutation must equal the plain sequential
    one exactly."""
    rng = np.random.default_rng(9)
    w, h = 200, 160
    idx = np.arange(w * h).reshape(h, w)
    e = [np.stack([idx[:, :-1].ravel(), idx[:, 1:].ravel()], 1),
         np.stack([idx[:-1, :].ravel(), idx[1:, :].ravel()], 1),
         np.stack([idx[:-1, :-1].ravel(), idx[1:, 1:].ravel()], 1)]
    g0 = w * h
    expander = g0 + np.stack([np.repeat(np.arange(30000), 4), rng.integers(0, 30000, 120000)], 1)
    extra = g0 + 30000 + rng.integers(0, 6000, (9000, 2))      # small components among the next 6000 nodes
    n = g0 + 30000 + 8000                                        # the last 2000 nodes are isolated
    e = np.concatenate(e + [expander, extra, e[0][:500]])        # repeats
    A = _shuffle(_csr(n, e), 3)                                  # asymmetric: each edge stored once
    perm = R.rcm_order_host(A.indptr, A.indices)
    assert sorted(perm.tolist()) == list(range(n))
    assert np.array_equal(perm, _rcm_reference(A + A.T))
