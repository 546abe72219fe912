"""Oracle global operator L_X (Section 4) and its application (Section 4.2).

For every node k: stencil P_k (oracle.stencils), shape parameter eps_k (given,
or searched to kappa_T as in Section 5), weights = first row of L_{P_k}
(oracle.weights).  The N x N sparse L_X has exactly n_k entries in row k, in
stencil order (Section 4: the weights "are arranged into a sparse N-by-N
differentiation matrix").  Application y = L_X u sums w_kj u[idx_kj] in
stencil order (Eq. kernel_mol, explicit part).

Pins: tests/test_oracle_operator.py (nnz = sum n_k, row sums, spherical
harmonic eigenfunctions, heat-equation decay, left-half-plane spectrum).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import stencils as _st
from . import weights as _w


@dataclass
class Operator:
    """Rows of L_X.  idx / w are padded to the widest stencil: entries past
    n[k] hold idx = row node and w = 0.0, which add exactly +0.0."""
    rows: np.ndarray     # (R,) node id of each row
    n: np.ndarray        # (R,) stencil size per row
    idx: np.ndarray      # (R, nmax) int64 stencil indices, centre first
    w: np.ndarray        # (R, nmax) float64 weights
    eps: np.ndarray      # (R,) shape parameter per stencil
    kappa: np.ndarray    # (R,) kappa(A(eps_k)); nan when eps was given
    evals: np.ndarray    # (R,) kappa evaluations used by the search (0 if given)

    @property
    def R(self) -> int:
        return len(self.rows)


def build_row(X, normals, idx, kernel, kappa_T=None, eps=None, xtol=1e-4):
    """Weights of one stencil; searches eps when ``eps`` is None."""
    P = X[idx]
    nr = normals[idx]
    if eps is None:
        eps, kap, ev = _w.search_eps(P, kernel, kappa_T, xtol)
    else:
        kap, ev = float("nan"), 0
    return _w.stencil_weights(P, nr, eps, kernel), float(eps), float(kap), int(ev)


def build_operator(X, normals, n_per_node, kernel, kappa_T=None, eps=None,
                   rows=None, stencil_idx=None, xtol=1e-4) -> Operator:
    """Rows ``rows`` (default all) of L_X.  ``eps`` may be a scalar or an (N,)
    array (fixed shape parameters) or None (search to ``kappa_T``).
    ``stencil_idx`` may pass precomputed stencils (list indexed by row)."""
    N = X.shape[0]
    ns = np.broadcast_to(np.asarray(n_per_node), (N,))
    rows = np.arange(N) if rows is None else np.asarray(rows, dtype=np.int64)
    idxs, ws, es, ks, evs = [], [], [], [], []
    for k in rows:
        idx = stencil_idx[k] if stencil_idx is not None else _st.stencil(X, k, int(ns[k]))
        ek = None if eps is None else float(np.broadcast_to(np.asarray(eps, dtype=float), (N,))[k])
        w, e, kap, ev = build_row(X, normals, idx, kernel, kappa_T, ek, xtol)
        idxs.append(np.asarray(idx, dtype=np.int64))
        ws.append(w)
        es.append(e)
        ks.append(kap)
        evs.append(ev)
    nk = np.array([len(i) for i in idxs], dtype=np.int64)
    nmax = int(nk.max()) if len(nk) else 0
    I = np.repeat(rows[:, None], nmax, axis=1).astype(np.int64)
    Wt = np.zeros((len(rows), nmax))
    for r, (i, w) in enumerate(zip(idxs, ws)):
        I[r, :len(i)] = i
        Wt[r, :len(w)] = w
    return Operator(rows, nk, I, Wt, np.array(es), np.array(ks), np.array(evs))


def apply(op: Operator, u: np.ndarray) -> np.ndarray:
    """y_k = sum_j w_kj u[idx_kj] for every row, accumulated in stencil order
    j = 1..n_k in float64 (padding adds +0.0)."""
    y = np.zeros(op.R)
    for j in range(op.idx.shape[1]):
        y = y + op.w[:, j] * u[op.idx[:, j]]
    return y


def dense(op: Operator, N: int) -> np.ndarray:
    """L_X as a dense N x N matrix (small N only; spectrum tests)."""
    L = np.zeros((N, N))
    for r in range(op.R):
        np.add.at(L[op.rows[r]], op.idx[r, :op.n[r]], op.w[r, :op.n[r]])
    return L


def sparse_matrix(op: Operator, N: int):
    """L_X as a scipy CSR matrix (N x N, Section 4: n_k entries in row k)."""
    import scipy.sparse as sps
    rows = np.repeat(op.rows, op.n)
    cols = np.concatenate([op.idx[r, :op.n[r]] for r in range(op.R)])
    vals = np.concatenate([op.w[r, :op.n[r]] for r in range(op.R)])
    return sps.csr_matrix((vals, (rows, cols)), shape=(N, N))
