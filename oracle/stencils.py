"""Oracle stencil selection (Section 4: a node and its n-1 nearest neighbours).

Section 4 takes, for node x_1, the n-1 nearest other nodes by Euclidean
distance in R^3 and puts the centre first; Section 4.1 uses a k-d tree only to
do that quickly.  The oracle does it by brute force: every squared distance,
then a sort.

Reading for ties (the paper is silent): the key is (d^2, j), compared
lexicographically, with d^2 = (dx*dx + dy*dy) + dz*dz evaluated left to right
in float64 with no fused multiply-add, dx = x_j - x_k.  The centre is entry 0
whatever the distances of duplicates.

Pins: tests/test_oracle_stencils.py (scipy cKDTree distances, hand cases with
ties, invariants).
"""
from __future__ import annotations

import numpy as np


def sq_dist(X: np.ndarray, k: int) -> np.ndarray:
    """Squared Euclidean distance from node k to every node, float64,
    evaluated as (dx*dx + dy*dy) + dz*dz (numpy elementwise ops never fuse)."""
    dx = X[:, 0] - X[k, 0]
    dy = X[:, 1] - X[k, 1]
    dz = X[:, 2] - X[k, 2]
    return dx * dx + dy * dy + dz * dz


def stencil(X: np.ndarray, k: int, n: int) -> np.ndarray:
    """Indices of stencil P_k: k first, then its n-1 nearest other nodes in
    ascending (d^2, index) order (Section 4, Section 4.1)."""
    N = X.shape[0]
    if n > N:
        raise ValueError("stencil size exceeds node count")
    d2 = sq_dist(X, k)
    others = np.concatenate([np.arange(k), np.arange(k + 1, N)])
    order = np.lexsort((others, d2[others]))  # primary d2, secondary index
    return np.concatenate([[k], others[order[: n - 1]]]).astype(np.int64)


def all_stencils(X: np.ndarray, n_per_node) -> list[np.ndarray]:
    """Stencil of every node; ``n_per_node`` is an int or an (N,) array."""
    N = X.shape[0]
    ns = np.broadcast_to(np.asarray(n_per_node), (N,))
    return [stencil(X, k, int(ns[k])) for k in range(N)]
