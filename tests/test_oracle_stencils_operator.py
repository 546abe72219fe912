"""Pins of the oracle's stencil selection (Section 4, Section 4.1) and of the
assembled operator (Section 4, Figure rcm) against an independent k-d tree,
hand-built tie cases, the paper's non-zero counts and the spectrum property
of Section 5."""
import json
import os

import numpy as np
import pytest

from oracle import stencils as ost
from oracle import operator as oop
from oracle import weights as ow
from paper_1404_0812_gb300 import workloads as W

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_knn_matches_kdtree_distances():
    from scipy.spatial import cKDTree
    ns = W.fibonacci_sphere(3000)
    tree = cKDTree(ns.X)
    d_ref, _ = tree.query(ns.X[::37], k=31)
    for r, k in enumerate(range(0, 3000, 37)):
        idx = ost.stencil(ns.X, k, 31)
        assert idx[0] == k
        d = np.linalg.norm(ns.X[idx] - ns.X[k], axis=1)
        np.testing.assert_allclose(d, d_ref[r], rtol=0, atol=1e-15)


def test_knn_tie_break_by_index():
    # unit square lattice: the 4 axis neighbours tie, then the 4 diagonals
    g = np.array([(i, j, 0.0) for i in range(5) for j in range(5)], dtype=np.float64)
    k = 12  # centre (2, 2)
    idx = ost.stencil(g, k, 9)
    assert list(idx) == [12, 7, 11, 13, 17, 6, 8, 16, 18]
    # a duplicate of the centre is the nearest other node (d^2 = 0)
    g2 = np.vstack([g, g[12:13]])
    assert list(ost.stencil(g2, 12, 3)) == [12, 25, 7]
    with pytest.raises(ValueError):
        ost.stencil(g, 0, 26)


def test_nnz_is_n_times_N():
    """Figure rcm: the share of non-zeros is n / N (0.31% for N = 10000 and
    0.62% for N = 5041 at n = 31); the oracle stores exactly n per row."""
    for key in ("rbc", "double_torus"):
        e = GOLDEN["nnz_fraction"][key]
        # the caption rounds to two decimals (31/5041 = 0.6150%, printed 0.62%)
        assert abs(100.0 * e["n"] / e["N"] - e["percent"]) < 0.006
    ns = W.icosahedral_sphere(2)
    op = oop.build_operator(ns.X, ns.normals, 13, ow.IMQ, eps=3.0)
    L = oop.dense(op, ns.N)
    assert np.count_nonzero(L) == 13 * ns.N


def test_apply_matches_dense_and_mixed_sizes():
    ns = W.icosahedral_sphere(2)
    nper = np.where(np.arange(ns.N) % 2 == 0, 11, 17)
    op = oop.build_operator(ns.X, ns.normals, nper, ow.GAUSSIAN, eps=2.0)
    assert list(op.n) == list(nper)
    u = W.uniform_field(ns.N, seed=3)
    np.testing.assert_allclose(oop.apply(op, u), oop.dense(op, ns.N) @ u, rtol=0,
                               atol=1e-12 * np.abs(op.w).sum(axis=1).max())


def test_node_generators_match_paper_counts():
    for lev, N in zip((3, 4), GOLDEN["icosahedral_node_counts"]["N"][:2]):
        ns = W.icosahedral_sphere(lev)
        assert ns.N == N
        np.testing.assert_allclose(np.linalg.norm(ns.X, axis=1), 1.0, atol=1e-15)
    for m, N in zip(GOLDEN["torus_node_counts"]["m"][:3], GOLDEN["torus_node_counts"]["N"][:3]):
        ns = W.torus_staggered(m)
        assert ns.N == N
        x, y, z = ns.X.T
        np.testing.assert_allclose((1 - np.sqrt(x * x + y * y)) ** 2 + z * z, 1 / 9, atol=1e-14)


def test_per_stencil_eps_spectrum_left_half_plane():
    """Section 5: with eps chosen per stencil for kappa_T the eigenvalues of
    L_X lie in the left half-plane (the zero eigenvalue of constants aside)."""
    ns = W.icosahedral_sphere(3)
    op = oop.build_operator(ns.X, ns.normals, 31, ow.GAUSSIAN, kappa_T=1e12)
    ev = np.linalg.eigvals(oop.dense(op, ns.N))
    assert ev.real.max() <= 1e-9 * np.abs(ev.real).max()
