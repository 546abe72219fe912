"""Oracle of the double-double build: Sections 2-5 in high precision.

Test infrastructure only (like the rest of ``oracle/``).  The same steps as
``oracle.weights`` -- kernel, augmented interpolation matrix A_P (Eq.
rbf_linsys), projected gradient matrices B^d (Eq. grad_x_f_interp),
G^d = B^d A_P^{-1}, L_P = sum_d G^d G^d (Eq. surface_lap_P1) and its first
row, kappa_2 = max|lambda| / min|lambda| (Section 5), the shape parameter as
the zero of F(eps) = ln(kappa / kappa_T) (Eq. target_cond) -- with every
operation in Python's decimal arithmetic at ``PREC`` significant digits, for
target condition numbers beyond float64: Section 6 computes its
kappa_T = 1e18 / 1e20 weights in quad precision and rounds them to float64,
as these functions do.  Float64 inputs convert exactly (Decimal(float)).

Written out here rather than taken from a library (the standard library has
no multiprecision linear algebra): the eigenvalues by the cyclic Jacobi
method (Rutishauser's rotation formulas, stopping when the off-diagonal
mass is below 1e-36 of the matrix's), and A_P^{-1} by Gauss-Jordan
elimination with partial pivoting.

Pins: tests/test_oracle_weights_hp.py (Jacobi eigenvalues against LAPACK on a
well-conditioned matrix, the two-node closed form of kappa and of its root at
kappa_T = 1e20, agreement with the float64 oracle where float64 suffices,
vanishing row sums and the Laplace-Beltrami eigenvalue of Y_3^2 at
kappa_T = 1e20).
"""
from __future__ import annotations

import decimal
import math
from decimal import Decimal

import numpy as np

from .weights import GAUSSIAN, IMQ, brent_root

PREC = 45


def _ctx():
    c = decimal.Context(prec=PREC, Emin=-999999, Emax=999999)
    return decimal.localcontext(c)


def _d(x: float) -> Decimal:
    return Decimal(float(x))


def _phi(kernel: int, e2r2: Decimal) -> Decimal:
    if kernel == GAUSSIAN:
        return (-e2r2).exp()
    if kernel == IMQ:
        return 1 / (1 + e2r2).sqrt()
    raise ValueError(kernel)


def _psi(kernel: int, e2: Decimal, e2r2: Decimal) -> Decimal:
    """phi'(r) / r in terms of eps^2 and (eps r)^2."""
    if kernel == GAUSSIAN:
        return -2 * e2 * (-e2r2).exp()
    s = 1 + e2r2
    return -e2 / (s * s.sqrt())


def interp_matrix_hp(P: np.ndarray, eps: float, kernel: int):
    """A_P(eps) (Eq. rbf_linsys) as a list of Decimal rows (call inside _ctx)."""
    X = [[_d(v) for v in row] for row in P]
    n = len(X)
    e2 = _d(eps) * _d(eps)
    A = [[Decimal(0)] * (n + 1) for _ in range(n + 1)]
    for i in range(n):
        for j in range(i + 1):
            r2 = sum((X[i][c] - X[j][c]) ** 2 for c in range(3))
            A[i][j] = A[j][i] = _phi(kernel, e2 * r2)
        A[i][n] = A[n][i] = Decimal(1)
    return A


def jacobi_eigenvalues(A) -> list:
    """Eigenvalues of the symmetric matrix A (Decimal rows) by cyclic Jacobi
    rotations (call inside _ctx; A is overwritten)."""
    m = len(A)
    total = sum(A[i][j] * A[i][j] for i in range(m) for j in range(m))
    tiny = total * Decimal(10) ** -72
    for _ in range(100):
        off = sum(A[i][j] * A[i][j] for i in range(m) for j in range(m) if i != j)
        if off <= tiny:
            break
        for p in range(m - 1):
            for q in range(p + 1, m):
                apq = A[p][q]
                if apq == 0:
                    continue
                # rotation that zeroes A[p][q]: theta = (a_qq - a_pp) / (2 a_pq),
                # t = sign(theta) / (|theta| + sqrt(theta^2 + 1))
                theta = (A[q][q] - A[p][p]) / (2 * apq)
                t = 1 / (abs(theta) + (theta * theta + 1).sqrt())
                if theta < 0:
                    t = -t
                c = 1 / (t * t + 1).sqrt()
                s = t * c
                for k in range(m):
                    akp, akq = A[k][p], A[k][q]
                    A[k][p] = c * akp - s * akq
                    A[k][q] = s * akp + c * akq
                for k in range(m):
                    apk, aqk = A[p][k], A[q][k]
                    A[p][k] = c * apk - s * aqk
                    A[q][k] = s * apk + c * aqk
    else:
        raise RuntimeError("Jacobi did not converge")
    return [A[i][i] for i in range(m)]


def cond2_hp(P: np.ndarray, eps: float, kernel: int) -> float:
    """kappa_2(A_P(eps)) = max|lambda| / min|lambda| (Section 5)."""
    with _ctx():
        lam = [abs(x) for x in jacobi_eigenvalues(interp_matrix_hp(P, eps, kernel))]
        return float(max(lam) / min(lam))


def inverse_hp(A):
    """A^{-1} by Gauss-Jordan elimination with partial pivoting (call inside
    _ctx)."""
    m = len(A)
    M = [list(A[i]) + [Decimal(1) if j == i else Decimal(0) for j in range(m)] for i in range(m)]
    for col in range(m):
        piv = max(range(col, m), key=lambda r: abs(M[r][col]))
        M[col], M[piv] = M[piv], M[col]
        pv = M[col][col]
        if pv == 0:
            raise ZeroDivisionError("singular matrix")
        M[col] = [v / pv for v in M[col]]
        for r in range(m):
            if r != col and M[r][col] != 0:
                f = M[r][col]
                M[r] = [a - f * b for a, b in zip(M[r], M[col])]
    return [row[m:] for row in M]


def search_eps_hp(P: np.ndarray, kernel: int, kappa_T: float, xtol: float = 1e-4, max_bracket: int = 60):
    """The float64 oracle's search (same start eps_0 = 1 / mean distance,
    doubling / halving bracket and Brent-Dekker root finder, Section 5) with
    kappa evaluated in high precision.  Returns (eps, kappa, evaluations)."""
    d = np.sqrt(np.sum((P[1:] - P[0]) ** 2, axis=1))
    e0 = 1.0 / float(np.mean(d))
    f = lambda e: math.log(cond2_hp(P, e, kernel) / kappa_T)
    f0 = f(e0)
    evals = 1
    a, fa = e0, f0
    step = 2.0 if f0 > 0.0 else 0.5
    for _ in range(max_bracket):
        b = a * step
        fb = f(b)
        evals += 1
        if fa * fb <= 0.0:
            break
        a, fa = b, fb
    else:
        raise RuntimeError("eps bracket not found")
    lo, flo, hi, fhi = (a, fa, b, fb) if a < b else (b, fb, a, fa)
    eps, k = brent_root(f, lo, hi, flo, fhi, xtol)
    return eps, cond2_hp(P, eps, kernel), evals + k


def stencil_weights_hp(P: np.ndarray, normals: np.ndarray, eps: float, kernel: int) -> np.ndarray:
    """First row of L_P = sum_d G^d G^d, G^d = B^d A_P^{-1} restricted to the
    node columns (Sections 3-4), in high precision, rounded to float64."""
    with _ctx():
        X = [[_d(v) for v in row] for row in P]
        Nn = [[_d(v) for v in row] for row in normals]
        n = len(X)
        e2 = _d(eps) * _d(eps)
        Ainv = inverse_hp(interp_matrix_hp(P, eps, kernel))
        G = []
        for dcomp in range(3):
            B = [[Decimal(0)] * (n + 1) for _ in range(n)]
            for i in range(n):
                for j in range(n):
                    # [P(x_i)(x_i - x_j)]_d = (x_i - x_j)_d - n_i,d (n_i . (x_i - x_j))
                    diff = [X[i][c] - X[j][c] for c in range(3)]
                    r2 = sum(v * v for v in diff)
                    nd = sum(Nn[i][c] * diff[c] for c in range(3))
                    B[i][j] = _psi(kernel, e2, e2 * r2) * (diff[dcomp] - Nn[i][dcomp] * nd)
            G.append([[sum(B[i][k] * Ainv[k][j] for k in range(n + 1)) for j in range(n)] for i in range(n)])
        w = [sum(G[dcomp][0][k] * G[dcomp][k][j] for dcomp in range(3) for k in range(n)) for j in range(n)]
        return np.array([float(v) for v in w])
