"""Oracle RBF-FD weights for the surface Laplacian (Sections 2-5).

Steps, in the paper's order and notation, all in float64:

1. Radial kernel phi(r) with shape parameter eps (Section 2): Gaussian
   exp(-(eps r)^2) or inverse multiquadric 1/sqrt(1 + (eps r)^2) (the paper's
   choice).  r is the straight-line distance in R^3.
2. Augmented interpolation matrix A_P (Eq. rbf_linsys on the stencil P):
   [[Phi, 1], [1^T, 0]], (n+1) x (n+1).
3. Projector P = I - n n^T at each node (Eq. proj_mat) and the surface
   gradient matrices B^d (Eq. grad_x_f_interp):
   (B^d)_{ij} = p^d(x_i) . grad phi(|x - x_j|) at x = x_i
             = psi(r_ij) [P(x_i)(x_i - x_j)]_d,  psi(r) = phi'(r)/r,
   with a zero column for the constant term.
4. G^d = B^d A^{-1} restricted to the n node columns (Section 4), one solve
   with A for the three right-hand-side blocks.
5. L_P = G^x G^x + G^y G^y + G^z G^z (Eq. surface_lap_P1); the weights are
   the first row (the centre).
6. Condition number in the 2-norm, kappa = max|lambda| / min|lambda| of the
   symmetric A_P (Section 5).
7. Shape parameter per stencil: the zero of F(eps) = log(kappa(A_P(eps)) /
   kappa_T) (Eq. target_cond), to an absolute tolerance of 1e-4 on eps
   (Section 5).  Readings (the paper names no root-finder, log base or
   bracket): natural log; Brent-Dekker on a bracket found by doubling or
   halving eps from eps_0 = 1 / (mean centre-to-neighbour distance); the
   tolerance is on eps.

Pins: tests/test_oracle_weights.py (n = 2 closed form of kappa and of its
root, LAPACK-independent brute-force checks, row sums, reproduction of
kernel shifts, rigid-motion / normal-sign / permutation invariance, scaling,
Laplace-Beltrami eigenfunctions on the sphere, the torus Laplacian of
Section 6).
"""
from __future__ import annotations

import math

import numpy as np

GAUSSIAN = 0
IMQ = 1
KERNELS = {"gaussian": GAUSSIAN, "imq": IMQ}


def phi(kernel: int, eps: float, r2: np.ndarray) -> np.ndarray:
    """phi(eps r) as a function of r^2 (Section 2)."""
    e2r2 = (eps * eps) * r2
    if kernel == GAUSSIAN:
        return np.exp(-e2r2)
    if kernel == IMQ:
        return 1.0 / np.sqrt(1.0 + e2r2)
    raise ValueError(kernel)


def psi(kernel: int, eps: float, r2: np.ndarray) -> np.ndarray:
    """phi'(r) / r, the radial factor of grad phi(|x - x_j|) (Eq. grad)."""
    e2 = eps * eps
    e2r2 = e2 * r2
    if kernel == GAUSSIAN:
        return -2.0 * e2 * np.exp(-e2r2)
    if kernel == IMQ:
        return -e2 / (1.0 + e2r2) ** 1.5
    raise ValueError(kernel)


def pair_sq_dist(P: np.ndarray) -> np.ndarray:
    """r_ij^2 over the stencil nodes P (n x 3)."""
    D = P[:, None, :] - P[None, :, :]
    return np.sum(D * D, axis=2)


def interp_matrix(P: np.ndarray, eps: float, kernel: int) -> np.ndarray:
    """A_P(eps) of Eq. rbf_linsys over the stencil (Section 4)."""
    n = P.shape[0]
    A = np.zeros((n + 1, n + 1))
    A[:n, :n] = phi(kernel, eps, pair_sq_dist(P))
    A[:n, n] = 1.0
    A[n, :n] = 1.0
    return A


def projectors(normals: np.ndarray) -> np.ndarray:
    """P(x_i) = I - n_i n_i^T (Eq. proj_mat), shape (n, 3, 3)."""
    return np.eye(3)[None, :, :] - normals[:, :, None] * normals[:, None, :]


def grad_matrices(P: np.ndarray, normals: np.ndarray, eps: float, kernel: int) -> np.ndarray:
    """B^x, B^y, B^z of Eq. grad_x_f_interp with the zero constant column.

    Returns (3, n, n+1): [d, i, j] = psi(r_ij) [P(x_i)(x_i - x_j)]_d.
    """
    n = P.shape[0]
    D = P[:, None, :] - P[None, :, :]                 # x_i - x_j
    Pr = projectors(normals)                          # (n,3,3)
    proj = np.einsum("ide,ije->dij", Pr, D)           # [P(x_i)(x_i - x_j)]_d
    B = np.zeros((3, n, n + 1))
    B[:, :, :n] = psi(kernel, eps, pair_sq_dist(P))[None, :, :] * proj
    return B


def cond2(A: np.ndarray) -> float:
    """2-norm condition number of the symmetric A_P: max|lambda| / min|lambda|
    (Section 5).  LAPACK symmetric eigenvalues are the library primitive."""
    lam = np.abs(np.linalg.eigvalsh(A))
    return float(lam.max() / lam.min())


def diff_matrices(P: np.ndarray, normals: np.ndarray, eps: float, kernel: int) -> np.ndarray:
    """G^d = B^d A_P^{-1}, keeping the n node columns (Section 4).  (3, n, n)."""
    n = P.shape[0]
    A = interp_matrix(P, eps, kernel)
    B = grad_matrices(P, normals, eps, kernel)
    # B^d A^{-1} = (A^{-1} B^{dT})^T since A is symmetric; one factorisation.
    rhs = np.concatenate([B[0].T, B[1].T, B[2].T], axis=1)   # (n+1, 3n)
    sol = np.linalg.solve(A, rhs)                            # A^{-1} B^T
    G = np.stack([sol[:, d * n:(d + 1) * n].T for d in range(3)])  # (3, n, n+1)
    return G[:, :, :n]


def local_laplacian(P: np.ndarray, normals: np.ndarray, eps: float, kernel: int) -> np.ndarray:
    """L_P = sum_d G^d G^d (Eq. surface_lap_P1), n x n."""
    G = diff_matrices(P, normals, eps, kernel)
    return G[0] @ G[0] + G[1] @ G[1] + G[2] @ G[2]


def stencil_weights(P: np.ndarray, normals: np.ndarray, eps: float, kernel: int) -> np.ndarray:
    """RBF-FD weights w_j of Eq. fd_weights: the first row of L_P."""
    return local_laplacian(P, normals, eps, kernel)[0].copy()


# ----------------------------------------------------------------------------
# shape parameter (Section 5, Eq. target_cond)
# ----------------------------------------------------------------------------

def target_F(P: np.ndarray, eps: float, kernel: int, kappa_T: float) -> float:
    """F(eps, kappa_T) = log(kappa(A_P(eps)) / kappa_T) (Eq. target_cond)."""
    return math.log(cond2(interp_matrix(P, eps, kernel)) / kappa_T)


def brent_root(f, a: float, b: float, fa: float, fb: float, xtol: float,
               maxiter: int = 200):
    """Brent-Dekker zero finder on a sign-changing bracket [a, b].

    The textbook method (Brent, "Algorithms for Minimization without
    Derivatives", 1973, ch. 4): inverse quadratic interpolation or secant
    steps, falling back to bisection whenever the interpolated step is not
    safely inside the bracket.  Stops when the bracket half-width is at most
    tol1 = 2 u |b| + xtol / 2 (u the float64 machine epsilon) or f(b) == 0.
    Returns (root, number of f evaluations).
    """
    if fa * fb > 0.0:
        raise ValueError("no sign change")
    u = np.finfo(np.float64).eps
    c, fc = a, fa
    d = e = b - a
    evals = 0
    for _ in range(maxiter):
        if fb * fc > 0.0:
            c, fc = a, fa
            d = e = b - a
        if abs(fc) < abs(fb):
            a, b, c = b, c, b
            fa, fb, fc = fb, fc, fb
        tol1 = 2.0 * u * abs(b) + 0.5 * xtol
        m = 0.5 * (c - b)
        if abs(m) <= tol1 or fb == 0.0:
            return b, evals
        if abs(e) >= tol1 and abs(fa) > abs(fb):
            s = fb / fa
            if a == c:                       # secant
                p = 2.0 * m * s
                q = 1.0 - s
            else:                            # inverse quadratic interpolation
                q = fa / fc
                r = fb / fc
                p = s * (2.0 * m * q * (q - r) - (b - a) * (r - 1.0))
                q = (q - 1.0) * (r - 1.0) * (s - 1.0)
            if p > 0.0:
                q = -q
            else:
                p = -p
            if 2.0 * p < min(3.0 * m * q - abs(tol1 * q), abs(e * q)):
                e, d = d, p / q
            else:
                d = e = m
        else:
            d = e = m
        a, fa = b, fb
        b = b + (d if abs(d) > tol1 else math.copysign(tol1, m))
        fb = f(b)
        evals += 1
    raise RuntimeError("Brent did not converge")


def search_eps(P: np.ndarray, kernel: int, kappa_T: float, xtol: float = 1e-4,
               max_bracket: int = 60):
    """Per-stencil shape parameter of Section 5.

    Bracket: start at eps_0 = 1 / mean(|x_j - x_1|, j >= 2); while F > 0
    (kappa too large, eps too small) double eps, while F < 0 halve it, until F
    changes sign.  Then Brent to an absolute eps tolerance ``xtol``.
    Returns (eps, kappa(A(eps)), number of kappa evaluations).
    """
    d = np.sqrt(np.sum((P[1:] - P[0]) ** 2, axis=1))
    e0 = 1.0 / float(np.mean(d))
    f = lambda e: target_F(P, e, kernel, kappa_T)
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
    evals += k
    return eps, cond2(interp_matrix(P, eps, kernel)), evals
