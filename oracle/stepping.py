"""Oracle method-of-lines stepping (Section 4.2, Section 7).

Semi-discrete system (Eq. kernel_mol; Eq. diffusion_scalar writes the
coefficient as nu, the text as delta: the same quantity):
    d/dt u = delta_u L_X u + f(u, v),   d/dt v = delta_v L_X v + g(u, v).

Time stepping (Section 7 names SBDF2 with the diffusion implicit; Section 6
steps the diffusion equations with BDF4; neither formula is printed, so the
standard semi-implicit BDF family SBDFk of Ascher, Ruuth and Wetton (SIAM J.
Numer. Anal. 32, 1995) is used):
    alpha_k u^{n+1} - dt delta L u^{n+1} = sum_j a_kj u^{n-j} + dt sum_j b_kj f^{n-j},
j = 0 .. k-1, with the coefficients in SBDF below; for k = 2 this is
    (3 I - 2 dt delta L) u^{n+1} = 4 u^n - u^{n-1} + 2 dt (2 f^n - f^{n-1})
(up to the factor 2).  A run of order k whose history holds fewer than k - 1
past levels takes its first steps at orders 1, 2, ... (IMEX Euler first), or
starts from caller-given past levels (Section 6 bootstraps BDF4 from the exact
solution).
Each implicit system is solved by BiCGSTAB (Section 4.2, Section 6), in the
textbook form of van der Vorst (1992) as laid out in the Barrett et al.
"Templates" book, with x0 = u^n and the relative residual ||b - A x||_2 /
||b||_2 as the stopping test -- or, as Section 7 does for its SBDF2 runs, by
a sparse LU factorisation of each implicit matrix computed once and two
triangular solves per step (solver="lu"; SuperLU through scipy, the library
primitive standing in for the paper's sparse LU).

Reaction terms: the paper's Turing kinetics (Eqs. turing1/turing2), and the
Schnakenberg and Gray-Scott kinetics of the synthetic workloads.

Pins: tests/test_oracle_stepping.py (BiCGSTAB against a dense solve; SBDF2
with L = -lambda I against its closed-form recurrence; constant steady states
stay constant; heat-equation decay of Y_3^2 on the sphere; every monomial of
each kinetics recovered exactly by interpolation on a grid; Gray-Scott's
double-root equilibrium (1/2, 1/5) and its Jacobians; the LU solver against
a dense solve and against BiCGSTAB).
"""
from __future__ import annotations

import numpy as np


def reaction(p: dict, u: np.ndarray, v: np.ndarray):
    """(f(u,v), g(u,v)) for the model named in p["model"]."""
    m = p["model"]
    if m == "none":
        return np.zeros_like(u), np.zeros_like(v)
    if m == "linear":   # f = lu u, g = lv v (closed-form test problems)
        return p["lu"] * u, p["lv"] * v
    if m == "schnakenberg":
        uuv = u * u * v
        return p["gamma"] * (p["a"] - u + uuv), p["gamma"] * (p["b"] - uuv)
    if m == "gray_scott":
        uvv = u * v * v
        return -uvv + p["F"] * (1.0 - u), uvv - (p["F"] + p["k"]) * v
    if m == "barrio":   # Eqs. turing1, turing2
        a, b, g, t1, t2 = p["alpha"], p["beta"], p["gamma"], p["tau1"], p["tau2"]
        f = a * u * (1.0 - t1 * v * v) + v * (1.0 - t2 * u)
        gg = b * v * (1.0 + (a * t1 / b) * u * v) + u * (g + t2 * v)
        return f, gg
    raise ValueError(m)


def bicgstab(matvec, b: np.ndarray, x0: np.ndarray, tol: float, maxit: int):
    """BiCGSTAB (van der Vorst 1992).  Returns (x, iterations, relres, ok).

    ok is False on breakdown (rho or omega exactly zero) or when maxit is hit.
    """
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros_like(b), 0, 0.0, True
    x = x0.copy()
    r = b - matvec(x)
    if np.linalg.norm(r) / bnorm <= tol:
        return x, 0, np.linalg.norm(r) / bnorm, True
    rhat = r.copy()
    rho_prev = alpha = omega = 1.0
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    for it in range(1, maxit + 1):
        rho = float(rhat @ r)
        if rho == 0.0:
            return x, it, np.linalg.norm(r) / bnorm, False
        beta = (rho / rho_prev) * (alpha / omega)
        p = r + beta * (p - omega * v)
        v = matvec(p)
        alpha = rho / float(rhat @ v)
        s = r - alpha * v
        if np.linalg.norm(s) / bnorm <= tol:
            x = x + alpha * p
            return x, it, np.linalg.norm(s) / bnorm, True
        t = matvec(s)
        tt = float(t @ t)
        if tt == 0.0:
            return x, it, np.linalg.norm(s) / bnorm, False
        omega = float(t @ s) / tt
        x = x + alpha * p + omega * s
        r = s - omega * t
        rel = np.linalg.norm(r) / bnorm
        if rel <= tol:
            return x, it, rel, True
        if omega == 0.0:
            return x, it, rel, False
        rho_prev = rho
    return x, maxit, np.linalg.norm(r) / bnorm, False


# SBDFk: k -> (alpha_k, a_k0 .. a_k,k-1 (on u^{n-j}), b_k0 .. b_k,k-1 (on f^{n-j}))
SBDF = {
    1: (1.0, (1.0,), (1.0,)),
    2: (3.0 / 2.0, (2.0, -1.0 / 2.0), (2.0, -1.0)),
    3: (11.0 / 6.0, (3.0, -3.0 / 2.0, 1.0 / 3.0), (3.0, -3.0, 1.0)),
    4: (25.0 / 12.0, (4.0, -3.0, 4.0 / 3.0, -1.0 / 4.0), (4.0, -6.0, 4.0, -1.0)),
}


def imex_run(L_apply, u0, v0, p: dict, nsteps: int, tol: float = 1e-12,
             maxit: int = 200, history=None, order: int = 2, source=None, t0: float = 0.0,
             solver: str = "bicgstab", L_matrix=None):
    """Advance (u, v) by ``nsteps`` SBDF steps of the given order (1..4).

    ``source`` = (rate, h_u, h_v) adds the forcing exp(rate t) h(x) to the
    species' equations, taken at the new time t^{n+1} (implicitly, as Section
    6 does for its forced diffusion tests); ``t0`` is the time of u0.

    ``L_apply(x)`` returns L_X x.  ``v0`` may be None for one species.
    ``solver="lu"`` solves every implicit system with a sparse LU of
    alpha_k I - dt delta L_X (``L_matrix``, scipy sparse), factorised once
    per (order, species); its iteration counts are 0.
    ``history``: None, one past level (u_prev, v_prev, f_prev, g_prev), or a
    list of past levels, most recent first (f, g the kinetics at that level;
    None entries for a missing second species).  Returns dict(u, v,
    history = the most recent past level, levels = all kept past levels,
    iters = list of (iters_u, iters_v)).
    """
    if order not in SBDF:
        raise ValueError("order must be 1, 2, 3 or 4")
    dt, du = p["dt"], p["delta_u"]
    dv = p.get("delta_v", 0.0)
    two = v0 is not None
    u = np.asarray(u0, dtype=np.float64).copy()
    v = np.asarray(v0, dtype=np.float64).copy() if two else np.zeros_like(u)
    if history is None:
        levels = []
    elif isinstance(history, tuple):
        levels = [history]
    else:
        levels = list(history)
    levels = [tuple(np.zeros_like(u) if x is None else np.asarray(x, dtype=np.float64) for x in lv)
              for lv in levels]
    iters = []
    factors = {}

    def lu_solve(k, c0, c, rhs):
        from scipy.sparse import identity
        from scipy.sparse.linalg import splu
        if (k, c) not in factors:
            n = L_matrix.shape[0]
            factors[(k, c)] = splu((c0 * identity(n) - c * L_matrix).tocsc())
        return factors[(k, c)].solve(rhs)

    for _ in range(nsteps):
        f, g = reaction(p, u, v)
        k = min(order, len(levels) + 1)
        alpha, a, b = SBDF[k]
        past = [(u, v, f, g)] + levels[:k - 1]
        bu = sum(a[j] * past[j][0] for j in range(k)) + dt * sum(b[j] * past[j][2] for j in range(k))
        bv = sum(a[j] * past[j][1] for j in range(k)) + dt * sum(b[j] * past[j][3] for j in range(k))
        if source is not None:
            rate, hu, hv = source
            amp = np.exp(rate * (t0 + (len(iters) + 1) * dt))
            if hu is not None:
                bu = bu + dt * amp * hu
            if hv is not None:
                bv = bv + dt * amp * hv
        c0, cl = alpha, dt
        if solver == "lu":
            un, iu = lu_solve(k, c0, cl * du, bu), 0
            vn, iv = (lu_solve(k, c0, cl * dv, bv), 0) if two else (v, 0)
        else:
            Au = lambda x: c0 * x - (cl * du) * L_apply(x)
            un, iu, ru, oku = bicgstab(Au, bu, u, tol, maxit)
            if not oku:
                raise RuntimeError(f"BiCGSTAB (u) failed: relres {ru}")
            if two:
                Av = lambda x: c0 * x - (cl * dv) * L_apply(x)
                vn, iv, rv, okv = bicgstab(Av, bv, v, tol, maxit)
                if not okv:
                    raise RuntimeError(f"BiCGSTAB (v) failed: relres {rv}")
            else:
                vn, iv = v, 0
        levels = ([(u, v, f, g)] + levels)[:order - 1]
        u, v = un, vn
        iters.append((iu, iv))
    return dict(u=u, v=v if two else None, history=levels[0] if levels else None, levels=levels,
                iters=iters, t=t0 + len(iters) * dt)
