"""Oracle method-of-lines stepping (Section 4.2, Section 7).

Semi-discrete system (Eq. kernel_mol; Eq. diffusion_scalar writes the
coefficient as nu, the text as delta: the same quantity):
    d/dt u = delta_u L_X u + f(u, v),   d/dt v = delta_v L_X v + g(u, v).

Time stepping (Section 7 names SBDF2 with the diffusion implicit; the formula
is not printed, so the standard second-order semi-implicit BDF is used):
    (3 I - 2 dt delta L) u^{n+1} = 4 u^n - u^{n-1} + 2 dt (2 f^n - f^{n-1}),
with a first step of IMEX Euler, (I - dt delta L) u^1 = u^0 + dt f^0.
Each implicit system is solved by BiCGSTAB (Section 4.2, Section 6), in the
textbook form of van der Vorst (1992) as laid out in the Barrett et al.
"Templates" book, with x0 = u^n and the relative residual ||b - A x||_2 /
||b||_2 as the stopping test.

Reaction terms: the paper's Turing kinetics (Eqs. turing1/turing2), and the
Schnakenberg and Gray-Scott kinetics of the synthetic workloads.

Pins: tests/test_oracle_stepping.py (BiCGSTAB against a dense solve; SBDF2
with L = -lambda I against its closed-form recurrence; constant steady states
stay constant; heat-equation decay of Y_3^2 on the sphere).
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


def imex_run(L_apply, u0, v0, p: dict, nsteps: int, tol: float = 1e-12,
             maxit: int = 200, history=None):
    """Advance (u, v) by ``nsteps`` IMEX steps (Euler first, then SBDF2).

    ``L_apply(x)`` returns L_X x.  ``v0`` may be None for one species.
    ``history`` = (u_prev, v_prev, f_prev, g_prev) continues an SBDF2 run.
    Returns dict(u, v, history, iters=list of (iters_u, iters_v)).
    """
    dt, du = p["dt"], p["delta_u"]
    dv = p.get("delta_v", 0.0)
    two = v0 is not None
    u = np.asarray(u0, dtype=np.float64).copy()
    v = np.asarray(v0, dtype=np.float64).copy() if two else np.zeros_like(u)
    hist = history
    iters = []
    for _ in range(nsteps):
        f, g = reaction(p, u, v)
        if hist is None:     # IMEX Euler
            c0, cl = 1.0, dt
            bu, bv = u + dt * f, v + dt * g
        else:                # SBDF2
            up, vp, fp, gp = hist
            c0, cl = 3.0, 2.0 * dt
            bu = 4.0 * u - up + 2.0 * dt * (2.0 * f - fp)
            bv = 4.0 * v - vp + 2.0 * dt * (2.0 * g - gp)
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
        hist = (u, v, f, g)
        u, v = un, vn
        iters.append((iu, iv))
    return dict(u=u, v=v if two else None, history=hist, iters=iters)
