"""Arbitration of float64 parity by the high-precision oracle (test helper).

At kappa_T = 1e12 the weights of a stencil carry float64 rounding amplified
by the condition of A_P, so two float64 computations of the same weights
(the CUDA build's Cholesky-based four-solve form and the oracle's LU-based
G^d) differ from each other, and neither equals the exact weights.  The
judge of both is the weights of the same stencil and eps in 45-digit
arithmetic (``oracle.weights_hp.stencil_weights_hp``, Sections 2-4): the
CUDA path passes when its error against that truth is no larger than the
float64 oracle's own, up to a factor (rounding errors of two different
orderings are not equal, only of the same size).

Errors, over a set of sampled rows k (stencil idx_k, eps_k):
  applied  e = max_k |w_k . u[idx_k] - w_hp,k . u[idx_k]| / max_k |w_hp,k . u[idx_k]|
           (the relative L-infinity error of the applied operator on the
           sampled rows, the parity metric of the float64 build), for each
           field u;
  weights  e = max_k max_j |w_kj - w_hp,kj| / max_j |w_hp,kj|.
Dot products are summed exactly (decimal) so that the metric itself adds no
rounding.  The 45-digit weights run in a pool of spawned processes (the
decimal arithmetic is slow at n = 101: ~10 s per row).
"""
from __future__ import annotations

import multiprocessing as mp
import os
from decimal import Decimal, localcontext

import numpy as np

from oracle import weights as ow
from oracle import weights_hp as ohp


def exact_dot(w, u) -> float:
    with localcontext() as c:
        c.prec = 60
        s = sum((Decimal(float(a)) * Decimal(float(b)) for a, b in zip(w, u)), Decimal(0))
        return float(s)


def _hp_row(args):
    P, nrm, eps, kernel = args
    return ohp.stencil_weights_hp(P, nrm, eps, kernel)


def hp_weights(jobs, procs=None):
    """45-digit weights for each (P, normals, eps, kernel) job, in order."""
    procs = procs or max(1, min(len(jobs), os.cpu_count() or 1, 16))
    if procs == 1 or len(jobs) == 1:
        return [_hp_row(j) for j in jobs]
    with mp.get_context("spawn").Pool(procs) as pool:
        return pool.map(_hp_row, jobs, chunksize=1)


def arbitrate(X, normals, rows, stencils, eps, kernel, w_gpu, fields):
    """Errors of the CUDA weights ``w_gpu`` (one array of n_k values per
    sampled row) and of the float64 oracle's against the 45-digit oracle.

    rows: node indices k; stencils: idx_k arrays; eps: eps_k; fields: dict
    name -> u (N values).  Returns dict with, per field, applied errors
    ("gpu", "f64") and the weight errors under "weights".
    """
    jobs = [(X[s], normals[s], float(e), kernel) for s, e in zip(stencils, eps)]
    w_hp = hp_weights(jobs)
    w_64 = [ow.stencil_weights(P, nr, e, kernel) for P, nr, e, _ in jobs]
    out = {}
    for name, u in fields.items():
        y_hp = np.array([exact_dot(wh, u[s]) for wh, s in zip(w_hp, stencils)])
        y_gp = np.array([exact_dot(wg, u[s]) for wg, s in zip(w_gpu, stencils)])
        y_64 = np.array([exact_dot(w6, u[s]) for w6, s in zip(w_64, stencils)])
        scale = np.abs(y_hp).max()
        out[name] = {"gpu": float(np.abs(y_gp - y_hp).max() / scale),
                     "f64": float(np.abs(y_64 - y_hp).max() / scale),
                     "gpu_vs_f64": float(np.abs(y_gp - y_64).max() / np.abs(y_64).max())}
    eg = max(float(np.abs(np.asarray(wg) - wh).max() / np.abs(wh).max()) for wg, wh in zip(w_gpu, w_hp))
    e6 = max(float(np.abs(w6 - wh).max() / np.abs(wh).max()) for w6, wh in zip(w_64, w_hp))
    out["weights"] = {"gpu": eg, "f64": e6}
    out["rows"] = len(rows)
    return out


def assert_no_worse_than_f64(res, factor=2.0, floor=1e-12):
    """The CUDA path's error against the truth is at most ``factor`` times
    the float64 oracle's, plus ``floor`` (for errors at the rounding level
    of the metric itself), for every field and for the weights."""
    for name, r in res.items():
        if not isinstance(r, dict):
            continue
        assert r["gpu"] <= factor * r["f64"] + floor, (name, r)


def _cond2_chunk(args):
    Ps, eps, kernel = args
    return [ow.cond2(ow.interp_matrix(P, e, kernel)) for P, e in zip(Ps, eps)]


def cond2_many(Ps, eps, kernel, procs=None, chunk=500):
    """The oracle's kappa_2(A_P(eps)) (Section 5) for many stencils, in a
    pool of spawned processes."""
    jobs = [(Ps[i:i + chunk], eps[i:i + chunk], kernel) for i in range(0, len(Ps), chunk)]
    procs = procs or max(1, min(len(jobs), os.cpu_count() or 1, 16))
    if procs == 1:
        return np.concatenate([_cond2_chunk(j) for j in jobs])
    with mp.get_context("spawn").Pool(procs) as pool:
        return np.concatenate(pool.map(_cond2_chunk, jobs, chunksize=1))
