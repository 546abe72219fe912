"""GPU parity of the double-double build (precision "dd") against the
high-precision oracle (oracle/weights_hp.py), at target condition numbers
float64 cannot reach (Section 6 computes its kappa_T = 1e18 / 1e20 weights in
quad precision), and against the float64 build where float64 suffices.

Tolerances: eps within 2 tol + 1e-5 eps (each search within tol of the root);
kappa at the returned eps by the oracle's definition within 1e-3 in log;
weights within 1e-9 of the row's largest (both are the same real numbers
rounded to float64 from ~1e-32 and ~1e-45 working precision; at kappa ~1e20
the residual rounding of the double-double solves is ~1e-12 relative)."""
import math

import numpy as np
import pytest
import torch

from oracle import operator as oop
from oracle import stencils as ost
from oracle import weights as ow
from oracle import weights_hp as hp
from paper_1404_0812_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def T(a, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


@pytest.fixture(scope="module")
def R():
    import paper_1404_0812_gb300 as R
    R._lib.load()
    return R


@pytest.mark.parametrize("kernel,n,kT", [("imq", 17, 1e20), ("gaussian", 11, 1e18)])
def test_dd_search_matches_high_precision_oracle(R, kernel, n, kT):
    ns = W.fibonacci_sphere(400)
    kid = ow.KERNELS[kernel]
    op = R.build_operator(T(ns.X), T(ns.normals), n, kernel=kernel, kappa_target=kT, precision="dd")
    info = {k: v.cpu().numpy() for k, v in R.get_stencil_info(op).items()}
    assert np.all(info["status"] == 0)
    assert np.all(np.abs(np.log(info["kappa"] / kT)) < 0.15)
    idx, w = R.get_rows(op)
    idx, w = idx.cpu().numpy(), w.cpu().numpy()
    for k in (0, 133, 399):
        sref = ost.stencil(ns.X, k, n)
        assert np.array_equal(idx[k, :n], sref.astype(np.int32))
        P, Nr = ns.X[sref], ns.normals[sref]
        e_ref, _, _ = hp.search_eps_hp(P, kid, kT)
        assert abs(info["eps"][k] - e_ref) <= 2e-4 + 1e-5 * e_ref
        assert abs(math.log(hp.cond2_hp(P, info["eps"][k], kid) / info["kappa"][k])) < 1e-3
        wref = hp.stencil_weights_hp(P, Nr, info["eps"][k], kid)
        assert np.abs(w[k, :n] - wref).max() <= 1e-9 * np.abs(wref).max()
        assert abs(w[k, :n].sum()) <= 1e-9 * np.abs(wref).sum()


def test_dd_fixed_eps_weights(R):
    """Weights at given eps (eps_override) in double-double at kappa ~1e20."""
    ns = W.fibonacci_sphere(400)
    n = 17
    rows = (5, 250)
    eps = np.full(ns.N, 1.0)
    for k in rows:
        sref = ost.stencil(ns.X, k, n)
        eps[k], _, _ = hp.search_eps_hp(ns.X[sref], ow.IMQ, 1e20)
    op = R.build_operator(T(ns.X), T(ns.normals), n, kernel="imq", eps_override=T(eps), precision="dd")
    _, w = R.get_rows(op)
    w = w.cpu().numpy()
    for k in rows:
        sref = ost.stencil(ns.X, k, n)
        wref = hp.stencil_weights_hp(ns.X[sref], ns.normals[sref], eps[k], ow.IMQ)
        assert np.abs(w[k, :n] - wref).max() <= 1e-9 * np.abs(wref).max()


def test_dd_equals_float64_where_float64_suffices(R):
    ns = W.icosahedral_sphere(3)
    X, Nr = T(ns.X), T(ns.normals)
    a = R.build_operator(X, Nr, 31, kernel="imq", kappa_target=1e10)
    b = R.build_operator(X, Nr, 31, kernel="imq", kappa_target=1e10, precision="dd")
    ea, eb = (R.get_stencil_info(o)["eps"].cpu().numpy() for o in (a, b))
    assert np.all(np.abs(ea - eb) <= 2e-4 + 1e-5 * ea)
    ref = oop.build_operator(ns.X, ns.normals, 31, ow.IMQ, eps=eb)
    u = W.sph_harm_y32(ns.X)
    y = R.apply(b, T(u)).cpu().numpy()
    assert np.abs(y - oop.apply(ref, u)).max() <= 1e-8 * np.abs(oop.apply(ref, u)).max()
