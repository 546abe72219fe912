"""The C-ABI library builds for sm_103a, loads, and exports every function
include/rbffd.h declares (no GPU needed: nothing is called)."""
import os
import re
import ctypes

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rbffd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rbffd_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_1404_0812_gb300 import _lib
    lib = _lib.load()
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # every declared function also has a ctypes signature in the binding
    assert set(names) <= set(_lib.SIGNATURES), set(names) - set(_lib.SIGNATURES)


def test_status_strings_without_gpu():
    from paper_1404_0812_gb300 import _lib
    lib = _lib.load()
    assert lib.rbffd_status_str(0) == b"ok"
    assert b"BiCGSTAB" in lib.rbffd_status_str(5)
    o = _lib.BuildOpts()
    lib.rbffd_build_opts_default(ctypes.byref(o))
    assert o.kappa_target == 1e12 and o.eps_tol == 1e-4 and o.kernel == _lib.IMQ
    assert (o.accept_lo, o.accept_hi) == (0.5, 2.0)


def test_argument_checks_need_no_gpu():
    """Entry points validate their arguments before touching the device:
    these return RBFFD_EINVAL (1) on a machine without a GPU."""
    from paper_1404_0812_gb300 import _lib
    lib = _lib.load()
    assert lib.rbffd_memory_pool_config(-1) == _lib.EINVAL
    assert lib.rbffd_fp64_peak(None, None) == _lib.EINVAL
    assert lib.rbffd_fp64_mma_peak(None, None) == _lib.EINVAL
    assert lib.rbffd_build_operator(None, None, 10, None, 5, None, None, None) == _lib.EINVAL
    assert b"NULL" in lib.rbffd_last_error() or b"invalid" in lib.rbffd_last_error()


def test_noalloc_binding_rejects_mismatched_shapes_before_the_call():
    """stencil_weights_noalloc checks every shape before anything reaches the
    library, whose kernel trusts N = nodes.shape[0], rows and n (a short
    array would be read or written past its end on the device).  CPU
    tensors: the shape check fires first, no GPU is touched."""
    import torch
    import paper_1404_0812_gb300 as R
    f64, i32 = torch.float64, torch.int32
    X, Nr = torch.zeros(50, 3, dtype=f64), torch.zeros(50, 3, dtype=f64)
    S, e, w = torch.zeros(8, 10, dtype=i32), torch.zeros(8, dtype=f64), torch.zeros(8, 10, dtype=f64)
    bad = [
        dict(nodes=torch.zeros(50, 2, dtype=f64)),        # not N x 3
        dict(nodes=torch.zeros(150, dtype=f64)),          # flat
        dict(normals=torch.zeros(49, 3, dtype=f64)),      # fewer normals than nodes
        dict(stencils=torch.zeros(80, dtype=i32)),        # not rows x n
        dict(eps=torch.zeros(7, dtype=f64)),              # shorter than rows
        dict(weights=torch.zeros(8, 9, dtype=f64)),       # smaller than rows x n
        dict(weights=torch.zeros(7, 10, dtype=f64)),
    ]
    for b in bad:
        kw = dict(nodes=X, normals=Nr, stencils=S, eps=e, weights=w)
        kw.update(b)
        with pytest.raises(ValueError, match="shape|must be"):
            R.stencil_weights_noalloc(**kw)
