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
