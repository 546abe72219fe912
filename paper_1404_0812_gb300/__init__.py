"""GB300-native RBF-FD discrete Laplace-Beltrami operator (sm_103a).

Python binding of the C ABI in ``include/rbffd.h``, with the same names:
``build_operator``, ``apply``, ``step_imex``, ``get_stencil_info``,
``get_eps``, ``get_ell``, ``get_rows``, ``destroy`` and the learned-eps calls.  The functions only
marshal arguments (torch tensors provide device memory and streams); all
arithmetic runs in the CUDA library, and a missing library is an error.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field

import torch

from . import _lib
from ._lib import (F32, F64, GAUSSIAN, IMQ, MODEL_BARRIO, MODEL_GRAY_SCOTT, MODEL_LINEAR,
                   MODEL_NONE, MODEL_SCHNAKENBERG, RbffdError)

KERNELS = {"gaussian": GAUSSIAN, "imq": IMQ}
MODELS = {"none": MODEL_NONE, "linear": MODEL_LINEAR, "schnakenberg": MODEL_SCHNAKENBERG,
          "gray_scott": MODEL_GRAY_SCOTT, "barrio": MODEL_BARRIO}


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dev(t, dtype):
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise ValueError(f"expected a contiguous CUDA {dtype} tensor")
    return t


class Operator:
    """Handle of a library-owned operator (rbffd_op)."""

    def __init__(self, handle, N, kernel):
        self.handle = handle
        self.N = N
        self.kernel = kernel

    @property
    def nnz(self) -> int:
        return int(_lib.load().rbffd_op_nnz(self.handle))

    @property
    def n_max(self) -> int:
        return int(_lib.load().rbffd_op_max_n(self.handle))

    def apply_bytes(self, dtype=F32) -> int:
        return int(_lib.load().rbffd_op_apply_bytes(self.handle, dtype))

    def __del__(self):
        try:
            destroy(self)
        except Exception:
            pass


def build_operator(nodes, normals, n=31, kernel="imq", kappa_target=1e12, eps_tol=1e-4,
                   max_evals=64, eps_override=None, mlps=None, accept=(0.5, 2.0),
                   block_threads=0, blocks_per_sm=0, stream=None, allow_failures=False,
                   eps_range=(0.0, 0.0), precision="f64"):
    """rbffd_build_operator.  ``n`` is an int or a CUDA int32 tensor (N,);
    ``mlps`` a list of EpsNet to warm-start the search; ``eps_range`` the
    search range of eps * r_s (0 = unbounded on that side); ``precision``
    "f64" or "dd" (double-double, for kappa_T beyond float64)."""
    lib = _lib.load()
    nodes = _dev(nodes, torch.float64)
    normals = _dev(normals, torch.float64)
    N = nodes.shape[0]
    o = _lib.BuildOpts()
    lib.rbffd_build_opts_default(C.byref(o))
    o.kernel = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
    o.kappa_target = float(kappa_target)
    o.eps_tol = float(eps_tol)
    o.max_evals = int(max_evals)
    o.accept_lo, o.accept_hi = float(accept[0]), float(accept[1])
    if eps_override is not None:
        eps_override = _dev(eps_override, torch.float64)
        o.eps_override = eps_override.data_ptr()
    if mlps:
        o.use_learned = 1
        for i, m in enumerate(mlps):
            o.mlp[i] = m.handle
    o.block_threads, o.blocks_per_sm = int(block_threads), int(blocks_per_sm)
    o.eps_lo, o.eps_hi = float(eps_range[0]), float(eps_range[1])
    o.precision = {"f64": _lib.PREC_F64, "dd": _lib.PREC_DD}[precision]
    if isinstance(n, torch.Tensor):
        npn = _dev(n, torch.int32)
        nptr, nu = C.c_void_p(npn.data_ptr()), 0
    else:
        nptr, nu = None, int(n)
    h = C.c_void_p()
    st = lib.rbffd_build_operator(C.c_void_p(nodes.data_ptr()), C.c_void_p(normals.data_ptr()), N,
                                  nptr, nu, C.byref(o), _stream(stream), C.byref(h))
    allow = (_lib.EPS_SEARCH_FAILED, _lib.ESINGULAR) if allow_failures else ()
    _lib.check(st, "rbffd_build_operator", allow)
    op = Operator(h, N, o.kernel)
    op.status = st
    return op


def autotune_build(nodes, normals, n=31, kernel="imq", kappa_target=1e12, sample=50_000,
                   cache_path=None, stream=None):
    """rbffd_autotune_build -> dict(block_threads, blocks_per_sm, ms)."""
    lib = _lib.load()
    nodes = _dev(nodes, torch.float64)
    normals = _dev(normals, torch.float64)
    o = _lib.BuildOpts()
    lib.rbffd_build_opts_default(C.byref(o))
    o.kernel = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
    o.kappa_target = float(kappa_target)
    if isinstance(n, torch.Tensor):
        nptr, nu = C.c_void_p(_dev(n, torch.int32).data_ptr()), 0
    else:
        nptr, nu = None, int(n)
    t, b, ms = C.c_int(), C.c_int(), C.c_double()
    path = None if cache_path is None else str(cache_path).encode()
    _lib.check(lib.rbffd_autotune_build(C.c_void_p(nodes.data_ptr()), C.c_void_p(normals.data_ptr()),
                                        nodes.shape[0], nptr, nu, C.byref(o), int(sample), path,
                                        _stream(stream), C.byref(t), C.byref(b), C.byref(ms)),
               "rbffd_autotune_build")
    return dict(block_threads=t.value, blocks_per_sm=b.value, ms=ms.value)


def stencil_weights_noalloc(nodes, normals, stencils, eps, kernel="imq", weights=None, stream=None):
    """rbffd_stencil_weights_noalloc: weights (rows x n float64) of caller-given
    stencils (rows x n int32, centre first) at caller-given eps, computed
    without any device allocation inside the library.  ``weights`` may be a
    preallocated CUDA float64 tensor.  Shapes are checked before anything
    reaches the library (the C call trusts N = nodes.shape[0], rows and n)."""
    _check_noalloc_shapes(nodes, normals, stencils, eps, weights)
    lib = _lib.load()
    nodes = _dev(nodes, torch.float64)
    normals = _dev(normals, torch.float64)
    stencils = _dev(stencils, torch.int32)
    eps = _dev(eps, torch.float64)
    rows, n = stencils.shape
    if weights is None:
        weights = torch.empty((rows, n), dtype=torch.float64, device=stencils.device)
    _dev(weights, torch.float64)
    here = torch.device("cuda", torch.cuda.current_device())
    for name, t in (("nodes", nodes), ("normals", normals), ("stencils", stencils), ("eps", eps),
                    ("weights", weights)):
        if t.device != here:
            raise ValueError(f"{name} is on {t.device}, not on the current device {here}")
    _lib.check(lib.rbffd_stencil_weights_noalloc(_ptr(nodes), _ptr(normals), nodes.shape[0], _ptr(stencils),
                                                 rows, n, _ptr(eps), KERNELS[kernel] if isinstance(kernel, str)
                                                 else int(kernel), _ptr(weights), _stream(stream)),
               "rbffd_stencil_weights_noalloc")
    return weights


def _check_noalloc_shapes(nodes, normals, stencils, eps, weights=None):
    """Shapes of rbffd_stencil_weights_noalloc's arguments: nodes and normals
    N x 3, stencils rows x n, eps (rows,), weights (rows, n) when given.
    Raises ValueError otherwise (a short array would be read or written past
    its end on the device)."""
    if nodes.dim() != 2 or nodes.shape[1] != 3:
        raise ValueError(f"nodes must be N x 3, got shape {tuple(nodes.shape)}")
    if tuple(normals.shape) != tuple(nodes.shape):
        raise ValueError(f"normals shape {tuple(normals.shape)} != nodes shape {tuple(nodes.shape)}")
    if stencils.dim() != 2:
        raise ValueError(f"stencils must be rows x n, got shape {tuple(stencils.shape)}")
    rows, n = stencils.shape
    if tuple(eps.shape) != (rows,):
        raise ValueError(f"eps shape {tuple(eps.shape)} != ({rows},)")
    if weights is not None and tuple(weights.shape) != (rows, n):
        raise ValueError(f"weights shape {tuple(weights.shape)} != ({rows}, {n})")


def apply(op: Operator, u, y=None, stream=None):
    """rbffd_apply: y = L_X u (float32 or float64 by u's dtype)."""
    lib = _lib.load()
    dt = F32 if u.dtype == torch.float32 else F64
    u = _dev(u, u.dtype)
    if y is None:
        y = torch.empty_like(u)
    _lib.check(lib.rbffd_apply(op.handle, _ptr(u), _ptr(y), dt, _stream(stream)), "rbffd_apply")
    return y


def get_stencil_info(op: Operator, stream=None):
    """rbffd_get_stencil_info -> dict(eps, kappa, evals, status) CUDA tensors."""
    lib = _lib.load()
    dev = torch.device("cuda")
    out = dict(eps=torch.empty(op.N, dtype=torch.float64, device=dev),
               kappa=torch.empty(op.N, dtype=torch.float64, device=dev),
               evals=torch.empty(op.N, dtype=torch.int32, device=dev),
               status=torch.empty(op.N, dtype=torch.int32, device=dev))
    _lib.check(lib.rbffd_get_stencil_info(op.handle, _ptr(out["eps"]), _ptr(out["kappa"]),
                                          _ptr(out["evals"]), _ptr(out["status"]), _stream(stream)),
               "rbffd_get_stencil_info")
    return out


def get_eps(op: Operator, stream=None):
    """rbffd_get_eps -> (eps float64, kappa float64, evals int32) CUDA tensors."""
    lib = _lib.load()
    eps = torch.empty(op.N, dtype=torch.float64, device="cuda")
    kappa = torch.empty(op.N, dtype=torch.float64, device="cuda")
    evals = torch.empty(op.N, dtype=torch.int32, device="cuda")
    _lib.check(lib.rbffd_get_eps(op.handle, _ptr(eps), _ptr(kappa), _ptr(evals), _stream(stream)),
               "rbffd_get_eps")
    return eps, kappa, evals


class _DeviceView:
    """Zero-copy wrapper of a library-owned device array (borrowed; valid
    while its operator lives)."""

    def __init__(self, ptr, count, typestr, owner):
        self.__cuda_array_interface__ = {"shape": (int(count),), "typestr": typestr,
                                         "data": (int(ptr or 0), False), "version": 2}
        self._owner = owner


def get_ell(op: Operator):
    """rbffd_get_ell -> dict with the sliced-ELL layout (ngroups, n, npad,
    row_begin, elem_begin, elems) and borrowed CUDA tensors row_node, idx,
    w64, w32 that alias the operator's storage (keep ``op`` alive)."""
    lib = _lib.load()
    v = _lib.EllView()
    _lib.check(lib.rbffd_get_ell(op.handle, C.byref(v)), "rbffd_get_ell")
    G = v.ngroups
    out = dict(ngroups=G, n=list(v.n[:G]), npad=list(v.npad[:G]), row_begin=list(v.row_begin[:G + 1]),
               elem_begin=list(v.elem_begin[:G + 1]), elems=int(v.elems))
    for name, count, ts in (("row_node", op.N, "<i4"), ("idx", v.elems, "<i4"),
                            ("w64", v.elems, "<f8"), ("w32", v.elems, "<f4")):
        out[name] = torch.as_tensor(_DeviceView(getattr(v, name), count, ts, op), device="cuda")
    return out


def morton_order(nodes, stream=None):
    """rbffd_morton_order -> CUDA int32 perm (perm[k] = original index of the
    k-th node in Z-order)."""
    nodes = _dev(nodes, torch.float64)
    perm = torch.empty(nodes.shape[0], dtype=torch.int32, device="cuda")
    _lib.check(_lib.load().rbffd_morton_order(_ptr(nodes), nodes.shape[0], _ptr(perm), _stream(stream)),
               "rbffd_morton_order")
    return perm


def rcm_order(op: Operator, stream=None):
    """rbffd_rcm_order -> CUDA int32 perm of op's stencil graph (Section 4.1's
    reverse Cuthill-McKee)."""
    perm = torch.empty(op.N, dtype=torch.int32, device="cuda")
    _lib.check(_lib.load().rbffd_rcm_order(op.handle, _ptr(perm), _stream(stream)), "rbffd_rcm_order")
    return perm


def rcm_order_host(rowptr, cols):
    """rbffd_rcm_order_host on a host CSR graph (numpy) -> numpy int32 perm."""
    import numpy as np
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    N = rowptr.shape[0] - 1
    perm = np.empty(N, dtype=np.int32)
    _lib.check(_lib.load(build=False).rbffd_rcm_order_host(rowptr.ctypes.data_as(C.c_void_p),
                                                           cols.ctypes.data_as(C.c_void_p), N,
                                                           perm.ctypes.data_as(C.c_void_p)),
               "rbffd_rcm_order_host")
    return perm


def get_rows(op: Operator, stream=None):
    """rbffd_get_rows -> (idx int32 N x n_max, w float64 N x n_max)."""
    lib = _lib.load()
    nm = op.n_max
    idx = torch.empty((op.N, nm), dtype=torch.int32, device="cuda")
    w = torch.empty((op.N, nm), dtype=torch.float64, device="cuda")
    _lib.check(lib.rbffd_get_rows(op.handle, _ptr(idx), _ptr(w), _stream(stream)), "rbffd_get_rows")
    return idx, w


def get_build_timings(op: Operator) -> dict:
    """rbffd_get_build_timings -> device ms of knn / guess / search / weights."""
    arr = (C.c_double * 4)()
    _lib.check(_lib.load().rbffd_get_build_timings(op.handle, arr), "rbffd_get_build_timings")
    return dict(knn=arr[0], guess=arr[1], search=arr[2], weights=arr[3])


def launch_count() -> int:
    """rbffd_launch_count: kernel launches issued by the library so far."""
    return int(_lib.load().rbffd_launch_count())


def destroy(op: Operator):
    if op is not None and op.handle:
        _lib.load().rbffd_destroy(op.handle)
        op.handle = None


@dataclass
class StepParams:
    model: str = "none"
    nspecies: int = 1
    dtype: torch.dtype = torch.float64
    dt: float = 1e-4
    delta_u: float = 1.0
    delta_v: float = 0.0
    coef: tuple = ()
    tol: float = 1e-12
    maxit: int = 200
    use_graph: bool = False
    order: int = 2          # SBDF order 1..4
    source_u: torch.Tensor | None = None   # forcing exp(source_rate t) h(x), taken at t^{n+1}
    source_v: torch.Tensor | None = None
    source_rate: float = 0.0
    solver: str = "bicgstab"   # or "lu": banded LU factors, two substitutions per step


@dataclass
class StepState:
    """Caller-owned CUDA vectors of one IMEX run (see rbffd_state)."""
    u: torch.Tensor
    v: torch.Tensor | None = None
    u_prev: torch.Tensor | None = None
    v_prev: torch.Tensor | None = None
    f_prev: torch.Tensor | None = None
    g_prev: torch.Tensor | None = None
    has_history: int = 0
    step: int = 0
    t: float = 0.0
    u_prev2: torch.Tensor | None = None
    v_prev2: torch.Tensor | None = None
    f_prev2: torch.Tensor | None = None
    g_prev2: torch.Tensor | None = None
    u_prev3: torch.Tensor | None = None
    v_prev3: torch.Tensor | None = None
    f_prev3: torch.Tensor | None = None
    g_prev3: torch.Tensor | None = None

    @staticmethod
    def create(u, v=None, order=2):
        z = lambda t: None if t is None else torch.zeros_like(t)
        s = StepState(u=u, v=v, u_prev=z(u), v_prev=z(v), f_prev=z(u), g_prev=z(v))
        if order >= 3:
            s.u_prev2, s.v_prev2, s.f_prev2, s.g_prev2 = z(u), z(v), z(u), z(v)
        if order >= 4:
            s.u_prev3, s.v_prev3, s.f_prev3, s.g_prev3 = z(u), z(v), z(u), z(v)
        return s


def model_coefs(p: dict):
    """(model name, coef tuple) from a reaction parameter dict."""
    m = p["model"]
    if m == "linear":
        return m, (p["lu"], p["lv"])
    if m == "schnakenberg":
        return m, (p["a"], p["b"], p["gamma"])
    if m == "gray_scott":
        return m, (p["F"], p["k"])
    if m == "barrio":
        return m, (p["alpha"], p["beta"], p["gamma"], p["tau1"], p["tau2"])
    return "none", ()


def step_imex(op: Operator, state: StepState, params: StepParams, nsteps: int, stream=None,
              allow_failure=False):
    """rbffd_step_imex; updates ``state`` in place and returns the report."""
    lib = _lib.load()
    sp = _lib.StepParams()
    sp.model = MODELS[params.model]
    sp.nspecies = params.nspecies
    sp.dtype = F32 if params.dtype == torch.float32 else F64
    sp.dt, sp.delta_u, sp.delta_v = params.dt, params.delta_u, params.delta_v
    for i, c in enumerate(params.coef):
        sp.coef[i] = c
    sp.tol, sp.maxit, sp.use_graph = params.tol, params.maxit, int(params.use_graph)
    sp.order = int(params.order)
    for name in ("source_u", "source_v"):
        h = getattr(params, name)
        if h is not None:
            setattr(sp, name, _dev(h, params.dtype).data_ptr())
    sp.source_rate = float(params.source_rate)
    sp.solver = {"bicgstab": _lib.SOLVER_BICGSTAB, "lu": _lib.SOLVER_BANDED_LU}[params.solver]
    cs = _lib.State(_ptr(state.u), _ptr(state.v), _ptr(state.u_prev), _ptr(state.v_prev),
                    _ptr(state.f_prev), _ptr(state.g_prev), state.has_history, state.step,
                    _ptr(state.u_prev2), _ptr(state.v_prev2), _ptr(state.f_prev2), _ptr(state.g_prev2),
                    _ptr(state.u_prev3), _ptr(state.v_prev3), _ptr(state.f_prev3), _ptr(state.g_prev3),
                    float(state.t))
    rep = _lib.StepReport()
    st = lib.rbffd_step_imex(op.handle, C.byref(cs), C.byref(sp), int(nsteps), _stream(stream),
                             C.byref(rep))
    state.has_history, state.step, state.t = cs.has_history, cs.step, cs.t
    allow = (_lib.SOLVER_NOT_CONVERGED,) if allow_failure else ()
    _lib.check(st, "rbffd_step_imex", allow)
    return dict(status=st, steps_done=rep.steps_done, max_iters_u=rep.max_iters_u,
                max_iters_v=rep.max_iters_v, total_iters=rep.total_iters,
                last_relres_u=rep.last_relres_u, last_relres_v=rep.last_relres_v,
                failed_step=rep.failed_step)


# ---------------------------------------------------------------------------
# direct solves (banded LU)
# ---------------------------------------------------------------------------

def op_bandwidth(op: Operator, stream=None):
    """rbffd_op_bandwidth -> (kl, ku) of op's matrix in node order."""
    kl, ku = C.c_int64(), C.c_int64()
    _lib.check(_lib.load().rbffd_op_bandwidth(op.handle, C.byref(kl), C.byref(ku), _stream(stream)),
               "rbffd_op_bandwidth")
    return kl.value, ku.value


class LU:
    """Handle of a library-owned banded LU factor (rbffd_lu) of
    alpha I - beta L_X."""

    def __init__(self, handle, N, dtype):
        self.handle = handle
        self.N = N
        self.dtype = dtype

    @property
    def bytes(self) -> int:
        return int(_lib.load().rbffd_lu_bytes(self.handle))

    def __del__(self):
        try:
            if self.handle:
                _lib.load().rbffd_lu_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


def lu_factor(op: Operator, alpha: float, beta: float, dtype=torch.float64, stream=None) -> LU:
    """rbffd_lu_factor: banded LU (partial pivoting) of alpha I - beta L_X."""
    h = C.c_void_p()
    _lib.check(_lib.load().rbffd_lu_factor(op.handle, float(alpha), float(beta),
                                           F32 if dtype == torch.float32 else F64, _stream(stream), C.byref(h)),
               "rbffd_lu_factor")
    return LU(h, op.N, dtype)


def lu_solve(lu: LU, b, x=None, stream=None):
    """rbffd_lu_solve: x = (alpha I - beta L_X)^{-1} b (x may be b)."""
    b = _dev(b, lu.dtype)
    if b.shape != (lu.N,):
        raise ValueError(f"b must have shape ({lu.N},)")
    if x is None:
        x = torch.empty_like(b)
    _dev(x, lu.dtype)
    _lib.check(_lib.load().rbffd_lu_solve(lu.handle, _ptr(b), _ptr(x), _stream(stream)), "rbffd_lu_solve")
    return x


def fp64_peak(stream=None) -> float:
    """FP64 FMA throughput of this GPU in GFLOP/s (microbenchmark)."""
    g = C.c_double()
    _lib.check(_lib.load().rbffd_fp64_peak(_stream(stream), C.byref(g)), "rbffd_fp64_peak")
    return g.value


def memory_pool_config(keep_bytes: int) -> None:
    """rbffd_memory_pool_config: bytes of transient scratch the library's
    pool keeps mapped between calls on the current device."""
    _lib.check(_lib.load().rbffd_memory_pool_config(int(keep_bytes)), "rbffd_memory_pool_config")


def release_memory() -> None:
    """rbffd_release_memory: return the pool's unused memory to the device."""
    _lib.check(_lib.load().rbffd_release_memory(), "rbffd_release_memory")


def memory_stats() -> dict:
    """rbffd_memory_stats: {"reserved": bytes mapped, "used": bytes in use}."""
    r, u = C.c_int64(), C.c_int64()
    _lib.check(_lib.load().rbffd_memory_stats(C.byref(r), C.byref(u)), "rbffd_memory_stats")
    return {"reserved": r.value, "used": u.value}


def fp64_mma_peak(stream=None) -> float:
    """FP64 tensor-path (mma.sync f64) throughput of this GPU in GFLOP/s."""
    g = C.c_double()
    _lib.check(_lib.load().rbffd_fp64_mma_peak(_stream(stream), C.byref(g)), "rbffd_fp64_mma_peak")
    return g.value


def selftest_barrier_timeout(stream=None) -> int:
    """rbffd_selftest_barrier_timeout; returns the status (TIMEOUT expected)."""
    return int(_lib.load().rbffd_selftest_barrier_timeout(_stream(stream)))


# ---------------------------------------------------------------------------
# learned eps warm start
# ---------------------------------------------------------------------------

class EpsNet:
    """Handle of a library-owned eps network (rbffd_mlp) for stencil size n."""

    def __init__(self, n: int, params=None):
        import numpy as np
        lib = _lib.load()
        self.n = int(n)
        self.P = int(lib.rbffd_mlp_param_count(self.n))
        h = C.c_void_p()
        buf = None
        if params is not None:
            buf = np.ascontiguousarray(np.asarray(params, dtype=np.float32).reshape(-1))
            if buf.size != self.P:
                raise ValueError(f"expected {self.P} parameters, got {buf.size}")
        _lib.check(lib.rbffd_mlp_create(self.n, None if buf is None else buf.ctypes.data_as(C.c_void_p),
                                        C.byref(h)), "rbffd_mlp_create")
        self.handle = h

    def params(self):
        import numpy as np
        out = np.empty(self.P, dtype=np.float32)
        _lib.check(_lib.load().rbffd_mlp_get_params(self.handle, out.ctypes.data_as(C.c_void_p)),
                   "rbffd_mlp_get_params")
        return out

    def load(self, params):
        """rbffd_mlp_load: replace the parameters (host float32, param_count
        values) and reset the Adam state."""
        import numpy as np
        buf = np.ascontiguousarray(np.asarray(params, dtype=np.float32).reshape(-1))
        if buf.size != self.P:
            raise ValueError(f"expected {self.P} parameters, got {buf.size}")
        _lib.check(_lib.load().rbffd_mlp_load(self.handle, buf.ctypes.data_as(C.c_void_p)),
                   "rbffd_mlp_load")

    def loss_grad(self, feats, target, stream=None):
        """rbffd_mlp_loss_grad -> (grad CUDA float32 tensor, loss float)."""
        feats = _dev(feats, torch.float32)
        target = _dev(target, torch.float32)
        g = torch.empty(self.P, dtype=torch.float32, device="cuda")
        l = torch.empty(1, dtype=torch.float32, device="cuda")
        _lib.check(_lib.load().rbffd_mlp_loss_grad(self.handle, _ptr(feats), _ptr(target),
                                                   target.shape[0], _ptr(g), _ptr(l), _stream(stream)),
                   "rbffd_mlp_loss_grad")
        return g, float(l.item())

    def train(self, feats, target, epochs=20, batch=1024, lr=1e-3, seed=0, stream=None):
        """rbffd_mlp_train -> list of per-epoch mean losses."""
        import numpy as np
        feats = _dev(feats, torch.float32)
        target = _dev(target, torch.float32)
        losses = np.zeros(epochs, dtype=np.float32)
        _lib.check(_lib.load().rbffd_mlp_train(self.handle, _ptr(feats), _ptr(target), target.shape[0],
                                               int(epochs), int(batch), float(lr), int(seed),
                                               _stream(stream), losses.ctypes.data_as(C.c_void_p)),
                   "rbffd_mlp_train")
        return losses.tolist()

    def predict(self, feats, stream=None):
        feats = _dev(feats, torch.float32)
        count = feats.shape[0]
        out = torch.empty(count, dtype=torch.float32, device="cuda")
        _lib.check(_lib.load().rbffd_mlp_predict(self.handle, _ptr(feats), count, _ptr(out),
                                                 _stream(stream)), "rbffd_mlp_predict")
        return out

    def __del__(self):
        try:
            if self.handle:
                _lib.load().rbffd_mlp_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


def features(op: Operator, nodes, normals, n: int, with_target=True, stream=None):
    """rbffd_features -> (feats count x 3n, target or None) for the rows of
    stencil size n, in node order."""
    lib = _lib.load()
    cnt = C.c_int64()
    # count = number of rows with this stencil size; ask first with a probe size
    N = op.N
    feats = torch.empty((N, 3 * n), dtype=torch.float32, device="cuda")
    target = torch.empty(N, dtype=torch.float32, device="cuda") if with_target else None
    _lib.check(lib.rbffd_features(op.handle, _ptr(_dev(nodes, torch.float64)),
                                  _ptr(_dev(normals, torch.float64)), int(n), _ptr(feats), _ptr(target),
                                  C.byref(cnt), _stream(stream)), "rbffd_features")
    c = int(cnt.value)
    return feats[:c], (target[:c] if with_target else None)
