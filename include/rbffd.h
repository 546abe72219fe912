/*
 * rbffd.h - C ABI of the GB300 (sm_103a) RBF-FD surface Laplace-Beltrami
 * library: batched per-stencil operator build with a per-stencil shape
 * parameter, fixed-width (sliced ELL) application, and IMEX (SBDF of order
 * 1-4 + BiCGSTAB) reaction-diffusion stepping.
 *
 * Method: Shankar, Wright, Kirby, Fogelson, "A Radial Basis Function
 * (RBF)-Finite Difference (FD) Method for Diffusion and Reaction-Diffusion
 * Equations on Surfaces".  Each entry point cites the section / equation
 * that defines what it computes.
 *
 * Conventions for every call:
 *  - Pointers marked "device" are CUDA device pointers on the current
 *    device; "host" pointers are ordinary host memory.  Arrays are dense and
 *    C-contiguous.  Node coordinates and normals are N x 3 row-major float64.
 *  - The caller owns every buffer it passes; the library owns what it
 *    allocates inside an rbffd_op / rbffd_mlp until the matching destroy,
 *    and the transient scratch of its calls, which lives in a library-owned
 *    memory pool (rbffd_memory_pool_config, rbffd_release_memory).
 *  - Work is queued on the given stream (a cudaStream_t passed as void*;
 *    NULL is the legacy default stream).  Calls that return data to host
 *    memory or a status depending on device results synchronise that stream.
 *  - Nothing throws across the ABI: every call returns an rbffd_status, and
 *    rbffd_last_error() gives a one-line message for the last failure on the
 *    calling thread.
 */
#ifndef RBFFD_H
#define RBFFD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RBFFD_OK = 0,
    RBFFD_EINVAL = 1,                 /* bad argument (size, pointer, option) */
    RBFFD_ECUDA = 2,                  /* a CUDA runtime call failed */
    RBFFD_ENOMEM = 3,                 /* device allocation failed */
    RBFFD_EPS_SEARCH_FAILED = 4,      /* some stencil's eps search found no root */
    RBFFD_SOLVER_NOT_CONVERGED = 5,   /* BiCGSTAB hit its cap or broke down */
    RBFFD_TIMEOUT = 6,                /* a bounded device-side wait gave up */
    RBFFD_NOT_IMPLEMENTED = 7,
    RBFFD_ESINGULAR = 8               /* a local interpolation matrix is not
                                         numerically positive definite */
} rbffd_status;

enum { RBFFD_GAUSSIAN = 0, RBFFD_IMQ = 1 };   /* Section 2 kernels */
enum { RBFFD_F32 = 0, RBFFD_F64 = 1 };        /* stepping / apply precision */
enum { RBFFD_PREC_F64 = 0, RBFFD_PREC_DD = 1 }; /* arithmetic of the operator build */
enum { RBFFD_MAX_GROUPS = 8, RBFFD_MAX_N = 128 };

/* Per-stencil status codes written by the build (rbffd_get_stencil_info). */
enum { RBFFD_STENCIL_OK = 0, RBFFD_STENCIL_NO_BRACKET = 1,
       RBFFD_STENCIL_NO_CONVERGENCE = 2, RBFFD_STENCIL_SINGULAR = 3,
       RBFFD_STENCIL_ACCEPTED_PREDICTION = 4 };

typedef struct rbffd_op rbffd_op;     /* opaque, library-owned operator */
typedef struct rbffd_mlp rbffd_mlp;   /* opaque, library-owned eps network */

/* Options of rbffd_build_operator. */
typedef struct {
    int kernel;               /* RBFFD_GAUSSIAN or RBFFD_IMQ (Section 2) */
    double kappa_target;      /* kappa_T of Eq. target_cond (> 1) */
    double eps_tol;           /* absolute tolerance on eps (Section 5: 1e-4) */
    int max_evals;            /* cap on kappa evaluations per stencil (e.g. 64) */
    int use_learned;          /* 1: first guess from the network in mlp[] whose
                                 stencil size matches the row's n */
    double accept_lo;         /* accept the prediction when kappa(A(eps_hat)) */
    double accept_hi;         /*   lies in [accept_lo, accept_hi] * kappa_T */
    const double* eps_override; /* device, N, or NULL: fixed eps per node (no
                                   search; kappa/evals reported as NaN/0) */
    const rbffd_mlp* mlp[RBFFD_MAX_GROUPS]; /* learned networks (may be NULL) */
    int block_threads;        /* 0 = autotuned / default launch shape */
    int blocks_per_sm;        /* 0 = autotuned / default launch shape */
    double eps_lo;            /* search range of the dimensionless eps * r_s */
    double eps_hi;            /*   (r_s = the stencil's largest centre distance);
                                 0 = unbounded on that side.  A stencil whose
                                 root lies outside gets RBFFD_STENCIL_NO_BRACKET */
    int precision;            /* RBFFD_PREC_F64 (default) or RBFFD_PREC_DD: the
                                 geometry, Phi, its factorisation, the A^{-1}
                                 solves and the weights in double-double
                                 arithmetic (unit roundoff ~1e-32) for kappa_T
                                 beyond float64 (Section 6 uses quad precision
                                 for kappa_T = 1e18 / 1e20); the weights are
                                 rounded to float64.  Much slower; the launch
                                 shape fields are ignored. */
} rbffd_build_opts;

/* Fill opts with defaults: IMQ, kappa_T 1e12, eps_tol 1e-4, max_evals 64,
 * no learned start, band [0.5, 2], unbounded eps range. */
void rbffd_build_opts_default(rbffd_build_opts* opts);

/*
 * rbffd_autotune_build - choose the launch shape (threads per block, resident
 * blocks per SM) of the build's lane-per-stencil kernels for this device and
 * workload (a systems addition; the paper has no GPU).  Builds the operator
 * on every (N / sample)-th node (same surface and stencil sizes, coarser
 * spacing; the sample is raised to at least 8 stencils per lane of the
 * largest candidate) with each candidate shape, times the search + weights phases with
 * CUDA events, and returns the fastest in *block_threads / *blocks_per_sm
 * (and its time in *best_ms, -1 when it came from the cache).  Arguments as
 * in rbffd_build_operator; cache_path (may be NULL) is a text file of
 * previous results keyed by device, stencil sizes, kernel and kappa_T; a hit
 * skips the timing.  Synchronises the stream.
 */
rbffd_status rbffd_autotune_build(const double* nodes, const double* normals, int64_t N,
                                  const int32_t* n_per_node, int n_uniform,
                                  const rbffd_build_opts* opts, int64_t sample,
                                  const char* cache_path, void* stream, int* block_threads,
                                  int* blocks_per_sm, double* best_ms);

/*
 * rbffd_build_operator - the discrete surface Laplacian L_X (Section 4).
 *
 * For every node k: its stencil P_k (k first, then its n_k - 1 nearest other
 * nodes by Euclidean distance in R^3, ties broken by node index; Section 4,
 * Section 4.1), a shape parameter eps_k (the zero of
 * F(eps) = ln(kappa_2(A_{P_k}(eps)) / kappa_T), Eq. target_cond, searched to
 * opts->eps_tol; Section 5) and the weights: the first row of
 * L_P = G^x G^x + G^y G^y + G^z G^z, G^d = B^d A^{-1} (Eqs. proj_mat,
 * grad_x_f_interp, surface_lap_P1).  The local linear algebra is float64,
 * except the short Lanczos estimate of max|lambda(A)| inside kappa_2, which
 * runs in float32 (its relative error, ~1e-6, moves ln kappa by as much and
 * eps_k by far less than eps_tol).
 *
 *   nodes      device, N x 3 float64, distinct points on the surface
 *   normals    device, N x 3 float64, unit normals (sign irrelevant)
 *   N          number of nodes (>= 2)
 *   n_per_node device int32 N (stencil size of each node, 2..128, at most 8
 *              distinct values) or NULL to use n_uniform for every node
 *   opts       options (NULL = defaults)
 *   stream     cudaStream_t (void*)
 *   out        receives the new operator (NULL on failure)
 *
 * Returns RBFFD_OK, RBFFD_EINVAL (bad sizes / options), RBFFD_ENOMEM,
 * RBFFD_ECUDA, or RBFFD_EPS_SEARCH_FAILED / RBFFD_ESINGULAR when at least one
 * stencil failed (the operator is still returned; per-stencil status is in
 * rbffd_get_stencil_info).  Synchronises the stream.
 */
rbffd_status rbffd_build_operator(const double* nodes, const double* normals, int64_t N,
                                  const int32_t* n_per_node, int n_uniform,
                                  const rbffd_build_opts* opts, void* stream,
                                  rbffd_op** out);

/*
 * rbffd_apply - y = L_X u (Eq. kernel_mol, explicit part; Section 4.2).
 *   u, y   device, N values of dtype (RBFFD_F32 uses the float32 copy of the
 *          weights, RBFFD_F64 the float64 weights); u and y must not alias.
 * Asynchronous on the stream.  Returns RBFFD_EINVAL on a bad dtype/pointer.
 */
rbffd_status rbffd_apply(const rbffd_op* op, const void* u, void* y, int dtype, void* stream);

/* IMEX stepping parameters (Section 4.2, Section 7). */
enum { RBFFD_MODEL_NONE = 0, RBFFD_MODEL_LINEAR = 1, RBFFD_MODEL_SCHNAKENBERG = 2,
       RBFFD_MODEL_GRAY_SCOTT = 3, RBFFD_MODEL_BARRIO = 4 };
typedef struct {
    int model;          /* reaction kinetics, see coef below */
    int nspecies;       /* 1 (u only, heat/forced diffusion) or 2 (u, v) */
    int dtype;          /* RBFFD_F32 or RBFFD_F64 state and arithmetic
                           (float32 dot products accumulate in float64, or,
                           for large operators, in compensated float32 --
                           Ogita-Rump-Oishi Dot2 -- of the same accuracy) */
    double dt;          /* time step */
    double delta_u, delta_v;   /* diffusion coefficients */
    double coef[8];     /* LINEAR: lu, lv.  SCHNAKENBERG: a, b, gamma.
                           GRAY_SCOTT: F, k.  BARRIO (Eqs. turing1/2):
                           alpha, beta, gamma, tau1, tau2 */
    double tol;         /* BiCGSTAB relative residual tolerance */
    int maxit;          /* BiCGSTAB iteration cap per solve */
    int use_graph;      /* 1: replay each step from a captured CUDA graph */
    int order;          /* SBDF order 1..4 (0 = 2, the SBDF2 of Section 7;
                           4 = the BDF4 of Section 6 with explicit kinetics) */
    const void* source_u;   /* device, N values of dtype, or NULL: a forcing   */
    const void* source_v;   /*   s(t, x) = exp(source_rate t) h(x) added to the */
    double source_rate;     /*   species' equation and taken at t^{n+1}, i.e.   */
                            /*   implicitly (Section 6's forced diffusion tests) */
    int solver;         /* RBFFD_SOLVER_BICGSTAB (0, Section 4.2 / Section 6) or
                           RBFFD_SOLVER_BANDED_LU (Section 7: each implicit
                           matrix factorised once, two substitutions per
                           step; see rbffd_lu_factor -- the nodes should be in
                           a bandwidth-reducing order).  tol / maxit apply to
                           BiCGSTAB only; an LU step reports 0 iterations */
} rbffd_step_params;

enum { RBFFD_SOLVER_BICGSTAB = 0, RBFFD_SOLVER_BANDED_LU = 1 };

/*
 * State of an IMEX run.  All vectors are caller-owned device arrays of N
 * values of params.dtype.  u, v: current solution (updated in place);
 * u_prev, v_prev, f_prev, g_prev: the past level n-1 (u^{n-1}, v^{n-1},
 * f(u^{n-1}, v^{n-1}), g(...)); *_prev2 and *_prev3 the levels n-2 and n-3
 * (needed for order 3 / 4 only, else may be NULL).  has_history = the number
 * of valid past levels: a step of order k uses min(k, has_history + 1)
 * (0 makes it IMEX Euler; a run without history climbs one order per step,
 * or the caller fills the past levels, e.g. from an exact solution, and sets
 * has_history = k - 1); the call updates it.  v and the v_ / g_ levels may
 * be NULL when nspecies = 1.
 */
typedef struct {
    void* u; void* v;
    void* u_prev; void* v_prev; void* f_prev; void* g_prev;
    int has_history;
    int64_t step;       /* steps taken so far (updated) */
    void* u_prev2; void* v_prev2; void* f_prev2; void* g_prev2;
    void* u_prev3; void* v_prev3; void* f_prev3; void* g_prev3;
    double t;           /* time of u (used by a source term; advanced by the call) */
} rbffd_state;

typedef struct {
    int64_t steps_done;
    int32_t max_iters_u, max_iters_v;   /* worst BiCGSTAB iteration counts */
    int64_t total_iters;                /* sum over solves */
    double last_relres_u, last_relres_v;
    int64_t failed_step;                /* -1 if none */
} rbffd_step_report;

/*
 * rbffd_step_imex - advance the semi-discrete reaction-diffusion system
 * d/dt u = delta_u L_X u + f(u,v), d/dt v = delta_v L_X v + g(u,v)
 * (Eq. kernel_mol; Eqs. turing1/turing2 for the paper's kinetics) by nsteps
 * steps of the semi-implicit BDF of params->order (SBDFk, Ascher-Ruuth-Wetton:
 * diffusion implicit, kinetics extrapolated), e.g. for k = 2
 *   (3 I - 2 dt delta L) u^{n+1} = 4 u^n - u^{n-1} + 2 dt (2 f^n - f^{n-1}),
 * and for k = 4
 *   (25 I - 12 dt delta L) u^{n+1} = 48 u^n - 36 u^{n-1} + 16 u^{n-2} - 3 u^{n-3}
 *                                    + 12 dt (4 f^n - 6 f^{n-1} + 4 f^{n-2} - f^{n-3})
 *                                    + 12 dt s(t^{n+1})
 * (s the optional source of params, zero without one),
 * each implicit system solved by BiCGSTAB from x0 = u^n (Section 4.2), or
 * by the banded LU factors (params->solver).  Operators with fewer than 1024
 * rows per SM: one cooperative persistent launch per step; larger ones:
 * BiCGSTAB as a sequence of kernels whose iteration loop runs on the device
 * (a WHILE node of the CUDA graph, or, with use_graph = 0, the same kernels
 * from a host loop).  Either path is replayed from a CUDA graph when
 * use_graph = 1 (captured at the first call, again whenever an argument
 * changes).  Synchronises the stream at the end and fills report (may be
 * NULL).  Returns RBFFD_SOLVER_NOT_CONVERGED (with report->failed_step) or
 * RBFFD_TIMEOUT when a bounded wait gave up.
 */
rbffd_status rbffd_step_imex(rbffd_op* op, rbffd_state* state, const rbffd_step_params* params,
                             int64_t nsteps, void* stream, rbffd_step_report* report);

/* ------------------------------------------------------------------------
 * Direct solves (Section 7 factors the SBDF2 matrix once by a sparse LU and
 * uses the triangular factors for a forward and a back substitution every
 * step).  M = alpha I - beta L_X in node order is factorised as a banded
 * matrix with partial pivoting (row interchanges; LAPACK's banded-LU
 * layout): lower / upper bandwidths kl / ku of L_X (rbffd_op_bandwidth), U
 * with upper bandwidth kl + ku.  Bandwidths come from the node numbering:
 * renumber by reverse Cuthill-McKee first (rbffd_rcm_order, Section 4.1);
 * the factor takes (2 kl + ku + 1) N + (kl + 1) N values of the dtype.
 * ---------------------------------------------------------------------- */
typedef struct rbffd_lu rbffd_lu;     /* opaque, library-owned factor */

/* Largest i - j (*kl) and j - i (*ku) over the nonzeros (i, j) of op's
 * matrix in node order.  Synchronises the stream. */
rbffd_status rbffd_op_bandwidth(const rbffd_op* op, int64_t* kl, int64_t* ku, void* stream);

/*
 * rbffd_lu_factor - factorise M = alpha I - beta L_X (for SBDF2 alpha = 3,
 * beta = 2 dt delta) in dtype (RBFFD_F32 with op's float32 weights,
 * RBFFD_F64 with its float64 weights).  Synchronises the stream.  Returns
 * RBFFD_ESINGULAR when a pivot column is exactly zero, RBFFD_EINVAL when
 * kl + ku is too large for the substitutions' shared-memory window (about
 * 3,200 in float64 / 6,400 in float32 at full prefetch depth, twice that at
 * half depth), RBFFD_ENOMEM when the band does not fit, RBFFD_TIMEOUT when a
 * bounded grid barrier gave up.  *out is NULL on failure.
 */
rbffd_status rbffd_lu_factor(const rbffd_op* op, double alpha, double beta, int dtype, void* stream,
                             rbffd_lu** out);
/* x = M^{-1} b (device vectors of N values of the factor's dtype, node
 * order; x may alias b).  Asynchronous on the stream. */
rbffd_status rbffd_lu_solve(const rbffd_lu* lu, const void* b, void* x, void* stream);
/* Device bytes held by the factor. */
int64_t rbffd_lu_bytes(const rbffd_lu* lu);
void rbffd_lu_destroy(rbffd_lu* lu);

/*
 * Per-stencil results of the build, in node order (device outputs, each
 * may be NULL): eps (float64 N, in the units of the node coordinates),
 * kappa (float64 N: kappa_2(A(eps)) at the returned eps, NaN when eps was
 * given), evals (int32 N: kappa evaluations used), status (int32 N: the
 * RBFFD_STENCIL_* codes).  Copies on the stream; asynchronous.
 */
rbffd_status rbffd_get_stencil_info(const rbffd_op* op, double* eps, double* kappa,
                                    int32_t* evals, int32_t* status, void* stream);

/* eps, kappa and evals of rbffd_get_stencil_info (Section 5), without the
 * status array (device outputs, each may be NULL; asynchronous copies).
 * Returns RBFFD_EINVAL when op is NULL, RBFFD_ECUDA when a copy fails. */
rbffd_status rbffd_get_eps(const rbffd_op* op, double* eps, double* kappa, int32_t* evals,
                           void* stream);

/*
 * Borrowed views of the operator's storage (Section 4.1's N x n weight
 * matrix, stored as sliced ELL), valid until rbffd_destroy(op).  Rows are
 * grouped by stencil size (groups by descending n); operator row r of group
 * g (row_begin[g] <= r < row_begin[g+1]) is row row_node[r] of L_X.  Entry j
 * (0 <= j < npad[g]) of the group's local row q = r - row_begin[g] is element
 *   elem_begin[g] + (q / 32) * 32 * npad[g] + (j / 4) * 128 + (q % 32) * 4 + j % 4
 * of idx (int32 column = node index), w64 (float64 weight) and w32 (its
 * float32 copy); entries j >= n[g] hold the row's own node and weight 0,
 * and the rows that pad a group's last slice of 32 hold index 0 and weight
 * 0 (every index is a valid node).  All pointers are device memory
 * owned by op; the call itself touches no device memory.  Returns
 * RBFFD_EINVAL on a NULL argument.
 */
typedef struct {
    int ngroups;
    int n[RBFFD_MAX_GROUPS];
    int npad[RBFFD_MAX_GROUPS];                /* n rounded up to a multiple of 4 */
    int64_t row_begin[RBFFD_MAX_GROUPS + 1];
    int64_t elem_begin[RBFFD_MAX_GROUPS + 1];
    int64_t elems;                             /* total elements, padding included */
    const int32_t* row_node;                   /* N */
    const int32_t* idx;
    const double* w64;
    const float* w32;
} rbffd_ell_view;
rbffd_status rbffd_get_ell(const rbffd_op* op, rbffd_ell_view* view);

/*
 * Operator rows in node order as dense padded arrays (device outputs):
 * idx int32 N x n_max and w float64 N x n_max (entries past a row's n_k
 * hold the row's own node and weight 0).  n_max = rbffd_op_max_n(op).
 */
rbffd_status rbffd_get_rows(const rbffd_op* op, int32_t* idx, double* w, void* stream);
/*
 * Device time of the phases of the last rbffd_build_operator that produced
 * op, from CUDA events recorded on its stream around the launches (ms):
 * [0] stencils (kNN), [1] learned first guess, [2] shape-parameter search
 * (which also forms the weights from its last factorisation), [3] weights
 * at given eps (eps_override builds only; 0 otherwise).  Host-side work
 * between launches is not included.
 */
rbffd_status rbffd_get_build_timings(const rbffd_op* op, double ms[4]);
/* Kernel launches issued by this library since it was loaded. */
int64_t rbffd_launch_count(void);
int64_t rbffd_op_nodes(const rbffd_op* op);
int rbffd_op_max_n(const rbffd_op* op);
int64_t rbffd_op_nnz(const rbffd_op* op);      /* sum of n_k (Section 4.1) */
/* Bytes one rbffd_apply of the given dtype must move: nnz * (weight + 4)
 * + 2 N * element size. */
int64_t rbffd_op_apply_bytes(const rbffd_op* op, int dtype);
void rbffd_destroy(rbffd_op* op);

/*
 * rbffd_stencil_weights_noalloc - surface-Laplacian weights for stencils and
 * shape parameters the caller already has, without allocating any memory.
 * (The paper has no counterpart: it is an interface for callers that may not
 * allocate, not a step of the method.)
 *
 * Who needs it: code that must not call cudaMalloc / cudaFree while it runs
 * -- for example a time loop on an evolving surface that re-forms weights
 * every step inside a region where another framework owns the whole device
 * heap, or an application that keeps the device running asynchronously and
 * cannot afford the implicit device-wide synchronisation that cudaMalloc and
 * cudaFree cause.  rbffd_build_operator allocates its operator and scratch;
 * this call allocates nothing: the caller passes inputs and outputs, and the
 * per-stencil working memory is a fixed 32 MiB array inside the library's
 * device image (every GPU that loads the library keeps it until exit).
 *
 *   nodes, normals  device, N x 3 float64 (normals unit, sign irrelevant)
 *   N               number of nodes (>= 2)
 *   stencils        device, rows x n int32, row-major, centre node first;
 *                   every index in [0, N)
 *   rows            number of stencils (0 is allowed)
 *   n               stencil size, 2 <= n <= min(N, 128); larger sizes are
 *                   rejected with RBFFD_EINVAL (the fixed array bounds n)
 *   eps             device, rows float64, shape parameter of each stencil in
 *                   the units of the coordinates
 *   kernel          RBFFD_GAUSSIAN or RBFFD_IMQ
 *   weights         device out, rows x n float64: the first row of
 *                   L_P = sum_d G^d G^d for each stencil (same arithmetic as
 *                   the weights of rbffd_build_operator)
 *
 * Returns RBFFD_ESINGULAR when some rows had an out-of-range index or a
 * local matrix that is not numerically positive definite (those rows are
 * NaN).  Synchronises the stream.  The first call on a device looks up the
 * array's device address (once per device, with that device current, kept
 * for the life of the process: after a cudaDeviceReset of that device the
 * kept address is stale and this call must not be used again); make that
 * first call before any stream capture.  All calls share the one array
 * and its failure counter, which keep the last call's contents: the counter
 * is cleared at the start of each call, and calls whose work overlaps on the
 * GPU (different streams or threads without ordering) race on the array.
 */
rbffd_status rbffd_stencil_weights_noalloc(const double* nodes, const double* normals, int64_t N,
                                           const int32_t* stencils, int64_t rows, int n,
                                           const double* eps, int kernel, double* weights,
                                           void* stream);

/* ------------------------------------------------------------------------
 * Locality orderings of the nodes (Section 4.1 reorders L_X by reverse
 * Cuthill-McKee for faster iterative solves).  Each returns perm (N int32,
 * perm[k] = the original index of the node placed k-th); the library never
 * reorders on its own: the caller applies perm to its node, normal and field
 * arrays (x_new[k] = x[perm[k]]) and builds on the reordered set.  The sorts
 * and searches run on the host (one-off O(N log N) / O(nnz) steps);
 * synchronous.  Errors: RBFFD_EINVAL (NULL argument, N out of range,
 * non-finite coordinates, a column index out of range), RBFFD_ECUDA.
 * ---------------------------------------------------------------------- */

/* Z-order (Morton) of the nodes: 21-bit quantisation of each coordinate
 * over the bounding cube, bits interleaved x-y-z, ties by index.
 * nodes: device N x 3 float64; perm: device out. */
rbffd_status rbffd_morton_order(const double* nodes, int64_t N, int32_t* perm, void* stream);
/* Reverse Cuthill-McKee (George-Liu) of op's stencil graph (node k linked
 * to its n_k - 1 neighbours, symmetrised): per connected component a
 * pseudo-peripheral start, breadth-first visits with neighbours in
 * increasing degree (ties by index), the whole order reversed.  perm: device
 * out, in op's node numbering. */
rbffd_status rbffd_rcm_order(const rbffd_op* op, int32_t* perm, void* stream);
/* The same on a host CSR graph (rowptr N+1 int64, cols int32, symmetrised
 * inside; self loops and repeats ignored); perm: host out.  Needs no GPU. */
rbffd_status rbffd_rcm_order_host(const int64_t* rowptr, const int32_t* cols, int64_t N, int32_t* perm);

/* ------------------------------------------------------------------------
 * Learned shape-parameter warm start (not in the paper; the paper's search
 * of Section 5 stays as the fallback and the arbiter).
 * Features of a stencil (3n floats): tangent-frame offsets (t1.d, t2.d,
 * nh.d) / r_s of every stencil node (centre first), with nh oriented so
 * sum nh.d <= 0, t1 the unit tangent part of the nearest neighbour's offset,
 * t2 = nh x t1, r_s the largest offset.  Target: ln(eps * r_s).
 * Network: 3n -> 64 -> 64 -> 1, GELU (erf form) hidden layers, float32.
 * Flat parameter layout: W1 (row-major 3n x 64), b1[64], W2 (64 x 64),
 * b2[64], W3[64], b3[1].
 * ---------------------------------------------------------------------- */

/* Number of float parameters for stencil size n. */
int64_t rbffd_mlp_param_count(int n);
/* Create a network for stencil size n from host float32 params (layout
 * above; NULL = zeros). */
rbffd_status rbffd_mlp_create(int n, const float* params_host, rbffd_mlp** out);
rbffd_status rbffd_mlp_get_params(const rbffd_mlp* mlp, float* params_host);
/* Replace a network's parameters with host float32 params (layout above;
 * param_count floats) and reset its Adam state.  Synchronous.  Returns
 * RBFFD_EINVAL on a NULL argument, RBFFD_ECUDA when the copy fails. */
rbffd_status rbffd_mlp_load(rbffd_mlp* mlp, const float* params_host);
void rbffd_mlp_destroy(rbffd_mlp* mlp);

/*
 * Features of the stencils of every node whose stencil size is n, in node
 * order (device out: count x 3n float32, count = number of such nodes,
 * returned in *count_host) and, when target is not NULL, the training target
 * ln(eps * r_s) from the operator's eps (device out: count float32).
 * nodes / normals must be the arrays the operator was built from.
 */
rbffd_status rbffd_features(const rbffd_op* op, const double* nodes, const double* normals,
                            int n, float* feats, float* target, int64_t* count_host,
                            void* stream);

/*
 * One forward + backward pass of the MSE loss over a batch (device inputs
 * feats count x 3n, target count; device outputs grad (param_count floats)
 * and loss (1 float)).  Used to check gradients against the oracle.
 */
rbffd_status rbffd_mlp_loss_grad(const rbffd_mlp* mlp, const float* feats, const float* target,
                                 int64_t count, float* grad, float* loss, void* stream);

/*
 * Adam training on the device: epochs passes over (feats, target) in
 * seeded shuffled mini-batches of `batch`; lr, beta1 0.9, beta2 0.999,
 * eps 1e-8.  loss_host (may be NULL) receives the mean loss of each epoch.
 * Synchronises the stream.
 */
rbffd_status rbffd_mlp_train(rbffd_mlp* mlp, const float* feats, const float* target,
                             int64_t count, int epochs, int batch, float lr, uint64_t seed,
                             void* stream, float* loss_host);

/* Predictions ln(eps * r_s) for count feature rows (device in / out). */
rbffd_status rbffd_mlp_predict(const rbffd_mlp* mlp, const float* feats, int64_t count,
                               float* out, void* stream);

/*
 * Failure-detection self test of the bounded grid barrier used by
 * rbffd_step_imex: launches one block that waits at the barrier for a second
 * arrival that never comes.  The wait gives up after about a second, the
 * kernel returns, and the call returns RBFFD_TIMEOUT with the CUDA context
 * still usable (any other status means the bound is broken).
 */
rbffd_status rbffd_selftest_barrier_timeout(void* stream);

/*
 * Transient device memory.  The scratch that calls need only while they run
 * (the search's per-lane matrices -- about 15 GB for a 1M-node build with
 * stencils up to n = 101 at the default launch shape -- the kNN grid, the
 * learned guesses, ...) comes from a stream-ordered memory pool that the
 * library owns, one per device, and goes back to it in stream order when the
 * call's work is done.  The pool keeps up to keep_bytes of that memory
 * mapped between calls (default 32 GiB), so that the next build does not map
 * it again; the rest is returned to the device at the next synchronisation.
 * Operators, ELL arrays and stepping workspaces are ordinary allocations
 * owned by the operator, not pool memory.
 *
 * rbffd_memory_pool_config: sets keep_bytes for the current device's pool
 *   (>= 0; 0 returns everything at each synchronisation).
 * rbffd_release_memory: returns all pool memory that no call is using to
 *   the device now (after the calls' streams have been synchronised).
 * rbffd_memory_stats: bytes the current device's pool holds mapped and
 *   bytes in use by calls in flight (either pointer may be NULL).
 * Errors: RBFFD_EINVAL for keep_bytes < 0, RBFFD_ECUDA when the pool cannot
 * be created or queried.
 */
rbffd_status rbffd_memory_pool_config(int64_t keep_bytes);
rbffd_status rbffd_release_memory(void);
rbffd_status rbffd_memory_stats(int64_t* reserved, int64_t* used);

/* ------------------------------------------------------------------------ */
const char* rbffd_status_str(rbffd_status s);
const char* rbffd_last_error(void);
/* Device FP64 FMA throughput microbenchmark (GFLOP/s, 2 flops per FMA),
 * used to report the build's roofline.  Synchronises the stream. */
rbffd_status rbffd_fp64_peak(void* stream, double* gflops);
/* Device FP64 tensor-path throughput microbenchmark (warp-level
 * mma.sync m16n8k16 f64; GFLOP/s, 2 flops per multiply-add).  Synchronises
 * the stream. */
rbffd_status rbffd_fp64_mma_peak(void* stream, double* gflops);

#ifdef __cplusplus
}
#endif
#endif /* RBFFD_H */
