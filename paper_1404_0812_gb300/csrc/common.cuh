// Internal declarations shared by the library's translation units.
// (Product code only; the CPU oracle never includes this.)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string>

#include "rbffd.h"

namespace rbffd {

// ---------------------------------------------------------------------------
// error reporting
// ---------------------------------------------------------------------------
void set_error(const char* fmt, ...);

#define RBFFD_CUDA_TRY(expr)                                                      \
    do {                                                                          \
        cudaError_t _e = (expr);                                                  \
        if (_e != cudaSuccess) {                                                  \
            (void)cudaGetLastError(); /* do not leave it for the next call */    \
            ::rbffd::set_error("%s:%d %s: %s", __FILE__, __LINE__, #expr,         \
                               cudaGetErrorString(_e));                           \
            return _e == cudaErrorMemoryAllocation ? RBFFD_ENOMEM : RBFFD_ECUDA;  \
        }                                                                         \
    } while (0)

#define RBFFD_CHECK_ARG(cond, msg)                                                \
    do {                                                                          \
        if (!(cond)) {                                                            \
            ::rbffd::set_error("invalid argument: %s", msg);                     \
            return RBFFD_EINVAL;                                                  \
        }                                                                         \
    } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// count of kernel launches issued by the library (reported to callers)
void note_launch(int k = 1);

// transient device memory from the library's per-device stream-ordered pool
// (kept mapped between calls up to a threshold); free with cudaFreeAsync
cudaError_t pool_alloc_bytes(void** p, size_t bytes, cudaStream_t st);
template <typename T>
inline cudaError_t pool_alloc(T** p, size_t bytes, cudaStream_t st) {
    return pool_alloc_bytes(reinterpret_cast<void**>(p), bytes, st);
}

// ---------------------------------------------------------------------------
// sliced ELL layout.  Rows are grouped by stencil size; within a group rows
// are cut into slices of 32 consecutive rows, and each row's entries are
// stored four at a time so that lane r of a warp reads its 4 consecutive
// entries with one 16-byte (int32 / float32) or two 16-byte (float64) loads
// and the warp's 32 lanes cover one contiguous span.
//   element(g, local row r, entry j) =
//     ell_off[g] + (r / 32) * 32 * npad[g] + (j / 4) * 128 + (r % 32) * 4 + j % 4
// npad[g] = n[g] rounded up to a multiple of 4.  Padding entries hold the
// row's own node (a valid index) and weight 0; padding rows of the last
// slice hold index 0 and weight 0.
// ---------------------------------------------------------------------------
constexpr int ELL_SLICE = 32;

__host__ __device__ inline int64_t ell_elem(int64_t off, int npad, int64_t r, int j) {
    return off + (r >> 5) * (int64_t)(ELL_SLICE * npad) + (int64_t)(j >> 2) * 128 +
           (r & 31) * 4 + (j & 3);
}

struct GroupInfo {
    int ngroups;
    int n[RBFFD_MAX_GROUPS];
    int npad[RBFFD_MAX_GROUPS];
    int64_t row_begin[RBFFD_MAX_GROUPS + 1];   // internal row ranges
    int64_t ell_off[RBFFD_MAX_GROUPS + 1];     // element offsets
};

// Bounded grid barrier of a cooperative launch (all blocks co-resident):
// every block adds 1 to *bar and waits until it reaches target (which grows
// by gridDim.x per barrier).  A block that has polled for about a second, or
// that sees *err set, gives up, sets *err and returns false, so that no wait
// can hang; the caller then leaves the kernel.
constexpr long long GRID_SYNC_MAX_POLLS = 20000000;   // ~1-2 s with 32 ns sleeps
__device__ __forceinline__ bool grid_sync(unsigned long long* bar, unsigned long long target, int* err) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        __threadfence();
        atomicAdd(bar, 1ull);
        long long polls = 0;
        while (*((volatile unsigned long long*)bar) < target) {
            if (++polls > GRID_SYNC_MAX_POLLS || *((volatile int*)err)) {
                ok = 0;
                atomicExch(err, 1);
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// exclusive prefix sum of n int32 values on the device (knn.cu)
rbffd_status exclusive_scan(const int32_t* in, int32_t* out, int64_t n, cudaStream_t st);

__host__ __device__ inline int group_of_row(const GroupInfo& gi, int64_t r) {
    int g = 0;
    while (g + 1 < gi.ngroups && r >= gi.row_begin[g + 1]) ++g;
    return g;
}

}  // namespace rbffd

struct rbffd_step_ws;   // stepping workspace (step.cu)

struct rbffd_op {
    int64_t N;
    int64_t nnz;
    int kernel;
    double kappa_target;
    rbffd::GroupInfo gi;        // groups sorted by descending n
    int n_max;
    int32_t* row_node;          // N: node of each internal row
    int32_t* idx;               // ELL indices
    double* w64;                // ELL weights (float64)
    float* w32;                 // ELL weights (float32 copy)
    int64_t ell_elems;
    double* eps;                // N node order
    double* kappa;              // N
    int32_t* evals;             // N
    int32_t* status;            // N
    rbffd_step_ws* step;        // lazily created stepping workspace
    double phase_ms[4];         // device time of build phases (events)
};

// banded LU of alpha I - beta L_X (lu.cu)
struct rbffd_lu {
    int64_t N, kl, ku, ldab;
    int dtype;                  // RBFFD_F32 / RBFFD_F64
    double alpha, beta;
    void* ab;                   // ldab x N band: factor rows above the diagonal
    void* lmul;                 // kl x N multipliers
    void* udiag;                // N
    int32_t* piv;               // N
    void* work;                 // 2 N + 16 values: b and y of rbffd_lu_solve
    int* err;                   // device flag: a bounded wait of the solve gave up
};

struct rbffd_mlp {
    int n;
    int D;                      // 3n
    int64_t P;                  // parameter count
    float* params;              // device, P floats
    // Adam state + scratch (allocated on first training call)
    float* adam_m;
    float* adam_v;
    int adam_t;                 // Adam steps taken
    float* partial;             // per-CTA gradient partials
    int64_t partial_rows;
    float* grad;                // P floats
    float* loss;                // device scalars
};

namespace rbffd {
// knn.cu: writes stencils (centre first, then n-1 nearest by (d^2, index))
// into op->idx in ELL layout.
rbffd_status knn_stencils(rbffd_op* op, const double* nodes, const double* normals,
                          cudaStream_t st);
// build.cu
rbffd_status build_search(rbffd_op* op, const double* nodes, const double* normals,
                          const rbffd_build_opts& o, const float* eps_guess_s, cudaStream_t st);
rbffd_status build_weights(rbffd_op* op, const double* nodes, const double* normals,
                           const rbffd_build_opts& o, const double* eps_node, cudaStream_t st);
// the same in double-double arithmetic: the search (eps_fixed == NULL) or the
// weights at the given node-order eps; per-stencil statuses as build_search
rbffd_status build_search_dd(rbffd_op* op, const double* nodes, const double* normals,
                             const rbffd_build_opts& o, const float* guess_rows, const double* eps_fixed,
                             cudaStream_t st);
// mlp.cu: predicted ln(eps * r_s) for every internal row of groups with a network
rbffd_status mlp_guess(const rbffd_op* op, const double* nodes, const double* normals,
                       const rbffd_build_opts& o, float* guess_rows, cudaStream_t st);
void step_ws_free(rbffd_step_ws* ws);
// lu.cu: bandwidths of op's matrix in node order; the banded LU of
// alpha I - beta L_X; the substitutions of one step for nspecies systems,
// the factor chosen on the device by the SBDF order in *ord_flag (1..4; NULL
// means order 1, i.e. fac[0]); vectors of vec_dtype, which may differ from
// the factors'; work: per species 2 N + 16 values of the factors' dtype plus
// 64 bytes; *err set when a bounded wait gave up
rbffd_status op_bandwidth(const rbffd_op* op, int64_t* kl, int64_t* ku, cudaStream_t st);
rbffd_status lu_factor(const rbffd_op* op, double alpha, double beta, int dtype, cudaStream_t st, rbffd_lu** out);
rbffd_status lu_solve_step(rbffd_lu* const (&fac)[4][2], int nspecies, const void* const b[2], void* const x[2],
                           int vec_dtype, const int* ord_flag, void* work, int* err, cudaStream_t st);
void lu_free(rbffd_lu* lu);
int sm_count();
}  // namespace rbffd
