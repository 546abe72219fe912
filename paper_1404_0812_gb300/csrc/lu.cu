// Direct solves of the implicit SBDF systems (Section 7 factors the SBDF2
// matrix once by a sparse LU and does a forward and a back substitution per
// step): banded LU with partial pivoting of M = alpha I - beta L_X in node
// order.  After a bandwidth-reducing renumbering (Section 4.1's reverse
// Cuthill-McKee, rbffd_rcm_order) L_X is banded with lower / upper
// bandwidths kl / ku; with row interchanges U has upper bandwidth kl + ku.
//
// Storage (column-major band, LAPACK's layout for a pivoted band LU):
// element (i, j) of the matrix being factorised at ab[j ldab + kl + ku + i - j]
// for j - kl - ku <= i <= j + kl, ldab = 2 kl + ku + 1 (the top kl rows hold
// U's fill-in).  The multipliers of column c go to lmul[c kl + i - c - 1]
// (rows c + 1 .. c + kl after the interchange of step c), U's diagonal to
// udiag[c] and the interchanged row to piv[c]; rows above the diagonal of
// column j of ab hold U(j - kl - ku .. j - 1, j).
//
// GPU design.  The factorisation is N dependent column steps; one
// cooperative launch runs them all, one bounded grid barrier per step.
// Every block finds the pivot of column c itself (the same deterministic
// argmax in every block), forms the multipliers in shared memory, and
// applies the interchange and the rank-1 update to the window columns
// c + 1 .. c + kl + ku that it owns (j mod blocks); the window (~kl (kl + ku)
// elements) stays in L2.  The substitutions are sequential in the rows; one
// 1024-thread block per species keeps the active window of the solution in
// a shared-memory ring and streams the factor's columns in with cp.async,
// D columns ahead, so each step costs one __syncthreads and a shared-memory
// update of kl (forward) or kl + ku (back) entries.
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <type_traits>

namespace rbffd {

void lu_free(rbffd_lu* lu) {
    if (!lu) return;
    cudaFree(lu->ab);
    cudaFree(lu->lmul);
    cudaFree(lu->udiag);
    cudaFree(lu->piv);
    delete lu;
}

namespace {

constexpr int FACTOR_THREADS = 256;
constexpr int SOLVE_THREADS = 1024;

__global__ void bandwidth_kernel(const int32_t* __restrict__ idx, const int32_t* __restrict__ row_node, GroupInfo gi,
                                 int* __restrict__ out) {
    const int64_t R = gi.row_begin[gi.ngroups];
    int lo = 0, up = 0;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < R; r += (int64_t)gridDim.x * blockDim.x) {
        const int g = group_of_row(gi, r);
        const int npad = gi.npad[g];
        const int64_t lr = r - gi.row_begin[g];
        const int i = row_node[r];
        for (int j = 0; j < npad; ++j) {
            const int c = idx[ell_elem(gi.ell_off[g], npad, lr, j)];
            lo = max(lo, i - c);
            up = max(up, c - i);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = max(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        up = max(up, __shfl_xor_sync(0xffffffffu, up, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(out, lo);
        atomicMax(out + 1, up);
    }
}

// ab (zeroed) <- alpha I - beta L_X, one thread per operator row
template <typename T>
__global__ void fill_kernel(const int32_t* __restrict__ idx, const T* __restrict__ w,
                            const int32_t* __restrict__ row_node, GroupInfo gi, int64_t kl, int64_t ku,
                            int64_t ldab, double alpha, double beta, T* __restrict__ ab) {
    const int64_t R = gi.row_begin[gi.ngroups];
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < R; r += (int64_t)gridDim.x * blockDim.x) {
        const int g = group_of_row(gi, r);
        const int npad = gi.npad[g];
        const int64_t lr = r - gi.row_begin[g];
        const int64_t i = row_node[r];
        for (int j = 0; j < npad; ++j) {
            const int64_t e = ell_elem(gi.ell_off[g], npad, lr, j);
            const int64_t c = idx[e];
            // padding entries are (i, i) with weight 0
            T* a = ab + c * ldab + kl + ku + i - c;
            *a = (T)((double)*a - beta * (double)w[e]);
        }
        T* d = ab + i * ldab + kl + ku;
        *d = (T)((double)*d + alpha);
    }
}

template <typename T>
struct FactorArgs {
    T* ab;
    T* lmul;
    T* udiag;
    int32_t* piv;
    int64_t N, kl, ku, ldab;
    int max_own;                 // owned window columns per block, at most
    unsigned long long* bar;
    int* flags;                  // [0] barrier gave up, [1] singular: 1 + first zero-pivot column
};

template <typename T>
__global__ void __launch_bounds__(FACTOR_THREADS) factor_kernel(FactorArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* l = reinterpret_cast<T*>(smem_raw);      // kl multipliers of the current column
    T* rc = l + a.kl;                           // per owned column: new row c (= old row p)
    T* rp = rc + a.max_own;                     //                   new row p (= old row c)
    __shared__ double red_v[FACTOR_THREADS / 32];
    __shared__ int64_t red_i[FACTOR_THREADS / 32];
    __shared__ int64_t s_pt;
    const int tid = threadIdx.x, G = gridDim.x, b = blockIdx.x;
    const int64_t N = a.N, kl = a.kl, ku = a.ku, ldab = a.ldab, W = kl + ku;
    unsigned long long target = 0;
    for (int64_t c = 0; c < N; ++c) {
        const int64_t rows = min(kl, N - 1 - c) + 1;   // rows c .. c + rows - 1 of column c
        const T* col = a.ab + c * ldab + kl + ku;        // col[t] = A(c + t, c)
        // pivot: largest |A(c + t, c)|, the smallest t among equals (the
        // same in every block)
        double bv = -1.0;
        int64_t bi = 0;
        // column c was last written by its owner block: read it through L2
        // (another SM's L1 may hold stale lines of it)
        for (int64_t t = tid; t < rows; t += FACTOR_THREADS) {
            const double v = fabs((double)__ldcg(col + t));
            if (v > bv) {
                bv = v;
                bi = t;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_down_sync(0xffffffffu, bv, o);
            const int64_t oi = __shfl_down_sync(0xffffffffu, bi, o);
            if (ov > bv || (ov == bv && oi < bi)) {
                bv = ov;
                bi = oi;
            }
        }
        if ((tid & 31) == 0) {
            red_v[tid >> 5] = bv;
            red_i[tid >> 5] = bi;
        }
        __syncthreads();
        if (tid == 0) {
            double v = red_v[0];
            int64_t i = red_i[0];
            for (int w = 1; w < FACTOR_THREADS / 32; ++w)
                if (red_v[w] > v || (red_v[w] == v && red_i[w] < i)) {
                    v = red_v[w];
                    i = red_i[w];
                }
            s_pt = i;
        }
        __syncthreads();
        const int64_t pt = s_pt, p = c + pt;
        const T pv = __ldcg(col + pt);
        if (!(pv != T(0)) || !isfinite((double)pv)) {   // every block sees the same pivot
            if (b == 0 && tid == 0) atomicCAS(a.flags + 1, 0, (int)(c + 1 < 0x7fffffff ? c + 1 : 0x7fffffff));
            return;
        }
        // multipliers of rows c + 1 .. c + rows - 1 after the interchange
        for (int64_t t = 1 + tid; t < rows; t += FACTOR_THREADS) {
            const T v = __ldcg(col + (t == pt ? 0 : t)) / pv;
            l[t - 1] = v;
            if (b == 0) a.lmul[c * kl + t - 1] = v;
        }
        if (b == 0 && tid == 0) {
            a.udiag[c] = pv;
            a.piv[c] = (int32_t)p;
        }
        // window columns j = c + 1 .. c + ncols owned by this block (j mod G == b)
        const int64_t ncols = min(W, N - 1 - c);
        const int64_t q0 = ((int64_t)b - (c + 1) % G + G) % G;
        const int64_t nown = q0 < ncols ? (ncols - 1 - q0) / G + 1 : 0;
        for (int64_t k = tid; k < nown; k += FACTOR_THREADS) {
            const int64_t j = c + 1 + q0 + k * G;
            T* cj = a.ab + j * ldab + kl + ku - j;   // cj[i] = A(i, j)
            rc[k] = cj[p];
            rp[k] = cj[c];
        }
        __syncthreads();
        // interchange + rank-1 update, rows c + 1 .. c + rows - 1 (consecutive
        // threads on consecutive rows of a column)
        const int64_t nb = rows - 1;
        for (int64_t e = tid; e < nown * nb; e += FACTOR_THREADS) {
            const int64_t k = e / nb, t = e - k * nb + 1;
            const int64_t j = c + 1 + q0 + k * G, i = c + t;
            T* aij = a.ab + j * ldab + kl + ku + i - j;
            const T v = i == p ? rp[k] : *aij;
            *aij = v - l[t - 1] * rc[k];
        }
        for (int64_t k = tid; k < nown; k += FACTOR_THREADS) {
            const int64_t j = c + 1 + q0 + k * G;
            a.ab[j * ldab + kl + ku + c - j] = rc[k];   // row c of U
        }
        if (!grid_sync(a.bar, target += G, a.flags)) return;
    }
}

// ---------------------------------------------------------------------------
// substitutions
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async_elem(float* s, const float* g) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((unsigned)__cvta_generic_to_shared(s)), "l"(g));
}
__device__ __forceinline__ void cp_async_elem(double* s, const double* g) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(s)), "l"(g));
}
__device__ __forceinline__ void cp_async_elem(int32_t* s, const int32_t* g) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((unsigned)__cvta_generic_to_shared(s)), "l"(g));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int K>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(K)); }

template <typename T>
struct SolveSys {
    const T* ab;
    const T* lmul;
    const T* udiag;
    const int32_t* piv;
};

template <typename T, typename TV>
struct SolveArgs {
    SolveSys<T> sys[4][2];       // factors by SBDF order (1..4) and species
    const TV* b[2];              // vectors of the caller's dtype (the
    TV* x[2];                    //   substitutions run in the factor's)
    int64_t N, kl, ku, ldab;
    const int* ord_flag;         // device: the SBDF order of the current step, or NULL (order 1)
    T* ywork;                    // 2 N values of T: forward results when TV != T
};

// x = M^{-1} b for species blockIdx.x: forward substitution with the row
// interchanges and L (column by column), then back substitution with U, in
// the factor's arithmetic T; b and x are of type TV (float32 vectors of a
// float32 time step are widened on load and rounded on store, and the
// forward result y is kept in x only when TV = T, else in ywork).
template <typename T, typename TV, int D>
__global__ void __launch_bounds__(SOLVE_THREADS) solve_kernel(SolveArgs<T, TV> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t N = a.N, kl = a.kl, ku = a.ku, ldab = a.ldab, KU = kl + ku;
    const int64_t W = KU + 2;                       // ring of the active rows
    T* win = reinterpret_cast<T*>(smem_raw);
    T* pf = win + W;                                // D staged columns of KU entries
    T* ps = pf + D * KU;                            // D staged scalars (U diagonal)
    T* pe = ps + D;                                 // D staged entering rows
    TV* pv = reinterpret_cast<TV*>((reinterpret_cast<uintptr_t>(pe + D) + 7) & ~(uintptr_t)7);   // D entering rows of b
    int32_t* pp = reinterpret_cast<int32_t*>(pv + D);   // D staged pivots
    const int tid = threadIdx.x, sp = blockIdx.x;
    const int ord = a.ord_flag ? *((volatile const int*)a.ord_flag) : 1;
    const SolveSys<T> f = a.sys[min(max(ord, 1), 4) - 1][sp];
    const TV* bvec = a.b[sp];
    TV* xo = a.x[sp];
    T* x = std::is_same<T, TV>::value ? reinterpret_cast<T*>(xo) : a.ywork + sp * N;

    // ---- forward: for c = 0 .. N-1: swap rows c and piv[c], then rows
    // c+1 .. c+kl -= L(., c) y_c.  Ring slot of row i: i mod (kl + 2).
    {
        const int64_t W1 = kl + 2;
        for (int64_t i = tid; i <= min(kl, N - 1); i += SOLVE_THREADS) win[i % W1] = (T)bvec[i];
        auto issue = [&](int64_t c) {
            if (c < N) {
                const int64_t s = c % D;
                const int64_t lim = min(kl, N - 1 - c);
                for (int64_t t = tid; t < lim; t += SOLVE_THREADS) cp_async_elem(pf + s * KU + t, f.lmul + c * kl + t);
                if (tid == 0) {
                    cp_async_elem(pp + s, f.piv + c);
                    if (c + 1 + kl < N) cp_async_elem(pv + s, bvec + c + 1 + kl);
                }
            }
            cp_async_commit();
        };
        for (int64_t c = 0; c < D - 1; ++c) issue(c);
        for (int64_t c = 0; c < N; ++c) {
            cp_async_wait<D - 2>();
            __syncthreads();
            const int64_t s = c % D;
            const int64_t p = pp[s];
            const T wc = win[c % W1];
            const T yc = p == c ? wc : win[p % W1];
            const int64_t lim = min(kl, N - 1 - c);
            for (int64_t t = tid; t <= kl; t += SOLVE_THREADS) {
                if (t < lim) {
                    const int64_t i = c + 1 + t;
                    const T v = i == p ? wc : win[i % W1];
                    win[i % W1] = v - pf[s * KU + t] * yc;
                } else if (t == kl && c + 1 + kl < N) {
                    win[(c + 1 + kl) % W1] = (T)pv[s];   // the row entering the window
                }
            }
            if (tid == 0) x[c] = yc;
            issue(c + D - 1);
        }
        cp_async_wait<0>();
        __syncthreads();
    }
    // ---- back: for j = N-1 .. 0: x_j = y_j / U_jj, rows j-1 .. j-KU -= U(., j) x_j
    {
        for (int64_t i = (N - 1 - KU > 0 ? N - 1 - KU : 0) + tid; i < N; i += SOLVE_THREADS) win[i % W] = x[i];
        auto issue = [&](int64_t j) {
            if (j >= 0) {
                const int64_t s = j % D;
                const int64_t lim = min(KU, j);
                // U(j - 1 - t, j) = ab[j ldab + KU - 1 - t]
                for (int64_t t = tid; t < lim; t += SOLVE_THREADS)
                    cp_async_elem(pf + s * KU + t, f.ab + j * ldab + KU - 1 - t);
                if (tid == 0) {
                    cp_async_elem(ps + s, f.udiag + j);
                    if (j - 1 - KU >= 0) cp_async_elem(pe + s, x + j - 1 - KU);
                }
            }
            cp_async_commit();
        };
        __syncthreads();
        for (int64_t j = N - 1; j > N - 1 - (D - 1); --j) issue(j);
        for (int64_t j = N - 1; j >= 0; --j) {
            cp_async_wait<D - 2>();
            __syncthreads();
            const int64_t s = j % D;
            const T xj = win[j % W] / ps[s];
            const int64_t lim = min(KU, j);
            for (int64_t t = tid; t <= KU; t += SOLVE_THREADS) {
                if (t < lim) {
                    const int64_t i = j - 1 - t;
                    win[i % W] -= pf[s * KU + t] * xj;
                } else if (t == KU && j - 1 - KU >= 0) {
                    win[(j - 1 - KU) % W] = pe[s];
                }
            }
            if (tid == 0) {
                x[j] = xj;
                if (!std::is_same<T, TV>::value) xo[j] = (TV)xj;
            }
            issue(j - (D - 1));
        }
        cp_async_wait<0>();
    }
}

template <typename T>
size_t solve_smem(int64_t kl, int64_t ku, int D) {
    const int64_t KU = kl + ku;
    return (size_t)(KU + 2 + (int64_t)D * KU + 2 * D) * sizeof(T) + (size_t)D * (sizeof(double) + sizeof(int32_t)) + 8;
}

// the deepest prefetch ring (8 or 4 columns) whose shared memory fits; 0
// when none does
template <typename T>
int solve_depth(int64_t kl, int64_t ku) {
    if (solve_smem<T>(kl, ku, 8) <= 227 * 1024) return 8;
    if (solve_smem<T>(kl, ku, 4) <= 227 * 1024) return 4;
    return 0;
}

template <typename T, typename TV, int D>
rbffd_status launch_solve_d(const SolveArgs<T, TV>& a, int nspecies, cudaStream_t st) {
    const size_t smem = solve_smem<T>(a.kl, a.ku, D);
    RBFFD_CUDA_TRY(cudaFuncSetAttribute(solve_kernel<T, TV, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
    solve_kernel<T, TV, D><<<nspecies, SOLVE_THREADS, smem, st>>>(a);
    note_launch();
    RBFFD_CUDA_TRY(cudaGetLastError());
    return RBFFD_OK;
}

template <typename T, typename TV>
rbffd_status launch_solve(const SolveArgs<T, TV>& a, int nspecies, cudaStream_t st) {
    const int D = solve_depth<T>(a.kl, a.ku);
    if (D == 8) return launch_solve_d<T, TV, 8>(a, nspecies, st);
    if (D == 4) return launch_solve_d<T, TV, 4>(a, nspecies, st);
    set_error("banded LU: bandwidth %lld + %lld too large for the substitutions' shared-memory window",
              (long long)a.kl, (long long)a.ku);
    return RBFFD_EINVAL;
}

template <typename T>
void fill_sys(SolveSys<T>& s, const rbffd_lu* lu) {
    s.ab = lu ? (const T*)lu->ab : nullptr;
    s.lmul = lu ? (const T*)lu->lmul : nullptr;
    s.udiag = lu ? (const T*)lu->udiag : nullptr;
    s.piv = lu ? lu->piv : nullptr;
}

template <typename T>
rbffd_status factor_t(const rbffd_op* op, rbffd_lu* lu, cudaStream_t st) {
    const int64_t N = lu->N, kl = lu->kl, ku = lu->ku, ldab = lu->ldab;
    RBFFD_CUDA_TRY(cudaMemsetAsync(lu->ab, 0, (size_t)ldab * N * sizeof(T), st));
    const T* w = std::is_same<T, float>::value ? (const T*)op->w32 : (const T*)op->w64;
    fill_kernel<T><<<(unsigned)std::min<int64_t>((N + 255) / 256, 65535), 256, 0, st>>>(
        op->idx, w, op->row_node, op->gi, kl, ku, ldab, lu->alpha, lu->beta, (T*)lu->ab);
    note_launch();
    RBFFD_CUDA_TRY(cudaGetLastError());
    // one block per SM (co-resident for the cooperative launch)
    const int G = std::max(1, sm_count());
    FactorArgs<T> a;
    a.ab = (T*)lu->ab;
    a.lmul = (T*)lu->lmul;
    a.udiag = (T*)lu->udiag;
    a.piv = lu->piv;
    a.N = N;
    a.kl = kl;
    a.ku = ku;
    a.ldab = ldab;
    a.max_own = (int)((kl + ku + G - 1) / G);
    const size_t smem = (size_t)(kl + 2 * a.max_own) * sizeof(T);
    RBFFD_CHECK_ARG(smem <= 200 * 1024, "banded LU: lower bandwidth too large for the factorisation's shared memory");
    unsigned long long* bar = nullptr;
    int* flags = nullptr;
    RBFFD_CUDA_TRY(pool_alloc(&bar, sizeof(unsigned long long), st));
    RBFFD_CUDA_TRY(pool_alloc(&flags, 2 * sizeof(int), st));
    RBFFD_CUDA_TRY(cudaMemsetAsync(bar, 0, sizeof(unsigned long long), st));
    RBFFD_CUDA_TRY(cudaMemsetAsync(flags, 0, 2 * sizeof(int), st));
    a.bar = bar;
    a.flags = flags;
    RBFFD_CUDA_TRY(cudaFuncSetAttribute(factor_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    RBFFD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, factor_kernel<T>, FACTOR_THREADS, smem));
    RBFFD_CHECK_ARG(per_sm >= 1, "banded LU: the factorisation kernel does not fit on an SM");
    void* args[] = {&a};
    RBFFD_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)factor_kernel<T>, dim3(G), dim3(FACTOR_THREADS), args,
                                               smem, st));
    note_launch();
    int hf[2] = {0, 0};
    RBFFD_CUDA_TRY(cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, st));
    RBFFD_CUDA_TRY(cudaStreamSynchronize(st));
    cudaFreeAsync(bar, st);
    cudaFreeAsync(flags, st);
    if (hf[1]) {
        set_error("banded LU: zero pivot in column %d (the matrix is singular)", hf[1] - 1);
        return RBFFD_ESINGULAR;
    }
    if (hf[0]) {
        set_error("banded LU: a grid barrier of the factorisation timed out");
        return RBFFD_TIMEOUT;
    }
    return RBFFD_OK;
}

}  // namespace

rbffd_status op_bandwidth(const rbffd_op* op, int64_t* kl, int64_t* ku, cudaStream_t st) {
    int* d = nullptr;
    RBFFD_CUDA_TRY(pool_alloc(&d, 2 * sizeof(int), st));
    RBFFD_CUDA_TRY(cudaMemsetAsync(d, 0, 2 * sizeof(int), st));
    const int64_t R = op->N;
    bandwidth_kernel<<<(unsigned)std::min<int64_t>((R + 255) / 256, 4096), 256, 0, st>>>(op->idx, op->row_node,
                                                                                           op->gi, d);
    note_launch();
    RBFFD_CUDA_TRY(cudaGetLastError());
    int h[2] = {0, 0};
    RBFFD_CUDA_TRY(cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, st));
    RBFFD_CUDA_TRY(cudaStreamSynchronize(st));
    cudaFreeAsync(d, st);
    *kl = h[0];
    *ku = h[1];
    return RBFFD_OK;
}

rbffd_status lu_factor(const rbffd_op* op, double alpha, double beta, int dtype, cudaStream_t st, rbffd_lu** out) {
    *out = nullptr;
    int64_t kl = 0, ku = 0;
    rbffd_status s = op_bandwidth(op, &kl, &ku, st);
    if (s != RBFFD_OK) return s;
    const size_t elem = dtype == RBFFD_F32 ? 4 : 8;
    if ((dtype == RBFFD_F32 ? solve_depth<float>(kl, ku) : solve_depth<double>(kl, ku)) == 0) {
        set_error("banded LU: bandwidths %lld / %lld too large for the substitutions (reorder the nodes, "
                  "e.g. by rbffd_rcm_order)", (long long)kl, (long long)ku);
        return RBFFD_EINVAL;
    }
    rbffd_lu* lu = new rbffd_lu();
    memset(lu, 0, sizeof(*lu));
    lu->N = op->N;
    lu->kl = kl;
    lu->ku = ku;
    lu->ldab = 2 * kl + ku + 1;
    lu->dtype = dtype;
    lu->alpha = alpha;
    lu->beta = beta;
    cudaError_t e = cudaMalloc(&lu->ab, (size_t)lu->ldab * lu->N * elem);
    if (e == cudaSuccess) e = cudaMalloc(&lu->lmul, (size_t)std::max<int64_t>(kl, 1) * lu->N * elem);
    if (e == cudaSuccess) e = cudaMalloc(&lu->udiag, (size_t)lu->N * elem);
    if (e == cudaSuccess) e = cudaMalloc(&lu->piv, (size_t)lu->N * sizeof(int32_t));
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        set_error("banded LU: %s (%lld x %lld band)", cudaGetErrorString(e), (long long)lu->ldab, (long long)lu->N);
        lu_free(lu);
        return e == cudaErrorMemoryAllocation ? RBFFD_ENOMEM : RBFFD_ECUDA;
    }
    s = dtype == RBFFD_F32 ? factor_t<float>(op, lu, st) : factor_t<double>(op, lu, st);
    if (s != RBFFD_OK) {
        lu_free(lu);
        return s;
    }
    *out = lu;
    return RBFFD_OK;
}

namespace {
template <typename T, typename TV>
rbffd_status solve_step_t(rbffd_lu* const (&fac)[4][2], const rbffd_lu* any, int nspecies, const void* const b[2],
                          void* const x[2], const int* ord_flag, void* ywork, cudaStream_t st) {
    SolveArgs<T, TV> a;
    memset(&a, 0, sizeof(a));
    for (int k = 0; k < 4; ++k)
        for (int s = 0; s < 2; ++s) fill_sys(a.sys[k][s], fac[k][s]);
    for (int s = 0; s < 2; ++s) {
        a.b[s] = (const TV*)b[s];
        a.x[s] = (TV*)x[s];
    }
    a.N = any->N;
    a.kl = any->kl;
    a.ku = any->ku;
    a.ldab = any->ldab;
    a.ord_flag = ord_flag;
    a.ywork = (T*)ywork;
    return launch_solve(a, nspecies, st);
}
}  // namespace

rbffd_status lu_solve_step(rbffd_lu* const (&fac)[4][2], int nspecies, const void* const b[2], void* const x[2],
                           int vec_dtype, const int* ord_flag, void* ywork, cudaStream_t st) {
    const rbffd_lu* any = nullptr;
    for (int k = 0; k < 4 && !any; ++k) any = fac[k][0];
    RBFFD_CHECK_ARG(any, "no LU factor");
    const bool f32 = any->dtype == RBFFD_F32, v32 = vec_dtype == RBFFD_F32;
    RBFFD_CHECK_ARG(f32 == v32 || ywork, "mixed-precision substitutions need a work vector");
    if (f32 && v32) return solve_step_t<float, float>(fac, any, nspecies, b, x, ord_flag, ywork, st);
    if (!f32 && !v32) return solve_step_t<double, double>(fac, any, nspecies, b, x, ord_flag, ywork, st);
    if (!f32 && v32) return solve_step_t<double, float>(fac, any, nspecies, b, x, ord_flag, ywork, st);
    return solve_step_t<float, double>(fac, any, nspecies, b, x, ord_flag, ywork, st);
}

}  // namespace rbffd

using namespace rbffd;

extern "C" {

rbffd_status rbffd_op_bandwidth(const rbffd_op* op, int64_t* kl, int64_t* ku, void* stream) {
    RBFFD_CHECK_ARG(op && kl && ku, "NULL argument");
    return op_bandwidth(op, kl, ku, as_stream(stream));
}

rbffd_status rbffd_lu_factor(const rbffd_op* op, double alpha, double beta, int dtype, void* stream,
                             rbffd_lu** out) {
    RBFFD_CHECK_ARG(out, "out is NULL");
    *out = nullptr;
    RBFFD_CHECK_ARG(op, "op is NULL");
    RBFFD_CHECK_ARG(dtype == RBFFD_F32 || dtype == RBFFD_F64, "dtype");
    RBFFD_CHECK_ARG(std::isfinite(alpha) && std::isfinite(beta), "alpha and beta must be finite");
    return lu_factor(op, alpha, beta, dtype, as_stream(stream), out);
}

rbffd_status rbffd_lu_solve(const rbffd_lu* lu, const void* b, void* x, void* stream) {
    RBFFD_CHECK_ARG(lu && b && x, "NULL argument");
    rbffd_lu* fac[4][2] = {};
    fac[0][0] = const_cast<rbffd_lu*>(lu);
    const void* bb[2] = {b, nullptr};
    void* xx[2] = {x, nullptr};
    return lu_solve_step(fac, 1, bb, xx, lu->dtype, nullptr, nullptr, as_stream(stream));
}

int64_t rbffd_lu_bytes(const rbffd_lu* lu) {
    if (!lu) return 0;
    const int64_t e = lu->dtype == RBFFD_F32 ? 4 : 8;
    return (lu->ldab + std::max<int64_t>(lu->kl, 1) + 1) * lu->N * e + lu->N * 4;
}

void rbffd_lu_destroy(rbffd_lu* lu) { lu_free(lu); }

}  // extern "C"
