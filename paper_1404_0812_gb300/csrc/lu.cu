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
// 256-thread block per species keeps the active window of the solution in
// a shared-memory ring and streams each factor column (with its multiplier,
// diagonal and pivot) into a ring of D shared-memory slots by bulk copies
// (cp.async.bulk, completing on one mbarrier per slot, every wait bounded),
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
    cudaFree(lu->work);
    cudaFree(lu->err);
    delete lu;
}

namespace {

constexpr int FACTOR_THREADS = 1024;
constexpr int SOLVE_THREADS = 256;

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
        // interchange + rank-1 update, rows c + 1 .. c + rows - 1: consecutive
        // threads on consecutive rows of a column, four rows per thread
        // loaded before any is stored (the window lives in L2: four loads
        // in flight per thread hide its latency)
        const int nb = (int)(rows - 1);
        const int pr = (int)(p - c);              // row p as an offset t (0: no interchange)
        for (int64_t k = 0; k < nown; ++k) {
            const int64_t j = c + 1 + q0 + k * G;
            T* __restrict__ cj = a.ab + j * ldab + kl + ku + c - j;   // cj[t] = A(c + t, j)
            const T u = rc[k], oldc = rp[k];
            for (int t0 = 1 + tid; t0 <= nb; t0 += 4 * FACTOR_THREADS) {
                T v[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int t = t0 + q * FACTOR_THREADS;
                    v[q] = t <= nb ? (t == pr ? oldc : cj[t]) : T(0);
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int t = t0 + q * FACTOR_THREADS;
                    if (t <= nb) cj[t] = v[q] - l[t - 1] * u;
                }
            }
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
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}\n" ::"r"(
                     smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
// one bulk copy global -> shared completing on bar (both ends 16-byte aligned,
// bytes a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
// bounded wait (about a second at most) for the given phase parity of bar:
// non-blocking tests with a short sleep between them; false when it gave up
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    for (long long it = 0; it < GRID_SYNC_MAX_POLLS; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(smem_addr(bar)), "r"(parity)
            : "memory");
        if (done) return true;
        if (it > 64) __nanosleep(32);
    }
    return false;
}

// the 16-byte-aligned span covering [p, p + bytes): its start and length
struct Span {
    const char* src;
    uint32_t bytes, off;   // off: bytes from the span's start to p
};
__device__ __forceinline__ Span span_of(const void* p, size_t bytes) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    const uintptr_t a0 = a & ~(uintptr_t)15, a1 = (a + bytes + 15) & ~(uintptr_t)15;
    return Span{reinterpret_cast<const char*>(a0), (uint32_t)(a1 - a0), (uint32_t)(a - a0)};
}

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
    T* work;                     // per species 2 N + 16 values of T: b, then the forward results y
    int* err;                    // set when a bounded wait gave up
};

constexpr int SLOT_PAD = 32;     // bytes of alignment slack in a staged column

// bytes of one staging slot: a column of up to KU values plus slack, and two
// 16-byte scalar spans (pivot or U diagonal; the row entering the window)
template <typename T>
__host__ __device__ inline size_t slot_bytes(int64_t KU) {
    return (((size_t)KU * sizeof(T) + SLOT_PAD + 15) & ~(size_t)15) + 32;
}

// x = M^{-1} b for species blockIdx.x: forward substitution with the row
// interchanges and L (column by column), then back substitution with U, in
// the factor's arithmetic T (b and x of type TV).  Each step's factor
// column and scalars arrive by bulk copies (TMA) D - 1 steps ahead into D
// shared-memory slots, each completing on its own mbarrier; the solution's
// active rows live in a shared-memory ring (slot of row i: i mod (kl + 2)
// forward, i mod (kl + ku + 2) back), one __syncthreads per step.
template <typename T, typename TV, int D>
__global__ void __launch_bounds__(SOLVE_THREADS) solve_kernel(SolveArgs<T, TV> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t N = a.N, kl = a.kl, ku = a.ku, ldab = a.ldab, KU = kl + ku;
    const int W = (int)KU + 2;
    T* win = reinterpret_cast<T*>(smem_raw);
    unsigned char* slots = smem_raw + (((size_t)W * sizeof(T) + 15) & ~(size_t)15);
    const size_t SB = slot_bytes<T>(KU);
    uint64_t* bar = reinterpret_cast<uint64_t*>(slots + D * SB);
    const int tid = threadIdx.x, sp = blockIdx.x;
    const int ord = a.ord_flag ? *((volatile const int*)a.ord_flag) : 1;
    const SolveSys<T> f = a.sys[min(max(ord, 1), 4) - 1][sp];
    const TV* bvec = a.b[sp];
    TV* xo = a.x[sp];
    T* wb = a.work + sp * (2 * N + 16);   // b in T
    T* wy = wb + N;                       // forward results
    // where a slot's data lands (offsets into the slot set by the producer)
    __shared__ uint32_t s_off[D][3];
    __shared__ int s_err;   // a bounded wait gave up (read after the step's barrier)
    if (tid == 0) s_err = 0;

    for (int64_t i = tid; i < N; i += SOLVE_THREADS) wb[i] = (T)bvec[i];
    // every writer orders its generic-proxy writes of wb before the bulk
    // copies (async proxy) that read them after the barrier
    asm volatile("fence.proxy.async.global;\n" ::: "memory");
    if (tid == 0) {
        for (int k = 0; k < D; ++k) mbar_init(bar + k);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    bool ok = true;

    // ---- forward: for c = 0 .. N-1: swap rows c and piv[c], then rows
    // c+1 .. c+kl -= L(., c) y_c
    {
        const int W1 = (int)kl + 2, KL = (int)kl;
        for (int64_t i = tid; i <= min(kl, N - 1); i += SOLVE_THREADS) win[i] = wb[i];
        auto issue = [&](int64_t c) {   // thread 0: stage column c
            if (c >= N) return;
            const int s = (int)(c & (D - 1));
            unsigned char* slot = slots + s * SB;
            const int lim = (int)min(kl, N - 1 - c);
            const Span col = span_of(f.lmul + c * kl, (size_t)max(lim, 1) * sizeof(T));
            const Span pv = span_of(f.piv + c, sizeof(int32_t));
            const bool enter = c + 1 + kl < N;
            const Span be = span_of(wb + (enter ? c + 1 + kl : c), sizeof(T));
            s_off[s][0] = col.off;
            s_off[s][1] = pv.off;
            s_off[s][2] = be.off;
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            mbar_expect_tx(bar + s, col.bytes + pv.bytes + be.bytes);
            bulk_g2s(slot, col.src, col.bytes, bar + s);
            bulk_g2s(slot + SB - 32, pv.src, pv.bytes, bar + s);
            bulk_g2s(slot + SB - 16, be.src, be.bytes, bar + s);
        };
        if (tid == 0)
            for (int64_t c = 0; c < D - 1; ++c) issue(c);
        __syncthreads();
        int cs = 0;   // ring slot of row c
        for (int64_t c = 0; c < N; ++c) {
            const int s = (int)(c & (D - 1));
            if (!mbar_wait(bar + s, (uint32_t)((c / D) & 1))) {
                s_err = 1;
                atomicExch(a.err, 1);
            }
            __syncthreads();
            if (s_err) {
                // leave only after the copies already issued have landed (bounded)
                if (tid == 0)
                    for (int64_t c2 = c + 1; c2 < min(c + D - 1, N); ++c2)
                        mbar_wait(bar + (c2 & (D - 1)), (uint32_t)((c2 / D) & 1));
                ok = false;
                break;
            }
            const unsigned char* slot = slots + s * SB;
            const T* col = reinterpret_cast<const T*>(slot + s_off[s][0]);
            const int dp = (int)(*reinterpret_cast<const int32_t*>(slot + SB - 32 + s_off[s][1]) - c);
            const T bent = *reinterpret_cast<const T*>(slot + SB - 16 + s_off[s][2]);
            const int ps_ = cs + dp < W1 ? cs + dp : cs + dp - W1;
            const T wc = win[cs];
            const T yc = dp == 0 ? wc : win[ps_];
            const int lim = (int)min(kl, N - 1 - c);
            for (int t = tid; t <= KL; t += SOLVE_THREADS) {
                int sl = cs + 1 + t;
                if (sl >= W1) sl -= W1;
                if (t < lim) {
                    const T v = t + 1 == dp ? wc : win[sl];
                    win[sl] = v - col[t] * yc;
                } else if (t == KL && c + 1 + kl < N) {
                    win[sl] = bent;   // the row entering the window
                }
            }
            if (tid == 0) {
                wy[c] = yc;
                issue(c + D - 1);
            }
            cs = cs + 1 == W1 ? 0 : cs + 1;
        }
    }
    // all staged copies of the forward phase have landed or were never
    // issued (columns >= N); its results y, written by thread 0, go to the
    // bulk copies of the back phase
    __syncthreads();
    if (!ok) return;
    if (tid == 0) asm volatile("fence.proxy.async.global;\n" ::: "memory");
    // ---- back: for j = N-1 .. 0: x_j = y_j / U_jj, rows j-1 .. j-KU -= U(., j) x_j
    {
        const int KUi = (int)KU;
        for (int64_t i = (N - 1 - KU > 0 ? N - 1 - KU : 0) + tid; i < N; i += SOLVE_THREADS) win[i % W] = wy[i];
        // the back phase continues the slots' phases: the forward phase used
        // slot k for columns c = k, k + D, ... < N
        auto uses = [&](int k) { return (N - 1 - k) >= 0 ? (N - 1 - k) / D + 1 : 0; };
        auto issue = [&](int64_t j, int64_t step) {   // thread 0: stage column j (the step-th of this phase)
            if (j < 0) return;
            const int s = (int)(step & (D - 1));
            unsigned char* slot = slots + s * SB;
            const int lim = (int)min(KU, j);
            const Span col = span_of(f.ab + j * ldab, (size_t)max(KUi, 1) * sizeof(T));
            const Span ud = span_of(f.udiag + j, sizeof(T));
            const bool enter = j - 1 - KU >= 0;
            const Span ye = span_of(wy + (enter ? j - 1 - KU : j), sizeof(T));
            (void)lim;
            s_off[s][0] = col.off;
            s_off[s][1] = ud.off;
            s_off[s][2] = ye.off;
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            mbar_expect_tx(bar + s, col.bytes + ud.bytes + ye.bytes);
            bulk_g2s(slot, col.src, col.bytes, bar + s);
            bulk_g2s(slot + SB - 32, ud.src, ud.bytes, bar + s);
            bulk_g2s(slot + SB - 16, ye.src, ye.bytes, bar + s);
        };
        __syncthreads();
        if (tid == 0)
            for (int64_t q = 0; q < D - 1; ++q) issue(N - 1 - q, q);
        __syncthreads();
        int js = (int)((N - 1) % W);   // ring slot of row j
        for (int64_t q = 0; q < N; ++q) {
            const int64_t j = N - 1 - q;
            const int s = (int)(q & (D - 1));
            if (!mbar_wait(bar + s, (uint32_t)((uses(s) + q / D) & 1))) {
                s_err = 1;
                atomicExch(a.err, 1);
            }
            __syncthreads();
            if (s_err) {
                if (tid == 0)
                    for (int64_t q2 = q + 1; q2 < min(q + D - 1, N); ++q2)
                        mbar_wait(bar + (q2 & (D - 1)), (uint32_t)((uses((int)(q2 & (D - 1))) + q2 / D) & 1));
                break;
            }
            const unsigned char* slot = slots + s * SB;
            // U(j - KU .. j - 1, j) staged in increasing row order: row j - 1 - t at KU - 1 - t
            const T* col = reinterpret_cast<const T*>(slot + s_off[s][0]);
            const T ujj = *reinterpret_cast<const T*>(slot + SB - 32 + s_off[s][1]);
            const T yent = *reinterpret_cast<const T*>(slot + SB - 16 + s_off[s][2]);
            const T xj = win[js] / ujj;
            const int lim = (int)min(KU, j);
            for (int t = tid; t <= KUi; t += SOLVE_THREADS) {
                int sl = js - 1 - t;
                if (sl < 0) sl += W;
                if (t < lim) {
                    win[sl] -= col[KUi - 1 - t] * xj;
                } else if (t == KUi && j - 1 - KU >= 0) {
                    win[sl] = yent;
                }
            }
            if (tid == 0) {
                xo[j] = (TV)xj;
                issue(j - (D - 1), q + D - 1);
            }
            js = js == 0 ? W - 1 : js - 1;
        }
    }
    __syncthreads();
}

template <typename T>
size_t solve_smem(int64_t kl, int64_t ku, int D) {
    const int64_t KU = kl + ku;
    return (((size_t)(KU + 2) * sizeof(T) + 15) & ~(size_t)15) + (size_t)D * slot_bytes<T>(KU) +
           (size_t)D * sizeof(uint64_t);
}

// the deepest staging ring (8 or 4 slots) whose shared memory fits; 0 when
// none does
template <typename T>
int solve_depth(int64_t kl, int64_t ku) {
    if (solve_smem<T>(kl, ku, 8) <= 220 * 1024) return 8;
    if (solve_smem<T>(kl, ku, 4) <= 220 * 1024) return 4;
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
    // every array the substitutions read by bulk copies is padded by 64
    // bytes: a copy's 16-byte-aligned span may reach past the last element
    const size_t pad = 64;
    cudaError_t e = cudaMalloc(&lu->ab, (size_t)lu->ldab * lu->N * elem + pad);
    if (e == cudaSuccess) e = cudaMalloc(&lu->lmul, (size_t)std::max<int64_t>(kl, 1) * lu->N * elem + pad);
    if (e == cudaSuccess) e = cudaMalloc(&lu->udiag, (size_t)lu->N * elem + pad);
    if (e == cudaSuccess) e = cudaMalloc(&lu->piv, (size_t)lu->N * sizeof(int32_t) + pad);
    if (e == cudaSuccess) e = cudaMalloc(&lu->work, (size_t)(2 * lu->N + 16) * elem + pad);
    if (e == cudaSuccess) e = cudaMalloc(&lu->err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(lu->err, 0, sizeof(int));
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
                          void* const x[2], const int* ord_flag, void* work, int* err, cudaStream_t st) {
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
    a.work = (T*)work;
    a.err = err;
    return launch_solve(a, nspecies, st);
}
}  // namespace

rbffd_status lu_solve_step(rbffd_lu* const (&fac)[4][2], int nspecies, const void* const b[2], void* const x[2],
                           int vec_dtype, const int* ord_flag, void* work, int* err, cudaStream_t st) {
    const rbffd_lu* any = nullptr;
    for (int k = 0; k < 4 && !any; ++k) any = fac[k][0];
    RBFFD_CHECK_ARG(any && work && err, "no LU factor / work vector / error flag");
    const bool f32 = any->dtype == RBFFD_F32, v32 = vec_dtype == RBFFD_F32;
    if (f32 && v32) return solve_step_t<float, float>(fac, any, nspecies, b, x, ord_flag, work, err, st);
    if (!f32 && !v32) return solve_step_t<double, double>(fac, any, nspecies, b, x, ord_flag, work, err, st);
    if (!f32 && v32) return solve_step_t<double, float>(fac, any, nspecies, b, x, ord_flag, work, err, st);
    return solve_step_t<float, double>(fac, any, nspecies, b, x, ord_flag, work, err, st);
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
    cudaStream_t st = as_stream(stream);
    rbffd_status s = lu_solve_step(fac, 1, bb, xx, lu->dtype, nullptr, lu->work, lu->err, st);
    if (s != RBFFD_OK) return s;
    int h = 0;
    RBFFD_CUDA_TRY(cudaMemcpyAsync(&h, lu->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    RBFFD_CUDA_TRY(cudaStreamSynchronize(st));
    if (h) {
        set_error("banded LU solve: a bounded wait for staged factor columns gave up");
        return RBFFD_TIMEOUT;
    }
    return RBFFD_OK;
}

int64_t rbffd_lu_bytes(const rbffd_lu* lu) {
    if (!lu) return 0;
    const int64_t e = lu->dtype == RBFFD_F32 ? 4 : 8;
    return (lu->ldab + std::max<int64_t>(lu->kl, 1) + 1) * lu->N * e + lu->N * 4;
}

void rbffd_lu_destroy(rbffd_lu* lu) { lu_free(lu); }

}  // extern "C"
