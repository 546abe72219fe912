// IMEX method-of-lines stepping (Section 4.2 method of lines; Section 7
// SBDF2 with the diffusion implicit; BiCGSTAB as Section 4.2 / Section 6 use).
//
//   d/dt u = delta_u L u + f(u, v),  d/dt v = delta_v L v + g(u, v)
//   SBDF2:  (3 I - 2 dt delta L) u^{n+1} = 4 u^n - u^{n-1} + 2 dt (2 f^n - f^{n-1})
//   first step without history: (I - dt delta L) u^1 = u^0 + dt f^0
//
// GPU design: one cooperative persistent launch per time step.  Every
// thread owns a fixed set of operator rows for the whole step; both species
// are solved together so each pass over the ELL matrix (the bytes that
// bound the step) serves two SpMVs.  Phases of BiCGSTAB are separated by a
// grid barrier of our own with a bounded spin (a block that waits longer
// than about a second sets an error flag and leaves, so nothing can hang);
// dot products are reduced per block in float64, written to per-phase
// slots, and every block sums the slots in the same fixed order, so all
// blocks hold bit-identical scalars.  Vectors written inside the launch are
// read with L1-bypassing loads.  The solution is updated in place in u
// (after the right-hand side is formed, u is only read by its own row).
// The launch can be captured once into a CUDA graph and replayed per step.
//
// Large operators take a second path with the same arithmetic per row:
// BiCGSTAB as a sequence of full-occupancy phase kernels under a device-side
// WHILE graph node (the phase-kernel section below says why and how).
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

// Loop state of the phase-kernel BiCGSTAB (device memory).  Each phase
// kernel reads it as its previous kernel left it; only the last block of a
// phase (by ticket) writes it, after every other block of that phase has
// finished reading.
struct PhaseCtl {
    double totR[6];              // phase R: |b|^2, |r0|^2 (u: 0, 1; v: 3, 4)
    double totB[2];              // (r-hat, q)
    double totC[2];              // |s|^2
    double totD[4];              // (t, s), (t, t) per species
    double totE[4];              // (r-hat, r), |r|^2 per species
    double bnorm[2], rho[2], rho_prev[2], alpha[2], omega[2], relres[2];
    int active[2], conv[2], fail[2], iters[2], zero[2];
    // the current iteration's scalars and decisions, each set once by the
    // last block of the phase that makes it (the phase kernels' threads only
    // read them: no per-thread float64 scalar arithmetic)
    double beta[2], alpha_n[2], omega_n[2];
    int actA[2], actB[2], early[2], actE[2];
    int it;                      // iterations done in this step
    int more;                    // the loop continues (host-loop mode reads it)
    unsigned int ticket;
};

struct rbffd_step_ws {
    int dtype;
    int64_t N;
    size_t elem;
    void* vec;                     // 2 species x 7 vectors (b, r, rh, p, q, s, t), each padded to a multiple of 4
    double* partial;               // phases x blocks x 8
    unsigned long long* bar;       // barrier counter
    int* flags;                    // [0] error (timeout), [1] not converged, [2] has_history,
                                   // [3] report slot of the next step, [4] order of the last step
    int* rep;                      // per step: iters_u, iters_v, failed
    double* rep_res;               // per step: relres_u, relres_v
    double* tstart;                // time of u at the start of the call (device copy)
    int64_t rep_cap;
    int blocks, threads;
    cudaGraphExec_t graph;            // captured step (memset + launch)
    cudaStream_t cap;                 // library-owned stream used only for capture
    unsigned char graph_args[1024];   // kernel arguments the graph holds
    size_t graph_args_size;
    int solver;                       // path the graph was captured with (0 cooperative, 1 LU, 2 phases)
    rbffd_lu* lu[4][2];               // banded LU factors by SBDF order and species
    rbffd_lu* graph_lu[4][2];         // the factors the captured graph's solve reads
    double* ywork;                    // the LU substitutions' work: per species 2 N + 16 float64
    PhaseCtl* ctl;                    // phase-kernel path: loop state
    double* pp;                       //   per-block partial sums
    int phased;                       // 1: BiCGSTAB as phase kernels (large operators)
};

namespace rbffd {

void step_ws_free(rbffd_step_ws* ws) {
    if (!ws) return;
    cudaFree(ws->vec);
    cudaFree(ws->partial);
    cudaFree(ws->bar);
    cudaFree(ws->flags);
    cudaFree(ws->rep);
    cudaFree(ws->rep_res);
    cudaFree(ws->tstart);
    if (ws->graph) cudaGraphExecDestroy(ws->graph);
    if (ws->cap) cudaStreamDestroy(ws->cap);
    for (auto& row : ws->lu)
        for (rbffd_lu* f : row) lu_free(f);
    cudaFree(ws->ywork);
    cudaFree(ws->ctl);
    cudaFree(ws->pp);
    delete ws;
}

namespace {

constexpr int NPHASE = 6;
constexpr int NSLOT = 8;

template <typename T>
struct Args {
    const int32_t* idx;
    const T* w;
    const int32_t* row_node;
    GroupInfo gi;
    int64_t N;
    T *u, *v, *up, *vp, *fp, *gp;
    T *up2, *vp2, *fp2, *gp2;   // levels n-2 and n-3 (SBDF3 / SBDF4 only)
    T *up3, *vp3, *fp3, *gp3;
    int order;         // SBDF order 1..4
    const T *su, *sv;  // source profiles h_u, h_v (or NULL): s(t) = exp(rate t) h
    double src_rate;
    const double* tstart;   // time of u when the call began
    T* vec;            // 2 x 7 vectors of ldv elements
    int64_t ldv;       // their stride: N rounded up to a multiple of 4 (16-byte aligned vectors)
    int vec4;          // the state u (and v) 16-byte aligned: the vector phases move 4 elements at a time
    int ns;
    int model;
    T c[8];
    T dt;
    T delta[2];
    double tol;
    int maxit;
    double* partial;
    unsigned long long* bar;
    int* flags;
    int* rep;
    double* rep_res;
    int rhs_only;      // 1: form the right-hand side b only (a direct solve follows)
    PhaseCtl* ctl;                         // phase-kernel path: loop state and totals
    double* pp;                            //   per-block partial sums (blocks x 8)
    cudaGraphConditionalHandle cond;       //   WHILE handle of the step graph (0: host loop)
};

enum { VB = 0, VR = 1, VRH = 2, VP = 3, VQ = 4, VS = 5, VT = 6 };

template <typename T>
__host__ __device__ __forceinline__ T* V(const Args<T>& a, int sp, int k) {
    return a.vec + ((int64_t)sp * 7 + k) * a.ldv;
}

template <typename T>
__device__ __forceinline__ T ldcg(const T* p) { return __ldcg(p); }

// block-reduce K doubles into partial[phase][block][0..K-1]
template <int K>
__device__ void block_partial(double (&v)[K], double* partial, int phase) {
    __shared__ double sh[K][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double x = v[k];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sh[k][wid] = x;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += sh[threadIdx.x][w];
        partial[((int64_t)phase * gridDim.x + blockIdx.x) * NSLOT + threadIdx.x] = s;
    }
}

// every block sums the per-block partials of a phase in block order
template <int K>
__device__ void grid_total(const double* partial, int phase, double (&out)[K]) {
    __shared__ double tot[K];
    if (threadIdx.x < K) {
        double s = 0.0;
        for (int b = 0; b < (int)gridDim.x; ++b)
            s += __ldcg(partial + ((int64_t)phase * gridDim.x + b) * NSLOT + threadIdx.x);
        tot[threadIdx.x] = s;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] = tot[k];
    __syncthreads();
}

template <typename T>
__device__ __forceinline__ void react(const Args<T>& a, T u, T v, T& f, T& g) {
    switch (a.model) {
        case RBFFD_MODEL_LINEAR: f = a.c[0] * u; g = a.c[1] * v; break;
        case RBFFD_MODEL_SCHNAKENBERG: {
            T uuv = u * u * v;
            f = a.c[2] * (a.c[0] - u + uuv);
            g = a.c[2] * (a.c[1] - uuv);
        } break;
        case RBFFD_MODEL_GRAY_SCOTT: {
            T uvv = u * v * v;
            f = -uvv + a.c[0] * (T(1) - u);
            g = uvv - (a.c[0] + a.c[1]) * v;
        } break;
        case RBFFD_MODEL_BARRIO: {   // Eqs. turing1, turing2
            T al = a.c[0], be = a.c[1], ga = a.c[2], t1 = a.c[3], t2 = a.c[4];
            f = al * u * (T(1) - t1 * v * v) + v * (T(1) - t2 * u);
            g = be * v * (T(1) + (al * t1 / be) * u * v) + u * (ga + t2 * v);
        } break;
        default: f = T(0); g = T(0);
    }
}

// (L x0)_row and (L x1)_row in one pass over the row (x read L1-bypassing:
// within one launch L1 is not coherent across SMs); software-pipelined so
// that a chunk's index and weight loads overlap the previous chunk's gathers
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

template <typename T>
__device__ __forceinline__ int4 ld_stream4(const int32_t* p) { return __ldcs(reinterpret_cast<const int4*>(p)); }
__device__ __forceinline__ void load4s(const float* p, float (&w)[4]) {
    float4 v = __ldcs(reinterpret_cast<const float4*>(p));
    w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
}
__device__ __forceinline__ void load4s(const double* p, double (&w)[4]) {
    double2 a = __ldcs(reinterpret_cast<const double2*>(p));
    double2 b = __ldcs(reinterpret_cast<const double2*>(p + 2));
    w[0] = a.x; w[1] = a.y; w[2] = b.x; w[3] = b.y;
}

constexpr int PF_CHUNKS = 6;   // ELL chunks prefetched into L2 ahead of use

// (L x0)_row and (L x1)_row in one pass over the row (x read L1-bypassing:
// within one launch L1 is not coherent across SMs); software-pipelined so
// that a chunk's index and weight loads overlap the previous chunk's
// gathers, with an L2 prefetch PF_CHUNKS chunks ahead that runs on into the
// thread's next row (rnext), and streaming (evict-first) loads of the
// single-use ELL so that the Krylov vectors stay in L2
template <typename T>
__device__ __forceinline__ void row_L2(const Args<T>& a, int64_t r, int64_t rnext, const T* x0, const T* x1,
                                       bool two, T& y0, T& y1) {
    int g = group_of_row(a.gi, r);
    const int npad = a.gi.npad[g], nch = npad >> 2;
    const int64_t base = ell_elem(a.gi.ell_off[g], npad, r - a.gi.row_begin[g], 0);
    int64_t nbase = -1;
    int nnch = 0;
    if (rnext < a.N) {
        const int gn = group_of_row(a.gi, rnext);
        nnch = a.gi.npad[gn] >> 2;
        nbase = ell_elem(a.gi.ell_off[gn], a.gi.npad[gn], rnext - a.gi.row_begin[gn], 0);
    }
    T s0 = T(0), s1 = T(0);
    int4 iv = __ldcs(reinterpret_cast<const int4*>(a.idx + base));
    T wv[4];
    load4s(a.w + base, wv);
    for (int c = 0; c < nch; ++c) {
        // L2 prefetch PF_CHUNKS ahead (into the next row past this one's end)
        {
            const int k = c + PF_CHUNKS;
            int64_t e = -1;
            if (k < nch) e = base + (int64_t)k * 128;
            else if (k - nch < nnch && nbase >= 0) e = nbase + (int64_t)(k - nch) * 128;
            if (e >= 0) {
                prefetch_l2(a.idx + e);
                prefetch_l2(a.w + e);
            }
        }
        // the next chunk's index and weight loads go out before this chunk's gathers
        int4 ivn = iv;
        T wn[4] = {wv[0], wv[1], wv[2], wv[3]};
        if (c + 1 < nch) {
            const int64_t en = base + (int64_t)(c + 1) * 128;
            ivn = __ldcs(reinterpret_cast<const int4*>(a.idx + en));
            load4s(a.w + en, wn);
        }
        const int ii[4] = {iv.x, iv.y, iv.z, iv.w};
        T g0[4], g1[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            g0[q] = ldcg(x0 + ii[q]);
            g1[q] = two ? ldcg(x1 + ii[q]) : T(0);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            s0 = fma(wv[q], g0[q], s0);
            s1 = fma(wv[q], g1[q], s1);
        }
        iv = ivn;
#pragma unroll
        for (int q = 0; q < 4; ++q) wv[q] = wn[q];
    }
    y0 = s0;
    y1 = two ? s1 : T(0);
}

// the SBDF order, report slot and coefficients of the current step (from
// the flags a previous launch left; the same in every block)
template <typename T>
struct StepCoef {
    int nhist, ord, slot;
    T c0, cl, k0, k1, samp;
};

template <typename T>
__device__ __forceinline__ StepCoef<T> step_coef(const Args<T>& a) {
    StepCoef<T> k;
    // past levels available -> the order of this step (SBDF1 .. SBDF4, the
    // first steps of a run without history climb one order per step)
    k.nhist = *((volatile int*)(a.flags + 2));
    k.ord = min(a.order, k.nhist + 1);
    k.slot = *((volatile int*)(a.flags + 3));
    // the SBDFk system scaled to integer coefficients:
    //   c0 u^{n+1} - cl delta L u^{n+1} = sum_j A_j u^{n-j} + cl sum_j B_j f^{n-j}
    // k = 1: c0 1, cl dt;  k = 2: 3, 2 dt;  k = 3: 11, 6 dt;  k = 4: 25, 12 dt
    const int ord = k.ord;
    k.c0 = ord == 1 ? T(1) : ord == 2 ? T(3) : ord == 3 ? T(11) : T(25);
    k.cl = (ord == 1 ? T(1) : ord == 2 ? T(2) : ord == 3 ? T(6) : T(12)) * a.dt;
    k.k0 = k.cl * a.delta[0];
    k.k1 = k.cl * a.delta[1];
    // the source is taken at the new time level t^{n+1} (implicitly)
    k.samp = (a.su || a.sv) ? (T)exp(a.src_rate * (*a.tstart + (double)(k.slot + 1) * (double)a.dt)) : T(0);
    return k;
}

// Dot-product accumulators.  The cooperative kernel sums in float64 (the
// float32 products are exact there).  The phase kernels sum float32 products
// with the compensated dot product Dot2 (Ogita, Rump & Oishi, "Accurate sum
// and dot product", SIAM J. Sci. Comput. 26 (2005), Algorithm 5.3): each
// product a b split exactly into p + e by an FMA (TwoProduct), the running
// sum carried by Knuth's error-free TwoSum, the rounding errors of both
// summed apart and added at the end.  The result is as accurate as the sum
// computed in twice the working precision, with float32 instructions only
// (the float64 pipe of this GPU is a small fraction of the float32 one).
struct Dot2 {
    float hi, lo;
};
__device__ __forceinline__ void acc_zero(Dot2& s) { s.hi = s.lo = 0.f; }
__device__ __forceinline__ void acc_zero(double& s) { s = 0.0; }
__device__ __forceinline__ void acc_add(Dot2& s, float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);                    // a b = p + e exactly
    const float x = __fadd_rn(s.hi, p);
    const float z = __fsub_rn(x, s.hi);
    const float t = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(x, z)), __fsub_rn(p, z));   // s.hi + p = x + t exactly
    s.hi = x;
    s.lo = __fadd_rn(s.lo, __fadd_rn(t, e));
}
__device__ __forceinline__ void acc_add(double& s, float a, float b) { s += (double)a * b; }
__device__ __forceinline__ void acc_add(double& s, double a, double b) { s += a * b; }
__device__ __forceinline__ double acc_value(const Dot2& s) { return (double)s.hi + (double)s.lo; }
__device__ __forceinline__ double acc_value(double s) { return s; }

// the phase kernels' accumulator for state type T
template <typename T>
struct PhaseAcc {
    using type = double;
};
template <>
struct PhaseAcc<float> {
    using type = Dot2;
};

// phase R of one row (node i, with (L u)_i = Lu, (L v)_i = Lv): kinetics,
// right-hand side b of the step's SBDF order, history rotation, r0 = b - A u,
// r-hat = r0, p = q = 0; accumulates |b|^2, |r0|^2 per species into d[0..1],
// d[3..4]
template <typename T, typename A>
__device__ __forceinline__ void rhs_row(const Args<T>& a, const StepCoef<T>& kc, int64_t i, T Lu, T Lv,
                                        A (&d)[6]) {
    const bool two = a.ns == 2;
    const int ord = kc.ord;
    const T c0 = kc.c0, cl = kc.cl, k0 = kc.k0, k1 = kc.k1, samp = kc.samp;
    T* u = a.u;
    T* v = two ? a.v : nullptr;
    T ui = u[i], vi = two ? v[i] : T(0);
    T f, g;
    react(a, ui, vi, f, g);
    T bu, bv = T(0);
    if (ord == 2) {
        bu = T(4) * ui - a.up[i] + T(2) * a.dt * (T(2) * f - a.fp[i]);
        if (two) bv = T(4) * vi - a.vp[i] + T(2) * a.dt * (T(2) * g - a.gp[i]);
    } else if (ord == 1) {
        bu = ui + a.dt * f;
        if (two) bv = vi + a.dt * g;
    } else if (ord == 3) {
        bu = (T(18) * ui - T(9) * a.up[i] + T(2) * a.up2[i]) +
             cl * (T(3) * f - T(3) * a.fp[i] + a.fp2[i]);
        if (two)
            bv = (T(18) * vi - T(9) * a.vp[i] + T(2) * a.vp2[i]) +
                 cl * (T(3) * g - T(3) * a.gp[i] + a.gp2[i]);
    } else {
        bu = (T(48) * ui - T(36) * a.up[i] + T(16) * a.up2[i] - T(3) * a.up3[i]) +
             cl * (T(4) * f - T(6) * a.fp[i] + T(4) * a.fp2[i] - a.fp3[i]);
        if (two)
            bv = (T(48) * vi - T(36) * a.vp[i] + T(16) * a.vp2[i] - T(3) * a.vp3[i]) +
                 cl * (T(4) * g - T(6) * a.gp[i] + T(4) * a.gp2[i] - a.gp3[i]);
    }
    if (a.su) bu += cl * samp * a.su[i];
    if (two && a.sv) bv += cl * samp * a.sv[i];
    // shift the history by one level (only the levels the order keeps)
    if (a.order >= 4) {
        a.up3[i] = a.up2[i];
        a.fp3[i] = a.fp2[i];
    }
    if (a.order >= 3) {
        a.up2[i] = a.up[i];
        a.fp2[i] = a.fp[i];
    }
    a.up[i] = ui;
    a.fp[i] = f;
    T ru = bu - (c0 * ui - k0 * Lu);
    V(a, 0, VB)[i] = bu;
    V(a, 0, VR)[i] = ru;
    V(a, 0, VRH)[i] = ru;
    V(a, 0, VP)[i] = T(0);
    V(a, 0, VQ)[i] = T(0);
    acc_add(d[0], bu, bu);
    acc_add(d[1], ru, ru);
    if (two) {
        if (a.order >= 4) {
            a.vp3[i] = a.vp2[i];
            a.gp3[i] = a.gp2[i];
        }
        if (a.order >= 3) {
            a.vp2[i] = a.vp[i];
            a.gp2[i] = a.gp[i];
        }
        a.vp[i] = vi;
        a.gp[i] = g;
        T rv = bv - (c0 * vi - k1 * Lv);
        V(a, 1, VB)[i] = bv;
        V(a, 1, VR)[i] = rv;
        V(a, 1, VRH)[i] = rv;
        V(a, 1, VP)[i] = T(0);
        V(a, 1, VQ)[i] = T(0);
        acc_add(d[3], bv, bv);
        acc_add(d[4], rv, rv);
    }
}

// NT threads per block: 1024 (one block per SM, <= 64 registers) for large
// operators (there only the LU step's right-hand side runs here), 256 for
// small ones
template <typename T, int NT>
__global__ void __launch_bounds__(NT) step_kernel(Args<T> a) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool two = a.ns == 2;
    const StepCoef<T> kc = step_coef(a);
    const int nhist = kc.nhist, ord = kc.ord, slot = kc.slot;
    const T c0 = kc.c0, k0 = kc.k0, k1 = kc.k1;
    unsigned long long target = 0;
    T* u = a.u;
    T* v = two ? a.v : nullptr;

    // ---- phase R: reaction, right-hand side, r0 = b - A u, history rotation
    {
        double d[6] = {0, 0, 0, 0, 0, 0};   // |b|^2, |r|^2, (rh, r) per species
        for (int64_t r = t0; r < a.N; r += stride) {
            int i = a.row_node[r];
            T Lu, Lv;
            row_L2(a, r, r + stride, u, v, two, Lu, Lv);
            rhs_row(a, kc, i, Lu, Lv, d);
        }
        block_partial<6>(d, a.partial, 0);
    }
    if (!grid_sync(a.bar, target += gridDim.x, a.flags)) return;
    if (a.rhs_only) {
        // the implicit systems are solved by the banded LU launch that
        // follows (every block has read flags[2..3] before the barrier)
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            int* rp = a.rep + (int64_t)slot * 3;
            rp[0] = rp[1] = rp[2] = 0;
            a.rep_res[(int64_t)slot * 2] = 0.0;
            a.rep_res[(int64_t)slot * 2 + 1] = 0.0;
            a.flags[2] = min(nhist + 1, max(a.order - 1, 1));
            a.flags[3] = slot + 1;
            a.flags[4] = ord;
        }
        return;
    }
    double tot[6];
    grid_total<6>(a.partial, 0, tot);

    double bnorm[2] = {sqrt(tot[0]), sqrt(tot[3])};
    double rho[2] = {tot[1], tot[4]};    // (rh, r0) = |r0|^2
    double rho_prev[2] = {1.0, 1.0}, alpha[2] = {1.0, 1.0}, omega[2] = {1.0, 1.0};
    bool active[2], conv[2] = {false, false}, fail[2] = {false, false};
    int iters[2] = {0, 0};
    double relres[2];
    for (int k = 0; k < 2; ++k) {
        bool exists = k == 0 || two;
        relres[k] = bnorm[k] > 0 ? sqrt(rho[k]) / bnorm[k] : 0.0;
        conv[k] = !exists || bnorm[k] == 0.0 || relres[k] <= a.tol;
        active[k] = !conv[k];
    }
    if (bnorm[0] == 0.0)   // b = 0: x = 0
        for (int64_t r = t0; r < a.N; r += stride) u[a.row_node[r]] = T(0);
    if (two && bnorm[1] == 0.0)
        for (int64_t r = t0; r < a.N; r += stride) v[a.row_node[r]] = T(0);

    int it = 0;
    while ((active[0] || active[1]) && it < a.maxit) {
        ++it;
        // ---- A: p = r + beta (p - omega q)
        double beta[2];
        for (int k = 0; k < 2; ++k) {
            beta[k] = (rho[k] / rho_prev[k]) * (alpha[k] / omega[k]);
            if (active[k] && (rho[k] == 0.0 || !isfinite(beta[k]))) {
                fail[k] = true;
                active[k] = false;
            }
        }
        for (int64_t r = t0; r < a.N; r += stride) {
            int i = a.row_node[r];
            for (int k = 0; k < 2; ++k) {
                if (!active[k]) continue;
                T* p = V(a, k, VP);
                p[i] = V(a, k, VR)[i] + (T)beta[k] * (p[i] - (T)omega[k] * V(a, k, VQ)[i]);
            }
        }
        if (!grid_sync(a.bar, target += gridDim.x, a.flags)) return;
        // ---- B: q = A p ; (rh, q)
        {
            double d[2] = {0, 0};
            for (int64_t r = t0; r < a.N; r += stride) {
                int i = a.row_node[r];
                T L0, L1;
                row_L2(a, r, r + stride, V(a, 0, VP), two ? V(a, 1, VP) : nullptr, two && active[1], L0, L1);
                if (active[0]) {
                    T q = c0 * V(a, 0, VP)[i] - k0 * L0;
                    V(a, 0, VQ)[i] = q;
                    d[0] += (double)V(a, 0, VRH)[i] * q;
                }
                if (active[1]) {
                    T q = c0 * V(a, 1, VP)[i] - k1 * L1;
                    V(a, 1, VQ)[i] = q;
                    d[1] += (double)V(a, 1, VRH)[i] * q;
                }
            }
            block_partial<2>(d, a.partial, 1);
        }
        if (!grid_sync(a.bar, target += gridDim.x, a.flags)) return;
        {
            double s[2];
            grid_total<2>(a.partial, 1, s);
            for (int k = 0; k < 2; ++k) {
                if (!active[k]) continue;
                alpha[k] = rho[k] / s[k];
                if (s[k] == 0.0 || !isfinite(alpha[k])) {
                    fail[k] = true;
                    active[k] = false;
                }
            }
        }
        // ---- C: s = r - alpha q ; |s|^2
        {
            double d[2] = {0, 0};
            for (int64_t r = t0; r < a.N; r += stride) {
                int i = a.row_node[r];
                for (int k = 0; k < 2; ++k) {
                    if (!active[k]) continue;
                    T s = V(a, k, VR)[i] - (T)alpha[k] * V(a, k, VQ)[i];
                    V(a, k, VS)[i] = s;
                    d[k] += (double)s * s;
                }
            }
            block_partial<2>(d, a.partial, 2);
        }
        if (!grid_sync(a.bar, target += gridDim.x, a.flags)) return;
        bool early[2] = {false, false};
        {
            double s[2];
            grid_total<2>(a.partial, 2, s);
            for (int k = 0; k < 2; ++k) {
                if (!active[k]) continue;
                double rr = sqrt(s[k]) / bnorm[k];
                if (rr <= a.tol) {
                    early[k] = true;
                    relres[k] = rr;
                }
            }
        }
        // ---- D: t = A s ; (t, s), (t, t)   (x += alpha p where s converged)
        {
            double d[4] = {0, 0, 0, 0};
            bool need0 = active[0] && !early[0], need1 = active[1] && !early[1];
            for (int64_t r = t0; r < a.N; r += stride) {
                int i = a.row_node[r];
                T L0 = T(0), L1 = T(0);
                if (need0 || need1)
                    row_L2(a, r, r + stride, V(a, 0, VS), two ? V(a, 1, VS) : nullptr, two && need1, L0, L1);
                for (int k = 0; k < 2; ++k) {
                    T* x = k == 0 ? u : v;
                    if (early[k]) {
                        x[i] += (T)alpha[k] * V(a, k, VP)[i];
                    } else if (active[k]) {
                        T s = V(a, k, VS)[i];
                        T t = c0 * s - (k == 0 ? k0 * L0 : k1 * L1);
                        V(a, k, VT)[i] = t;
                        d[2 * k] += (double)t * s;
                        d[2 * k + 1] += (double)t * t;
                    }
                }
            }
            block_partial<4>(d, a.partial, 3);
        }
        for (int k = 0; k < 2; ++k)
            if (early[k]) {
                active[k] = false;
                conv[k] = true;
                iters[k] = it;
            }
        if (!grid_sync(a.bar, target += gridDim.x, a.flags)) return;
        {
            double s[4];
            grid_total<4>(a.partial, 3, s);
            for (int k = 0; k < 2; ++k) {
                if (!active[k]) continue;
                omega[k] = s[2 * k] / s[2 * k + 1];
                if (s[2 * k + 1] == 0.0 || !isfinite(omega[k])) {
                    fail[k] = true;
                    active[k] = false;
                }
            }
        }
        // ---- E: x += alpha p + omega s ; r = s - omega t ; (rh, r), |r|^2
        {
            double d[4] = {0, 0, 0, 0};
            for (int64_t r = t0; r < a.N; r += stride) {
                int i = a.row_node[r];
                for (int k = 0; k < 2; ++k) {
                    if (!active[k]) continue;
                    T* x = k == 0 ? u : v;
                    T s = V(a, k, VS)[i];
                    x[i] += (T)alpha[k] * V(a, k, VP)[i] + (T)omega[k] * s;
                    T rn = s - (T)omega[k] * V(a, k, VT)[i];
                    V(a, k, VR)[i] = rn;
                    d[2 * k] += (double)V(a, k, VRH)[i] * rn;
                    d[2 * k + 1] += (double)rn * rn;
                }
            }
            block_partial<4>(d, a.partial, 4);
        }
        if (!grid_sync(a.bar, target += gridDim.x, a.flags)) return;
        {
            double s[4];
            grid_total<4>(a.partial, 4, s);
            for (int k = 0; k < 2; ++k) {
                if (!active[k]) continue;
                rho_prev[k] = rho[k];
                rho[k] = s[2 * k];
                relres[k] = sqrt(s[2 * k + 1]) / bnorm[k];
                if (relres[k] <= a.tol) {
                    active[k] = false;
                    conv[k] = true;
                    iters[k] = it;
                } else if (omega[k] == 0.0) {
                    fail[k] = true;
                    active[k] = false;
                }
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        bool bad = false;
        for (int k = 0; k < 2; ++k) {
            if (active[k]) {   // hit maxit
                iters[k] = it;
                bad = true;
            }
            if (fail[k]) bad = true;
        }
        int* rp = a.rep + (int64_t)slot * 3;
        rp[0] = iters[0];
        rp[1] = iters[1];
        rp[2] = bad ? 1 : 0;
        a.rep_res[(int64_t)slot * 2] = relres[0];
        a.rep_res[(int64_t)slot * 2 + 1] = relres[1];
        if (bad) atomicExch(a.flags + 1, 1);
        a.flags[2] = min(nhist + 1, max(a.order - 1, 1));   // past levels now stored
        a.flags[3] = slot + 1;   // every block read the slot before the first barrier
        a.flags[4] = ord;
    }
}

// ---------------------------------------------------------------------------
// Phase-kernel BiCGSTAB for large operators, replayed from a CUDA graph: the
// right-hand side (R), then a device-side WHILE loop whose body is one
// BiCGSTAB iteration as five kernels (A: p; B: q = A p; C: s; D: t = A s;
// E: x, r), then the report (F).  Kernel boundaries make the vectors
// coherent, so the SpMV gathers go through L1 (neighbouring rows share most
// of their stencil nodes) -- inside one cooperative launch they must bypass
// it -- and no grid barrier is needed.  Reductions: block partials, then the
// phase's last block (by ticket) sums them in block order (deterministic)
// and sets the scalars the next phase reads; the last block of E commits
// the iteration and sets the loop condition.
// ---------------------------------------------------------------------------
constexpr int PT = 256;     // threads per block of the SpMV phase kernels (R, B, D)
constexpr int PT_MINB = 4;  // their resident blocks per SM (<= 64 registers a thread: no spills)
constexpr int PV = 256;    // threads per block of the vector phase kernels (A, C, E)
constexpr int PV_BPS = 4;   //   and their blocks per SM
constexpr int VG = 2;       // four-element groups a thread of phases A and C loads together

// (L x0)_r and (L x1)_r through L1 (x is not written by this kernel); the
// next chunk's index and weight loads go out before this chunk's gathers,
// so that a thread has two chunks of the matrix in flight, and with
// ROW_PF > 0 an L2 prefetch ROW_PF chunks ahead runs on into the thread's
// next row (rnext)
constexpr int ROW_PF = 2;

template <typename T>
__device__ __forceinline__ void row_L1(const Args<T>& a, int64_t r, int64_t rnext, const T* __restrict__ x0,
                                       const T* __restrict__ x1, bool two, T& y0, T& y1) {
    const int g = group_of_row(a.gi, r);
    const int npad = a.gi.npad[g], nch = npad >> 2;
    const int64_t base = ell_elem(a.gi.ell_off[g], npad, r - a.gi.row_begin[g], 0);
    int64_t nbase = -1;
    int nnch = 0;
    if (ROW_PF > 0 && rnext < a.N) {
        const int gn = group_of_row(a.gi, rnext);
        nnch = a.gi.npad[gn] >> 2;
        nbase = ell_elem(a.gi.ell_off[gn], a.gi.npad[gn], rnext - a.gi.row_begin[gn], 0);
    }
    T s0 = T(0), s1 = T(0);
    int4 iv = __ldcs(reinterpret_cast<const int4*>(a.idx + base));
    T wv[4];
    load4s(a.w + base, wv);
    for (int c = 0; c < nch; ++c) {
        if (ROW_PF > 0) {
            const int k = c + ROW_PF;
            int64_t e = -1;
            if (k < nch) e = base + (int64_t)k * 128;
            else if (k - nch < nnch && nbase >= 0) e = nbase + (int64_t)(k - nch) * 128;
            if (e >= 0) {
                prefetch_l2(a.idx + e);
                prefetch_l2(a.w + e);
            }
        }
        int4 ivn = iv;
        T wn[4] = {wv[0], wv[1], wv[2], wv[3]};
        if (c + 1 < nch) {
            const int64_t en = base + (int64_t)(c + 1) * 128;
            ivn = __ldcs(reinterpret_cast<const int4*>(a.idx + en));
            load4s(a.w + en, wn);
        }
        const int ii[4] = {iv.x, iv.y, iv.z, iv.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            s0 = fma(wv[q], __ldg(x0 + ii[q]), s0);
            if (two) s1 = fma(wv[q], __ldg(x1 + ii[q]), s1);
        }
        iv = ivn;
#pragma unroll
        for (int q = 0; q < 4; ++q) wv[q] = wn[q];
    }
    y0 = s0;
    y1 = two ? s1 : T(0);
}

constexpr int RED_ROUNDS = 4;   // rounds of partials the last block loads at once

// K sums per block (each thread's accumulators, in float64 from here on)
// into pp[block][0..K-1]; the last block of the grid sums them in block
// order into tot[0..K-1] and returns true.  Blocks of NTB <= 1024 threads.
template <int K, int NTB, typename A>
__device__ bool phase_reduce(const A (&v)[K], double* pp, double* tot, unsigned int* ticket) {
    __shared__ double sh[K][NTB / 32];
    __shared__ int last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double x = acc_value(v[k]);
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sh[k][wid] = x;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        double t = 0.0;
        for (int w = 0; w < NTB / 32; ++w) t += sh[threadIdx.x][w];
        pp[(int64_t)blockIdx.x * 8 + threadIdx.x] = t;
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return false;
    __threadfence();
    // fixed order: thread t sums blocks t, t + NTB, ...; then a fixed tree
    // over the threads' sums.  The loads of the first RED_ROUNDS rounds go
    // out together (one L2 round trip instead of one per round and sum)
    __shared__ double acc[K][NTB];
    double part[K][RED_ROUNDS];
#pragma unroll
    for (int u = 0; u < RED_ROUNDS; ++u) {
        const int64_t b = threadIdx.x + (int64_t)u * NTB;
#pragma unroll
        for (int k = 0; k < K; ++k) part[k][u] = b < gridDim.x ? __ldcg(pp + b * 8 + k) : 0.0;
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double t = 0.0;
#pragma unroll
        for (int u = 0; u < RED_ROUNDS; ++u)
            if (threadIdx.x + (int64_t)u * NTB < gridDim.x) t += part[k][u];
        for (int64_t b = threadIdx.x + (int64_t)RED_ROUNDS * NTB; b < gridDim.x; b += NTB) t += __ldcg(pp + b * 8 + k);
        acc[k][threadIdx.x] = t;
    }
    __syncthreads();
    for (int h = NTB / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h)
#pragma unroll
            for (int k = 0; k < K; ++k) acc[k][threadIdx.x] += acc[k][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x < K) tot[threadIdx.x] = acc[threadIdx.x][0];
    if (threadIdx.x == 0) *ticket = 0u;
    __syncthreads();
    return true;
}

__device__ __forceinline__ void set_more(PhaseCtl* c, cudaGraphConditionalHandle h, int more) {
    c->more = more;
    if (h) cudaGraphSetConditional(h, (unsigned)more);
}

// beta and the A-decision of the next iteration, from the committed state
__device__ __forceinline__ void next_iteration(PhaseCtl* c) {
    for (int k = 0; k < 2; ++k) {
        c->beta[k] = (c->rho[k] / c->rho_prev[k]) * (c->alpha[k] / c->omega[k]);
        c->actA[k] = c->active[k] && !(c->rho[k] == 0.0 || !isfinite(c->beta[k]));
        c->actB[k] = c->early[k] = c->actE[k] = 0;
    }
}

// R: right-hand side and r0 (the cooperative kernel's phase R, per row)
template <typename T>
__global__ void __launch_bounds__(PT, PT_MINB) phase_R(Args<T> a) {
    const StepCoef<T> kc = step_coef(a);
    const bool two = a.ns == 2;
    typename PhaseAcc<T>::type d[6];
    for (auto& x : d) acc_zero(x);
    for (int64_t r = blockIdx.x * (int64_t)PT + threadIdx.x; r < a.N; r += (int64_t)gridDim.x * PT) {
        const int64_t i = a.row_node[r];
        T Lu, Lv;
        row_L1(a, r, r + (int64_t)gridDim.x * PT, a.u, two ? a.v : a.u, two, Lu, Lv);
        rhs_row(a, kc, i, Lu, Lv, d);
    }
    PhaseCtl* c = a.ctl;
    if (phase_reduce<6, PT>(d, a.pp, c->totR, &c->ticket) && threadIdx.x == 0) {
        int more = 0;
        for (int k = 0; k < 2; ++k) {
            const bool exists = k == 0 || two;
            const double bn = sqrt(c->totR[3 * k]), rr = c->totR[3 * k + 1];
            c->bnorm[k] = bn;
            c->rho[k] = rr;   // (r-hat, r0) = |r0|^2
            c->rho_prev[k] = c->alpha[k] = c->omega[k] = 1.0;
            c->relres[k] = bn > 0 ? sqrt(rr) / bn : 0.0;
            c->conv[k] = !exists || bn == 0.0 || c->relres[k] <= a.tol;
            c->active[k] = !c->conv[k];
            c->fail[k] = 0;
            c->iters[k] = 0;
            c->zero[k] = exists && bn == 0.0;   // b = 0: x = 0
            more |= c->active[k];
        }
        c->it = 0;
        next_iteration(c);
        set_more(c, a.cond, more && a.maxit > 0);
    }
}

// The vector phases move groups of four consecutive elements with 16-byte
// loads and stores (every internal vector starts on a 16-byte boundary; the
// state u, v when the caller's are aligned, else a plain element loop): a
// quarter of the memory instructions and of the index arithmetic of an
// element loop, whose instruction count bounded them.  A thread visits
// groups g0, g0 + S, ... (S = the grid's threads), VG at a time with all
// their loads issued first; the last N mod 4 elements go element by
// element.  The dot products are summed per thread in that order.

__device__ __forceinline__ void ld4v(const float* p, float (&w)[4]) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
}
__device__ __forceinline__ void ld4v(const double* p, double (&w)[4]) {
    const double2 a = *reinterpret_cast<const double2*>(p);
    const double2 b = *reinterpret_cast<const double2*>(p + 2);
    w[0] = a.x; w[1] = a.y; w[2] = b.x; w[3] = b.y;
}
__device__ __forceinline__ void st4v(float* p, const float (&w)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(w[0], w[1], w[2], w[3]);
}
__device__ __forceinline__ void st4v(double* p, const double (&w)[4]) {
    *reinterpret_cast<double2*>(p) = make_double2(w[0], w[1]);
    *reinterpret_cast<double2*>(p + 2) = make_double2(w[2], w[3]);
}

// A: p = r + beta (p - omega q)
template <typename T>
__global__ void __launch_bounds__(PV, PV_BPS) phase_A(Args<T> a) {
    const PhaseCtl* c = a.ctl;
    const int64_t S = (int64_t)gridDim.x * PV, t0 = blockIdx.x * (int64_t)PV + threadIdx.x;
    for (int k = 0; k < a.ns; ++k) {
        if (!c->actA[k]) continue;
        const T beta = (T)c->beta[k], omega = (T)c->omega[k];
        T* __restrict__ p = V(a, k, VP);
        const T* __restrict__ r = V(a, k, VR);
        const T* __restrict__ q = V(a, k, VQ);
        int64_t i = t0;
        if (a.vec4) {
            const int64_t G = a.N >> 2;
            for (int64_t g0 = t0; g0 < G; g0 += VG * S) {
                T rv[VG][4], pv[VG][4], qv[VG][4];
#pragma unroll
                for (int u = 0; u < VG; ++u)
                    if (g0 + u * S < G) {
                        const int64_t e = 4 * (g0 + u * S);
                        ld4v(r + e, rv[u]);
                        ld4v(p + e, pv[u]);
                        ld4v(q + e, qv[u]);
                    }
#pragma unroll
                for (int u = 0; u < VG; ++u)
                    if (g0 + u * S < G) {
#pragma unroll
                        for (int j = 0; j < 4; ++j) pv[u][j] = rv[u][j] + beta * (pv[u][j] - omega * qv[u][j]);
                        st4v(p + 4 * (g0 + u * S), pv[u]);
                    }
            }
            i = 4 * G + t0;
        }
        for (; i < a.N; i += S) p[i] = r[i] + beta * (p[i] - omega * q[i]);
    }
}

// B: q = A p ; (r-hat, q).  With B_BACK it visits the rows from the last
// 32-row slice to the first (lanes keep their order within a slice): R and D
// run forward, so every pass over the matrix starts on the rows the pass
// before it ended on, which are still in L2.
constexpr bool B_BACK = true;

__device__ __forceinline__ int64_t back_row(int64_t k, int64_t Np) { return Np - 32 - (k & ~(int64_t)31) + (k & 31); }

template <typename T>
__global__ void __launch_bounds__(PT, PT_MINB) phase_B(Args<T> a) {
    PhaseCtl* c = a.ctl;
    const bool a0 = c->actA[0], a1 = a.ns == 2 && c->actA[1];
    const StepCoef<T> kc = step_coef(a);
    typename PhaseAcc<T>::type d[2];
    for (auto& x : d) acc_zero(x);
    const int64_t S = (int64_t)gridDim.x * PT, Np = (a.N + 31) & ~(int64_t)31;
    for (int64_t k = blockIdx.x * (int64_t)PT + threadIdx.x; (a0 || a1) && k < Np; k += S) {
        const int64_t r = B_BACK ? back_row(k, Np) : k;
        if (r >= a.N) continue;
        const int64_t rn = k + S >= Np ? a.N : (B_BACK ? back_row(k + S, Np) : k + S);
        const int64_t i = a.row_node[r];
        T L0, L1;
        row_L1(a, r, rn, V(a, 0, VP), a.ns == 2 ? V(a, 1, VP) : V(a, 0, VP), a1, L0, L1);
        if (a0) {
            const T q = kc.c0 * V(a, 0, VP)[i] - kc.k0 * L0;
            V(a, 0, VQ)[i] = q;
            acc_add(d[0], V(a, 0, VRH)[i], q);
        }
        if (a1) {
            const T q = kc.c0 * V(a, 1, VP)[i] - kc.k1 * L1;
            V(a, 1, VQ)[i] = q;
            acc_add(d[1], V(a, 1, VRH)[i], q);
        }
    }
    if (phase_reduce<2, PT>(d, a.pp, c->totB, &c->ticket) && threadIdx.x == 0)
        for (int k = 0; k < 2; ++k) {
            c->alpha_n[k] = c->actA[k] ? c->rho[k] / c->totB[k] : 0.0;
            c->actB[k] = c->actA[k] && !(c->totB[k] == 0.0 || !isfinite(c->alpha_n[k]));
        }
}

// C: s = r - alpha q ; |s|^2
template <typename T>
__global__ void __launch_bounds__(PV, PV_BPS) phase_C(Args<T> a) {
    PhaseCtl* c = a.ctl;
    typename PhaseAcc<T>::type d[2];
    for (auto& x : d) acc_zero(x);
    const int64_t S = (int64_t)gridDim.x * PV, t0 = blockIdx.x * (int64_t)PV + threadIdx.x;
    for (int k = 0; k < a.ns; ++k) {
        if (!c->actB[k]) continue;
        const T alpha = (T)c->alpha_n[k];
        const T* __restrict__ r = V(a, k, VR);
        const T* __restrict__ q = V(a, k, VQ);
        T* __restrict__ sv = V(a, k, VS);
        int64_t i = t0;
        if (a.vec4) {
            const int64_t G = a.N >> 2;
            for (int64_t g0 = t0; g0 < G; g0 += VG * S) {
                T rv[VG][4], qv[VG][4];
#pragma unroll
                for (int u = 0; u < VG; ++u)
                    if (g0 + u * S < G) {
                        const int64_t e = 4 * (g0 + u * S);
                        ld4v(r + e, rv[u]);
                        ld4v(q + e, qv[u]);
                    }
#pragma unroll
                for (int u = 0; u < VG; ++u)
                    if (g0 + u * S < G) {
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            rv[u][j] = rv[u][j] - alpha * qv[u][j];
                            acc_add(d[k], rv[u][j], rv[u][j]);
                        }
                        st4v(sv + 4 * (g0 + u * S), rv[u]);
                    }
            }
            i = 4 * G + t0;
        }
        for (; i < a.N; i += S) {
            const T x = r[i] - alpha * q[i];
            sv[i] = x;
            acc_add(d[k], x, x);
        }
    }
    if (phase_reduce<2, PV>(d, a.pp, c->totC, &c->ticket) && threadIdx.x == 0)
        for (int k = 0; k < 2; ++k) c->early[k] = c->actB[k] && sqrt(c->totC[k]) / c->bnorm[k] <= a.tol;
}

// D: t = A s ; (t, s), (t, t)   (x += alpha p where s already converged)
template <typename T>
__global__ void __launch_bounds__(PT, PT_MINB) phase_D(Args<T> a) {
    PhaseCtl* c = a.ctl;
    const StepCoef<T> kc = step_coef(a);
    const bool two = a.ns == 2;
    const bool e0 = c->early[0], e1 = two && c->early[1];
    const bool b0 = c->actB[0], b1 = two && c->actB[1];
    const bool need0 = b0 && !e0, need1 = b1 && !e1;
    typename PhaseAcc<T>::type d[4];
    for (auto& x : d) acc_zero(x);
    for (int64_t r = blockIdx.x * (int64_t)PT + threadIdx.x; (b0 || b1) && r < a.N; r += (int64_t)gridDim.x * PT) {
        const int64_t i = a.row_node[r];
        T L0 = T(0), L1 = T(0);
        if (need0 || need1) row_L1(a, r, r + (int64_t)gridDim.x * PT, V(a, 0, VS), two ? V(a, 1, VS) : V(a, 0, VS), need1, L0, L1);
        for (int k = 0; k < a.ns; ++k) {
            T* x = k == 0 ? a.u : a.v;
            if (k == 0 ? e0 : e1) {
                x[i] += (T)c->alpha_n[k] * V(a, k, VP)[i];
            } else if (k == 0 ? b0 : b1) {
                const T sv = V(a, k, VS)[i];
                const T t = kc.c0 * sv - (k == 0 ? kc.k0 * L0 : kc.k1 * L1);
                V(a, k, VT)[i] = t;
                acc_add(d[2 * k], t, sv);
                acc_add(d[2 * k + 1], t, t);
            }
        }
    }
    if (phase_reduce<4, PT>(d, a.pp, c->totD, &c->ticket) && threadIdx.x == 0)
        for (int k = 0; k < 2; ++k) {
            c->omega_n[k] = c->totD[2 * k] / c->totD[2 * k + 1];
            c->actE[k] = c->actB[k] && !c->early[k] && !(c->totD[2 * k + 1] == 0.0 || !isfinite(c->omega_n[k]));
        }
}

// E: x += alpha p + omega s ; r = s - omega t ; (r-hat, r), |r|^2; the last
// block commits the iteration and decides whether the loop continues
template <typename T>
__device__ __forceinline__ void e_update(T alpha, T omega, T& x, T p, T s, T t, T& r) {
    x = x + (alpha * p + omega * s);
    r = s - omega * t;
}

template <typename T>
__global__ void __launch_bounds__(PV, PV_BPS) phase_E(Args<T> a) {
    PhaseCtl* c = a.ctl;
    typename PhaseAcc<T>::type d[4];
    for (auto& x : d) acc_zero(x);
    const int64_t S = (int64_t)gridDim.x * PV, t0 = blockIdx.x * (int64_t)PV + threadIdx.x;
    for (int k = 0; k < a.ns; ++k) {
        if (!c->actE[k]) continue;
        const T alpha = (T)c->alpha_n[k], omega = (T)c->omega_n[k];
        T* __restrict__ x = k == 0 ? a.u : a.v;
        const T* __restrict__ p = V(a, k, VP);
        const T* __restrict__ sv = V(a, k, VS);
        const T* __restrict__ t = V(a, k, VT);
        const T* __restrict__ rh = V(a, k, VRH);
        T* __restrict__ r = V(a, k, VR);
        int64_t i = t0;
        if (a.vec4) {
            const int64_t G = a.N >> 2;
            for (int64_t g = t0; g < G; g += S) {
                const int64_t e = 4 * g;
                T xv[4], pv[4], s_[4], tv[4], hv[4], rn[4];
                ld4v(x + e, xv);
                ld4v(p + e, pv);
                ld4v(sv + e, s_);
                ld4v(t + e, tv);
                ld4v(rh + e, hv);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    e_update(alpha, omega, xv[j], pv[j], s_[j], tv[j], rn[j]);
                    acc_add(d[2 * k], hv[j], rn[j]);
                    acc_add(d[2 * k + 1], rn[j], rn[j]);
                }
                st4v(x + e, xv);
                st4v(r + e, rn);
            }
            i = 4 * G + t0;
        }
        for (; i < a.N; i += S) {
            T xi = x[i], rn;
            e_update(alpha, omega, xi, p[i], sv[i], t[i], rn);
            x[i] = xi;
            r[i] = rn;
            acc_add(d[2 * k], rh[i], rn);
            acc_add(d[2 * k + 1], rn, rn);
        }
    }
    if (phase_reduce<4, PV>(d, a.pp, c->totE, &c->ticket) && threadIdx.x == 0) {
        const int it = c->it + 1;
        int more = 0;
        for (int k = 0; k < 2; ++k) {
            if (!c->active[k]) continue;
            if (!c->actA[k] || !c->actB[k]) {
                c->fail[k] = 1;
                c->active[k] = 0;
            } else if (c->early[k]) {
                c->relres[k] = sqrt(c->totC[k]) / c->bnorm[k];
                c->conv[k] = 1;
                c->active[k] = 0;
                c->iters[k] = it;
            } else if (!c->actE[k]) {
                c->fail[k] = 1;
                c->active[k] = 0;
            } else {
                c->rho_prev[k] = c->rho[k];
                c->rho[k] = c->totE[2 * k];
                c->alpha[k] = c->alpha_n[k];
                c->omega[k] = c->omega_n[k];
                c->relres[k] = sqrt(c->totE[2 * k + 1]) / c->bnorm[k];
                if (c->relres[k] <= a.tol) {
                    c->conv[k] = 1;
                    c->active[k] = 0;
                    c->iters[k] = it;
                } else if (c->omega_n[k] == 0.0) {
                    c->fail[k] = 1;
                    c->active[k] = 0;
                }
            }
            more |= c->active[k];
        }
        c->it = it;
        next_iteration(c);
        set_more(c, a.cond, more && it < a.maxit);
    }
}

// F: report of the step, history flags, x = 0 where b = 0
template <typename T>
__global__ void __launch_bounds__(PT) phase_F(Args<T> a) {
    const PhaseCtl* c = a.ctl;
    for (int k = 0; k < a.ns; ++k) {
        if (!c->zero[k]) continue;
        T* x = k == 0 ? a.u : a.v;
        for (int64_t i = blockIdx.x * (int64_t)PT + threadIdx.x; i < a.N; i += (int64_t)gridDim.x * PT) x[i] = T(0);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const StepCoef<T> kc = step_coef(a);
        int iters[2] = {c->iters[0], c->iters[1]};
        bool bad = false;
        for (int k = 0; k < 2; ++k) {
            if (c->active[k]) {   // hit maxit
                iters[k] = c->it;
                bad = true;
            }
            if (c->fail[k]) bad = true;
        }
        int* rp = a.rep + (int64_t)kc.slot * 3;
        rp[0] = iters[0];
        rp[1] = iters[1];
        rp[2] = bad ? 1 : 0;
        a.rep_res[(int64_t)kc.slot * 2] = c->relres[0];
        a.rep_res[(int64_t)kc.slot * 2 + 1] = c->relres[1];
        if (bad) atomicExch(a.flags + 1, 1);
        a.flags[2] = min(kc.nhist + 1, max(a.order - 1, 1));
        a.flags[3] = kc.slot + 1;
        a.flags[4] = kc.ord;
    }
}

__global__ void lonely_barrier(unsigned long long* bar, int* err) {
    // a second arrival never comes: the bounded wait must give up
    grid_sync(bar, 2ull * gridDim.x, err);
}

template <typename T>
void fill_args(Args<T>& a, rbffd_op* op, rbffd_state* s, const rbffd_step_params* p, rbffd_step_ws* ws) {
    a.idx = op->idx;
    a.w = std::is_same<T, float>::value ? (const T*)op->w32 : (const T*)op->w64;
    a.row_node = op->row_node;
    a.gi = op->gi;
    a.N = op->N;
    a.u = (T*)s->u;
    a.v = (T*)s->v;
    a.up = (T*)s->u_prev;
    a.vp = (T*)s->v_prev;
    a.fp = (T*)s->f_prev;
    a.gp = (T*)s->g_prev;
    a.up2 = (T*)s->u_prev2;
    a.vp2 = (T*)s->v_prev2;
    a.fp2 = (T*)s->f_prev2;
    a.gp2 = (T*)s->g_prev2;
    a.up3 = (T*)s->u_prev3;
    a.vp3 = (T*)s->v_prev3;
    a.fp3 = (T*)s->f_prev3;
    a.gp3 = (T*)s->g_prev3;
    a.order = p->order == 0 ? 2 : p->order;
    a.su = (const T*)p->source_u;
    a.sv = p->nspecies == 2 ? (const T*)p->source_v : nullptr;
    a.src_rate = p->source_rate;
    a.tstart = ws->tstart;
    a.vec = (T*)ws->vec;
    a.ldv = (op->N + 3) & ~(int64_t)3;
    a.vec4 = ((uintptr_t)s->u % 16 == 0 && (p->nspecies == 1 || (uintptr_t)s->v % 16 == 0)) ? 1 : 0;
    a.ns = p->nspecies;
    a.model = p->model;
    for (int i = 0; i < 8; ++i) a.c[i] = (T)p->coef[i];
    a.dt = (T)p->dt;
    a.delta[0] = (T)p->delta_u;
    a.delta[1] = (T)p->delta_v;
    a.tol = p->tol;
    a.maxit = p->maxit;
    a.partial = ws->partial;
    a.bar = ws->bar;
    a.flags = ws->flags;
    a.rep = ws->rep;
    a.rep_res = ws->rep_res;
    a.rhs_only = p->solver == RBFFD_SOLVER_BANDED_LU ? 1 : 0;
    a.ctl = ws->ctl;
    a.pp = ws->pp;
    a.cond = 0;
}

template <typename T>
rbffd_status launch_step(Args<T>& a, rbffd_step_ws* ws, cudaStream_t st) {
    RBFFD_CUDA_TRY(cudaMemsetAsync(ws->bar, 0, sizeof(unsigned long long), st));
    void* args[] = {&a};
    const void* fn = ws->threads == 1024 ? (const void*)step_kernel<T, 1024> : (const void*)step_kernel<T, 256>;
    RBFFD_CUDA_TRY(cudaLaunchCooperativeKernel(fn, dim3(ws->blocks),
                                               dim3(ws->threads), args, 0, st));
    note_launch();
    if (a.rhs_only) {
        // (c0 I - cl delta L) x = b by the cached LU factors of the step's
        // order (read on the device from flags[4]); x overwrites u, v
        const void* b[2] = {V(a, 0, VB), a.ns == 2 ? V(a, 1, VB) : nullptr};
        void* x[2] = {a.u, a.ns == 2 ? a.v : nullptr};
        rbffd_status r = lu_solve_step(ws->lu, a.ns, b, x, std::is_same<T, float>::value ? RBFFD_F32 : RBFFD_F64,
                                       ws->flags + 4, ws->ywork, ws->flags, st);
        if (r != RBFFD_OK) return r;
    }
    return RBFFD_OK;
}

// resident-sized grids, grid-stride loops: the SpMV phases PT_MINB blocks
// of PT threads per SM (their register bound makes exactly that many fit:
// one wave, no partial second one), the vector phases one block of PV
// threads per SM.  (A grid of one thread per row or element ran slower:
// the per-block reduction and ticket then cost more than a block's work.)
// The per-block partials (pp) hold ceil(N / PT) blocks, more than either grid.
template <typename T>
void phase_grids(const Args<T>& a, unsigned* g_rows, unsigned* g_vec) {
    *g_rows = (unsigned)std::max<int64_t>(1, std::min<int64_t>((a.N + PT - 1) / PT, (int64_t)sm_count() * PT_MINB));
    *g_vec = (unsigned)std::max<int64_t>(1, std::min<int64_t>((a.N + PV - 1) / PV, (int64_t)sm_count() * PV_BPS));
}

// One step of the phase-kernel path from the host (no graph): R, then the
// iterations while the loop state says so (the condition is read back after
// each iteration), then F -- the same kernels and arithmetic as the graph.
template <typename T>
rbffd_status phased_step_host(Args<T>& a, rbffd_step_ws* ws, cudaStream_t st) {
    unsigned gr, gv;
    phase_grids(a, &gr, &gv);
    a.cond = 0;
    phase_R<T><<<gr, PT, 0, st>>>(a);
    note_launch();
    RBFFD_CUDA_TRY(cudaGetLastError());
    for (;;) {
        int more = 0;
        RBFFD_CUDA_TRY(cudaMemcpyAsync(&more, &ws->ctl->more, sizeof(int), cudaMemcpyDeviceToHost, st));
        RBFFD_CUDA_TRY(cudaStreamSynchronize(st));
        if (!more) break;
        phase_A<T><<<gv, PV, 0, st>>>(a);
        phase_B<T><<<gr, PT, 0, st>>>(a);
        phase_C<T><<<gv, PV, 0, st>>>(a);
        phase_D<T><<<gr, PT, 0, st>>>(a);
        phase_E<T><<<gv, PV, 0, st>>>(a);
        note_launch(5);
        RBFFD_CUDA_TRY(cudaGetLastError());
    }
    phase_F<T><<<gr, PT, 0, st>>>(a);
    note_launch();
    RBFFD_CUDA_TRY(cudaGetLastError());
    return RBFFD_OK;
}

// The step as a graph: R -> WHILE (condition set on the device) { A B C D E } -> F
template <typename T>
rbffd_status build_phase_graph(Args<T> a, cudaGraphExec_t* out) {
    unsigned gr, gv;
    phase_grids(a, &gr, &gv);
    cudaGraph_t g = nullptr;
    RBFFD_CUDA_TRY(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 0, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        RBFFD_CUDA_TRY(e);
    }
    a.cond = h;
    void* args[] = {&a};
    auto kernel = [&](cudaGraph_t graph, const void* fn, bool vec, cudaGraphNode_t* dep, cudaGraphNode_t* node) {
        cudaKernelNodeParams kp;
        memset(&kp, 0, sizeof(kp));
        kp.func = const_cast<void*>(fn);
        kp.gridDim = dim3(vec ? gv : gr);
        kp.blockDim = dim3(vec ? PV : PT);
        kp.kernelParams = args;
        return cudaGraphAddKernelNode(node, graph, dep, dep ? 1 : 0, &kp);
    };
    cudaGraphNode_t nR, nW, nF;
    e = kernel(g, (const void*)phase_R<T>, false, nullptr, &nR);
    // (the parameter union has no default constructor: zeroed raw storage)
    alignas(cudaGraphNodeParams) unsigned char cp_raw[sizeof(cudaGraphNodeParams)];
    memset(cp_raw, 0, sizeof(cp_raw));
    cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_raw);
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    if (e == cudaSuccess) e = cudaGraphAddNode(&nW, g, &nR, nullptr, 1, &cp);
    if (e == cudaSuccess) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        cudaGraphNode_t n1, n2, n3, n4, n5;
        e = kernel(body, (const void*)phase_A<T>, true, nullptr, &n1);
        if (e == cudaSuccess) e = kernel(body, (const void*)phase_B<T>, false, &n1, &n2);
        if (e == cudaSuccess) e = kernel(body, (const void*)phase_C<T>, true, &n2, &n3);
        if (e == cudaSuccess) e = kernel(body, (const void*)phase_D<T>, false, &n3, &n4);
        if (e == cudaSuccess) e = kernel(body, (const void*)phase_E<T>, true, &n4, &n5);
    }
    if (e == cudaSuccess) e = kernel(g, (const void*)phase_F<T>, false, &nW, &nF);
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    RBFFD_CUDA_TRY(e);
    return RBFFD_OK;
}

// nsteps launches, directly or by replaying one captured graph of a step
template <typename T>
rbffd_status run_steps(Args<T>& a, rbffd_step_ws* ws, int64_t nsteps, bool use_graph, cudaStream_t st) {
    static_assert(sizeof(Args<T>) <= sizeof(ws->graph_args), "graph key too small");
    if (ws->phased && !a.rhs_only) {
        if (!use_graph) {
            for (int64_t k = 0; k < nsteps; ++k) {
                rbffd_status r = phased_step_host(a, ws, st);
                if (r != RBFFD_OK) return r;
            }
            return RBFFD_OK;
        }
        a.cond = 0;   // the graph key holds the arguments without the handle
        if (!ws->graph || ws->graph_args_size != sizeof(a) || memcmp(ws->graph_args, &a, sizeof(a)) != 0 ||
            ws->solver != 2) {
            if (ws->graph) {
                cudaGraphExecDestroy(ws->graph);
                ws->graph = nullptr;
            }
            rbffd_status r = build_phase_graph(a, &ws->graph);
            if (r != RBFFD_OK) return r;
            memcpy(ws->graph_args, &a, sizeof(a));
            ws->graph_args_size = sizeof(a);
            ws->solver = 2;
        }
        for (int64_t k = 0; k < nsteps; ++k) {
            RBFFD_CUDA_TRY(cudaGraphLaunch(ws->graph, st));
            note_launch(2);   // R and F; the loop body's five per iteration are counted from the report
        }
        return RBFFD_OK;
    }
    if (!use_graph) {
        for (int64_t k = 0; k < nsteps; ++k) {
            rbffd_status r = launch_step(a, ws, st);
            if (r != RBFFD_OK) return r;
        }
        return RBFFD_OK;
    }
    // the graph holds the kernels' arguments, the LU solve's factor pointers
    // included: any change recaptures it
    if (!ws->graph || ws->graph_args_size != sizeof(a) || memcmp(ws->graph_args, &a, sizeof(a)) != 0 ||
        ws->solver != a.rhs_only || memcmp(ws->graph_lu, ws->lu, sizeof(ws->lu)) != 0 || ws->solver == 2) {
        if (ws->graph) {
            cudaGraphExecDestroy(ws->graph);
            ws->graph = nullptr;
        }
        // capture on a private stream (the caller's may be the legacy default
        // stream, which cannot be captured); replay on the caller's stream
        if (!ws->cap) RBFFD_CUDA_TRY(cudaStreamCreateWithFlags(&ws->cap, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        RBFFD_CUDA_TRY(cudaStreamBeginCapture(ws->cap, cudaStreamCaptureModeThreadLocal));
        rbffd_status r = launch_step(a, ws, ws->cap);
        cudaError_t e = cudaStreamEndCapture(ws->cap, &g);
        if (r != RBFFD_OK) return r;
        RBFFD_CUDA_TRY(e);
        e = cudaGraphInstantiate(&ws->graph, g, 0);
        cudaGraphDestroy(g);
        RBFFD_CUDA_TRY(e);
        memcpy(ws->graph_args, &a, sizeof(a));
        ws->graph_args_size = sizeof(a);
        ws->solver = a.rhs_only;
        memcpy(ws->graph_lu, ws->lu, sizeof(ws->lu));
    }
    for (int64_t k = 0; k < nsteps; ++k) {
        RBFFD_CUDA_TRY(cudaGraphLaunch(ws->graph, st));
        note_launch();
    }
    return RBFFD_OK;
}

}  // namespace
}  // namespace rbffd

using namespace rbffd;

extern "C" rbffd_status rbffd_step_imex(rbffd_op* op, rbffd_state* s, const rbffd_step_params* p,
                                        int64_t nsteps, void* stream, rbffd_step_report* report) {
    RBFFD_CHECK_ARG(op && s && p, "NULL argument");
    RBFFD_CHECK_ARG(p->dtype == RBFFD_F32 || p->dtype == RBFFD_F64, "dtype");
    RBFFD_CHECK_ARG(p->nspecies == 1 || p->nspecies == 2, "nspecies must be 1 or 2");
    RBFFD_CHECK_ARG(s->u && s->u_prev && s->f_prev, "u / u_prev / f_prev are NULL");
    RBFFD_CHECK_ARG(p->nspecies == 1 || (s->v && s->v_prev && s->g_prev), "v state is NULL");
    RBFFD_CHECK_ARG(p->dt > 0 && p->tol > 0 && p->maxit > 0 && nsteps >= 0, "dt / tol / maxit / nsteps");
    RBFFD_CHECK_ARG(p->model >= RBFFD_MODEL_NONE && p->model <= RBFFD_MODEL_BARRIO, "model");
    RBFFD_CHECK_ARG(p->model != RBFFD_MODEL_BARRIO || p->coef[1] != 0.0, "Barrio model needs beta != 0");
    const int order = p->order == 0 ? 2 : p->order;
    RBFFD_CHECK_ARG(order >= 1 && order <= 4, "order must be 1..4 (0 = 2)");
    RBFFD_CHECK_ARG(order < 3 || (s->u_prev2 && s->f_prev2 &&
                                  (p->nspecies == 1 || (s->v_prev2 && s->g_prev2))),
                    "SBDF3/4 need u_prev2 / f_prev2 (and v_prev2 / g_prev2)");
    RBFFD_CHECK_ARG(order < 4 || (s->u_prev3 && s->f_prev3 &&
                                  (p->nspecies == 1 || (s->v_prev3 && s->g_prev3))),
                    "SBDF4 needs u_prev3 / f_prev3 (and v_prev3 / g_prev3)");
    RBFFD_CHECK_ARG(s->has_history >= 0, "has_history must be >= 0");
    RBFFD_CHECK_ARG(p->solver == RBFFD_SOLVER_BICGSTAB || p->solver == RBFFD_SOLVER_BANDED_LU, "solver");
    cudaStream_t st = as_stream(stream);
    const size_t elem = p->dtype == RBFFD_F32 ? 4 : 8;
    rbffd_step_ws* ws = op->step;
    if (ws && ws->elem != elem) {
        step_ws_free(ws);
        ws = op->step = nullptr;
    }
    if (!ws) {
        ws = new rbffd_step_ws();
        memset(ws, 0, sizeof(*ws));
        op->step = ws;
        ws->elem = elem;
        ws->N = op->N;
        // The cooperative kernel's shape.  Large operators (a row per thread
        // at one 1024-thread block per SM) run BiCGSTAB as phase kernels and
        // use the cooperative launch only for the right-hand side of an LU
        // step; there one 1024-thread block per SM meets at each grid barrier
        // (measured when BiCGSTAB still ran in it, 1M-node operator: 2.67 ms
        // per step against 3.08 ms with 2 x 512 and 3.22 ms with 2 x 256
        // threads per SM; 4 x 256 was slower still, 3.94 ms -- the barrier's
        // cost grows with its blocks).  Smaller operators keep 256-thread
        // blocks (about four rows per thread) so that they still spread over
        // the SMs.
        ws->threads = op->N >= (int64_t)1024 * sm_count() ? 1024 : 256;
        int dev = 0, per_sm = 0;
        RBFFD_CUDA_TRY(cudaGetDevice(&dev));
        const void* fn = elem == 4 ? (ws->threads == 1024 ? (const void*)step_kernel<float, 1024>
                                                          : (const void*)step_kernel<float, 256>)
                                   : (ws->threads == 1024 ? (const void*)step_kernel<double, 1024>
                                                          : (const void*)step_kernel<double, 256>);
        RBFFD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, ws->threads, 0));
        int64_t maxb = (int64_t)std::max(1, per_sm) * sm_count();
        const int64_t rows_per_block = ws->threads == 1024 ? 1024 : 4 * 256;
        int64_t want = (op->N + rows_per_block - 1) / rows_per_block;
        ws->blocks = (int)std::max<int64_t>(1, std::min(maxb, std::max<int64_t>(want, 1)));
        RBFFD_CUDA_TRY(cudaMalloc(&ws->vec, 2 * 7 * ((op->N + 3) & ~(int64_t)3) * elem));
        RBFFD_CUDA_TRY(cudaMalloc(&ws->partial, (size_t)NPHASE * ws->blocks * NSLOT * sizeof(double)));
        RBFFD_CUDA_TRY(cudaMalloc(&ws->bar, sizeof(unsigned long long)));
        RBFFD_CUDA_TRY(cudaMalloc(&ws->flags, 5 * sizeof(int)));
        RBFFD_CUDA_TRY(cudaMalloc(&ws->tstart, sizeof(double)));
        // large operators: BiCGSTAB as phase kernels under a device-side
        // loop (SpMV gathers through L1, full occupancy); small ones: the
        // cooperative kernel (a few blocks, latency-bound, where one launch
        // per step wins)
        ws->phased = ws->threads == 1024 ? 1 : 0;
        RBFFD_CUDA_TRY(cudaMalloc(&ws->ctl, sizeof(PhaseCtl)));
        RBFFD_CUDA_TRY(cudaMemset(ws->ctl, 0, sizeof(PhaseCtl)));
        RBFFD_CUDA_TRY(cudaMalloc(&ws->pp, (size_t)std::max<int64_t>(1, (op->N + PT - 1) / PT) * 8 * sizeof(double)));
        ws->rep_cap = 0;
    }
    if (ws->rep_cap < std::max<int64_t>(nsteps, 1)) {
        cudaFree(ws->rep);
        cudaFree(ws->rep_res);
        ws->rep_cap = std::max<int64_t>(nsteps, 1);
        RBFFD_CUDA_TRY(cudaMalloc(&ws->rep, ws->rep_cap * 3 * sizeof(int)));
        RBFFD_CUDA_TRY(cudaMalloc(&ws->rep_res, ws->rep_cap * 2 * sizeof(double)));
    }
    const int kept = std::max(order - 1, 1);   // past levels the order stores
    int hflags[5] = {0, 0, std::min(s->has_history, kept), 0, 0};   // slot counter starts at 0
    if (p->solver == RBFFD_SOLVER_BANDED_LU) {
        // factor (c0 I - cl delta L) for every SBDF order this call steps
        // with (orders climb while history builds up) and species, once per
        // (order, dt, delta, dtype); factors live with the workspace
        int h = std::min(s->has_history, kept);
        bool need[4] = {false, false, false, false};
        for (int64_t k = 0; k < nsteps && k < 4; ++k) {
            need[std::min(order, h + 1) - 1] = true;
            h = std::min(h + 1, kept);
        }
        if (nsteps > 4) need[std::min(order, h + 1) - 1] = true;
        const double c0s[4] = {1.0, 3.0, 11.0, 25.0}, cls[4] = {1.0, 2.0, 6.0, 12.0};
        const double del[2] = {p->delta_u, p->delta_v};
        for (int o = 0; o < 4; ++o) {
            if (!need[o]) continue;
            for (int sp = 0; sp < p->nspecies; ++sp) {
                const double alpha = c0s[o], beta = cls[o] * p->dt * del[sp];
                rbffd_lu*& f = ws->lu[o][sp];
                // float64 factors whatever the step's dtype: a float32 band
                // LU loses several digits to its growth and rounding, while
                // the substitutions are latency-bound, not FP64-bound
                if (f && (f->alpha != alpha || f->beta != beta)) {
                    lu_free(f);
                    f = nullptr;
                }
                if (!f) {
                    rbffd_status fs = lu_factor(op, alpha, beta, RBFFD_F64, st, &f);
                    if (fs != RBFFD_OK) return fs;
                }
            }
        }
        if (!ws->ywork) RBFFD_CUDA_TRY(cudaMalloc(&ws->ywork, (2 * (2 * op->N + 16)) * sizeof(double) + 64));
    }
    RBFFD_CUDA_TRY(cudaMemcpyAsync(ws->flags, hflags, sizeof(hflags), cudaMemcpyHostToDevice, st));
    RBFFD_CUDA_TRY(cudaMemcpyAsync(ws->tstart, &s->t, sizeof(double), cudaMemcpyHostToDevice, st));
    RBFFD_CUDA_TRY(cudaMemsetAsync(ws->rep, 0, ws->rep_cap * 3 * sizeof(int), st));
    rbffd_status rs;
    if (elem == 4) {
        Args<float> a;
        memset(&a, 0, sizeof(a));
        fill_args(a, op, s, p, ws);
        rs = run_steps(a, ws, nsteps, p->use_graph != 0, st);
    } else {
        Args<double> a;
        memset(&a, 0, sizeof(a));
        fill_args(a, op, s, p, ws);
        rs = run_steps(a, ws, nsteps, p->use_graph != 0, st);
    }
    if (rs != RBFFD_OK) return rs;
    std::vector<int> rep(std::max<int64_t>(nsteps, 1) * 3);
    std::vector<double> res(std::max<int64_t>(nsteps, 1) * 2);
    RBFFD_CUDA_TRY(cudaMemcpyAsync(hflags, ws->flags, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
    if (nsteps > 0) {
        RBFFD_CUDA_TRY(cudaMemcpyAsync(rep.data(), ws->rep, nsteps * 3 * sizeof(int), cudaMemcpyDeviceToHost, st));
        RBFFD_CUDA_TRY(cudaMemcpyAsync(res.data(), ws->rep_res, nsteps * 2 * sizeof(double),
                                       cudaMemcpyDeviceToHost, st));
    }
    RBFFD_CUDA_TRY(cudaStreamSynchronize(st));
    rbffd_step_report r;
    memset(&r, 0, sizeof(r));
    r.failed_step = -1;
    for (int64_t k = 0; k < nsteps; ++k) {
        r.max_iters_u = std::max(r.max_iters_u, rep[3 * k]);
        r.max_iters_v = std::max(r.max_iters_v, rep[3 * k + 1]);
        r.total_iters += rep[3 * k] + rep[3 * k + 1];
        if (rep[3 * k + 2] && r.failed_step < 0) r.failed_step = s->step + k;
        r.last_relres_u = res[2 * k];
        r.last_relres_v = res[2 * k + 1];
    }
    if (ws->phased && p->use_graph && p->solver == RBFFD_SOLVER_BICGSTAB)
        for (int64_t k = 0; k < nsteps; ++k) note_launch(5 * std::max(rep[3 * k], rep[3 * k + 1]));
    r.steps_done = nsteps;
    s->has_history = (int)std::min<int64_t>((int64_t)std::min(s->has_history, kept) + nsteps, kept);
    s->step += nsteps;
    s->t += (double)nsteps * p->dt;
    if (report) *report = r;
    if (hflags[0]) {
        set_error("grid barrier timed out (blocks not co-resident?)");
        return RBFFD_TIMEOUT;
    }
    if (hflags[1]) {
        set_error("BiCGSTAB failed at step %lld", (long long)r.failed_step);
        return RBFFD_SOLVER_NOT_CONVERGED;
    }
    return RBFFD_OK;
}

extern "C" rbffd_status rbffd_selftest_barrier_timeout(void* stream) {
    cudaStream_t st = as_stream(stream);
    unsigned long long* bar = nullptr;
    int* err = nullptr;
    RBFFD_CUDA_TRY(cudaMalloc(&bar, sizeof(unsigned long long)));
    RBFFD_CUDA_TRY(cudaMalloc(&err, sizeof(int)));
    RBFFD_CUDA_TRY(cudaMemsetAsync(bar, 0, sizeof(unsigned long long), st));
    RBFFD_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
    lonely_barrier<<<1, 32, 0, st>>>(bar, err);
    note_launch();
    RBFFD_CUDA_TRY(cudaGetLastError());
    int h = 0;
    RBFFD_CUDA_TRY(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    RBFFD_CUDA_TRY(cudaStreamSynchronize(st));
    cudaFree(bar);
    cudaFree(err);
    if (h) {
        set_error("grid barrier wait gave up as designed");
        return RBFFD_TIMEOUT;
    }
    return RBFFD_OK;
}
