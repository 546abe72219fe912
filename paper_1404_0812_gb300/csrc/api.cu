// C ABI entry points (include/rbffd.h): argument checks, operator storage,
// and the order of the build phases.  The arithmetic lives in knn.cu,
// build.cu, apply.cu, step.cu and mlp.cu.
#include "common.cuh"

#include <algorithm>
#include <atomic>
#include <mutex>
#include <cmath>
#include <cstdarg>
#include <map>
#include <vector>

namespace rbffd {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

static std::atomic<int64_t> g_launches{0};
void note_launch(int k) { g_launches.fetch_add(k); }

// ---- the library's stream-ordered memory pools (one per device)
namespace {
constexpr int MAX_DEVICES = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[MAX_DEVICES] = {};
constexpr uint64_t POOL_KEEP_DEFAULT = 32ull << 30;

cudaError_t device_pool(cudaMemPool_t* out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        e = cudaMemPoolCreate(&pool, &props);
        if (e != cudaSuccess) return e;
        uint64_t keep = POOL_KEEP_DEFAULT;
        e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(pool);
            return e;
        }
        g_pool[dev] = pool;
    }
    *out = g_pool[dev];
    return cudaSuccess;
}
}  // namespace

cudaError_t pool_alloc_bytes(void** p, size_t bytes, cudaStream_t st) {
    cudaMemPool_t pool = nullptr;
    cudaError_t e = device_pool(&pool);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

int sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

rbffd_status apply_launch(const rbffd_op* op, const void* u, void* y, int dtype, cudaStream_t st);

namespace {

__global__ void iota_kernel(int32_t* a, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) a[i] = (int32_t)i;
}

// ---- rows grouped by stencil size on the device: a counting sort by size,
// stable in node order (rows of a group keep the nodes' order)
constexpr int GROUP_CHUNK = 4096;   // nodes per block of the two grouping kernels
constexpr int GROUP_THREADS = 256;

// hist[v] = nodes with stencil size v (2 <= v <= RBFFD_MAX_N); sizes outside
// that range are counted in hist[RBFFD_MAX_N + 1]
__global__ void size_histogram(const int32_t* __restrict__ np, int64_t N, unsigned long long* __restrict__ hist) {
    __shared__ unsigned int h[RBFFD_MAX_N + 2];
    for (int i = threadIdx.x; i < RBFFD_MAX_N + 2; i += blockDim.x) h[i] = 0u;
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int v = np[i];
        atomicAdd(&h[(v >= 2 && v <= RBFFD_MAX_N) ? v : RBFFD_MAX_N + 1], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < RBFFD_MAX_N + 2; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[i], (unsigned long long)h[i]);
}

struct SizeToGroup {
    int8_t g[RBFFD_MAX_N + 1];   // group of each stencil size present
};

// counts[g * nchunks + c] = nodes of chunk c (GROUP_CHUNK consecutive nodes)
// in group g
__global__ void chunk_group_counts(const int32_t* __restrict__ np, int64_t N, SizeToGroup map, int G,
                                   int64_t nchunks, int32_t* __restrict__ counts) {
    __shared__ int cnt[RBFFD_MAX_GROUPS];
    if (threadIdx.x < RBFFD_MAX_GROUPS) cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t c = blockIdx.x;
    const int64_t lo = c * GROUP_CHUNK, hi = min(N, lo + GROUP_CHUNK);
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) atomicAdd(&cnt[map.g[np[i]]], 1);
    __syncthreads();
    if (threadIdx.x < G) counts[threadIdx.x * nchunks + c] = cnt[threadIdx.x];
}

// row_node[start[g * nchunks + c] + rank] = i, rank = the number of earlier
// nodes of chunk c in group g (warp ballots, then warp totals in order)
__global__ void __launch_bounds__(GROUP_THREADS)
chunk_group_scatter(const int32_t* __restrict__ np, int64_t N, SizeToGroup map, int G, int64_t nchunks,
                    const int32_t* __restrict__ start, int32_t* __restrict__ row_node) {
    __shared__ int base[RBFFD_MAX_GROUPS];
    __shared__ int wsum[GROUP_THREADS / 32][RBFFD_MAX_GROUPS];
    const int64_t c = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x < G) base[threadIdx.x] = start[threadIdx.x * nchunks + c];
    __syncthreads();
    const int64_t lo = c * GROUP_CHUNK, hi = min(N, lo + GROUP_CHUNK);
    for (int64_t i0 = lo; i0 < hi; i0 += GROUP_THREADS) {   // uniform across the block
        const int64_t i = i0 + threadIdx.x;
        const int g = i < hi ? map.g[np[i]] : -1;
        int rank = 0;
        for (int k = 0; k < G; ++k) {
            const unsigned m = __ballot_sync(0xffffffffu, g == k);
            if (g == k) rank = __popc(m & ((1u << lane) - 1u));
            if (lane == 0) wsum[warp][k] = __popc(m);
        }
        __syncthreads();
        if (g >= 0) {
            int off = base[g] + rank;
            for (int w = 0; w < warp; ++w) off += wsum[w][g];
            row_node[off] = (int32_t)i;
        }
        __syncthreads();
        if (threadIdx.x < G) {
            int tot = 0;
            for (int w = 0; w < GROUP_THREADS / 32; ++w) tot += wsum[w][threadIdx.x];
            base[threadIdx.x] += tot;
        }
        __syncthreads();
    }
}

__global__ void init_info(double* eps, double* kappa, int32_t* evals, int32_t* status,
                          const double* eps_override, int64_t N) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    eps[i] = eps_override ? eps_override[i] : NAN;
    kappa[i] = NAN;
    evals[i] = 0;
    status[i] = RBFFD_STENCIL_OK;
}

__global__ void count_status(const int32_t* status, int64_t N, int* bad) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    int s = status[i];
    if (s != RBFFD_STENCIL_OK && s != RBFFD_STENCIL_ACCEPTED_PREDICTION) atomicAdd(bad, 1);
}

__global__ void rows_kernel(const int32_t* __restrict__ idx, const double* __restrict__ w,
                            const int32_t* __restrict__ row_node, GroupInfo gi, int nmax, int64_t R,
                            int32_t* __restrict__ out_idx, double* __restrict__ out_w) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= R) return;
    int g = group_of_row(gi, r);
    int n = gi.n[g], npad = gi.npad[g];
    int64_t lr = r - gi.row_begin[g];
    int node = row_node[r];
    for (int j = 0; j < nmax; ++j) {
        int32_t id = node;
        double wv = 0.0;
        if (j < n) {
            int64_t e = ell_elem(gi.ell_off[g], npad, lr, j);
            id = idx[e];
            wv = w[e];
        }
        if (out_idx) out_idx[(int64_t)node * nmax + j] = id;
        if (out_w) out_w[(int64_t)node * nmax + j] = wv;
    }
}

// number of stencils whose status is neither OK nor an accepted prediction
// (synchronises the stream)
cudaError_t failed_stencils(const rbffd_op* op, cudaStream_t st, int* count) {
    int* bad = nullptr;
    cudaError_t e = pool_alloc(&bad, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(int), st);
    if (e == cudaSuccess) {
        count_status<<<(unsigned)((op->N + 255) / 256), 256, 0, st>>>(op->status, op->N, bad);
        note_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(count, bad, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (bad) cudaFreeAsync(bad, st);
    return e;
}

void free_op(rbffd_op* op) {
    if (!op) return;
    cudaFree(op->row_node);
    cudaFree(op->idx);
    cudaFree(op->w64);
    cudaFree(op->w32);
    cudaFree(op->eps);
    cudaFree(op->kappa);
    cudaFree(op->evals);
    cudaFree(op->status);
    if (op->step) step_ws_free(op->step);
    delete op;
}

}  // namespace
}  // namespace rbffd

using namespace rbffd;

extern "C" {

const char* rbffd_last_error(void) { return g_err; }

const char* rbffd_status_str(rbffd_status s) {
    switch (s) {
        case RBFFD_OK: return "ok";
        case RBFFD_EINVAL: return "invalid argument";
        case RBFFD_ECUDA: return "CUDA error";
        case RBFFD_ENOMEM: return "out of device memory";
        case RBFFD_EPS_SEARCH_FAILED: return "shape-parameter search failed for some stencils";
        case RBFFD_SOLVER_NOT_CONVERGED: return "BiCGSTAB did not converge";
        case RBFFD_TIMEOUT: return "device-side wait timed out";
        case RBFFD_NOT_IMPLEMENTED: return "not implemented";
        case RBFFD_ESINGULAR: return "local interpolation matrix not positive definite";
    }
    return "unknown status";
}

void rbffd_build_opts_default(rbffd_build_opts* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->kernel = RBFFD_IMQ;
    o->kappa_target = 1e12;
    o->eps_tol = 1e-4;
    o->max_evals = 64;
    o->use_learned = 0;
    o->accept_lo = 0.5;
    o->accept_hi = 2.0;
}

rbffd_status rbffd_build_operator(const double* nodes, const double* normals, int64_t N,
                                  const int32_t* n_per_node, int n_uniform,
                                  const rbffd_build_opts* opts_in, void* stream, rbffd_op** out) {
    RBFFD_CHECK_ARG(out != nullptr, "out is NULL");
    *out = nullptr;
    (void)cudaGetLastError();   // an earlier failure elsewhere is not ours
    RBFFD_CHECK_ARG(nodes != nullptr && normals != nullptr, "nodes / normals are NULL");
    RBFFD_CHECK_ARG(N >= 2 && N < (int64_t)1 << 31, "N must be in [2, 2^31)");
    rbffd_build_opts o;
    if (opts_in) o = *opts_in; else rbffd_build_opts_default(&o);
    RBFFD_CHECK_ARG(o.kernel == RBFFD_GAUSSIAN || o.kernel == RBFFD_IMQ, "kernel");
    RBFFD_CHECK_ARG(o.eps_override || (o.kappa_target > 1.0 && std::isfinite(o.kappa_target)),
                    "kappa_target must be > 1");
    RBFFD_CHECK_ARG(o.eps_override || o.eps_tol > 0.0, "eps_tol must be > 0");
    RBFFD_CHECK_ARG(o.eps_override || o.max_evals >= 2, "max_evals must be >= 2");
    RBFFD_CHECK_ARG(!o.use_learned || (o.accept_lo > 0 && o.accept_hi >= o.accept_lo), "accept band");
    RBFFD_CHECK_ARG(o.eps_lo >= 0.0 && o.eps_hi >= 0.0 && std::isfinite(o.eps_lo) && std::isfinite(o.eps_hi),
                    "eps_lo / eps_hi must be finite and >= 0");
    RBFFD_CHECK_ARG(o.eps_lo == 0.0 || o.eps_hi == 0.0 || o.eps_lo < o.eps_hi, "eps_lo must be < eps_hi");
    RBFFD_CHECK_ARG(o.precision == RBFFD_PREC_F64 || o.precision == RBFFD_PREC_DD, "precision");
    cudaStream_t st = as_stream(stream);

    // ---- stencil-size groups (sorted by descending n; stable node order)
    std::map<int, int64_t> counts;
    if (n_per_node) {
        // histogram of the sizes on the device; only the 130 counts come back
        unsigned long long* hist_d = nullptr;
        unsigned long long hist[RBFFD_MAX_N + 2];
        RBFFD_CUDA_TRY(pool_alloc(&hist_d, sizeof(hist), st));
        RBFFD_CUDA_TRY(cudaMemsetAsync(hist_d, 0, sizeof(hist), st));
        const int64_t hb = std::min<int64_t>((N + 255) / 256, (int64_t)sm_count() * 8);
        size_histogram<<<(unsigned)hb, 256, 0, st>>>(n_per_node, N, hist_d);
        note_launch();
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(hist, hist_d, sizeof(hist), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        cudaFreeAsync(hist_d, st);
        RBFFD_CUDA_TRY(e);
        RBFFD_CHECK_ARG(hist[RBFFD_MAX_N + 1] == 0, "stencil size must be in [2, 128]");
        for (int v = 2; v <= RBFFD_MAX_N; ++v)
            if (hist[v]) counts[v] = (int64_t)hist[v];
    } else {
        counts[n_uniform] = N;
    }
    RBFFD_CHECK_ARG((int)counts.size() <= RBFFD_MAX_GROUPS, "more than 8 distinct stencil sizes");
    for (auto& kv : counts) {
        RBFFD_CHECK_ARG(kv.first >= 2 && kv.first <= RBFFD_MAX_N, "stencil size must be in [2, 128]");
        RBFFD_CHECK_ARG(kv.first <= N, "stencil size exceeds the number of nodes");
    }
    rbffd_op* op = new rbffd_op();
    memset(op, 0, sizeof(*op));
    op->N = N;
    op->kernel = o.kernel;
    op->kappa_target = o.kappa_target;
    GroupInfo& gi = op->gi;
    gi.ngroups = (int)counts.size();
    {
        int g = 0;
        int64_t row = 0, elem = 0;
        for (auto it = counts.rbegin(); it != counts.rend(); ++it, ++g) {
            gi.n[g] = it->first;
            gi.npad[g] = (it->first + 3) / 4 * 4;
            gi.row_begin[g] = row;
            gi.ell_off[g] = elem;
            row += it->second;
            elem += (it->second + ELL_SLICE - 1) / ELL_SLICE * ELL_SLICE * gi.npad[g];
            op->nnz += it->second * it->first;
            op->n_max = std::max(op->n_max, it->first);
        }
        gi.row_begin[g] = row;
        gi.ell_off[g] = elem;
        op->ell_elems = elem;
    }
    auto fail = [&](rbffd_status s) {
        free_op(op);
        return s;
    };
#define TRY_OP(expr)                                                                   \
    do {                                                                               \
        cudaError_t _e = (expr);                                                       \
        if (_e != cudaSuccess) {                                                       \
            set_error("%s: %s", #expr, cudaGetErrorString(_e));                       \
            return fail(_e == cudaErrorMemoryAllocation ? RBFFD_ENOMEM : RBFFD_ECUDA); \
        }                                                                              \
    } while (0)
    TRY_OP(cudaMalloc(&op->row_node, N * sizeof(int32_t)));
    TRY_OP(cudaMalloc(&op->idx, op->ell_elems * sizeof(int32_t)));
    TRY_OP(cudaMalloc(&op->w64, op->ell_elems * sizeof(double)));
    TRY_OP(cudaMalloc(&op->w32, op->ell_elems * sizeof(float)));
    TRY_OP(cudaMalloc(&op->eps, N * sizeof(double)));
    TRY_OP(cudaMalloc(&op->kappa, N * sizeof(double)));
    TRY_OP(cudaMalloc(&op->evals, N * sizeof(int32_t)));
    TRY_OP(cudaMalloc(&op->status, N * sizeof(int32_t)));
    TRY_OP(cudaMemsetAsync(op->idx, 0, op->ell_elems * sizeof(int32_t), st));
    TRY_OP(cudaMemsetAsync(op->w64, 0, op->ell_elems * sizeof(double), st));
    TRY_OP(cudaMemsetAsync(op->w32, 0, op->ell_elems * sizeof(float), st));
    if (n_per_node) {
        SizeToGroup map;
        memset(&map, -1, sizeof(map));
        for (int g = 0; g < gi.ngroups; ++g) map.g[gi.n[g]] = (int8_t)g;
        const int64_t nchunks = (N + GROUP_CHUNK - 1) / GROUP_CHUNK;
        const int64_t ncnt = nchunks * gi.ngroups;
        int32_t *cnt = nullptr, *start = nullptr;
        TRY_OP(pool_alloc(&cnt, ncnt * sizeof(int32_t), st));
        TRY_OP(pool_alloc(&start, ncnt * sizeof(int32_t), st));
        chunk_group_counts<<<(unsigned)nchunks, GROUP_THREADS, 0, st>>>(n_per_node, N, map, gi.ngroups, nchunks,
                                                                       cnt);
        note_launch();
        cudaError_t e = cudaGetLastError();
        rbffd_status rs = RBFFD_OK;
        if (e == cudaSuccess) rs = exclusive_scan(cnt, start, ncnt, st);
        if (e == cudaSuccess && rs == RBFFD_OK) {
            chunk_group_scatter<<<(unsigned)nchunks, GROUP_THREADS, 0, st>>>(n_per_node, N, map, gi.ngroups,
                                                                             nchunks, start, op->row_node);
            note_launch();
            e = cudaGetLastError();
        }
        cudaFreeAsync(cnt, st);
        cudaFreeAsync(start, st);
        TRY_OP(e);
        if (rs != RBFFD_OK) return fail(rs);
    } else {
        iota_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(op->row_node, N);
        note_launch();
        TRY_OP(cudaGetLastError());
    }
    init_info<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(op->eps, op->kappa, op->evals, op->status,
                                                           o.eps_override, N);
    note_launch();
    TRY_OP(cudaGetLastError());

    cudaEvent_t ev[5];
    for (int i = 0; i < 5; ++i) TRY_OP(cudaEventCreate(&ev[i]));
    struct EvGuard {
        cudaEvent_t* e;
        ~EvGuard() {
            for (int i = 0; i < 5; ++i) cudaEventDestroy(e[i]);
        }
    } evguard{ev};
    TRY_OP(cudaEventRecord(ev[0], st));
    // ---- stencils
    rbffd_status s = knn_stencils(op, nodes, normals, st);
    if (s != RBFFD_OK) return fail(s);
    TRY_OP(cudaEventRecord(ev[1], st));

    // ---- shape parameters
    rbffd_status search_status = RBFFD_OK;
    if (!o.eps_override) {
        float* guess = nullptr;
        if (o.use_learned) {
            TRY_OP(pool_alloc(&guess, N * sizeof(float), st));
            s = mlp_guess(op, nodes, normals, o, guess, st);
            if (s != RBFFD_OK) {
                cudaFreeAsync(guess, st);
                return fail(s);
            }
        }
        TRY_OP(cudaEventRecord(ev[2], st));
        s = o.precision == RBFFD_PREC_DD ? build_search_dd(op, nodes, normals, o, guess, nullptr, st)
                                         : build_search(op, nodes, normals, o, guess, st);
        TRY_OP(cudaEventRecord(ev[3], st));
        TRY_OP(cudaEventRecord(ev[4], st));   // no separate weights phase
        if (guess) cudaFreeAsync(guess, st);
        if (s != RBFFD_OK) return fail(s);
        int hb = 0;
        TRY_OP(failed_stencils(op, st, &hb));
        if (hb) {
            set_error("eps search failed for %d stencils", hb);
            search_status = RBFFD_EPS_SEARCH_FAILED;
        }
    }
    else {
        TRY_OP(cudaEventRecord(ev[2], st));
        TRY_OP(cudaEventRecord(ev[3], st));
    }
    // ---- weights (the search writes them itself from its last factorisation)
    if (o.eps_override) {
        if (o.precision == RBFFD_PREC_DD) {
            s = build_search_dd(op, nodes, normals, o, nullptr, op->eps, st);
            if (s != RBFFD_OK) return fail(s);
            int hb = 0;
            TRY_OP(failed_stencils(op, st, &hb));
            if (hb) {
                set_error("%d stencils have a local matrix that is not numerically positive definite", hb);
                s = RBFFD_ESINGULAR;
            }
        } else {
            s = build_weights(op, nodes, normals, o, op->eps, st);
        }
        if (s != RBFFD_OK && s != RBFFD_ESINGULAR) return fail(s);
        TRY_OP(cudaEventRecord(ev[4], st));
    } else {
        s = RBFFD_OK;
    }
    TRY_OP(cudaStreamSynchronize(st));
    for (int i = 0; i < 4; ++i) {
        float ms = 0.f;
        TRY_OP(cudaEventElapsedTime(&ms, ev[i], ev[i + 1]));
        op->phase_ms[i] = ms;
    }
    *out = op;
    if (search_status != RBFFD_OK) return search_status;
    return s;
#undef TRY_OP
}

rbffd_status rbffd_apply(const rbffd_op* op, const void* u, void* y, int dtype, void* stream) {
    RBFFD_CHECK_ARG(op && u && y, "NULL argument");
    RBFFD_CHECK_ARG(dtype == RBFFD_F32 || dtype == RBFFD_F64, "dtype");
    RBFFD_CHECK_ARG(u != y, "u and y alias");
    return apply_launch(op, u, y, dtype, as_stream(stream));   // counts its launch
}

rbffd_status rbffd_get_stencil_info(const rbffd_op* op, double* eps, double* kappa, int32_t* evals,
                                    int32_t* status, void* stream) {
    RBFFD_CHECK_ARG(op, "op is NULL");
    cudaStream_t st = as_stream(stream);
    if (eps) RBFFD_CUDA_TRY(cudaMemcpyAsync(eps, op->eps, op->N * 8, cudaMemcpyDeviceToDevice, st));
    if (kappa) RBFFD_CUDA_TRY(cudaMemcpyAsync(kappa, op->kappa, op->N * 8, cudaMemcpyDeviceToDevice, st));
    if (evals) RBFFD_CUDA_TRY(cudaMemcpyAsync(evals, op->evals, op->N * 4, cudaMemcpyDeviceToDevice, st));
    if (status) RBFFD_CUDA_TRY(cudaMemcpyAsync(status, op->status, op->N * 4, cudaMemcpyDeviceToDevice, st));
    return RBFFD_OK;
}

rbffd_status rbffd_get_eps(const rbffd_op* op, double* eps, double* kappa, int32_t* evals, void* stream) {
    return rbffd_get_stencil_info(op, eps, kappa, evals, nullptr, stream);
}

rbffd_status rbffd_get_ell(const rbffd_op* op, rbffd_ell_view* v) {
    RBFFD_CHECK_ARG(op && v, "NULL argument");
    memset(v, 0, sizeof(*v));
    v->ngroups = op->gi.ngroups;
    for (int g = 0; g < op->gi.ngroups; ++g) {
        v->n[g] = op->gi.n[g];
        v->npad[g] = op->gi.npad[g];
    }
    for (int g = 0; g <= op->gi.ngroups; ++g) {
        v->row_begin[g] = op->gi.row_begin[g];
        v->elem_begin[g] = op->gi.ell_off[g];
    }
    v->elems = op->ell_elems;
    v->row_node = op->row_node;
    v->idx = op->idx;
    v->w64 = op->w64;
    v->w32 = op->w32;
    return RBFFD_OK;
}

rbffd_status rbffd_get_rows(const rbffd_op* op, int32_t* idx, double* w, void* stream) {
    RBFFD_CHECK_ARG(op, "op is NULL");
    cudaStream_t st = as_stream(stream);
    rows_kernel<<<(unsigned)((op->N + 127) / 128), 128, 0, st>>>(op->idx, op->w64, op->row_node, op->gi,
                                                                 op->n_max, op->N, idx, w);
    note_launch();
    RBFFD_CUDA_TRY(cudaGetLastError());
    return RBFFD_OK;
}

rbffd_status rbffd_get_build_timings(const rbffd_op* op, double ms[4]) {
    RBFFD_CHECK_ARG(op && ms, "NULL argument");
    for (int i = 0; i < 4; ++i) ms[i] = op->phase_ms[i];
    return RBFFD_OK;
}
int64_t rbffd_launch_count(void) { return g_launches.load(); }
int64_t rbffd_op_nodes(const rbffd_op* op) { return op ? op->N : 0; }
int rbffd_op_max_n(const rbffd_op* op) { return op ? op->n_max : 0; }
int64_t rbffd_op_nnz(const rbffd_op* op) { return op ? op->nnz : 0; }
int64_t rbffd_op_apply_bytes(const rbffd_op* op, int dtype) {
    if (!op) return 0;
    int64_t ws = dtype == RBFFD_F32 ? 4 : 8;
    return op->nnz * (ws + 4) + 2 * op->N * ws;
}
void rbffd_destroy(rbffd_op* op) { free_op(op); }

}  // extern "C"

extern "C" rbffd_status rbffd_memory_pool_config(int64_t keep_bytes) {
    RBFFD_CHECK_ARG(keep_bytes >= 0, "keep_bytes must be >= 0");
    cudaMemPool_t pool = nullptr;
    RBFFD_CUDA_TRY(device_pool(&pool));
    uint64_t keep = (uint64_t)keep_bytes;
    RBFFD_CUDA_TRY(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
    return RBFFD_OK;
}

extern "C" rbffd_status rbffd_release_memory(void) {
    cudaMemPool_t pool = nullptr;
    RBFFD_CUDA_TRY(device_pool(&pool));
    RBFFD_CUDA_TRY(cudaMemPoolTrimTo(pool, 0));
    return RBFFD_OK;
}

extern "C" rbffd_status rbffd_memory_stats(int64_t* reserved, int64_t* used) {
    cudaMemPool_t pool = nullptr;
    RBFFD_CUDA_TRY(device_pool(&pool));
    uint64_t r = 0, u = 0;
    RBFFD_CUDA_TRY(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &r));
    RBFFD_CUDA_TRY(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &u));
    if (reserved) *reserved = (int64_t)r;
    if (used) *used = (int64_t)u;
    return RBFFD_OK;
}
