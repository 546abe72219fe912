// Launch-shape autotuner for the operator build (threads per block and
// resident blocks per SM of the lane-per-stencil search and weights
// kernels).  It builds the operator on a strided subsample of the caller's
// nodes (every k-th node: the same surface, the same stencil sizes, coarser
// spacing) with each candidate shape, times the search and weights phases
// with CUDA events, and keeps the fastest.  Results can be cached in a text
// file, one line per (device, stencil sizes, kernel, kappa_T) key.
#include "common.cuh"

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

namespace rbffd {
namespace {

__global__ void gather_stride(const double* __restrict__ X, const double* __restrict__ NR,
                              const int32_t* __restrict__ np, int64_t stride, int64_t m,
                              double* __restrict__ Xo, double* __restrict__ No, int32_t* __restrict__ npo) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m) return;
    int64_t k = i * stride;
    for (int a = 0; a < 3; ++a) {
        Xo[3 * i + a] = X[3 * k + a];
        No[3 * i + a] = NR[3 * k + a];
    }
    if (np) npo[i] = np[k];
}

std::string tune_key(const std::vector<int>& sizes, int kernel, double kT) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp p;
    cudaGetDeviceProperties(&p, dev);
    char buf[512];
    std::string s = std::string(p.name) + "|sm" + std::to_string(p.multiProcessorCount) + "|n";
    for (int n : sizes) s += std::to_string(n) + ",";
    snprintf(buf, sizeof(buf), "|k%d|kT%.3g", kernel, kT);
    s += buf;
    for (auto& c : s)
        if (c == ' ') c = '_';
    return s;
}

bool cache_lookup(const char* path, const std::string& key, int* t, int* b) {
    if (!path) return false;
    FILE* f = fopen(path, "r");
    if (!f) return false;
    char line[1024];
    bool found = false;
    while (fgets(line, sizeof(line), f)) {
        char k[900];
        int tt, bb;
        if (sscanf(line, "%899s %d %d", k, &tt, &bb) == 3 && key == k) {
            *t = tt;
            *b = bb;
            found = true;
        }
    }
    fclose(f);
    return found;
}

void cache_store(const char* path, const std::string& key, int t, int b, double ms) {
    if (!path) return;
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d %d %.4f\n", key.c_str(), t, b, ms);
    fclose(f);
}

}  // namespace
}  // namespace rbffd

using namespace rbffd;

extern "C" rbffd_status rbffd_autotune_build(const double* nodes, const double* normals, int64_t N,
                                             const int32_t* n_per_node, int n_uniform,
                                             const rbffd_build_opts* opts_in, int64_t sample,
                                             const char* cache_path, void* stream, int* block_threads,
                                             int* blocks_per_sm, double* best_ms) {
    RBFFD_CHECK_ARG(nodes && normals && block_threads && blocks_per_sm, "NULL argument");
    RBFFD_CHECK_ARG(N >= 2 && sample >= 2, "N and sample must be >= 2");
    rbffd_build_opts o;
    if (opts_in) o = *opts_in; else rbffd_build_opts_default(&o);
    cudaStream_t st = as_stream(stream);
    // stencil sizes present (for the cache key)
    std::vector<int> sizes;
    if (n_per_node) {
        std::vector<int32_t> hn(N);
        RBFFD_CUDA_TRY(cudaMemcpyAsync(hn.data(), n_per_node, N * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        RBFFD_CUDA_TRY(cudaStreamSynchronize(st));
        std::vector<char> seen(RBFFD_MAX_N + 1, 0);
        for (int32_t v : hn) {
            RBFFD_CHECK_ARG(v >= 2 && v <= RBFFD_MAX_N, "stencil size must be in [2, 128]");
            seen[v] = 1;
        }
        for (int v = 2; v <= RBFFD_MAX_N; ++v)
            if (seen[v]) sizes.push_back(v);
    } else {
        sizes.push_back(n_uniform);
    }
    std::string key = tune_key(sizes, o.kernel, o.kappa_target);
    int ct, cb;
    if (cache_lookup(cache_path, key, &ct, &cb)) {
        *block_threads = ct;
        *blocks_per_sm = cb;
        if (best_ms) *best_ms = -1.0;
        return RBFFD_OK;
    }
    // every candidate must see several stencils per lane, or the timing
    // measures the tail of the persistent loop instead of its throughput
    const int cand_t[] = {128, 64, 128, 64};
    const int cand_b[] = {4, 8, 3, 6};
    const int ncand = 4;
    int64_t max_lanes = 0;
    for (int c = 0; c < ncand; ++c) max_lanes = std::max<int64_t>(max_lanes, (int64_t)cand_t[c] * cand_b[c] * sm_count());
    sample = std::min<int64_t>(N, std::max<int64_t>(sample, 8 * max_lanes));
    int64_t stride = std::max<int64_t>(1, N / sample);
    int64_t m = (N + stride - 1) / stride;
    double *Xs = nullptr, *Ns = nullptr;
    int32_t* Ps = nullptr;
    RBFFD_CUDA_TRY(cudaMalloc(&Xs, m * 3 * sizeof(double)));
    RBFFD_CUDA_TRY(cudaMalloc(&Ns, m * 3 * sizeof(double)));
    if (n_per_node) RBFFD_CUDA_TRY(cudaMalloc(&Ps, m * sizeof(int32_t)));
    gather_stride<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(nodes, normals, n_per_node, stride, m, Xs, Ns, Ps);
    note_launch();
    RBFFD_CUDA_TRY(cudaGetLastError());
    double best = 1e300;
    int bt = 128, bb = 2;
    rbffd_status result = RBFFD_OK;
    for (int c = 0; c < ncand; ++c) {
        const int t = cand_t[c], b = cand_b[c];
        {
            rbffd_build_opts oc = o;
            oc.eps_override = nullptr;
            oc.block_threads = t;
            oc.blocks_per_sm = b;
            double tot = 0.0;
            for (int rep = 0; rep < 2; ++rep) {   // first repetition warms up
                rbffd_op* op = nullptr;
                rbffd_status s = rbffd_build_operator(Xs, Ns, m, Ps, n_uniform, &oc, stream, &op);
                if (s != RBFFD_OK && s != RBFFD_EPS_SEARCH_FAILED && s != RBFFD_ESINGULAR) {
                    if (op) rbffd_destroy(op);
                    if (s == RBFFD_ENOMEM) {   // shape too large for this device: skip it
                        tot = 1e300;
                        break;
                    }
                    result = s;
                    break;
                }
                double ms[4];
                rbffd_get_build_timings(op, ms);
                if (rep == 1) tot = ms[2] + ms[3];
                rbffd_destroy(op);
            }
            if (result != RBFFD_OK) break;
            if (tot < best) {
                best = tot;
                bt = t;
                bb = b;
            }
        }
        if (result != RBFFD_OK) break;
    }
    cudaFree(Xs);
    cudaFree(Ns);
    cudaFree(Ps);
    if (result != RBFFD_OK) return result;
    *block_threads = bt;
    *blocks_per_sm = bb;
    if (best_ms) *best_ms = best;
    cache_store(cache_path, key, bt, bb, best);
    return RBFFD_OK;
}
