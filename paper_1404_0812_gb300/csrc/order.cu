// Locality orderings of the nodes.  Section 4.1 reorders L_X by reverse
// Cuthill-McKee (George and Liu) for faster iterative solves; a Morton
// (Z-order) key of the coordinates is the geometric alternative, available
// before any stencil exists.  Both return a permutation perm with perm[k] =
// the original index of the node placed k-th; the caller applies it to its
// node, normal and field arrays (x_new[k] = x[perm[k]]) and builds on the
// reordered set.  The sorts and the breadth-first search run on the host:
// they are one-off, O(N log N) / O(nnz) steps ahead of the build.
#include "common.cuh"

#include <algorithm>
#include <cstring>
#include <numeric>
#include <thread>
#include <vector>

namespace rbffd {
namespace {

__global__ void bbox_blocks(const double* __restrict__ X, int64_t N, double* __restrict__ out) {
    __shared__ double lo[3][128], hi[3][128];
    double l[3] = {INFINITY, INFINITY, INFINITY}, h[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        for (int a = 0; a < 3; ++a) {
            double v = X[3 * i + a];
            l[a] = fmin(l[a], v);
            h[a] = fmax(h[a], v);
        }
    for (int a = 0; a < 3; ++a) {
        lo[a][threadIdx.x] = l[a];
        hi[a][threadIdx.x] = h[a];
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double a0 = INFINITY, a1 = -INFINITY;
        for (int t = 0; t < (int)blockDim.x; ++t) {
            a0 = fmin(a0, lo[threadIdx.x][t]);
            a1 = fmax(a1, hi[threadIdx.x][t]);
        }
        out[6 * blockIdx.x + threadIdx.x] = a0;
        out[6 * blockIdx.x + 3 + threadIdx.x] = a1;
    }
}

// spread the low 21 bits of v to every third bit
__device__ __forceinline__ uint64_t spread3(uint64_t v) {
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x1f00000000ffffull;
    v = (v | (v << 16)) & 0x1f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

__global__ void morton_keys(const double* __restrict__ X, int64_t N, double x0, double y0, double z0,
                            double scale, uint64_t* __restrict__ key) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double c[3] = {X[3 * i] - x0, X[3 * i + 1] - y0, X[3 * i + 2] - z0};
    uint64_t q[3];
    for (int a = 0; a < 3; ++a) {
        double t = c[a] * scale;   // in [0, 2^21 - 1]
        q[a] = (uint64_t)fmin(fmax(t, 0.0), 2097151.0);
    }
    key[i] = spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2);
}

__global__ void stencil_rows(const int32_t* __restrict__ idx, const int32_t* __restrict__ row_node, GroupInfo gi,
                             int64_t R, int nmax, int32_t* __restrict__ out, int32_t* __restrict__ deg) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= R) return;
    int g = group_of_row(gi, r);
    int n = gi.n[g], npad = gi.npad[g];
    int64_t lr = r - gi.row_begin[g];
    int node = row_node[r];
    for (int j = 0; j < nmax; ++j)
        out[(int64_t)node * nmax + j] = j < n ? idx[ell_elem(gi.ell_off[g], npad, lr, j)] : -1;
    deg[node] = n;
}

}  // namespace
}  // namespace rbffd

using namespace rbffd;

extern "C" rbffd_status rbffd_morton_order(const double* nodes, int64_t N, int32_t* perm, void* stream) {
    RBFFD_CHECK_ARG(nodes && perm, "NULL argument");
    RBFFD_CHECK_ARG(N >= 1 && N < (int64_t)1 << 31, "N must be in [1, 2^31)");
    cudaStream_t st = as_stream(stream);
    const int nb = (int)std::min<int64_t>(1024, (N + 127) / 128);
    double* part = nullptr;
    uint64_t* key = nullptr;
    RBFFD_CUDA_TRY(pool_alloc(&part, (size_t)nb * 6 * sizeof(double), st));
    bbox_blocks<<<nb, 128, 0, st>>>(nodes, N, part);
    note_launch();
    RBFFD_CUDA_TRY(cudaGetLastError());
    std::vector<double> hp((size_t)nb * 6);
    RBFFD_CUDA_TRY(cudaMemcpyAsync(hp.data(), part, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    RBFFD_CUDA_TRY(cudaStreamSynchronize(st));
    cudaFreeAsync(part, st);
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int b = 0; b < nb; ++b)
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(lo[a], hp[6 * b + a]);
            hi[a] = std::max(hi[a], hp[6 * b + 3 + a]);
        }
    double ext = std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
    RBFFD_CHECK_ARG(std::isfinite(ext), "non-finite node coordinates");
    const double scale = ext > 0.0 ? 2097151.0 / ext : 0.0;   // one cube: the Z-order keeps proportions
    RBFFD_CUDA_TRY(pool_alloc(&key, (size_t)N * sizeof(uint64_t), st));
    morton_keys<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(nodes, N, lo[0], lo[1], lo[2], scale, key);
    note_launch();
    RBFFD_CUDA_TRY(cudaGetLastError());
    std::vector<uint64_t> hk((size_t)N);
    RBFFD_CUDA_TRY(cudaMemcpyAsync(hk.data(), key, (size_t)N * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    RBFFD_CUDA_TRY(cudaStreamSynchronize(st));
    cudaFreeAsync(key, st);
    std::vector<int32_t> p((size_t)N);
    std::iota(p.begin(), p.end(), 0);
    std::sort(p.begin(), p.end(), [&](int32_t a, int32_t b) { return hk[a] < hk[b] || (hk[a] == hk[b] && a < b); });
    RBFFD_CUDA_TRY(cudaMemcpyAsync(perm, p.data(), (size_t)N * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    RBFFD_CUDA_TRY(cudaStreamSynchronize(st));
    return RBFFD_OK;
}

extern "C" rbffd_status rbffd_rcm_order_host(const int64_t* rowptr, const int32_t* cols, int64_t N, int32_t* perm) {
    RBFFD_CHECK_ARG(rowptr && perm && (cols || N == 0), "NULL argument");
    RBFFD_CHECK_ARG(N >= 0 && N < (int64_t)1 << 31, "N must be in [0, 2^31)");
    for (int64_t i = 0; i < N; ++i)
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e)
            RBFFD_CHECK_ARG(cols[e] >= 0 && cols[e] < N, "column index out of range");
    // passes over disjoint ranges of nodes, on the host's cores
    auto for_nodes = [&](auto&& body) {
        const int64_t nt = std::max<int64_t>(1, std::min<int64_t>(std::thread::hardware_concurrency(), N / 4096));
        std::vector<std::thread> pool;
        for (int64_t t = 1; t < nt; ++t) pool.emplace_back([&, t] { body(N * t / nt, N * (t + 1) / nt); });
        body(0, N / nt);
        for (auto& th : pool) th.join();
    };
    // symmetrised adjacency in one flat array: node i's slots are
    // nb[off[i] .. off[i + 1]) (its out- and in-edges, self loops dropped);
    // after the repeats are removed its neighbours are the first deg[i].
    // Each thread scans every edge and fills only the slots of its own
    // nodes, so no two threads write the same place.
    std::vector<int64_t> off((size_t)N + 1, 0);
    for_nodes([&](int64_t lo, int64_t hi) {
        for (int64_t i = 0; i < N; ++i)
            for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
                const int64_t j = cols[e];
                if (j == i) continue;
                if (i >= lo && i < hi) off[(size_t)i + 1]++;
                if (j >= lo && j < hi) off[(size_t)j + 1]++;
            }
    });
    for (int64_t i = 0; i < N; ++i) off[(size_t)i + 1] += off[(size_t)i];
    std::vector<int32_t> nb((size_t)off[(size_t)N]);
    for_nodes([&](int64_t lo, int64_t hi) {
        std::vector<int64_t> fill(off.begin() + lo, off.begin() + hi);
        for (int64_t i = 0; i < N; ++i)
            for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
                const int64_t j = cols[e];
                if (j == i) continue;
                if (i >= lo && i < hi) nb[(size_t)fill[(size_t)(i - lo)]++] = (int32_t)j;
                if (j >= lo && j < hi) nb[(size_t)fill[(size_t)(j - lo)]++] = (int32_t)i;
            }
    });
    std::vector<int32_t> deg((size_t)N);
    for_nodes([&](int64_t lo, int64_t hi) {
        for (int64_t i = lo; i < hi; ++i) {
            int32_t* a = nb.data() + off[(size_t)i];
            int32_t* b = nb.data() + off[(size_t)i + 1];
            std::sort(a, b);
            deg[(size_t)i] = (int32_t)(std::unique(a, b) - a);
        }
    });
    // neighbours in increasing degree (ties by index), the Cuthill-McKee
    // visiting order: sorted as 64-bit keys (degree, index)
    for_nodes([&](int64_t lo, int64_t hi) {
        std::vector<uint64_t> key;
        for (int64_t i = lo; i < hi; ++i) {
            int32_t* a = nb.data() + off[(size_t)i];
            const int32_t d = deg[(size_t)i];
            key.resize((size_t)d);
            for (int32_t k = 0; k < d; ++k) key[(size_t)k] = ((uint64_t)(uint32_t)deg[(size_t)a[k]] << 32) | (uint32_t)a[k];
            std::sort(key.begin(), key.end());
            for (int32_t k = 0; k < d; ++k) a[k] = (int32_t)(key[(size_t)k] & 0xffffffffu);
        }
    });
    auto adj_begin = [&](int32_t v) { return nb.data() + off[(size_t)v]; };
    auto adj_end = [&](int32_t v) { return nb.data() + off[(size_t)v] + deg[(size_t)v]; };
    std::vector<int32_t> level((size_t)N, -1), order;
    order.reserve((size_t)N);
    std::vector<char> done((size_t)N, 0);
    std::vector<int32_t> queue;
    queue.reserve((size_t)N);
    // BFS from s over the unvisited component: levels and the last level.
    // Level-synchronous: each frontier (comp[fb, fe), all at level depth) is
    // expanded by the host's threads, a node joining the next frontier through
    // an atomic claim of its level.  Levels, depth and the component's node
    // set are those of a sequential BFS; only the order of comp differs, and
    // nothing below depends on it (every choice is by (degree, index)).
    const int64_t hw = std::max<int64_t>(1, (int64_t)std::thread::hardware_concurrency());
    auto bfs_levels = [&](int32_t s, std::vector<int32_t>& comp, int& depth) {
        comp.clear();
        comp.push_back(s);
        level[s] = 0;
        depth = 0;
        size_t fb = 0, fe = 1;
        std::vector<std::vector<int32_t>> part;
        while (fb < fe) {
            const int32_t next = depth + 1;
            const int64_t F = (int64_t)(fe - fb);
            const int64_t nt = std::max<int64_t>(1, std::min<int64_t>(hw, F / 512));
            part.assign((size_t)nt, {});
            auto expand = [&](int64_t t) {
                std::vector<int32_t>& out = part[(size_t)t];
                for (size_t h = fb + (size_t)(F * t / nt); h < fb + (size_t)(F * (t + 1) / nt); ++h) {
                    const int32_t v = comp[h];
                    for (const int32_t* pw = adj_begin(v); pw != adj_end(v); ++pw) {
                        int32_t* lw = &level[(size_t)*pw];
                        int32_t expect = -1;
                        if (__atomic_load_n(lw, __ATOMIC_RELAXED) < 0 &&
                            __atomic_compare_exchange_n(lw, &expect, next, false, __ATOMIC_RELAXED, __ATOMIC_RELAXED))
                            out.push_back(*pw);
                    }
                }
            };
            std::vector<std::thread> pool;
            for (int64_t t = 1; t < nt; ++t) pool.emplace_back(expand, t);
            expand(0);
            for (auto& th : pool) th.join();
            fb = fe;
            for (const auto& p : part) comp.insert(comp.end(), p.begin(), p.end());
            fe = comp.size();
            if (fe > fb) depth = next;
        }
    };
    std::vector<int32_t> comp;
    for (int64_t seed = 0; seed < N; ++seed) {
        if (done[(size_t)seed]) continue;
        // pseudo-peripheral start (George-Liu): from a minimum-degree node of
        // the component, move to a minimum-degree node of the deepest BFS
        // level while the eccentricity grows
        int depth;
        bfs_levels((int32_t)seed, comp, depth);
        int32_t start = (int32_t)seed;
        for (int32_t v : comp)
            if (deg[v] < deg[start] || (deg[v] == deg[start] && v < start)) start = v;
        for (int32_t v : comp) level[v] = -1;
        int d0 = -1;
        for (int it = 0; it < 8; ++it) {
            bfs_levels(start, comp, depth);
            int32_t best = -1;
            for (int32_t v : comp)
                if (level[v] == depth && (best < 0 || deg[v] < deg[best] || (deg[v] == deg[best] && v < best))) best = v;
            for (int32_t v : comp) level[v] = -1;
            if (depth <= d0) break;
            d0 = depth;
            if (best == start) break;
            start = best;
        }
        // Cuthill-McKee BFS from the start
        queue.clear();
        queue.push_back(start);
        done[(size_t)start] = 1;
        for (size_t h = 0; h < queue.size(); ++h) {
            int32_t v = queue[h];
            order.push_back(v);
            for (const int32_t* pw = adj_begin(v); pw != adj_end(v); ++pw)
                if (!done[(size_t)*pw]) {
                    done[(size_t)*pw] = 1;
                    queue.push_back(*pw);
                }
        }
    }
    // reversed
    for (int64_t k = 0; k < N; ++k) perm[k] = order[(size_t)(N - 1 - k)];
    return RBFFD_OK;
}

extern "C" rbffd_status rbffd_rcm_order(const rbffd_op* op, int32_t* perm, void* stream) {
    RBFFD_CHECK_ARG(op && perm, "NULL argument");
    cudaStream_t st = as_stream(stream);
    const int64_t N = op->N;
    const int nmax = op->n_max;
    int32_t *rows = nullptr, *deg = nullptr;
    RBFFD_CUDA_TRY(pool_alloc(&rows, (size_t)N * nmax * sizeof(int32_t), st));
    RBFFD_CUDA_TRY(pool_alloc(&deg, (size_t)N * sizeof(int32_t), st));
    stencil_rows<<<(unsigned)((N + 127) / 128), 128, 0, st>>>(op->idx, op->row_node, op->gi, N, nmax, rows, deg);
    note_launch();
    RBFFD_CUDA_TRY(cudaGetLastError());
    std::vector<int32_t> hr((size_t)N * nmax), hd((size_t)N);
    RBFFD_CUDA_TRY(cudaMemcpyAsync(hr.data(), rows, hr.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    RBFFD_CUDA_TRY(cudaMemcpyAsync(hd.data(), deg, hd.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    RBFFD_CUDA_TRY(cudaStreamSynchronize(st));
    cudaFreeAsync(rows, st);
    cudaFreeAsync(deg, st);
    // CSR of the stencil graph: node k -> its n_k - 1 neighbours
    std::vector<int64_t> rp((size_t)N + 1, 0);
    for (int64_t k = 0; k < N; ++k) rp[(size_t)k + 1] = rp[(size_t)k] + std::max(0, hd[(size_t)k] - 1);
    std::vector<int32_t> cols((size_t)rp[(size_t)N]);
    for (int64_t k = 0; k < N; ++k)
        for (int j = 1; j < hd[(size_t)k]; ++j) cols[(size_t)(rp[(size_t)k] + j - 1)] = hr[(size_t)k * nmax + j];
    std::vector<int32_t> hp((size_t)N);
    rbffd_status s = rbffd_rcm_order_host(rp.data(), cols.data(), N, hp.data());
    if (s != RBFFD_OK) return s;
    RBFFD_CUDA_TRY(cudaMemcpyAsync(perm, hp.data(), (size_t)N * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    RBFFD_CUDA_TRY(cudaStreamSynchronize(st));
    return RBFFD_OK;
}
