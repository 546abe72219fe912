// Stencil selection (Section 4: a node and its n-1 nearest neighbours by
// Euclidean distance in R^3; Section 4.1 uses a k-d tree for speed).
//
// GPU design: a uniform grid of cubic cells replaces the k-d tree.  Nodes
// are counting-sorted by cell (histogram, exclusive scan, scatter); one
// thread per query then scans Chebyshev rings of cells around its own cell,
// keeping the n-1 best (d^2, index) keys in an insertion-sorted list, and
// stops once every unvisited cell is provably farther than the current
// (n-1)-th key.  d^2 = (dx*dx + dy*dy) + dz*dz is evaluated with explicit
// round-to-nearest operations and no fused multiply-add, so the key (and
// therefore every tie-break by index) is bit-reproducible.
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace rbffd {
namespace {

constexpr int BB_THREADS = 256;

__global__ void bbox_partial(const double* __restrict__ X, const double* __restrict__ NR, int64_t N,
                             double* __restrict__ part, int* __restrict__ bad) {
    __shared__ double s[6][BB_THREADS];
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        double nn = 0.0;
        for (int a = 0; a < 3; ++a) {
            double v = X[3 * i + a];
            double nv = NR[3 * i + a];
            if (!isfinite(v) || !isfinite(nv)) atomicExch(bad, 1);
            nn += nv * nv;
            lo[a] = fmin(lo[a], v);
            hi[a] = fmax(hi[a], v);
        }
        if (!(nn > 0.0)) atomicExch(bad, 1);
    }
    for (int a = 0; a < 3; ++a) {
        s[a][threadIdx.x] = lo[a];
        s[3 + a][threadIdx.x] = hi[a];
    }
    __syncthreads();
    for (int w = BB_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            for (int a = 0; a < 3; ++a) {
                s[a][threadIdx.x] = fmin(s[a][threadIdx.x], s[a][threadIdx.x + w]);
                s[3 + a][threadIdx.x] = fmax(s[3 + a][threadIdx.x], s[3 + a][threadIdx.x + w]);
            }
        }
        __syncthreads();
    }
    if (threadIdx.x < 6) part[blockIdx.x * 6 + threadIdx.x] = s[threadIdx.x][0];
}

// one block: each thread folds a strided subset of the per-block partials,
// then a shared-memory tree (min and max are exact: any order gives the
// same box)
__global__ void __launch_bounds__(BB_THREADS) bbox_final(const double* __restrict__ part, int nb,
                                                        double* __restrict__ out) {
    __shared__ double s[6][BB_THREADS];
    double v[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
    for (int b = threadIdx.x; b < nb; b += BB_THREADS)
        for (int a = 0; a < 3; ++a) {
            v[a] = fmin(v[a], part[b * 6 + a]);
            v[3 + a] = fmax(v[3 + a], part[b * 6 + 3 + a]);
        }
    for (int a = 0; a < 6; ++a) s[a][threadIdx.x] = v[a];
    __syncthreads();
    for (int w = BB_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int a = 0; a < 3; ++a) {
                s[a][threadIdx.x] = fmin(s[a][threadIdx.x], s[a][threadIdx.x + w]);
                s[3 + a][threadIdx.x] = fmax(s[3 + a][threadIdx.x], s[3 + a][threadIdx.x + w]);
            }
        __syncthreads();
    }
    if (threadIdx.x < 6) out[threadIdx.x] = s[threadIdx.x][0];
}

struct Grid {
    double lo[3];
    double h, inv_h;
    int G[3];
    double delta;   // bound on the float32 error of one coordinate difference
};

__device__ inline int cell_coord(double x, double lo, double inv_h, int G) {
    int c = (int)floor((x - lo) * inv_h);
    return c < 0 ? 0 : (c >= G ? G - 1 : c);
}

__global__ void cell_of_nodes(const double* __restrict__ X, int64_t N, Grid g,
                              int32_t* __restrict__ cell, int32_t* __restrict__ count) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    int cx = cell_coord(X[3 * i], g.lo[0], g.inv_h, g.G[0]);
    int cy = cell_coord(X[3 * i + 1], g.lo[1], g.inv_h, g.G[1]);
    int cz = cell_coord(X[3 * i + 2], g.lo[2], g.inv_h, g.G[2]);
    int c = (cz * g.G[1] + cy) * g.G[0] + cx;
    cell[i] = c;
    atomicAdd(&count[c], 1);
}

// -- exclusive scan of int32 counts (three-phase, recursive over block sums)
constexpr int SCAN_T = 1024;

__global__ void scan_block(const int32_t* __restrict__ in, int32_t* __restrict__ out, int64_t n,
                           int32_t* __restrict__ block_sum) {
    __shared__ int32_t s[SCAN_T];
    int64_t i = blockIdx.x * (int64_t)SCAN_T + threadIdx.x;
    int32_t v = i < n ? in[i] : 0;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < SCAN_T; off <<= 1) {
        int32_t t = threadIdx.x >= off ? s[threadIdx.x - off] : 0;
        __syncthreads();
        s[threadIdx.x] += t;
        __syncthreads();
    }
    if (i < n) out[i] = s[threadIdx.x] - v;   // exclusive
    if (threadIdx.x == SCAN_T - 1) block_sum[blockIdx.x] = s[SCAN_T - 1];
}

__global__ void scan_add(int32_t* __restrict__ out, int64_t n, const int32_t* __restrict__ block_off) {
    int64_t i = blockIdx.x * (int64_t)SCAN_T + threadIdx.x;
    if (i < n) out[i] += block_off[blockIdx.x];
}


__global__ void scatter_nodes(const double* __restrict__ X, int64_t N,
                              const int32_t* __restrict__ cell, const int32_t* __restrict__ start,
                              int32_t* __restrict__ cursor, int32_t* __restrict__ sidx,
                              double* __restrict__ sx, float4* __restrict__ sxf) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    int c = cell[i];
    int p = start[c] + atomicAdd(&cursor[c], 1);
    sidx[p] = (int32_t)i;
    sx[3 * (int64_t)p] = X[3 * i];
    sx[3 * (int64_t)p + 1] = X[3 * i + 1];
    sx[3 * (int64_t)p + 2] = X[3 * i + 2];
    sxf[p] = make_float4((float)X[3 * i], (float)X[3 * i + 1], (float)X[3 * i + 2], 0.f);
}

__global__ void invert_rows(const int32_t* __restrict__ row_node, int64_t N, int32_t* __restrict__ node_row) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r < N) node_row[row_node[r]] = (int32_t)r;
}

// Bit-reproducible squared distance: no contraction into FMA.
__device__ __forceinline__ double sq_dist(double ax, double ay, double az, double bx, double by,
                                          double bz) {
    double dx = __dsub_rn(bx, ax), dy = __dsub_rn(by, ay), dz = __dsub_rn(bz, az);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// (d^2, index) order.  d^2 >= +0 is never NaN, so its IEEE bit pattern read
// as a signed 64-bit integer orders exactly as the double does; comparing the
// integers keeps the insertion sort off the (slow) float64 pipe.
__device__ __forceinline__ bool key_less(long long ka, int ia, long long kb, int ib) {
    return ka < kb || (ka == kb && ia < ib);
}

// Shell sort of (key, index) pairs by key_less (gaps 23, 10, 4, 1): the
// (unique) pairs end in the same order as incremental insertion would give.
__device__ void sort_keys(long long* k, int* v, int n) {
    const int gaps[4] = {23, 10, 4, 1};
    for (int gi = 0; gi < 4; ++gi) {
        const int gap = gaps[gi];
        for (int i = gap; i < n; ++i) {
            const long long tk = k[i];
            const int tv = v[i];
            int j = i;
            while (j >= gap && key_less(tk, tv, k[j - gap], v[j - gap])) {
                k[j] = k[j - gap];
                v[j] = v[j - gap];
                j -= gap;
            }
            k[j] = tk;
            v[j] = tv;
        }
    }
}

// One thread per query, queries taken in cell-sorted order so that the 32
// queries of a warp share nearby cells.
__global__ void __launch_bounds__(128)
knn_query(const double* __restrict__ X, const int32_t* __restrict__ node_row, int64_t nrows_total,
          GroupInfo gi, Grid g, const int32_t* __restrict__ start,
          const int32_t* __restrict__ sidx, const double* __restrict__ sx, const float4* __restrict__ sxf,
          int32_t* __restrict__ ell_idx, int* __restrict__ err) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nrows_total) return;
    const int q = sidx[t];
    const int64_t r = node_row[q];
    int grp = group_of_row(gi, r);
    int n = gi.n[grp];
    int K = n - 1;
    int64_t lr = r - gi.row_begin[grp];
    double qx = X[3 * (int64_t)q], qy = X[3 * (int64_t)q + 1], qz = X[3 * (int64_t)q + 2];
    const float qxf = (float)qx, qyf = (float)qy, qzf = (float)qz;
    float kth_f = INFINITY;   // float32 bound on the current (n-1)-th key
    int c0[3] = {cell_coord(qx, g.lo[0], g.inv_h, g.G[0]), cell_coord(qy, g.lo[1], g.inv_h, g.G[1]),
                 cell_coord(qz, g.lo[2], g.inv_h, g.G[2])};
    double qc[3] = {qx, qy, qz};

    long long bk[RBFFD_MAX_N];   // d^2 bit patterns of the current list
    int bi[RBFFD_MAX_N];
    int cnt = 0;
    int smax = max(g.G[0], max(g.G[1], g.G[2]));
    for (int s = 0; s <= smax; ++s) {
        int lo3[3], hi3[3];
        for (int a = 0; a < 3; ++a) {
            lo3[a] = c0[a] - s;
            hi3[a] = c0[a] + s;
        }
        for (int cz = max(lo3[2], 0); cz <= min(hi3[2], g.G[2] - 1); ++cz) {
            for (int cy = max(lo3[1], 0); cy <= min(hi3[1], g.G[1] - 1); ++cy) {
                bool yz_shell = (cz == lo3[2] || cz == hi3[2] || cy == lo3[1] || cy == hi3[1]);
                int step = yz_shell ? 1 : (hi3[0] - lo3[0]);
                for (int cx = lo3[0]; cx <= hi3[0]; cx += (step > 0 ? step : 1)) {
                    if (cx < 0 || cx >= g.G[0]) continue;
                    int c = (cz * g.G[1] + cy) * g.G[0] + cx;
                    int p0 = start[c], p1 = start[c + 1];
                    for (int p = p0; p < p1; ++p) {
                        // float32 screen.  With every coordinate difference off by
                        // at most delta in float32, |d2_f32 - d2| <= 2 sqrt(3) delta |d|
                        // + 3 delta^2 + 2e-7 d2, so a candidate whose float32 d2
                        // exceeds the bound below cannot enter the exact top list
                        float4 c = __ldg(sxf + p);
                        float fx = c.x - qxf, fy = c.y - qyf, fz = c.z - qzf;
                        float d2f = fx * fx + fy * fy + fz * fz;
                        if (d2f > kth_f) continue;   // certainly beyond the current list
                        int j = sidx[p];
                        if (j == q) continue;
                        double d2 = sq_dist(qx, qy, qz, sx[3 * (int64_t)p], sx[3 * (int64_t)p + 1],
                                            sx[3 * (int64_t)p + 2]);
                        const long long kd = __double_as_longlong(d2);
                        if (cnt < K) {
                            // the first K candidates arrive in no useful order:
                            // gather them unsorted and sort once when the list fills
                            bk[cnt] = kd;
                            bi[cnt] = j;
                            if (++cnt == K) {
                                sort_keys(bk, bi, K);
                                double kth = __longlong_as_double(bk[K - 1]);
                                kth_f = (float)(kth * (1.0 + 1e-6) + 4.0 * g.delta * sqrt(kth) +
                                                4.0 * g.delta * g.delta) * (1.0f + 1e-6f);
                            }
                            continue;
                        }
                        if (!key_less(kd, j, bk[K - 1], bi[K - 1])) continue;
                        // later candidates come from outer shells and land near the end
                        int i = K - 1;
                        while (i > 0 && key_less(kd, j, bk[i - 1], bi[i - 1])) {
                            bk[i] = bk[i - 1];
                            bi[i] = bi[i - 1];
                            --i;
                        }
                        bk[i] = kd;
                        bi[i] = j;
                        if (cnt == K) {
                            double kth = __longlong_as_double(bk[K - 1]);
                            kth_f = (float)(kth * (1.0 + 1e-6) + 4.0 * g.delta * sqrt(kth) +
                                            4.0 * g.delta * g.delta) * (1.0f + 1e-6f);
                        }
                    }
                }
            }
        }
        // distance from q to the outside of the visited cube (sides clipped by
        // the grid have no nodes beyond them)
        bool all = true;
        double bound = INFINITY;
        for (int a = 0; a < 3; ++a) {
            if (lo3[a] > 0) {
                all = false;
                bound = fmin(bound, qc[a] - (g.lo[a] + lo3[a] * g.h));
            }
            if (hi3[a] < g.G[a] - 1) {
                all = false;
                bound = fmin(bound, (g.lo[a] + (hi3[a] + 1) * g.h) - qc[a]);
            }
        }
        if (all) break;
        if (cnt == K) {
            double b = bound * (1.0 - 1e-12);
            if (b > 0.0 && __longlong_as_double(bk[K - 1]) < b * b) break;
        }
    }
    if (cnt < K) {
        atomicExch(err, 1);
        return;
    }
    int npad = gi.npad[grp];
    int64_t off = gi.ell_off[grp];
    ell_idx[ell_elem(off, npad, lr, 0)] = q;
    for (int j = 0; j < K; ++j) ell_idx[ell_elem(off, npad, lr, j + 1)] = bi[j];
    for (int j = n; j < npad; ++j) ell_idx[ell_elem(off, npad, lr, j)] = q;
}

}  // namespace

// Exclusive prefix sum of n int32 counts on the device (three-phase,
// recursive over block sums); temporaries from the library's pool.
rbffd_status exclusive_scan(const int32_t* in, int32_t* out, int64_t n, cudaStream_t st) {
    int64_t nb = (n + SCAN_T - 1) / SCAN_T;
    int32_t *bs = nullptr, *bo = nullptr;
    RBFFD_CUDA_TRY(pool_alloc(&bs, nb * sizeof(int32_t), st));
    RBFFD_CUDA_TRY(pool_alloc(&bo, nb * sizeof(int32_t), st));
    scan_block<<<(unsigned)nb, SCAN_T, 0, st>>>(in, out, n, bs);
    note_launch();
    RBFFD_CUDA_TRY(cudaGetLastError());
    if (nb > 1) {
        rbffd_status r = exclusive_scan(bs, bo, nb, st);
        if (r != RBFFD_OK) return r;
        scan_add<<<(unsigned)nb, SCAN_T, 0, st>>>(out, n, bo);
        note_launch();
        RBFFD_CUDA_TRY(cudaGetLastError());
    }
    RBFFD_CUDA_TRY(cudaFreeAsync(bs, st));
    RBFFD_CUDA_TRY(cudaFreeAsync(bo, st));
    return RBFFD_OK;
}

rbffd_status knn_stencils(rbffd_op* op, const double* nodes, const double* normals,
                          cudaStream_t st) {
    const int64_t N = op->N;
    // bounding box (and a finiteness check of nodes and normals)
    int nb = (int)std::min<int64_t>(1024, (N + BB_THREADS - 1) / BB_THREADS);
    double* part = nullptr;
    double* bb_d = nullptr;
    RBFFD_CUDA_TRY(pool_alloc(&part, (size_t)nb * 6 * sizeof(double), st));
    RBFFD_CUDA_TRY(pool_alloc(&bb_d, 7 * sizeof(double), st));
    RBFFD_CUDA_TRY(cudaMemsetAsync(bb_d + 6, 0, sizeof(int), st));
    bbox_partial<<<nb, BB_THREADS, 0, st>>>(nodes, normals, N, part, reinterpret_cast<int*>(bb_d + 6));
    note_launch();
    bbox_final<<<1, BB_THREADS, 0, st>>>(part, nb, bb_d);
    note_launch();
    RBFFD_CUDA_TRY(cudaGetLastError());
    double bb[7];
    RBFFD_CUDA_TRY(cudaMemcpyAsync(bb, bb_d, sizeof(bb), cudaMemcpyDeviceToHost, st));
    RBFFD_CUDA_TRY(cudaStreamSynchronize(st));
    RBFFD_CUDA_TRY(cudaFreeAsync(part, st));
    RBFFD_CUDA_TRY(cudaFreeAsync(bb_d, st));
    int bad = 0;
    memcpy(&bad, &bb[6], sizeof(int));
    if (bad) {
        set_error("node coordinates or normals are not finite, or a normal is zero");
        return RBFFD_EINVAL;
    }

    // cell size: nodes sample a surface, so about N h^2 / D^2 nodes share a
    // cell of side h on a surface of extent D; aim for ~4 per occupied cell.
    // Small cells keep the candidate lists short and the shells' stopping
    // radius close to the k-th distance; the empty cells they add are cheap
    // to skip.  1M-node sphere, stencils of 31 / 101 / both mixed: 6.8 / 33.7
    // / 19.0 ms at ~4 per cell against 9.7 / 48.1 / 27.7 ms at ~16 (the
    // result does not depend on the cell size).
    Grid g;
    double ext[3], diag2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        ext[a] = bb[3 + a] - bb[a];
        diag2 += ext[a] * ext[a];
    }
    double D = std::sqrt(diag2);
    double h = D > 0 ? D * std::sqrt(4.0 / (double)N) : 1.0;
    int64_t total = 1;
    for (;;) {
        total = 1;
        for (int a = 0; a < 3; ++a) {
            int64_t Ga = (int64_t)std::floor(ext[a] / h) + 1;
            g.G[a] = (int)std::min<int64_t>(Ga, 1024);
            total *= g.G[a];
        }
        if (total <= (int64_t)1 << 27 && g.G[0] < 1024 && g.G[1] < 1024 && g.G[2] < 1024) break;
        h *= 1.25;
    }
    for (int a = 0; a < 3; ++a) g.lo[a] = bb[a];
    g.h = h;
    g.inv_h = 1.0 / h;
    // float32 rounding of two coordinates of magnitude <= M and of their
    // difference: at most 2^-24 (2 M + |dx|) <= 2^-23 * 1.5 M; doubled margin
    double M = 0.0;
    for (int a = 0; a < 6; ++a) M = std::max(M, std::fabs(bb[a]));
    g.delta = 4.0 * 1.5 * M * std::ldexp(1.0, -24);

    int32_t *cell = nullptr, *count = nullptr, *start = nullptr, *cursor = nullptr, *sidx = nullptr;
    double* sx = nullptr;
    float4* sxf = nullptr;
    int32_t* node_row = nullptr;
    int* err = nullptr;
    RBFFD_CUDA_TRY(pool_alloc(&cell, N * sizeof(int32_t), st));
    RBFFD_CUDA_TRY(pool_alloc(&count, (total + 1) * sizeof(int32_t), st));
    RBFFD_CUDA_TRY(pool_alloc(&start, (total + 1) * sizeof(int32_t), st));
    RBFFD_CUDA_TRY(pool_alloc(&cursor, total * sizeof(int32_t), st));
    RBFFD_CUDA_TRY(pool_alloc(&sidx, N * sizeof(int32_t), st));
    RBFFD_CUDA_TRY(pool_alloc(&sx, N * 3 * sizeof(double), st));
    RBFFD_CUDA_TRY(pool_alloc(&sxf, N * sizeof(float4), st));
    RBFFD_CUDA_TRY(pool_alloc(&node_row, N * sizeof(int32_t), st));
    RBFFD_CUDA_TRY(pool_alloc(&err, sizeof(int), st));
    RBFFD_CUDA_TRY(cudaMemsetAsync(count, 0, (total + 1) * sizeof(int32_t), st));
    RBFFD_CUDA_TRY(cudaMemsetAsync(cursor, 0, total * sizeof(int32_t), st));
    RBFFD_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
    unsigned nbN = (unsigned)((N + 255) / 256);
    cell_of_nodes<<<nbN, 256, 0, st>>>(nodes, N, g, cell, count);
    note_launch();
    RBFFD_CUDA_TRY(cudaGetLastError());
    rbffd_status rs = exclusive_scan(count, start, total + 1, st);
    if (rs != RBFFD_OK) return rs;
    scatter_nodes<<<nbN, 256, 0, st>>>(nodes, N, cell, start, cursor, sidx, sx, sxf);
    note_launch();
    invert_rows<<<nbN, 256, 0, st>>>(op->row_node, N, node_row);
    note_launch();
    RBFFD_CUDA_TRY(cudaGetLastError());
    knn_query<<<(unsigned)((N + 127) / 128), 128, 0, st>>>(nodes, node_row, N, op->gi, g, start,
                                                            sidx, sx, sxf, op->idx, err);
    note_launch();
    RBFFD_CUDA_TRY(cudaGetLastError());
    int herr = 0;
    RBFFD_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    RBFFD_CUDA_TRY(cudaStreamSynchronize(st));
    cudaFreeAsync(cell, st);
    cudaFreeAsync(count, st);
    cudaFreeAsync(start, st);
    cudaFreeAsync(cursor, st);
    cudaFreeAsync(sidx, st);
    cudaFreeAsync(sx, st);
    cudaFreeAsync(sxf, st);
    cudaFreeAsync(node_row, st);
    cudaFreeAsync(err, st);
    if (herr) {
        set_error("stencil search found fewer than n-1 neighbours");
        return RBFFD_EINVAL;
    }
    return RBFFD_OK;
}

}  // namespace rbffd
