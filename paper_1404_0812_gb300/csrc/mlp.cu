// Learned shape-parameter warm start (not in the paper; it feeds the
// Section 5 search a first guess, and the search stays the arbiter).
//
// Features (float64 geometry, stored float32): tangent-frame offsets
// (t1.d, t2.d, nh.d) / r_s of every stencil node, with nh oriented so that
// sum nh.d <= 0, t1 = unit tangent part of the nearest neighbour's offset,
// t2 = nh x t1.  Network 3n -> 64 -> 64 -> 1 with GELU (erf form), float32.
//
// GPU design: one CTA of 256 threads owns a tile of 64 samples and runs the
// whole forward and backward pass in shared memory (4x4 register tiles for
// the three dense products); each CTA writes its gradient contribution to
// its own row of a partial buffer, and a second kernel sums the rows in a
// fixed order (deterministic) and applies Adam.  The products are far too
// small (64 x 64 x <=303 per tile) for tensor-core tiles to pay, and the
// network is specified in float32, so they run on the FP32 pipes.
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <random>
#include <vector>

namespace rbffd {
namespace {

constexpr int H = 64;      // hidden width
constexpr int TS = 64;     // samples per CTA tile
constexpr int NT = 256;    // threads per CTA

__host__ __device__ inline int64_t param_count(int D) {
    return (int64_t)D * H + H + H * H + H + H + 1;
}

struct View {
    const float *W1, *b1, *W2, *b2, *W3, *b3;
};
__device__ inline View view(const float* p, int D) {
    View v;
    v.W1 = p;
    v.b1 = v.W1 + (int64_t)D * H;
    v.W2 = v.b1 + H;
    v.b2 = v.W2 + H * H;
    v.W3 = v.b2 + H;
    v.b3 = v.W3 + H;
    return v;
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
    return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// ---------------------------------------------------------------------------
// features of the rows [0, count) of group g (internal row order = node order
// within the group)
// ---------------------------------------------------------------------------
__global__ void features_kernel(const double* __restrict__ X, const double* __restrict__ NR,
                                const int32_t* __restrict__ idx, const int32_t* __restrict__ row_node,
                                GroupInfo gi, int g, const double* __restrict__ eps,
                                float* __restrict__ feats, float* __restrict__ target) {
    const int64_t count = gi.row_begin[g + 1] - gi.row_begin[g];
    int64_t lr = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (lr >= count) return;
    const int n = gi.n[g], npad = gi.npad[g];
    const int64_t off = gi.ell_off[g];
    int c = idx[ell_elem(off, npad, lr, 0)];
    double cx = X[3 * (int64_t)c], cy = X[3 * (int64_t)c + 1], cz = X[3 * (int64_t)c + 2];
    double nx = NR[3 * (int64_t)c], ny = NR[3 * (int64_t)c + 1], nz = NR[3 * (int64_t)c + 2];
    double inv = rsqrt(nx * nx + ny * ny + nz * nz);
    nx *= inv; ny *= inv; nz *= inv;
    double rs2 = 0.0, sn = 0.0;
    for (int j = 1; j < n; ++j) {
        int k = idx[ell_elem(off, npad, lr, j)];
        double dx = X[3 * (int64_t)k] - cx, dy = X[3 * (int64_t)k + 1] - cy, dz = X[3 * (int64_t)k + 2] - cz;
        rs2 = fmax(rs2, dx * dx + dy * dy + dz * dz);
        sn += nx * dx + ny * dy + nz * dz;
    }
    if (sn > 0.0) { nx = -nx; ny = -ny; nz = -nz; }
    double rs = sqrt(rs2), irs = 1.0 / rs;
    int k1 = idx[ell_elem(off, npad, lr, 1)];
    double ax = X[3 * (int64_t)k1] - cx, ay = X[3 * (int64_t)k1 + 1] - cy, az = X[3 * (int64_t)k1 + 2] - cz;
    double an = nx * ax + ny * ay + nz * az;
    double t1x = ax - an * nx, t1y = ay - an * ny, t1z = az - an * nz;
    double it = rsqrt(t1x * t1x + t1y * t1y + t1z * t1z);
    t1x *= it; t1y *= it; t1z *= it;
    double t2x = ny * t1z - nz * t1y, t2y = nz * t1x - nx * t1z, t2z = nx * t1y - ny * t1x;
    // the projections in float32: each offset is formed in float64 (no
    // cancellation) and rounded once, the frame vectors carry the 1 / r_s
    // scale; the float32 features then differ from float64 projections by
    // a few float32 roundings (~1e-7 of their size), and the float64 pipe
    // (a small fraction of the float32 one here) does only the subtractions
    const float f1x = (float)(t1x * irs), f1y = (float)(t1y * irs), f1z = (float)(t1z * irs);
    const float f2x = (float)(t2x * irs), f2y = (float)(t2y * irs), f2z = (float)(t2z * irs);
    const float f3x = (float)(nx * irs), f3y = (float)(ny * irs), f3z = (float)(nz * irs);
    float* f = feats + lr * (int64_t)(3 * n);
    for (int j = 0; j < n; ++j) {
        int k = idx[ell_elem(off, npad, lr, j)];
        const float dx = (float)(X[3 * (int64_t)k] - cx), dy = (float)(X[3 * (int64_t)k + 1] - cy),
                    dz = (float)(X[3 * (int64_t)k + 2] - cz);
        f[3 * j] = fmaf(f1x, dx, fmaf(f1y, dy, f1z * dz));
        f[3 * j + 1] = fmaf(f2x, dx, fmaf(f2y, dy, f2z * dz));
        f[3 * j + 2] = fmaf(f3x, dx, fmaf(f3y, dy, f3z * dz));
    }
    if (target) target[lr] = (float)log(eps[row_node[gi.row_begin[g] + lr]] * rs);
}

// ---------------------------------------------------------------------------
// one tile: forward (mode 0: write predictions) or forward + backward
// (mode 1: per-CTA gradient partial and loss partial)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT)
mlp_tile(const float* __restrict__ params, int D, const float* __restrict__ feats,
         const float* __restrict__ target, const int32_t* __restrict__ sel, int64_t count,
         float inv_B, int mode, float* __restrict__ pred, float* __restrict__ partial,
         float* __restrict__ loss_part) {
    extern __shared__ float sm[];
    float* Xs = sm;                     // TS x D
    float* Z1 = Xs + TS * D;            // TS x H
    float* H1 = Z1 + TS * H;
    float* Z2 = H1 + TS * H;
    float* H2 = Z2 + TS * H;
    float* ys = H2 + TS * H;            // TS
    float* dys = ys + TS;               // TS
    const View P = view(params, D);
    const int t = threadIdx.x;
    const int64_t s0 = (int64_t)blockIdx.x * TS;
    const int ns = (int)((count - s0) < TS ? (count - s0) : TS);

    for (int e = t; e < TS * D; e += NT) {
        int s = e / D, d = e - s * D;
        float v = 0.f;
        if (s < ns) {
            int64_t row = sel ? sel[s0 + s] : s0 + s;
            v = feats[row * D + d];
        }
        Xs[e] = v;
    }
    __syncthreads();
    const int sa = (t >> 4) * 4;    // 4 samples
    const int ha = (t & 15) * 4;    // 4 hidden units
    {   // Z1 = X W1 + b1
        float acc[4][4];
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) acc[a][b] = P.b1[ha + b];
        for (int d = 0; d < D; ++d) {
            float4 w = __ldg(reinterpret_cast<const float4*>(P.W1 + (int64_t)d * H + ha));
            for (int a = 0; a < 4; ++a) {
                float x = Xs[(sa + a) * D + d];
                acc[a][0] = fmaf(x, w.x, acc[a][0]);
                acc[a][1] = fmaf(x, w.y, acc[a][1]);
                acc[a][2] = fmaf(x, w.z, acc[a][2]);
                acc[a][3] = fmaf(x, w.w, acc[a][3]);
            }
        }
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) {
                Z1[(sa + a) * H + ha + b] = acc[a][b];
                H1[(sa + a) * H + ha + b] = gelu(acc[a][b]);
            }
    }
    __syncthreads();
    {   // Z2 = H1 W2 + b2
        float acc[4][4];
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) acc[a][b] = P.b2[ha + b];
        for (int k = 0; k < H; ++k) {
            float4 w = __ldg(reinterpret_cast<const float4*>(P.W2 + k * H + ha));
            for (int a = 0; a < 4; ++a) {
                float x = H1[(sa + a) * H + k];
                acc[a][0] = fmaf(x, w.x, acc[a][0]);
                acc[a][1] = fmaf(x, w.y, acc[a][1]);
                acc[a][2] = fmaf(x, w.z, acc[a][2]);
                acc[a][3] = fmaf(x, w.w, acc[a][3]);
            }
        }
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) {
                Z2[(sa + a) * H + ha + b] = acc[a][b];
                H2[(sa + a) * H + ha + b] = gelu(acc[a][b]);
            }
    }
    __syncthreads();
    if (t < TS) {
        float y = P.b3[0];
        for (int h = 0; h < H; ++h) y = fmaf(H2[t * H + h], P.W3[h], y);
        ys[t] = y;
        if (mode == 0 && t < ns) pred[s0 + t] = y;
    }
    if (mode == 0) return;
    __syncthreads();
    if (t < TS) {
        float r = 0.f;
        if (t < ns) {
            int64_t row = sel ? sel[s0 + t] : s0 + t;
            r = ys[t] - target[row];
        }
        dys[t] = 2.f * r * inv_B;
        ys[t] = r * r;   // reuse for the loss
    }
    __syncthreads();
    const int64_t Pc = param_count(D);
    float* G = partial + (int64_t)blockIdx.x * Pc;
    float* gW1 = G;
    float* gb1 = gW1 + (int64_t)D * H;
    float* gW2 = gb1 + H;
    float* gb2 = gW2 + H * H;
    float* gW3 = gb2 + H;
    float* gb3 = gW3 + H;
    if (t < H) {            // dW3, loss
        float g = 0.f;
        for (int s = 0; s < TS; ++s) g = fmaf(H2[s * H + t], dys[s], g);
        gW3[t] = g;
    } else if (t == H) {
        float g = 0.f, l = 0.f;
        for (int s = 0; s < TS; ++s) {
            g += dys[s];
            l += ys[s];
        }
        gb3[0] = g;
        loss_part[blockIdx.x] = l;
    }
    __syncthreads();
    // dZ2 = dy W3^T * gelu'(Z2)  (in place in Z2)
    for (int e = t; e < TS * H; e += NT) {
        int s = e / H, h = e - s * H;
        Z2[e] = dys[s] * P.W3[h] * gelu_grad(Z2[e]);
    }
    __syncthreads();
    {   // dW2 = H1^T dZ2 ; dZ1 = (dZ2 W2^T) * gelu'(Z1) into H2
        const int ka = (t >> 4) * 4;
        float acc[4][4] = {};
        for (int s = 0; s < TS; ++s) {
            float4 dz = *reinterpret_cast<const float4*>(Z2 + s * H + ha);
            for (int a = 0; a < 4; ++a) {
                float x = H1[s * H + ka + a];
                acc[a][0] = fmaf(x, dz.x, acc[a][0]);
                acc[a][1] = fmaf(x, dz.y, acc[a][1]);
                acc[a][2] = fmaf(x, dz.z, acc[a][2]);
                acc[a][3] = fmaf(x, dz.w, acc[a][3]);
            }
        }
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) gW2[(ka + a) * H + ha + b] = acc[a][b];
        // dH1[s][k] = sum_h dZ2[s][h] W2[k][h]; thread: samples sa..+3, k = ha..+3
        float dh[4][4] = {};
        for (int h = 0; h < H; ++h) {
            float w0 = P.W2[(ha + 0) * H + h], w1 = P.W2[(ha + 1) * H + h];
            float w2 = P.W2[(ha + 2) * H + h], w3 = P.W2[(ha + 3) * H + h];
            for (int a = 0; a < 4; ++a) {
                float dz = Z2[(sa + a) * H + h];
                dh[a][0] = fmaf(dz, w0, dh[a][0]);
                dh[a][1] = fmaf(dz, w1, dh[a][1]);
                dh[a][2] = fmaf(dz, w2, dh[a][2]);
                dh[a][3] = fmaf(dz, w3, dh[a][3]);
            }
        }
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b)
                H2[(sa + a) * H + ha + b] = dh[a][b] * gelu_grad(Z1[(sa + a) * H + ha + b]);
    }
    __syncthreads();
    if (t < H) {            // db2, db1
        float g2 = 0.f, g1 = 0.f;
        for (int s = 0; s < TS; ++s) {
            g2 += Z2[s * H + t];
            g1 += H2[s * H + t];
        }
        gb2[t] = g2;
        gb1[t] = g1;
    }
    // dW1 = X^T dZ1
    for (int d = t >> 4; d < D; d += NT / 16) {
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int s = 0; s < TS; ++s) {
            float x = Xs[s * D + d];
            float4 dz = *reinterpret_cast<const float4*>(H2 + s * H + ha);
            acc[0] = fmaf(x, dz.x, acc[0]);
            acc[1] = fmaf(x, dz.y, acc[1]);
            acc[2] = fmaf(x, dz.z, acc[2]);
            acc[3] = fmaf(x, dz.w, acc[3]);
        }
        for (int b = 0; b < 4; ++b) gW1[(int64_t)d * H + ha + b] = acc[b];
    }
}

// grad[p] = sum over tiles of partial[c][p] (fixed order); optionally Adam.
__global__ void reduce_grad(const float* __restrict__ partial, int ntiles, int64_t P,
                            const float* __restrict__ loss_part, float* __restrict__ grad,
                            float* __restrict__ loss_out, float* __restrict__ params,
                            float* __restrict__ m, float* __restrict__ v, int adam_t, float lr,
                            int loss_slot) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P;
         p += (int64_t)gridDim.x * blockDim.x) {
        float g = 0.f;
        for (int c = 0; c < ntiles; ++c) g += partial[(int64_t)c * P + p];
        if (grad) grad[p] = g;
        if (params) {
            const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
            float mm = b1 * m[p] + (1.f - b1) * g;
            float vv = b2 * v[p] + (1.f - b2) * g * g;
            m[p] = mm;
            v[p] = vv;
            float mh = mm / (1.f - powf(b1, (float)adam_t));
            float vh = vv / (1.f - powf(b2, (float)adam_t));
            params[p] -= lr * mh / (sqrtf(vh) + eps);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && loss_out) {
        float l = 0.f;
        for (int c = 0; c < ntiles; ++c) l += loss_part[c];
        loss_out[loss_slot] = l;
    }
}

size_t tile_smem(int D) { return (size_t)(TS * D + 4 * TS * H + 2 * TS) * sizeof(float); }

rbffd_status ensure_smem(int D) {
    RBFFD_CUDA_TRY(cudaFuncSetAttribute(mlp_tile, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)tile_smem(D)));
    return RBFFD_OK;
}

rbffd_status ensure_train_ws(rbffd_mlp* m, int64_t tiles) {
    if (!m->adam_m) {
        RBFFD_CUDA_TRY(cudaMalloc(&m->adam_m, m->P * sizeof(float)));
        RBFFD_CUDA_TRY(cudaMalloc(&m->adam_v, m->P * sizeof(float)));
        RBFFD_CUDA_TRY(cudaMemset(m->adam_m, 0, m->P * sizeof(float)));
        RBFFD_CUDA_TRY(cudaMemset(m->adam_v, 0, m->P * sizeof(float)));
    }
    if (m->partial_rows < tiles) {
        cudaFree(m->partial);
        cudaFree(m->loss);
        m->partial = nullptr;
        RBFFD_CUDA_TRY(cudaMalloc(&m->partial, tiles * m->P * sizeof(float)));
        RBFFD_CUDA_TRY(cudaMalloc(&m->loss, (tiles + 4096) * sizeof(float)));
        m->partial_rows = tiles;
    }
    return RBFFD_OK;
}

rbffd_status predict_launch(const rbffd_mlp* m, const float* feats, int64_t count, float* out,
                            cudaStream_t st) {
    if (count <= 0) return RBFFD_OK;
    rbffd_status s = ensure_smem(m->D);
    if (s != RBFFD_OK) return s;
    unsigned tiles = (unsigned)((count + TS - 1) / TS);
    mlp_tile<<<tiles, NT, tile_smem(m->D), st>>>(m->params, m->D, feats, nullptr, nullptr, count, 0.f,
                                                 0, out, nullptr, nullptr);
    note_launch();
    RBFFD_CUDA_TRY(cudaGetLastError());
    return RBFFD_OK;
}

__global__ void scatter_guess(const float* __restrict__ pred, int64_t count, int64_t row0,
                              float* __restrict__ guess) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < count) guess[row0 + i] = pred[i];
}

__global__ void fill_nan(float* a, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) a[i] = NAN;
}

}  // namespace

rbffd_status mlp_guess(const rbffd_op* op, const double* nodes, const double* normals,
                       const rbffd_build_opts& o, float* guess_rows, cudaStream_t st) {
    fill_nan<<<(unsigned)((op->N + 255) / 256), 256, 0, st>>>(guess_rows, op->N);
    note_launch();
    RBFFD_CUDA_TRY(cudaGetLastError());
    for (int g = 0; g < op->gi.ngroups; ++g) {
        const rbffd_mlp* net = nullptr;
        for (int i = 0; i < RBFFD_MAX_GROUPS; ++i)
            if (o.mlp[i] && o.mlp[i]->n == op->gi.n[g]) net = o.mlp[i];
        if (!net) continue;
        int64_t count = op->gi.row_begin[g + 1] - op->gi.row_begin[g];
        float *feats = nullptr, *pred = nullptr;
        RBFFD_CUDA_TRY(pool_alloc(&feats, count * net->D * sizeof(float), st));
        RBFFD_CUDA_TRY(pool_alloc(&pred, count * sizeof(float), st));
        features_kernel<<<(unsigned)((count + 127) / 128), 128, 0, st>>>(
            nodes, normals, op->idx, op->row_node, op->gi, g, nullptr, feats, nullptr);
        note_launch();
        RBFFD_CUDA_TRY(cudaGetLastError());
        rbffd_status s = predict_launch(net, feats, count, pred, st);
        if (s != RBFFD_OK) return s;
        scatter_guess<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(pred, count, op->gi.row_begin[g],
                                                                       guess_rows);
        note_launch();
        RBFFD_CUDA_TRY(cudaGetLastError());
        cudaFreeAsync(feats, st);
        cudaFreeAsync(pred, st);
    }
    return RBFFD_OK;
}

}  // namespace rbffd

using namespace rbffd;

extern "C" {

int64_t rbffd_mlp_param_count(int n) { return param_count(3 * n); }

rbffd_status rbffd_mlp_create(int n, const float* params_host, rbffd_mlp** out) {
    RBFFD_CHECK_ARG(out, "out is NULL");
    *out = nullptr;
    RBFFD_CHECK_ARG(n >= 2 && n <= RBFFD_MAX_N, "n must be in [2, 128]");
    rbffd_mlp* m = new rbffd_mlp();
    memset(m, 0, sizeof(*m));
    m->n = n;
    m->D = 3 * n;
    m->P = param_count(m->D);
    cudaError_t e = cudaMalloc(&m->params, m->P * sizeof(float));
    if (e == cudaSuccess)
        e = params_host ? cudaMemcpy(m->params, params_host, m->P * sizeof(float), cudaMemcpyHostToDevice)
                        : cudaMemset(m->params, 0, m->P * sizeof(float));
    if (e != cudaSuccess) {
        set_error("rbffd_mlp_create: %s", cudaGetErrorString(e));
        cudaFree(m->params);
        delete m;
        return RBFFD_ECUDA;
    }
    *out = m;
    return RBFFD_OK;
}

rbffd_status rbffd_mlp_get_params(const rbffd_mlp* m, float* params_host) {
    RBFFD_CHECK_ARG(m && params_host, "NULL argument");
    RBFFD_CUDA_TRY(cudaMemcpy(params_host, m->params, m->P * sizeof(float), cudaMemcpyDeviceToHost));
    return RBFFD_OK;
}

rbffd_status rbffd_mlp_load(rbffd_mlp* m, const float* params_host) {
    RBFFD_CHECK_ARG(m && params_host, "NULL argument");
    RBFFD_CUDA_TRY(cudaMemcpy(m->params, params_host, m->P * sizeof(float), cudaMemcpyHostToDevice));
    // new parameters start a new optimisation: Adam's moments and step count reset
    if (m->adam_m) RBFFD_CUDA_TRY(cudaMemset(m->adam_m, 0, m->P * sizeof(float)));
    if (m->adam_v) RBFFD_CUDA_TRY(cudaMemset(m->adam_v, 0, m->P * sizeof(float)));
    m->adam_t = 0;
    return RBFFD_OK;
}

void rbffd_mlp_destroy(rbffd_mlp* m) {
    if (!m) return;
    cudaFree(m->params);
    cudaFree(m->adam_m);
    cudaFree(m->adam_v);
    cudaFree(m->partial);
    cudaFree(m->grad);
    cudaFree(m->loss);
    delete m;
}

rbffd_status rbffd_features(const rbffd_op* op, const double* nodes, const double* normals, int n,
                            float* feats, float* target, int64_t* count_host, void* stream) {
    RBFFD_CHECK_ARG(op && nodes && normals && feats, "NULL argument");
    cudaStream_t st = as_stream(stream);
    int g = -1;
    for (int i = 0; i < op->gi.ngroups; ++i)
        if (op->gi.n[i] == n) g = i;
    RBFFD_CHECK_ARG(g >= 0, "no stencil of that size in the operator");
    int64_t count = op->gi.row_begin[g + 1] - op->gi.row_begin[g];
    if (count_host) *count_host = count;
    features_kernel<<<(unsigned)((count + 127) / 128), 128, 0, st>>>(nodes, normals, op->idx, op->row_node,
                                                                     op->gi, g, op->eps, feats, target);
    note_launch();
    RBFFD_CUDA_TRY(cudaGetLastError());
    return RBFFD_OK;
}

rbffd_status rbffd_mlp_loss_grad(const rbffd_mlp* mc, const float* feats, const float* target,
                                 int64_t count, float* grad, float* loss, void* stream) {
    RBFFD_CHECK_ARG(mc && feats && target && grad && count > 0, "NULL argument");
    rbffd_mlp* m = const_cast<rbffd_mlp*>(mc);
    cudaStream_t st = as_stream(stream);
    int64_t tiles = (count + TS - 1) / TS;
    rbffd_status s = ensure_train_ws(m, tiles);
    if (s != RBFFD_OK) return s;
    s = ensure_smem(m->D);
    if (s != RBFFD_OK) return s;
    mlp_tile<<<(unsigned)tiles, NT, tile_smem(m->D), st>>>(m->params, m->D, feats, target, nullptr, count,
                                                           1.f / (float)count, 1, nullptr, m->partial,
                                                           m->loss + 4096);
    note_launch();
    RBFFD_CUDA_TRY(cudaGetLastError());
    reduce_grad<<<(unsigned)((m->P + 255) / 256), 256, 0, st>>>(m->partial, (int)tiles, m->P, m->loss + 4096,
                                                                grad, m->loss, nullptr, nullptr, nullptr, 0,
                                                                0.f, 0);
    note_launch();
    RBFFD_CUDA_TRY(cudaGetLastError());
    if (loss) {
        // mean squared error = sum of squares / count
        float hl = 0.f;
        RBFFD_CUDA_TRY(cudaMemcpyAsync(&hl, m->loss, sizeof(float), cudaMemcpyDeviceToHost, st));
        RBFFD_CUDA_TRY(cudaStreamSynchronize(st));
        hl /= (float)count;
        RBFFD_CUDA_TRY(cudaMemcpyAsync(loss, &hl, sizeof(float), cudaMemcpyHostToDevice, st));
        RBFFD_CUDA_TRY(cudaStreamSynchronize(st));
    }
    return RBFFD_OK;
}

rbffd_status rbffd_mlp_train(rbffd_mlp* m, const float* feats, const float* target, int64_t count,
                             int epochs, int batch, float lr, uint64_t seed, void* stream,
                             float* loss_host) {
    RBFFD_CHECK_ARG(m && feats && target && count > 0 && epochs > 0 && batch > 0, "bad argument");
    RBFFD_CHECK_ARG(count < (int64_t)1 << 31, "too many samples");
    cudaStream_t st = as_stream(stream);
    int64_t tiles_per_batch = (batch + TS - 1) / TS;
    rbffd_status s = ensure_train_ws(m, tiles_per_batch);
    if (s != RBFFD_OK) return s;
    s = ensure_smem(m->D);
    if (s != RBFFD_OK) return s;
    int32_t* perm_d = nullptr;
    RBFFD_CUDA_TRY(pool_alloc(&perm_d, count * sizeof(int32_t), st));
    std::vector<int32_t> perm(count);
    for (int64_t i = 0; i < count; ++i) perm[i] = (int32_t)i;
    std::mt19937_64 rng(seed);
    int64_t steps_per_epoch = (count + batch - 1) / batch;
    RBFFD_CHECK_ARG(steps_per_epoch <= 4096, "count / batch must be <= 4096");
    std::vector<float> lossv(steps_per_epoch);
    for (int ep = 0; ep < epochs; ++ep) {
        for (int64_t i = count - 1; i > 0; --i) {
            int64_t j = (int64_t)(rng() % (uint64_t)(i + 1));
            std::swap(perm[i], perm[j]);
        }
        RBFFD_CUDA_TRY(cudaMemcpyAsync(perm_d, perm.data(), count * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        for (int64_t b = 0; b < steps_per_epoch; ++b) {
            int64_t b0 = b * batch;
            int64_t nb = std::min<int64_t>(batch, count - b0);
            unsigned tiles = (unsigned)((nb + TS - 1) / TS);
            ++m->adam_t;   // the step counter lives with the network's moments
            mlp_tile<<<tiles, NT, tile_smem(m->D), st>>>(m->params, m->D, feats, target, perm_d + b0, nb,
                                                         1.f / (float)nb, 1, nullptr, m->partial,
                                                         m->loss + 4096);
            note_launch();
            reduce_grad<<<(unsigned)((m->P + 255) / 256), 256, 0, st>>>(
                m->partial, (int)tiles, m->P, m->loss + 4096, nullptr, m->loss, m->params, m->adam_m,
                m->adam_v, m->adam_t, lr, (int)b);
            note_launch();
        }
        RBFFD_CUDA_TRY(cudaGetLastError());
        RBFFD_CUDA_TRY(cudaMemcpyAsync(lossv.data(), m->loss, steps_per_epoch * sizeof(float),
                                       cudaMemcpyDeviceToHost, st));
        RBFFD_CUDA_TRY(cudaStreamSynchronize(st));
        if (loss_host) {
            double tot = 0.0;
            for (float l : lossv) tot += l;
            loss_host[ep] = (float)(tot / (double)count);
        }
    }
    cudaFreeAsync(perm_d, st);
    RBFFD_CUDA_TRY(cudaStreamSynchronize(st));
    return RBFFD_OK;
}

rbffd_status rbffd_mlp_predict(const rbffd_mlp* m, const float* feats, int64_t count, float* out,
                               void* stream) {
    RBFFD_CHECK_ARG(m && feats && out, "NULL argument");
    return predict_launch(m, feats, count, out, as_stream(stream));
}

}  // extern "C"
