// FP64 throughput microbenchmarks.  rbffd_fp64_peak (FMA on the FP64 pipe)
// is the denominator of the build's roofline ("alu" bound): each thread runs
// 8 independent FMA chains.  rbffd_fp64_mma_peak measures the FP64 tensor
// path (warp-level mma.sync m16n8k16 f64, 8 independent accumulators per
// warp), the only FP64 matrix instruction of this architecture, to show
// whether moving the build's small factorisations onto it could pay.
#include "common.cuh"

namespace rbffd {
namespace {

__global__ void fp64_fma_loop(double* out, int iters, double a, double b) {
    double x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = threadIdx.x * 1e-3 + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == 12345.678) out[0] = s;   // keeps the chains alive
}

// D = A B + D on 16 x 8 tiles with k = 16, eight independent accumulators
// (eight MMAs in flight per warp, 64 warps per SM: no dependency stall)
__global__ void fp64_mma_loop(double* out, int iters) {
    double a[8], b[4], c[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = 1e-3 * (threadIdx.x + i);
#pragma unroll
    for (int i = 0; i < 4; ++i) b[i] = 1e-3 * ((int)threadIdx.x - i);
#pragma unroll
    for (int q = 0; q < 8; ++q)
#pragma unroll
        for (int i = 0; i < 4; ++i) c[q][i] = 0.0;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < 8; ++q)
            asm volatile(
                "mma.sync.aligned.m16n8k16.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, "
                "{%4,%5,%6,%7,%8,%9,%10,%11}, {%12,%13,%14,%15}, {%0,%1,%2,%3};"
                : "+d"(c[q][0]), "+d"(c[q][1]), "+d"(c[q][2]), "+d"(c[q][3])
                : "d"(a[0]), "d"(a[1]), "d"(a[2]), "d"(a[3]), "d"(a[4]), "d"(a[5]), "d"(a[6]), "d"(a[7]),
                  "d"(b[0]), "d"(b[1]), "d"(b[2]), "d"(b[3]));
    }
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q)
#pragma unroll
        for (int i = 0; i < 4; ++i) s += c[q][i];
    if (s == 12345.678) out[0] = s;   // keeps the chains alive
}

}  // namespace
}  // namespace rbffd

extern "C" rbffd_status rbffd_fp64_peak(void* stream, double* gflops) {
    using namespace rbffd;
    RBFFD_CHECK_ARG(gflops, "gflops is NULL");
    cudaStream_t st = as_stream(stream);
    double* out = nullptr;
    RBFFD_CUDA_TRY(pool_alloc(&out, sizeof(double), st));
    const int threads = 256, blocks = sm_count() * 8, iters = 4096;
    cudaEvent_t e0, e1;
    RBFFD_CUDA_TRY(cudaEventCreate(&e0));
    RBFFD_CUDA_TRY(cudaEventCreate(&e1));
    fp64_fma_loop<<<blocks, threads, 0, st>>>(out, 64, 0.999999, 1e-7);   // warm-up
    float best = 1e30f;
    note_launch();
    for (int rep = 0; rep < 3; ++rep) {
        RBFFD_CUDA_TRY(cudaEventRecord(e0, st));
        fp64_fma_loop<<<blocks, threads, 0, st>>>(out, iters, 0.999999, 1e-7);
        note_launch();
        RBFFD_CUDA_TRY(cudaEventRecord(e1, st));
        RBFFD_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.f;
        RBFFD_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        best = ms < best ? ms : best;
    }
    RBFFD_CUDA_TRY(cudaGetLastError());
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(out, st);
    double flops = 2.0 * 8.0 * (double)iters * threads * (double)blocks;
    *gflops = flops / (best * 1e-3) / 1e9;
    return RBFFD_OK;
}

extern "C" rbffd_status rbffd_fp64_mma_peak(void* stream, double* gflops) {
    using namespace rbffd;
    RBFFD_CHECK_ARG(gflops, "gflops is NULL");
    cudaStream_t st = as_stream(stream);
    double* out = nullptr;
    RBFFD_CUDA_TRY(pool_alloc(&out, sizeof(double), st));
    const int threads = 256, blocks = sm_count() * 8, iters = 1024;
    cudaEvent_t e0, e1;
    RBFFD_CUDA_TRY(cudaEventCreate(&e0));
    RBFFD_CUDA_TRY(cudaEventCreate(&e1));
    fp64_mma_loop<<<blocks, threads, 0, st>>>(out, 16);   // warm-up
    note_launch();
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
        RBFFD_CUDA_TRY(cudaEventRecord(e0, st));
        fp64_mma_loop<<<blocks, threads, 0, st>>>(out, iters);
        note_launch();
        RBFFD_CUDA_TRY(cudaEventRecord(e1, st));
        RBFFD_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.f;
        RBFFD_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        best = ms < best ? ms : best;
    }
    RBFFD_CUDA_TRY(cudaGetLastError());
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(out, st);
    // 2 * 16 * 8 * 16 flops per warp-level mma, 8 per iteration per warp
    const double warps = (double)blocks * threads / 32.0;
    double flops = 2.0 * 16.0 * 8.0 * 16.0 * 8.0 * (double)iters * warps;
    *gflops = flops / (best * 1e-3) / 1e9;
    return RBFFD_OK;
}
