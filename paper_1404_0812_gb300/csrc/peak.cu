// FP64 FMA throughput microbenchmark: the denominator of the build's
// roofline ("alu" bound).  Each thread runs 8 independent FMA chains.
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
