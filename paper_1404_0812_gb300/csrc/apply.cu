// y = L_X u (Eq. kernel_mol, explicit part; Section 4.2: O(N) per apply).
//
// One thread per operator row over the sliced ELL layout: each lane reads
// its row's entries four at a time (one 16-byte load of indices, one or two
// 16-byte loads of weights), the 32 lanes of a warp cover one contiguous
// span, and the gathers of u go through the read-only path (u is small
// enough to stay in L2).  The result is scattered to the row's node.
#include "common.cuh"

namespace rbffd {
namespace {

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
    __device__ static inline void load(const float* p, float (&w)[4]) {
        float4 v = *reinterpret_cast<const float4*>(p);
        w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
    }
};
template <>
struct Vec4<double> {
    __device__ static inline void load(const double* p, double (&w)[4]) {
        double2 a = *reinterpret_cast<const double2*>(p);
        double2 b = *reinterpret_cast<const double2*>(p + 2);
        w[0] = a.x; w[1] = a.y; w[2] = b.x; w[3] = b.y;
    }
};

template <typename T>
__global__ void __launch_bounds__(256)
apply_kernel(const int32_t* __restrict__ idx, const T* __restrict__ w,
             const int32_t* __restrict__ row_node, GroupInfo gi, const T* __restrict__ u,
             T* __restrict__ y, int64_t R) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= R) return;
    int g = group_of_row(gi, r);
    const int npad = gi.npad[g];
    const int64_t lr = r - gi.row_begin[g];
    const int64_t base = ell_elem(gi.ell_off[g], npad, lr, 0);
    T acc = T(0);
    for (int jb = 0; jb < npad; jb += 4) {
        const int64_t e = base + (int64_t)(jb >> 2) * 128;
        int4 iv = __ldg(reinterpret_cast<const int4*>(idx + e));
        T wv[4];
        Vec4<T>::load(w + e, wv);
        acc = fma(wv[0], __ldg(u + iv.x), acc);
        acc = fma(wv[1], __ldg(u + iv.y), acc);
        acc = fma(wv[2], __ldg(u + iv.z), acc);
        acc = fma(wv[3], __ldg(u + iv.w), acc);
    }
    y[row_node[r]] = acc;
}

}  // namespace

rbffd_status apply_launch(const rbffd_op* op, const void* u, void* y, int dtype, cudaStream_t st) {
    const int64_t R = op->N;
    unsigned blocks = (unsigned)((R + 255) / 256);
    if (dtype == RBFFD_F32)
        apply_kernel<float><<<blocks, 256, 0, st>>>(op->idx, op->w32, op->row_node, op->gi,
                                                     (const float*)u, (float*)y, R);
    else
        apply_kernel<double><<<blocks, 256, 0, st>>>(op->idx, op->w64, op->row_node, op->gi,
                                                      (const double*)u, (double*)y, R);
    note_launch();
    RBFFD_CUDA_TRY(cudaGetLastError());
    return RBFFD_OK;
}

}  // namespace rbffd
