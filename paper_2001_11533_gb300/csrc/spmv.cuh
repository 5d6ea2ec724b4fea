// spmv.cuh -- row access shared by every SpMV-class kernel.
//
// An operator is applied either as SELL-32 (tpr = 1: one thread per row,
// slices of 32 rows stored column-major so a warp's loads coalesce; best for
// the short rows of the fine P1 matrices) or as CSR with tpr = 2..32 lanes
// cooperating on one row (strided loads inside the row, butterfly sum inside
// the lane group; best for the long rows of the coarse Galerkin matrices and
// of S^T).  The choice is made per matrix from its mean row length.  Both
// forms sum in a fixed order, so results are reproducible run to run.
#pragma once

#include "internal.cuh"
#include "df.cuh"

template <typename T>
struct MatView {
    int rows, cols, tpr;
    const int *ptr; // SELL slice pointers (tpr = 1) or CSR row pointers
    const int *ci;
    const T *v;
};

template <typename T>
inline MatView<T> view(const DevCsr &a);
template <>
inline MatView<double> view<double>(const DevCsr &a)
{
    if (a.tpr <= 1) return {a.rows, a.cols, 1, a.sl_ptr, a.sl_ci, a.sl_v};
    return {a.rows, a.cols, a.tpr, a.rp, a.ci, a.v};
}
template <>
inline MatView<float> view<float>(const DevCsr &a)
{
    if (a.tpr <= 1) return {a.rows, a.cols, 1, a.sl_ptr, a.sl_ci, a.sl_v32};
    return {a.rows, a.cols, a.tpr, a.rp, a.ci, a.v32};
}

// row owned by this thread (tpr = 1) or lane group
template <int TPR>
__device__ __forceinline__ int my_row()
{
    return (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / TPR);
}

template <int TPR>
__device__ __forceinline__ bool row_leader()
{
    return TPR == 1 || (threadIdx.x & (TPR - 1)) == 0;
}

// sum_j a_rj * xf(j); every lane of the group returns the row's value.  All
// lanes of a warp must call this (rows past the end contribute zero).
template <typename T, int TPR, typename F>
__device__ __forceinline__ T row_sum(const MatView<T> &m, int row, F xf)
{
    T acc = (T)0;
    if (TPR == 1) {
        if (row < m.rows) {
            int s = row >> 5, lane = row & 31;
            int end = m.ptr[s + 1];
#pragma unroll 4
            for (int k = m.ptr[s] + lane; k < end; k += 32) acc += m.v[k] * xf(m.ci[k]);
        }
    } else {
        int lane = threadIdx.x & (TPR - 1);
        if (row < m.rows) {
            int end = m.ptr[row + 1];
#pragma unroll 4
            for (int k = m.ptr[row] + lane; k < end; k += TPR) acc += m.v[k] * xf(m.ci[k]);
        }
#pragma unroll
        for (int o = TPR / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, TPR);
    }
    return acc;
}

// a z added to acc, a = ahi + alo (FP32 parts of an FP64 value)
template <typename Z>
__device__ __forceinline__ void df_term(DF &acc, float ahi, float alo, Z z);
template <>
__device__ __forceinline__ void df_term<float>(DF &acc, float ahi, float alo, float z) { df_fma(acc, ahi, alo, z); }
template <>
__device__ __forceinline__ void df_term<double>(DF &acc, float ahi, float alo, double z)
{
    float zhi = (float)z;
    float zlo = (float)(z - (double)zhi);
    df_fma2(acc, ahi, alo, zhi, zlo);
}

// sum_j a_rj z_j in double-float (normalised); every lane of the group returns it
template <typename Z, int TPR>
__device__ __forceinline__ DF row_sum_dfv(const MatView<float> &m, const float *__restrict__ lo, int row,
                                          const Z *__restrict__ z)
{
    DF acc = {0.f, 0.f};
    if (TPR == 1) {
        if (row < m.rows) {
            int s = row >> 5, lane = row & 31;
            int end = m.ptr[s + 1];
#pragma unroll 4
            for (int k = m.ptr[s] + lane; k < end; k += 32) df_term<Z>(acc, m.v[k], lo[k], __ldg(&z[m.ci[k]]));
        }
    } else {
        int lane = threadIdx.x & (TPR - 1);
        if (row < m.rows) {
            int end = m.ptr[row + 1];
#pragma unroll 4
            for (int k = m.ptr[row] + lane; k < end; k += TPR) df_term<Z>(acc, m.v[k], lo[k], __ldg(&z[m.ci[k]]));
        }
#pragma unroll
        for (int o = TPR / 2; o > 0; o >>= 1) {
            DF other = {__shfl_xor_sync(0xffffffffu, acc.hi, o, TPR), __shfl_xor_sync(0xffffffffu, acc.lo, o, TPR)};
            df_merge(acc, other);
        }
    }
    DF r;
    quick_two_sum(acc.hi, acc.lo, r.hi, r.lo);
    return r;
}

template <typename Z, int TPR>
__device__ __forceinline__ double row_sum_df(const MatView<float> &m, const float *__restrict__ lo, int row,
                                             const Z *__restrict__ z)
{
    DF acc = {0.f, 0.f};
    if (TPR == 1) {
        if (row < m.rows) {
            int s = row >> 5, lane = row & 31;
            int end = m.ptr[s + 1];
#pragma unroll 4
            for (int k = m.ptr[s] + lane; k < end; k += 32) df_term<Z>(acc, m.v[k], lo[k], __ldg(&z[m.ci[k]]));
        }
    } else {
        int lane = threadIdx.x & (TPR - 1);
        if (row < m.rows) {
            int end = m.ptr[row + 1];
#pragma unroll 4
            for (int k = m.ptr[row] + lane; k < end; k += TPR) df_term<Z>(acc, m.v[k], lo[k], __ldg(&z[m.ci[k]]));
        }
#pragma unroll
        for (int o = TPR / 2; o > 0; o >>= 1) {
            DF other = {__shfl_xor_sync(0xffffffffu, acc.hi, o, TPR), __shfl_xor_sync(0xffffffffu, acc.lo, o, TPR)};
            df_merge(acc, other);
        }
    }
    return (double)acc.hi + (double)acc.lo;
}

inline int rows_grid(int rows, int tpr, int tpb = 256) { return ceil_div((int64_t)rows * (tpr < 1 ? 1 : tpr), tpb); }

// run KERNEL<T, TPR><<<grid, 256, 0, stream>>>(args...) with TPR = m.tpr
#define LAUNCH_TPR(KERNEL, T, tpr, rows, stream, ...)                                                     \
    do {                                                                                                  \
        int g_ = rows_grid(rows, tpr);                                                                    \
        switch (tpr) {                                                                                    \
        case 2: KERNEL<T, 2><<<g_, 256, 0, stream>>>(__VA_ARGS__); break;                                 \
        case 4: KERNEL<T, 4><<<g_, 256, 0, stream>>>(__VA_ARGS__); break;                                 \
        case 8: KERNEL<T, 8><<<g_, 256, 0, stream>>>(__VA_ARGS__); break;                                 \
        case 16: KERNEL<T, 16><<<g_, 256, 0, stream>>>(__VA_ARGS__); break;                               \
        case 32: KERNEL<T, 32><<<g_, 256, 0, stream>>>(__VA_ARGS__); break;                               \
        default: KERNEL<T, 1><<<g_, 256, 0, stream>>>(__VA_ARGS__); break;                                \
        }                                                                                                 \
    } while (0)
