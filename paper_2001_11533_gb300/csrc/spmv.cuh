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
    int wmax;       // most entries one lane visits in a row (DevCsr::wmax)
    int ellw;       // SELL with one width for all slices (DevCsr::ellw), else 0
    const int *ptr; // SELL slice pointers (tpr = 1) or CSR row pointers
    const int *ci;
    const T *v;
    const short *d16; // SELL: column - row as int16 (DevCsr::sl_ci16), else null
};

template <typename T>
inline MatView<T> view(const DevCsr &a);
template <>
inline MatView<double> view<double>(const DevCsr &a)
{
    if (a.tpr <= 1) return {a.rows, a.cols, 1, a.wmax, a.ellw, a.sl_ptr, a.sl_ci, a.sl_v, a.sl_ci16};
    return {a.rows, a.cols, a.tpr, a.wmax, 0, a.rp, a.ci, a.v, nullptr};
}
template <>
inline MatView<float> view<float>(const DevCsr &a)
{
    if (a.tpr <= 1) return {a.rows, a.cols, 1, a.wmax, a.ellw, a.sl_ptr, a.sl_ci, a.sl_v32, a.sl_ci16};
    return {a.rows, a.cols, a.tpr, a.wmax, 0, a.rp, a.ci, a.v32, nullptr};
}

// A lane's entries of a row are read ROW_UNROLL at a time: all value and
// index loads of the chunk first, then all its gathers, then the sum in entry
// order (so the result does not depend on the chunking): two memory round
// trips per chunk instead of one per entry or small group of entries.
#define ROW_UNROLL 8

// column of stored entry k of `row`
template <typename T>
__device__ __forceinline__ int col_of(const MatView<T> &m, int row, int k)
{
    return m.d16 ? row + (int)m.d16[k] : m.ci[k];
}

// entry range of this lane in `row` (SELL: stride 32 inside the slice; CSR:
// stride STEP = TPR inside the row)
template <typename T, int TPR>
__device__ __forceinline__ void lane_range(const MatView<T> &m, int row, int &k, int &end)
{
    if (TPR == 1) {
        int s = row >> 5;
        if (m.ellw > 0) {
            int base = s * 32 * m.ellw;
            k = base + (row & 31);
            end = base + 32 * m.ellw;
        } else {
            k = m.ptr[s] + (row & 31);
            end = m.ptr[s + 1];
        }
    } else {
        k = m.ptr[row] + (int)(threadIdx.x & (TPR - 1));
        end = m.ptr[row + 1];
    }
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
    constexpr int STEP = TPR == 1 ? 32 : TPR;
    T acc = (T)0;
    if (row < m.rows) {
        int k, end;
        lane_range<T, TPR>(m, row, k, end);
        auto chunk = [&](int k0) {
            T vv[ROW_UNROLL];
            int cc[ROW_UNROLL];
#pragma unroll
            for (int j = 0; j < ROW_UNROLL; j++) {
                bool ok = k0 + STEP * j < end;
                vv[j] = ok ? m.v[k0 + STEP * j] : (T)0;
                cc[j] = ok ? col_of(m, row, k0 + STEP * j) : 0;
            }
            T xv[ROW_UNROLL];
#pragma unroll
            for (int j = 0; j < ROW_UNROLL; j++) xv[j] = k0 + STEP * j < end ? xf(cc[j]) : (T)0;
#pragma unroll
            for (int j = 0; j < ROW_UNROLL; j++)
                if (k0 + STEP * j < end) acc += vv[j] * xv[j];
        };
        if (m.wmax <= ROW_UNROLL) chunk(k);
        else
            for (; k < end; k += STEP * ROW_UNROLL) chunk(k);
    }
    if (TPR > 1) {
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

// sum_j a_rj z_j in double-float, not normalised; every lane of the group
// returns it
template <typename Z, int TPR>
__device__ __forceinline__ DF row_sum_df_acc(const MatView<float> &m, const float *__restrict__ lo, int row,
                                             const Z *__restrict__ z)
{
    constexpr int STEP = TPR == 1 ? 32 : TPR;
    DF acc = {0.f, 0.f};
    if (row < m.rows) {
        int k, end;
        lane_range<float, TPR>(m, row, k, end);
        auto chunk = [&](int k0) {
            float vh[ROW_UNROLL], vl[ROW_UNROLL];
            int cc[ROW_UNROLL];
#pragma unroll
            for (int j = 0; j < ROW_UNROLL; j++) {
                bool ok = k0 + STEP * j < end;
                vh[j] = ok ? m.v[k0 + STEP * j] : 0.f;
                vl[j] = ok ? lo[k0 + STEP * j] : 0.f;
                cc[j] = ok ? col_of(m, row, k0 + STEP * j) : 0;
            }
            Z zv[ROW_UNROLL];
#pragma unroll
            for (int j = 0; j < ROW_UNROLL; j++) zv[j] = k0 + STEP * j < end ? __ldg(&z[cc[j]]) : (Z)0;
#pragma unroll
            for (int j = 0; j < ROW_UNROLL; j++)
                if (k0 + STEP * j < end) df_term<Z>(acc, vh[j], vl[j], zv[j]);
        };
        if (m.wmax <= ROW_UNROLL) chunk(k);
        else
            for (; k < end; k += STEP * ROW_UNROLL) chunk(k);
    }
    if (TPR > 1) {
#pragma unroll
        for (int o = TPR / 2; o > 0; o >>= 1) {
            DF other = {__shfl_xor_sync(0xffffffffu, acc.hi, o, TPR), __shfl_xor_sync(0xffffffffu, acc.lo, o, TPR)};
            df_merge(acc, other);
        }
    }
    return acc;
}

// sum_j a_rj z_j in double-float (normalised)
template <typename Z, int TPR>
__device__ __forceinline__ DF row_sum_dfv(const MatView<float> &m, const float *__restrict__ lo, int row,
                                          const Z *__restrict__ z)
{
    DF acc = row_sum_df_acc<Z, TPR>(m, lo, row, z);
    DF r;
    quick_two_sum(acc.hi, acc.lo, r.hi, r.lo);
    return r;
}

template <typename Z, int TPR>
__device__ __forceinline__ double row_sum_df(const MatView<float> &m, const float *__restrict__ lo, int row,
                                             const Z *__restrict__ z)
{
    DF acc = row_sum_df_acc<Z, TPR>(m, lo, row, z);
    return (double)acc.hi + (double)acc.lo;
}

// ---- point-wise V-cycle arithmetic with explicit rounding, shared by the
// level-by-level kernels and the fused coarse cycle so both give the same bits
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float rsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double rsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rfma(double a, double b, double c) { return __fma_rn(a, b, c); }

// Chebyshev step at one row: d' = c_d d + c_r D^-1 (b - A x), x' = x + d'
template <typename T>
__device__ __forceinline__ void cheb_point(T br, T ax, T ir, T dr, T xr, T cdv, T crv, T &dn, T &xn)
{
    T res = rmul(rsub(br, ax), ir);
    dn = rfma(cdv, dr, rmul(crv, res));
    xn = radd(xr, dn);
}

// first step from zero: c D^-1 b
template <typename T>
__device__ __forceinline__ T cheb_first_point(T br, T ir, T c)
{
    return rmul(c, rmul(br, ir));
}

// one row of a dense FP32 inverse (rows padded to ld, 16-byte aligned) times
// b; the whole warp returns the sum
template <bool VEC>
__device__ __forceinline__ float dense_row32(const float *__restrict__ inv, int ld, int row, int n, const float *b,
                                             int lane)
{
    const float4 *r4 = reinterpret_cast<const float4 *>(inv + (int64_t)row * ld);
    int full = n >> 2;
    float a0 = 0.f, a1 = 0.f;
    for (int k = lane; k < full; k += 32) {
        float4 r = r4[k], v;
        if (VEC) v = __ldcg(reinterpret_cast<const float4 *>(b) + k);
        else v = make_float4(__ldcg(b + 4 * k), __ldcg(b + 4 * k + 1), __ldcg(b + 4 * k + 2), __ldcg(b + 4 * k + 3));
        a0 = fmaf(r.x, v.x, a0);
        a1 = fmaf(r.y, v.y, a1);
        a0 = fmaf(r.z, v.z, a0);
        a1 = fmaf(r.w, v.w, a1);
    }
    for (int k = (full << 2) + lane; k < n; k += 32) a0 = fmaf(inv[(int64_t)row * ld + k], __ldcg(b + k), a0);
    float acc = a0 + a1;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    return acc;
}

inline int rows_grid(int rows, int tpr, int tpb = 256) { return ceil_div((int64_t)rows * (tpr < 1 ? 1 : tpr), tpb); }

// launch KERNEL<T, TPR> (grid of 256-thread blocks, programmatic dependent launch) with TPR = m.tpr
#define LAUNCH_TPR(KERNEL, T, tpr, rows, stream, ...)                                                     \
    do {                                                                                                  \
        int g_ = rows_grid(rows, tpr);                                                                    \
        switch (tpr) {                                                                                    \
        case 2: pdl_launch(KERNEL<T, 2>, dim3(g_), dim3(256), 0, stream, __VA_ARGS__); break;                                 \
        case 4: pdl_launch(KERNEL<T, 4>, dim3(g_), dim3(256), 0, stream, __VA_ARGS__); break;                                 \
        case 8: pdl_launch(KERNEL<T, 8>, dim3(g_), dim3(256), 0, stream, __VA_ARGS__); break;                                 \
        case 16: pdl_launch(KERNEL<T, 16>, dim3(g_), dim3(256), 0, stream, __VA_ARGS__); break;                               \
        case 32: pdl_launch(KERNEL<T, 32>, dim3(g_), dim3(256), 0, stream, __VA_ARGS__); break;                               \
        default: pdl_launch(KERNEL<T, 1>, dim3(g_), dim3(256), 0, stream, __VA_ARGS__); break;                                \
        }                                                                                                 \
    } while (0)
