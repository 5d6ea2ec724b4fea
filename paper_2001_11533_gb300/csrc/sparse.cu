// sparse.cu -- SELL-32 sparse kernels of the hot path: SpMV, the Chebyshev /
// l1-Jacobi smoother step fused with its residual, the V-cycle residual,
// prolongation-add, and the dense coarsest-level GEMV.
//
// Layout (SELL-C-sigma with C = 32, sigma = 1; Kreutzer et al., SIAM J. Sci.
// Comput. 36, 2014): rows are cut into slices of 32 consecutive rows; a slice
// of width w stores w columns of 32 entries each, entry (row, k) at
// sl_ptr[slice] + 32*k + lane.  One thread owns one row, so a warp reads 32
// consecutive values and 32 consecutive column indices per step (coalesced),
// and gathers x through the read-only cache.  Entries keep the CSR order, so
// padding (value 0, column = the row's last column) only adds exact zeros.
#include <mutex>

#include "internal.cuh"
#include "spmv.cuh"
#include "bulk.cuh"
#include "util.cuh"

// ------------------------------------------------------------------ conversion
__global__ void k_slice_width(int rows, const int *__restrict__ rp, int nslices, int *__restrict__ wcnt)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nslices) return;
    int w = 0;
    for (int l = 0; l < 32; l++) {
        int r = s * 32 + l;
        if (r < rows) w = max(w, rp[r + 1] - rp[r]);
    }
    wcnt[s] = 32 * w;
}

__global__ void k_sell_fill(int rows, const int *__restrict__ rp, const int *__restrict__ ci,
                            const double *__restrict__ v, const int *__restrict__ slp,
                            int *__restrict__ sci, double *__restrict__ sv, float *__restrict__ sv32,
                            int nslices)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nslices * 32) return;
    int s = r >> 5, lane = r & 31;
    int base = slp[s], w = (slp[s + 1] - base) >> 5;
    int beg = 0, len = 0;
    if (r < rows) {
        beg = rp[r];
        len = rp[r + 1] - beg;
    }
    int padc = len > 0 ? ci[beg + len - 1] : 0;
    for (int k = 0; k < w; k++) {
        int idx = base + 32 * k + lane;
        if (k < len) {
            sci[idx] = ci[beg + k];
            sv[idx] = v[beg + k];
            sv32[idx] = (float)v[beg + k];
        } else {
            sci[idx] = padc;
            sv[idx] = 0.0;
            sv32[idx] = 0.0f;
        }
    }
}

__global__ void k_fill_int(int n, int v, int *__restrict__ x)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = v;
}

// column - row of every stored entry of a uniform-width SELL matrix as int16;
// *bad set if some entry of a real row does not fit (padding rows store 0)
__global__ void k_sell_delta(int rows, int nslices, int w, const int *__restrict__ sci, short *__restrict__ d16,
                             int *__restrict__ bad)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nslices * 32) return;
    int64_t base = (int64_t)(r >> 5) * 32 * w + (r & 31);
    for (int j = 0; j < w; j++) {
        int64_t k = base + 32 * j;
        int d = r < rows ? sci[k] - r : 0;
        if (d < -32768 || d > 32767) {
            atomicOr(bad, 1);
            d = 0;
        }
        d16[k] = (short)d;
    }
}

int csr_to_sell(Arena &ar, DevCsr &a, int /*want32*/, cudaStream_t s)
{
    a.nslices = ceil_div(a.rows, 32);
    int ns = a.nslices;
    TRY(ar.alloc(&a.sl_ptr, ns + 1));
    Scratch sc;
    int *w = nullptr;
    TRY(sc.alloc(&w, ns + 1));
    if (ns > 0) {
        k_slice_width<<<ceil_div(ns, 256), 256, 0, s>>>(a.rows, a.rp, ns, w);
        LAUNCH_CHECK();
    }
    int total = 0;
    TRY(exclusive_scan<int>(w, a.sl_ptr, ns, s, &total));
    // one width for all slices when that pads by at most 5 %: the kernels
    // then compute where a slice starts instead of loading it
    a.ellw = 0;
    int widest = a.wmax < (1 << 30) ? a.wmax : 0;
    if (ns > 0 && widest > 0 && (int64_t)32 * widest * ns <= (int64_t)total + total / 20 &&
        (int64_t)32 * widest * ns < (1ll << 31)) {
        k_fill_int<<<ceil_div(ns, 256), 256, 0, s>>>(ns, 32 * widest, w);
        LAUNCH_CHECK();
        TRY(exclusive_scan<int>(w, a.sl_ptr, ns, s, &total));
        a.ellw = widest;
    }
    a.sell_nnz = total;
    a.sl_ci16 = nullptr;
    TRY(ar.alloc(&a.sl_ci, total));
    TRY(ar.alloc(&a.sl_v, total));
    TRY(ar.alloc(&a.sl_v32, total));
    if (ns > 0) {
        k_sell_fill<<<ceil_div(ns * 32, 256), 256, 0, s>>>(a.rows, a.rp, a.ci, a.v, a.sl_ptr, a.sl_ci,
                                                          a.sl_v, a.sl_v32, ns);
        LAUNCH_CHECK();
    }
    // int16 column offsets for uniform-width SELL when every entry fits
    if (a.ellw > 0 && ns > 0) {
        int *bad = nullptr;
        short *d16 = nullptr;
        TRY(sc.alloc(&bad, 1));
        TRY(ar.alloc(&d16, total));
        CU(cudaMemsetAsync(bad, 0, sizeof(int), s));
        k_sell_delta<<<ceil_div(ns * 32, 256), 256, 0, s>>>(a.rows, ns, a.ellw, a.sl_ci, d16, bad);
        LAUNCH_CHECK();
        int hb = 0;
        CU(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        if (!hb) a.sl_ci16 = d16;
    }
    CU(cudaStreamSynchronize(s));
    return AMGH_OK;
}

// ------------------------------------------------------------------ transpose
// t = a^T with ascending columns: count entries per column, scan, scatter
// every entry to its column's segment through an atomic cursor, then sort
// each row of t by column.  The atomics only decide a temporary order; after
// the per-row sort the result is the same on every run.
__global__ void k_col_count(int nnz, const int *__restrict__ ci, int *__restrict__ cnt)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nnz) atomicAdd(&cnt[ci[k]], 1);
}

__global__ void k_transpose_fill(int rows, const int *__restrict__ rp, const int *__restrict__ ci,
                                 const double *__restrict__ v, const int *__restrict__ trp,
                                 int *__restrict__ cursor, int *__restrict__ tci, double *__restrict__ tv)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows) return;
    for (int k = rp[i]; k < rp[i + 1]; k++) {
        int c = ci[k];
        int pos = trp[c] + atomicAdd(&cursor[c], 1);
        tci[pos] = i;
        tv[pos] = v[k];
    }
}

// Sort every row of (ci, v) by column: rows of at most 32 entries (or more
// than SORT_WARP_MAX) by one thread with insertion sort, the others by one
// warp with a bitonic network in shared memory.  Columns within a row are
// distinct, so the result does not depend on the order of equal keys.
#define SORT_WARP_MAX 1024
#define SORT_WARPS 4
__global__ void k_sort_rows_warp(int rows, const int *__restrict__ rp, int *__restrict__ ci, double *__restrict__ v)
{
    __shared__ int ks[SORT_WARPS][SORT_WARP_MAX];
    __shared__ double vs[SORT_WARPS][SORT_WARP_MAX];
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int r = blockIdx.x * SORT_WARPS + w;
    if (r >= rows) return; // warp-uniform
    int b = rp[r], L = rp[r + 1] - b;
    if (L <= 32 || L > SORT_WARP_MAX) return;
    int P = 64;
    while (P < L) P <<= 1;
    int *key = ks[w];
    double *val = vs[w];
    for (int q = lane; q < P; q += 32) {
        key[q] = q < L ? ci[b + q] : 0x7fffffff;
        val[q] = q < L ? v[b + q] : 0.0;
    }
    __syncwarp();
    for (int kk = 2; kk <= P; kk <<= 1)
        for (int jj = kk >> 1; jj > 0; jj >>= 1) {
            for (int a = lane; a < P; a += 32) {
                int c = a ^ jj;
                if (c > a) {
                    bool up = (a & kk) == 0;
                    int ka = key[a], kc = key[c];
                    if ((ka > kc) == up) {
                        key[a] = kc;
                        key[c] = ka;
                        double t = val[a];
                        val[a] = val[c];
                        val[c] = t;
                    }
                }
            }
            __syncwarp();
        }
    for (int q = lane; q < L; q += 32) {
        ci[b + q] = key[q];
        v[b + q] = val[q];
    }
}

__global__ void k_sort_rows(int rows, const int *__restrict__ rp, int *__restrict__ ci, double *__restrict__ v)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    int b = rp[r], e = rp[r + 1];
    if (e - b > 32 && e - b <= SORT_WARP_MAX) return; // the warp kernel's rows
    for (int k = b + 1; k < e; k++) {
        int c = ci[k];
        double x = v[k];
        int j = k - 1;
        while (j >= b && ci[j] > c) {
            ci[j + 1] = ci[j];
            v[j + 1] = v[j];
            j--;
        }
        ci[j + 1] = c;
        v[j + 1] = x;
    }
}

int csr_transpose(Arena &ar, const DevCsr &a, DevCsr &t, cudaStream_t s)
{
    t.rows = a.cols;
    t.cols = a.rows;
    t.nnz = a.nnz;
    Scratch sc;
    int *cnt = nullptr, *cur = nullptr;
    TRY(sc.alloc(&cnt, t.rows + 1));
    TRY(sc.alloc(&cur, t.rows + 1));
    CU(cudaMemsetAsync(cnt, 0, sizeof(int) * (t.rows + 1), s));
    CU(cudaMemsetAsync(cur, 0, sizeof(int) * (t.rows + 1), s));
    if (a.nnz > 0) {
        k_col_count<<<ceil_div(a.nnz, 256), 256, 0, s>>>(a.nnz, a.ci, cnt);
        LAUNCH_CHECK();
    }
    TRY(ar.alloc(&t.rp, t.rows + 1));
    TRY(exclusive_scan<int>(cnt, t.rp, t.rows, s, nullptr));
    TRY(ar.alloc(&t.ci, t.nnz));
    TRY(ar.alloc(&t.v, t.nnz));
    if (a.rows > 0) {
        k_transpose_fill<<<ceil_div(a.rows, 256), 256, 0, s>>>(a.rows, a.rp, a.ci, a.v, t.rp, cur, t.ci, t.v);
        LAUNCH_CHECK();
    }
    if (t.rows > 0) {
        k_sort_rows<<<ceil_div(t.rows, 128), 128, 0, s>>>(t.rows, t.rp, t.ci, t.v);
        LAUNCH_CHECK();
        k_sort_rows_warp<<<ceil_div(t.rows, SORT_WARPS), 32 * SORT_WARPS, 0, s>>>(t.rows, t.rp, t.ci, t.v);
        LAUNCH_CHECK();
    }
    CU(cudaStreamSynchronize(s));
    return AMGH_OK;
}

// ------------------------------------------------------------------ operator layout
__global__ void k_to_f32(int64_t n, const double *__restrict__ a, float *__restrict__ b)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

int to_f32(amgh_problem *p, const double *a, int64_t n, float *b)
{
    if (n <= 0) return AMGH_OK;
    k_to_f32<<<ceil_div(n, 256), 256, 0, p->stream>>>(n, a, b);
    LAUNCH_CHECK();
    return AMGH_OK;
}

__global__ void k_row_max(int rows, const int *__restrict__ rp, int *__restrict__ out)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    int len = r < rows ? rp[r + 1] - rp[r] : 0;
    for (int o = 16; o > 0; o >>= 1) len = max(len, __shfl_xor_sync(0xffffffffu, len, o));
    if ((threadIdx.x & 31) == 0 && len > 0) atomicMax(out, len);
}

// longest row of a (host value; setup only)
static int max_row_length(const DevCsr &a, cudaStream_t s, int *out)
{
    *out = 0;
    if (a.rows == 0) return AMGH_OK;
    Scratch sc;
    int *d = nullptr;
    TRY(sc.alloc(&d, 1));
    CU(cudaMemsetAsync(d, 0, sizeof(int), s));
    k_row_max<<<ceil_div(a.rows, 256), 256, 0, s>>>(a.rows, a.rp, d);
    LAUNCH_CHECK();
    CU(cudaMemcpyAsync(out, d, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    return AMGH_OK;
}

__global__ void k_count_nonzero(int rows, const int *__restrict__ rp, const double *__restrict__ v, int *__restrict__ cnt)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows) return;
    int c = 0;
    for (int k = rp[i]; k < rp[i + 1]; k++) c += v[k] != 0.0;
    cnt[i] = c;
}

__global__ void k_drop_zeros(int rows, const int *__restrict__ rp, const int *__restrict__ ci,
                             const double *__restrict__ v, const int *__restrict__ rp2, int *__restrict__ ci2,
                             double *__restrict__ v2)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows) return;
    int q = rp2[i];
    for (int k = rp[i]; k < rp[i + 1]; k++)
        if (v[k] != 0.0) {
            ci2[q] = ci[k];
            v2[q] = v[k];
            q++;
        }
}

static int prepare_layout(Arena &ar, DevCsr &a, cudaStream_t s, int force_tpr);

// Solve-phase layout of a.  Entries whose value is exactly zero (the P1
// stiffness of the Kuhn cube stores 8 of its 15 entries per row as exact
// zeros) are left out of the SELL copy: a zero term adds nothing to any row
// sum, so the products are unchanged while the matrix stream shrinks.  The
// canonical CSR (rp, ci, v) keeps every entry for the setup.
int prepare_operator(Arena &ar, DevCsr &a, cudaStream_t s, int force_tpr)
{
    if (a.rows > 0 && a.nnz > 0 && force_tpr <= 1) {
        Scratch sc;
        int *cnt = nullptr, *rp2 = nullptr;
        TRY(sc.alloc(&cnt, a.rows + 1));
        TRY(sc.alloc(&rp2, a.rows + 1));
        k_count_nonzero<<<ceil_div(a.rows, 256), 256, 0, s>>>(a.rows, a.rp, a.v, cnt);
        LAUNCH_CHECK();
        int nz = 0;
        TRY(exclusive_scan<int>(cnt, rp2, a.rows, s, &nz));
        if ((double)nz < 0.95 * a.nnz) {
            DevCsr c = a;
            c.rp = rp2;
            c.nnz = nz;
            TRY(sc.alloc(&c.ci, nz));
            TRY(sc.alloc(&c.v, nz));
            k_drop_zeros<<<ceil_div(a.rows, 256), 256, 0, s>>>(a.rows, a.rp, a.ci, a.v, rp2, c.ci, c.v);
            LAUNCH_CHECK();
            int longest = 0;
            TRY(max_row_length(c, s, &longest));
            const double avg = (double)nz / a.rows;
            const bool uniform = (double)longest * a.rows <= 1.05 * nz;
            if (!(avg > 16.0 || (avg > 12.0 && !uniform))) { // SELL-32 for the compacted rows
                c.tpr = 1;
                c.wmax = longest;
                TRY(csr_to_sell(ar, c, 1, s));
                a.tpr = 1;
                a.wmax = c.wmax;
                a.nslices = c.nslices;
                a.sell_nnz = c.sell_nnz;
                a.ellw = c.ellw;
                a.sl_ptr = c.sl_ptr;
                a.sl_ci = c.sl_ci;
                a.sl_v = c.sl_v;
                a.sl_v32 = c.sl_v32;
                a.sl_ci16 = c.sl_ci16;
                a.nnz_solve = nz;
                CU(cudaStreamSynchronize(s));
                return AMGH_OK;
            }
        }
    }
    return prepare_layout(ar, a, s, force_tpr);
}

static int prepare_layout(Arena &ar, DevCsr &a, cudaStream_t s, int force_tpr)
{
    double avg = a.rows > 0 ? (double)a.nnz / a.rows : 0.0;
    int longest = 0;
    TRY(max_row_length(a, s, &longest));
    // SELL-32 for short rows, and for rows up to 16 long when every row has
    // nearly the longest length (uniform-width SELL: the staged smoother);
    // otherwise CSR with 4..32 lanes per row
    bool uniform = (double)longest * a.rows <= 1.05 * a.nnz;
    int tpr = 1;
    if (force_tpr > 0) tpr = force_tpr;
    else if (avg > 96.0) tpr = 32;
    else if (avg > 48.0) tpr = 16;
    else if (avg > 24.0) tpr = 8;
    else if (avg > 16.0 || (avg > 12.0 && !uniform)) tpr = 4;
    a.tpr = tpr;
    // SELL pads every row of a slice to the slice's longest row
    a.wmax = tpr == 1 ? longest : ceil_div(longest, tpr);
    if (tpr == 1) return csr_to_sell(ar, a, 1, s);
    TRY(ar.alloc(&a.v32, a.nnz));
    if (a.nnz > 0) {
        k_to_f32<<<ceil_div(a.nnz, 256), 256, 0, s>>>(a.nnz, a.v, a.v32);
        LAUNCH_CHECK();
    }
    CU(cudaStreamSynchronize(s));
    return AMGH_OK;
}

__global__ void k_lo_parts(int64_t n, const double *__restrict__ v, const float *__restrict__ hi,
                           float *__restrict__ lo)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) lo[i] = (float)(v[i] - (double)hi[i]);
}

int build_lo_parts(Arena &ar, DevCsr &a, cudaStream_t s)
{
    int64_t n = a.tpr <= 1 ? a.sell_nnz : a.nnz;
    const double *v = a.tpr <= 1 ? a.sl_v : a.v;
    const float *hi = a.tpr <= 1 ? a.sl_v32 : a.v32;
    TRY(ar.alloc(&a.lo32, n));
    if (n > 0) {
        k_lo_parts<<<ceil_div(n, 256), 256, 0, s>>>(n, v, hi, a.lo32);
        LAUNCH_CHECK();
    }
    CU(cudaStreamSynchronize(s));
    return AMGH_OK;
}

// ------------------------------------------------------------------ SpMV family
#define SKIP_RETURN() \
    if (skip && *skip) return

template <typename T, int TPR>
__global__ void k_spmv(MatView<T> A, const T *__restrict__ x, T *__restrict__ y, const int *__restrict__ skip)
{
    pdl_enter();
    SKIP_RETURN();
    int r = my_row<TPR>();
    T v = row_sum<T, TPR>(A, r, [&](int c) { return __ldg(&x[c]); });
    if (r < A.rows && row_leader<TPR>()) y[r] = v;
}

// y = A1 x1 + c A2 x2
template <typename T, int TPR>
__global__ void k_spmv2(MatView<T> A1, const T *__restrict__ x1, MatView<T> A2, const T *__restrict__ x2, T c,
                        T *__restrict__ y, const int *__restrict__ skip)
{
    pdl_enter();
    SKIP_RETURN();
    int r = my_row<TPR>();
    T a = row_sum<T, TPR>(A1, r, [&](int j) { return __ldg(&x1[j]); });
    // A2 may use another layout; it is read row-wise by the group leader's lanes
    T b = row_sum<T, TPR>(A2, r, [&](int j) { return __ldg(&x2[j]); });
    if (r < A1.rows && row_leader<TPR>()) y[r] = a + c * b;
}

// smoother step: d = cd d + cr D^-1 (b - A x); xn = x + d
template <typename T, int TPR>
__global__ void k_cheb_step(MatView<T> A, const T *__restrict__ invd, const T *__restrict__ b,
                            const T *__restrict__ x, T *__restrict__ d, T *__restrict__ xn, T cdv, T crv,
                            const int *__restrict__ skip)
{
    pdl_enter();
    SKIP_RETURN();
    int r = my_row<TPR>();
    bool lead = r < A.rows && row_leader<TPR>();
    // row-local operands first, so their loads overlap the row's
    T br = 0, ir = 0, dr = 0, xr = 0;
    if (lead) {
        br = b[r];
        ir = invd[r];
        dr = d[r];
        xr = x[r];
    }
    T ax = row_sum<T, TPR>(A, r, [&](int c) { return __ldg(&x[c]); });
    if (lead) {
        T dn, xv;
        cheb_point(br, ax, ir, dr, xr, cdv, crv, dn, xv);
        d[r] = dn;
        xn[r] = xv;
    }
}

// first smoother step from x = 0: d = c D^-1 b; x = d
template <typename T>
__global__ void k_cheb_first(int n, const T *__restrict__ invd, const T *__restrict__ b, T *__restrict__ d,
                             T *__restrict__ x, T c, const int *__restrict__ skip)
{
    pdl_enter();
    SKIP_RETURN();
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    T v = cheb_first_point(b[r], invd[r], c);
    d[r] = v;
    x[r] = v;
}

// ------------------------------------------------------------------ staged ELL smoother
// Level-0 Chebyshev step on a uniform-width SELL matrix (FP32 values, int16
// offsets or int32 columns): each block's 8 slices of the matrix are one
// contiguous range, brought into shared memory by the copy engine in one
// transaction while the threads load their rows' b, D^-1, d and x; then
// each thread gathers x at its row's columns, summing in the same order as
// row_sum in the register-loading kernel.  A copy that has not landed
// after g_bulk_first_polls polls sets g_bulk_timeout and the block computes
// nothing: it then waits (again bounded, with a far larger limit) for its
// copies to land before it exits, so that no copy is still writing into
// shared memory that a later block on the SM may own.  The host turns the
// flag into AMGH_ERR_TIMEOUT for the whole call: every value that call
// produced is invalid.
#define ELL_SLICES 8
#define ELL_MAX_W 16
#define BULK_POLLS (1 << 16)
#define BULK_DRAIN_POLLS (1 << 22)
__device__ int g_bulk_timeout = 0;
// poll limit of the first wait; lowered only by amgh_debug_limits (tests of
// the timeout path), read by every block so captured graphs see changes
__device__ int g_bulk_first_polls = BULK_POLLS;

template <bool D16>
__global__ void __launch_bounds__(32 * ELL_SLICES)
    k_cheb_step_ell(int rows, int nslices, int W, const float *__restrict__ v, const void *__restrict__ cols,
                    const float *__restrict__ invd, const float *__restrict__ b, const float *__restrict__ x,
                    float *__restrict__ d, float *__restrict__ xn, float cdv, float crv, const int *__restrict__ skip)
{
    pdl_enter();
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char ell_sm[];
    __shared__ __align__(8) uint64_t bar;
    const int first_polls = *(volatile int *)&g_bulk_first_polls; // issued early: off the wait's path
    const int s0 = blockIdx.x * ELL_SLICES;
    const int ns = min(ELL_SLICES, nslices - s0);
    const int64_t first = (int64_t)s0 * 32 * W;
    const uint32_t nent = (uint32_t)ns * 32 * W;
    float *sv = (float *)ell_sm;
    unsigned char *sc = ell_sm + (size_t)ELL_SLICES * 32 * W * sizeof(float);
    const uint32_t ib = D16 ? 2 : 4;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_expect_tx(&bar, nent * (4 + ib));
        bulk_g2s(sv, v + first, nent * 4, &bar);
        bulk_g2s(sc, (const unsigned char *)cols + first * ib, nent * ib, &bar);
    }
    const int row = s0 * 32 + (int)threadIdx.x;
    const bool ok = row < rows;
    float br = 0.f, ir = 0.f, dr = 0.f, xr = 0.f;
    if (ok) {
        br = b[row];
        ir = invd[row];
        dr = d[row];
        xr = x[row];
    }
    __syncthreads(); // the barrier is initialised before anyone polls it
    if (!mbar_wait(&bar, 0, first_polls)) {
        if (threadIdx.x == 0) atomicExch(&g_bulk_timeout, 1);
        mbar_wait(&bar, 0, BULK_DRAIN_POLLS); // let the copies into this block's memory finish
        return;
    }
    if (!ok) return;
    const int base = ((int)threadIdx.x >> 5) * 32 * W + ((int)threadIdx.x & 31);
    float xv[ELL_MAX_W];
#pragma unroll
    for (int j = 0; j < ELL_MAX_W; j++) {
        if (j < W) {
            int k = base + 32 * j;
            int c = D16 ? row + (int)((const short *)sc)[k] : ((const int *)sc)[k];
            xv[j] = __ldg(&x[c]);
        }
    }
    float ax = 0.f;
#pragma unroll
    for (int j = 0; j < ELL_MAX_W; j++)
        if (j < W) ax += sv[base + 32 * j] * xv[j];
    float dn, xv2;
    cheb_point(br, ax, ir, dr, xr, cdv, crv, dn, xv2);
    d[row] = dn;
    xn[row] = xv2;
}

template <typename T, int TPR>
__global__ void k_residual(MatView<T> A, const T *__restrict__ b, const T *__restrict__ x, T *__restrict__ res,
                           const int *__restrict__ skip)
{
    pdl_enter();
    SKIP_RETURN();
    int r = my_row<TPR>();
    bool lead = r < A.rows && row_leader<TPR>();
    T br = lead ? b[r] : (T)0;
    T ax = row_sum<T, TPR>(A, r, [&](int c) { return __ldg(&x[c]); });
    if (lead) res[r] = rsub(br, ax);
}

// restriction b_c = S^T r fused with the first smoother step of the coarse
// level from zero: d_c = x_c = c0 D_c^-1 b_c
template <typename T, int TPR>
__global__ void k_restrict_first(MatView<T> St, const T *__restrict__ r, T *__restrict__ bc,
                                 const T *__restrict__ invd, T *__restrict__ d, T *__restrict__ x, T c0,
                                 const int *__restrict__ skip)
{
    pdl_enter();
    SKIP_RETURN();
    int i = my_row<TPR>();
    bool lead = i < St.rows && row_leader<TPR>();
    T ir = lead ? invd[i] : (T)0;
    T b = row_sum<T, TPR>(St, i, [&](int c) { return __ldg(&r[c]); });
    if (lead) {
        bc[i] = b;
        T v = cheb_first_point(b, ir, c0);
        d[i] = v;
        x[i] = v;
    }
}

template <typename T, int TPR>
__global__ void k_prolong_add(MatView<T> S, const T *__restrict__ e, T *__restrict__ x,
                              const int *__restrict__ skip)
{
    pdl_enter();
    SKIP_RETURN();
    int i = my_row<TPR>();
    bool lead = i < S.rows && row_leader<TPR>();
    T xi = lead ? x[i] : (T)0;
    T v = row_sum<T, TPR>(S, i, [&](int c) { return __ldg(&e[c]); });
    if (lead) x[i] = radd(xi, v);
}

// x = inv b, one warp per row of the dense explicit inverse
template <typename T>
__global__ void k_dense_gemv(int n, const double *__restrict__ inv, const T *__restrict__ b, T *__restrict__ x,
                             const int *__restrict__ skip)
{
    pdl_enter();
    SKIP_RETURN();
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= n) return;
    const double *row = inv + (int64_t)warp * n;
    double acc = 0.0;
    for (int k = lane; k < n; k += 32) acc += row[k] * (double)b[k];
    acc = warp_sum(acc);
    if (lane == 0) x[warp] = (T)acc;
}

// FP32 copy, one warp per row, 16-byte loads of the padded row and (VEC) of
// b (the last partial group of four read element by element)
template <bool VEC>
__global__ void k_dense_gemv32(int n, int ld, const float *__restrict__ inv, const float *__restrict__ b,
                               float *__restrict__ x, const int *__restrict__ skip)
{
    pdl_enter();
    SKIP_RETURN();
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= n) return;
    float acc = dense_row32<VEC>(inv, ld, warp, n, b, lane);
    if (lane == 0) x[warp] = acc;
}

__global__ void k_pad32(int n, int ld, const double *__restrict__ inv, float *__restrict__ out)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * ld) return;
    int i = (int)(e / ld), j = (int)(e % ld);
    out[e] = j < n ? (float)inv[(int64_t)i * n + j] : 0.f;
}

static const int TPB = 256;

int dense_gemv32(amgh_problem *p, int n, int ld, const float *inv32, const float *b, float *x, const int *skip)
{
    if (n == 0) return AMGH_OK;
    int g = ceil_div((int64_t)n * 32, TPB);
    timer_begin(p, KC_COARSE);
    if (((uintptr_t)b & 15) == 0) pdl_launch(k_dense_gemv32<true>, dim3(g), dim3(TPB), 0, p->stream, n, ld, inv32, b, x, skip);
    else pdl_launch(k_dense_gemv32<false>, dim3(g), dim3(TPB), 0, p->stream, n, ld, inv32, b, x, skip);
    LAUNCH_CHECK();
    timer_end(p, KC_COARSE, 4.0 * n * (double)n + 8.0 * n);
    return AMGH_OK;
}

int dense_make32(amgh_problem *p, Arena &ar, Dense &d)
{
    if (d.n == 0) return AMGH_OK;
    d.ld32 = (d.n + 3) & ~3;
    TRY(ar.alloc(&d.inv32, (int64_t)d.n * d.ld32));
    if ((uintptr_t)d.inv32 & 15) return AMGH_ERR_CUDA; // pool blocks are 256-byte aligned
    k_pad32<<<ceil_div((int64_t)d.n * d.ld32, TPB), TPB, 0, p->stream>>>(d.n, d.ld32, d.inv, d.inv32);
    LAUNCH_CHECK();
    return AMGH_OK;
}

double spmv_bytes(const DevCsr &a, int vb)
{
    // index bytes per entry and slice / row pointers as the kernels read them
    const double nnz = a.nnz_solve >= 0 ? a.nnz_solve : a.nnz;
    if (a.tpr <= 1 && a.ellw > 0)
        return nnz * (vb + (a.sl_ci16 ? 2 : 4)) + (double)vb * (a.rows + a.cols);
    return nnz * (vb + 4) + 4.0 * (a.rows + 1) + (double)vb * (a.rows + a.cols);
}

// ------------------------------------------------------------------ autotuning
// Rows per lane group (tpr: 1 = SELL-32, else lanes per CSR row) of a state
// matrix A picked by timing what the V-cycle does with it: four back-to-back
// FP32 Chebyshev steps (so launch overlap between kernels is part of the
// measurement), after writing a buffer larger than L2 when the matrix itself
// would not stay in L2.  The choice is remembered for matrices of the same
// shape (rows, columns, entries, longest row) for the rest of the process.
__global__ void k_fill_f32(int n, float v, float *__restrict__ x)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = v;
}

struct TuneKey {
    int rows, cols, nnz, longest, dev;
    bool operator==(const TuneKey &o) const
    {
        return rows == o.rows && cols == o.cols && nnz == o.nnz && longest == o.longest && dev == o.dev;
    }
};

#define TUNE_COLD_BYTES (32ll << 20)
#define TUNE_FLUSH_BYTES (256ll << 20)

static int tune_tpr(amgh_problem *p, const DevCsr &a, int *best)
{
    static std::mutex mu;
    static std::vector<std::pair<TuneKey, int>> cache;
    cudaStream_t s = p->stream;
    int longest = 0, dev = 0;
    TRY(max_row_length(a, s, &longest));
    CU(cudaGetDevice(&dev));
    TuneKey key = {a.rows, a.cols, a.nnz, longest, dev};
    {
        std::lock_guard<std::mutex> lock(mu);
        for (auto &e : cache)
            if (e.first == key) {
                *best = e.second;
                return AMGH_OK;
            }
    }
    int n = a.rows;
    bool cold = (int64_t)a.nnz * 8 > TUNE_COLD_BYTES;
    Scratch sc;
    float *x = nullptr, *xn = nullptr, *d = nullptr, *b = nullptr, *invd = nullptr;
    unsigned char *flush = nullptr;
    TRY(sc.alloc(&x, n));
    TRY(sc.alloc(&xn, n));
    TRY(sc.alloc(&d, n));
    TRY(sc.alloc(&b, n));
    TRY(sc.alloc(&invd, n));
    if (cold) TRY(sc.alloc(&flush, TUNE_FLUSH_BYTES));
    for (float *v : {x, xn, d, b, invd}) {
        k_fill_f32<<<ceil_div(n, 256), 256, 0, s>>>(n, 0.5f, v);
        LAUNCH_CHECK();
    }
    double mean = (double)a.nnz / n;
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    int pick = 0, st = AMGH_OK;
    for (int c : {1, 2, 4, 8, 16, 32}) {
        if (c > 1 && c > 2 * mean) break;
        DevCsr t;
        t.rows = a.rows;
        t.cols = a.cols;
        t.nnz = a.nnz;
        t.rp = a.rp;
        t.ci = a.ci;
        t.v = a.v;
        Arena tar;
        st = prepare_operator(tar, t, s, c);
        float total = 0.f;
        for (int rep = 0; rep < 3 && st == AMGH_OK; rep++) {
            if (cold) CU(cudaMemsetAsync(flush, rep, TUNE_FLUSH_BYTES, s));
            MatView<float> V = view<float>(t);
            cudaEventRecord(e0, s);
            for (int k = 0; k < 4; k++)
                LAUNCH_TPR(k_cheb_step, float, c, n, s, V, (const float *)invd, (const float *)b,
                           (const float *)(k & 1 ? xn : x), d, k & 1 ? x : xn, 0.5f, 0.5f, (const int *)nullptr);
            cudaEventRecord(e1, s);
            float ms = 0.f;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                st = AMGH_ERR_CUDA;
            if (rep > 0) total += ms; // the first repetition warms the caches of a small matrix
        }
        if (st == AMGH_OK && total < best_ms) {
            best_ms = total;
            pick = c;
        }
        cudaStreamSynchronize(s);
        tar.free_all();
        if (st) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    *best = pick;
    std::lock_guard<std::mutex> lock(mu);
    cache.push_back({key, pick});
    return AMGH_OK;
}

#define TUNE_MIN_ROWS 4096

int prepare_tuned(amgh_problem *p, Arena &ar, DevCsr &a, int is_state_matrix)
{
    int tpr = 0;
    if (p->aopts.autotune && is_state_matrix && a.rows >= TUNE_MIN_ROWS && a.nnz > 0) TRY(tune_tpr(p, a, &tpr));
    return prepare_operator(ar, a, p->stream, tpr);
}

template <typename T>
int spmv_t(amgh_problem *p, const DevCsr &a, const T *x, T *y, const int *skip, int cls)
{
    if (a.rows == 0) return AMGH_OK;
    timer_begin(p, cls);
    MatView<T> A = view<T>(a);
    LAUNCH_TPR(k_spmv, T, A.tpr, A.rows, p->stream, A, x, y, skip);
    LAUNCH_CHECK();
    timer_end(p, cls, spmv_bytes(a, sizeof(T)));
    return AMGH_OK;
}
template int spmv_t<double>(amgh_problem *, const DevCsr &, const double *, double *, const int *, int);
template int spmv_t<float>(amgh_problem *, const DevCsr &, const float *, float *, const int *, int);

int spmv(amgh_problem *p, const DevCsr &a, const double *x, double *y, const int *skip, int cls)
{
    return spmv_t<double>(p, a, x, y, skip, cls);
}
int spmv32(amgh_problem *p, const DevCsr &a, const float *x, float *y, const int *skip, int cls)
{
    return spmv_t<float>(p, a, x, y, skip, cls);
}

int bulk_set_first_polls(int polls)
{
    int v = polls > 0 ? polls : BULK_POLLS;
    if (polls == 0) v = 0;
    CU(cudaMemcpyToSymbol(g_bulk_first_polls, &v, sizeof(int)));
    return AMGH_OK;
}

// nonzero once a staged copy has timed out (then cleared)
int bulk_timeout_check(cudaStream_t s)
{
    int h = 0;
    CU(cudaMemcpyFromSymbolAsync(&h, g_bulk_timeout, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (!h) return AMGH_OK;
    int zero = 0;
    CU(cudaMemcpyToSymbolAsync(g_bulk_timeout, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s));
    CU(cudaStreamSynchronize(s));
    return AMGH_ERR_TIMEOUT;
}

int spmv2(amgh_problem *p, const DevCsr &a1, const double *x1, const DevCsr &a2, const double *x2, double c,
          double *y, const int *skip)
{
    if (a1.rows == 0) return AMGH_OK;
    // both operands use the layout of a1 (a2 is re-viewed with a1's lane count)
    MatView<double> A1 = view<double>(a1), A2 = view<double>(a2);
    if (A1.tpr != A2.tpr) {
        // mixed layouts: two passes through y
        TRY(spmv_t<double>(p, a2, x2, y, skip, KC_SPMV));
        TRY(vec_axpby_spmv(p, a1, x1, c, y, skip));
        return AMGH_OK;
    }
    timer_begin(p, KC_SPMV);
    LAUNCH_TPR(k_spmv2, double, A1.tpr, A1.rows, p->stream, A1, x1, A2, x2, c, y, skip);
    LAUNCH_CHECK();
    timer_end(p, KC_SPMV, spmv_bytes(a1, 8) + spmv_bytes(a2, 8) - 8.0 * a1.rows);
    return AMGH_OK;
}

// y = A x + c y  (used when the two operands of spmv2 have different layouts)
template <typename T, int TPR>
__global__ void k_spmv_axpy(MatView<T> A, const T *__restrict__ x, T c, T *__restrict__ y,
                            const int *__restrict__ skip)
{
    pdl_enter();
    SKIP_RETURN();
    int r = my_row<TPR>();
    T v = row_sum<T, TPR>(A, r, [&](int j) { return __ldg(&x[j]); });
    if (r < A.rows && row_leader<TPR>()) y[r] = v + c * y[r];
}

int vec_axpby_spmv(amgh_problem *p, const DevCsr &a, const double *x, double c, double *y, const int *skip)
{
    MatView<double> A = view<double>(a);
    timer_begin(p, KC_SPMV);
    LAUNCH_TPR(k_spmv_axpy, double, A.tpr, A.rows, p->stream, A, x, c, y, skip);
    LAUNCH_CHECK();
    timer_end(p, KC_SPMV, spmv_bytes(a, 8) + 8.0 * a.rows);
    return AMGH_OK;
}

template <typename T>
int cheb_first(amgh_problem *p, int n, const T *invd, const T *b, T *d, T *x, double c, const int *skip)
{
    if (n == 0) return AMGH_OK;
    timer_begin(p, KC_CHEB);
    pdl_launch(k_cheb_first<T>, dim3(ceil_div(n, TPB)), dim3(TPB), 0, p->stream, n, invd, b, d, x, (T)c, skip);
    LAUNCH_CHECK();
    timer_end(p, KC_CHEB, 4.0 * sizeof(T) * n);
    return AMGH_OK;
}

template <typename T>
int cheb_step(amgh_problem *p, const DevCsr &a, const T *invd, const T *b, const T *x, T *d, T *xn, double cdv,
              double crv, const int *skip, int lvl0)
{
    if (a.rows == 0) return AMGH_OK;
    const int cls = lvl0 ? KC_CHEB0 : KC_CHEB;
    timer_begin(p, cls);
    MatView<T> A = view<T>(a);
    const void *ellcols = a.sl_ci16 ? (const void *)a.sl_ci16 : (const void *)a.sl_ci;
    if (sizeof(T) == sizeof(float) && a.tpr <= 1 && a.ellw > 0 && a.ellw <= ELL_MAX_W &&
        ((uintptr_t)a.sl_v32 & 15) == 0 && ((uintptr_t)ellcols & 15) == 0) {
        size_t smem = (size_t)ELL_SLICES * 32 * a.ellw * (sizeof(float) + (a.sl_ci16 ? 2 : 4));
        dim3 g(ceil_div(a.nslices, ELL_SLICES)), blk(32 * ELL_SLICES);
        const float *fi = (const float *)invd, *fb = (const float *)b, *fx = (const float *)x;
        float *fd = (float *)d, *fxn = (float *)xn;
        if (a.sl_ci16)
            pdl_launch(k_cheb_step_ell<true>, g, blk, smem, p->stream, a.rows, a.nslices, a.ellw, a.sl_v32,
                       (const void *)a.sl_ci16, fi, fb, fx, fd, fxn, (float)cdv, (float)crv, skip);
        else
            pdl_launch(k_cheb_step_ell<false>, g, blk, smem, p->stream, a.rows, a.nslices, a.ellw, a.sl_v32,
                       (const void *)a.sl_ci, fi, fb, fx, fd, fxn, (float)cdv, (float)crv, skip);
    } else {
        LAUNCH_TPR(k_cheb_step, T, A.tpr, A.rows, p->stream, A, invd, b, x, d, xn, (T)cdv, (T)crv, skip);
    }
    LAUNCH_CHECK();
    // algorithmic bytes: matrix + x gather + b, invd, d (read+write), xn
    timer_end(p, cls, spmv_bytes(a, sizeof(T)) + 4.0 * sizeof(T) * a.rows);
    return AMGH_OK;
}

template <typename T>
int residual(amgh_problem *p, const DevCsr &a, const T *b, const T *x, T *r, const int *skip, int lvl0)
{
    if (a.rows == 0) return AMGH_OK;
    const int cls = lvl0 ? KC_RESID0 : KC_RESID;
    timer_begin(p, cls);
    MatView<T> A = view<T>(a);
    LAUNCH_TPR(k_residual, T, A.tpr, A.rows, p->stream, A, b, x, r, skip);
    LAUNCH_CHECK();
    timer_end(p, cls, spmv_bytes(a, sizeof(T)) + sizeof(T) * (double)a.rows);
    return AMGH_OK;
}

template <typename T>
int restrict_first(amgh_problem *p, const DevCsr &st, const T *r, T *bc, const T *invd_c, T *d_c, T *x_c,
                   double c0, const int *skip)
{
    if (st.rows == 0) return AMGH_OK;
    MatView<T> A = view<T>(st);
    const int cls = st.cols == p->m ? KC_RESTRICT0 : KC_RESTRICT;
    timer_begin(p, cls);
    LAUNCH_TPR(k_restrict_first, T, A.tpr, A.rows, p->stream, A, r, bc, invd_c, d_c, x_c, (T)c0, skip);
    LAUNCH_CHECK();
    // S^T r, then D_c^-1 read and d_c, x_c written on the coarse level
    timer_end(p, cls, spmv_bytes(st, sizeof(T)) + 3.0 * sizeof(T) * st.rows);
    return AMGH_OK;
}

template <typename T>
int prolong_add(amgh_problem *p, const DevCsr &s, const T *e, T *x, const int *skip)
{
    if (s.rows == 0) return AMGH_OK;
    MatView<T> A = view<T>(s);
    const int cls = s.rows == p->m ? KC_PROLONG0 : KC_PROLONG;
    timer_begin(p, cls);
    LAUNCH_TPR(k_prolong_add, T, A.tpr, A.rows, p->stream, A, e, x, skip);
    LAUNCH_CHECK();
    // S e, and x read before it is written
    timer_end(p, cls, spmv_bytes(s, sizeof(T)) + sizeof(T) * (double)s.rows);
    return AMGH_OK;
}

template <typename T>
int dense_gemv(amgh_problem *p, int n, const double *inv, const T *b, T *x, const int *skip)
{
    if (n == 0) return AMGH_OK;
    timer_begin(p, KC_COARSE);
    pdl_launch(k_dense_gemv<T>, dim3(ceil_div((int64_t)n * 32, TPB)), dim3(TPB), 0, p->stream, n, inv, b, x, skip);
    LAUNCH_CHECK();
    timer_end(p, KC_COARSE, 8.0 * n * (double)n + 2.0 * sizeof(T) * n);
    return AMGH_OK;
}

#define INST(T)                                                                                              \
    template int cheb_first<T>(amgh_problem *, int, const T *, const T *, T *, T *, double, const int *);        \
    template int cheb_step<T>(amgh_problem *, const DevCsr &, const T *, const T *, const T *, T *, T *, double, \
                              double, const int *, int);                                                    \
    template int residual<T>(amgh_problem *, const DevCsr &, const T *, const T *, T *, const int *, int);       \
    template int prolong_add<T>(amgh_problem *, const DevCsr &, const T *, T *, const int *);                  \
    template int restrict_first<T>(amgh_problem *, const DevCsr &, const T *, T *, const T *, T *, T *, double, \
                                   const int *);                                                            \
    template int dense_gemv<T>(amgh_problem *, int, const double *, const T *, T *, const int *);
INST(double)
INST(float)
