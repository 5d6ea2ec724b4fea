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
#include "internal.cuh"
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
    a.sell_nnz = total;
    TRY(ar.alloc(&a.sl_ci, total));
    TRY(ar.alloc(&a.sl_v, total));
    TRY(ar.alloc(&a.sl_v32, total));
    if (ns > 0) {
        k_sell_fill<<<ceil_div(ns * 32, 256), 256, 0, s>>>(a.rows, a.rp, a.ci, a.v, a.sl_ptr, a.sl_ci,
                                                          a.sl_v, a.sl_v32, ns);
        LAUNCH_CHECK();
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

// sort every row of (ci, v) by column (insertion sort; rows are short)
__global__ void k_sort_rows(int rows, const int *__restrict__ rp, int *__restrict__ ci, double *__restrict__ v)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    int b = rp[r], e = rp[r + 1];
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
    }
    CU(cudaStreamSynchronize(s));
    return AMGH_OK;
}

// ------------------------------------------------------------------ SpMV family
template <typename T>
static inline const T *h_sell_vals(const DevCsr &a);
template <>
inline const double *h_sell_vals<double>(const DevCsr &a) { return a.sl_v; }
template <>
inline const float *h_sell_vals<float>(const DevCsr &a) { return a.sl_v32; }

// row dot product of SELL row r with x
template <typename T>
__device__ __forceinline__ T sell_row(int r, const int *__restrict__ slp, const int *__restrict__ sci,
                                      const T *__restrict__ sv, const T *__restrict__ x)
{
    int s = r >> 5, lane = r & 31;
    int beg = slp[s] + lane, end = slp[s + 1];
    T acc = (T)0;
    for (int k = beg; k < end; k += 32) acc += sv[k] * __ldg(&x[sci[k]]);
    return acc;
}

#define SKIP_RETURN() \
    if (skip && *skip) return

template <typename T>
__global__ void k_spmv(int rows, const int *__restrict__ slp, const int *__restrict__ sci,
                       const T *__restrict__ sv, const T *__restrict__ x, T *__restrict__ y,
                       const int *__restrict__ skip)
{
    SKIP_RETURN();
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    y[r] = sell_row<T>(r, slp, sci, sv, x);
}

// y = A1 x1 + c A2 x2
__global__ void k_spmv2(int rows, const int *__restrict__ slp1, const int *__restrict__ sci1,
                        const double *__restrict__ sv1, const double *__restrict__ x1,
                        const int *__restrict__ slp2, const int *__restrict__ sci2,
                        const double *__restrict__ sv2, const double *__restrict__ x2, double c,
                        double *__restrict__ y, const int *__restrict__ skip)
{
    SKIP_RETURN();
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    double a = sell_row<double>(r, slp1, sci1, sv1, x1);
    double b = sell_row<double>(r, slp2, sci2, sv2, x2);
    y[r] = a + c * b;
}

// smoother step: d = cd d + cr D^-1 (b - A x); xn = x + d
template <typename T>
__global__ void k_cheb_step(int rows, const int *__restrict__ slp, const int *__restrict__ sci,
                            const T *__restrict__ sv, const T *__restrict__ invd, const T *__restrict__ b,
                            const T *__restrict__ x, T *__restrict__ d, T *__restrict__ xn, T cdv, T crv,
                            const int *__restrict__ skip)
{
    SKIP_RETURN();
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    T ax = sell_row<T>(r, slp, sci, sv, x);
    T res = (b[r] - ax) * invd[r];
    T dn = cdv * d[r] + crv * res;
    d[r] = dn;
    xn[r] = x[r] + dn;
}

// first smoother step from x = 0: d = c D^-1 b; x = d
template <typename T>
__global__ void k_cheb_first(int n, const T *__restrict__ invd, const T *__restrict__ b,
                             T *__restrict__ d, T *__restrict__ x, T c, const int *__restrict__ skip)
{
    SKIP_RETURN();
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    T v = c * (b[r] * invd[r]);
    d[r] = v;
    x[r] = v;
}

template <typename T>
__global__ void k_residual(int rows, const int *__restrict__ slp, const int *__restrict__ sci,
                           const T *__restrict__ sv, const T *__restrict__ b, const T *__restrict__ x,
                           T *__restrict__ r, const int *__restrict__ skip)
{
    SKIP_RETURN();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows) return;
    r[i] = b[i] - sell_row<T>(i, slp, sci, sv, x);
}

// restriction b_c = S^T r fused with the first smoother step of the coarse
// level from zero: d_c = x_c = c0 D_c^-1 b_c
template <typename T>
__global__ void k_restrict_first(int rows, const int *__restrict__ slp, const int *__restrict__ sci,
                                 const T *__restrict__ sv, const T *__restrict__ r, T *__restrict__ bc,
                                 const T *__restrict__ invd, T *__restrict__ d, T *__restrict__ x, T c0,
                                 const int *__restrict__ skip)
{
    SKIP_RETURN();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows) return;
    T b = sell_row<T>(i, slp, sci, sv, r);
    bc[i] = b;
    T v = c0 * (b * invd[i]);
    d[i] = v;
    x[i] = v;
}

template <typename T>
__global__ void k_prolong_add(int rows, const int *__restrict__ slp, const int *__restrict__ sci,
                              const T *__restrict__ sv, const T *__restrict__ e, T *__restrict__ x,
                              const int *__restrict__ skip)
{
    SKIP_RETURN();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows) return;
    x[i] = x[i] + sell_row<T>(i, slp, sci, sv, e);
}

// x = inv b, one warp per row of the dense explicit inverse
template <typename T>
__global__ void k_dense_gemv(int n, const double *__restrict__ inv, const T *__restrict__ b,
                             T *__restrict__ x, const int *__restrict__ skip)
{
    SKIP_RETURN();
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= n) return;
    const double *row = inv + (int64_t)warp * n;
    double acc = 0.0;
    for (int k = lane; k < n; k += 32) acc += row[k] * (double)b[k];
    acc = warp_sum(acc);
    if (lane == 0) x[warp] = (T)acc;
}

static const int TPB = 256;

static double spmv_bytes(const DevCsr &a, int vb)
{
    return (double)a.nnz * (vb + 4) + 4.0 * (a.rows + 1) + (double)vb * (a.rows + a.cols);
}

template <typename T>
int spmv_t(amgh_problem *p, const DevCsr &a, const T *x, T *y, const int *skip, int timed)
{
    if (a.rows == 0) return AMGH_OK;
    timer_begin(p, timed);
    k_spmv<T><<<ceil_div(a.rows, TPB), TPB, 0, p->stream>>>(a.rows, a.sl_ptr, a.sl_ci, h_sell_vals<T>(a), x,
                                                            y, skip);
    LAUNCH_CHECK();
    timer_end(p, timed, spmv_bytes(a, sizeof(T)));
    return AMGH_OK;
}
template int spmv_t<double>(amgh_problem *, const DevCsr &, const double *, double *, const int *, int);
template int spmv_t<float>(amgh_problem *, const DevCsr &, const float *, float *, const int *, int);

int spmv(amgh_problem *p, const DevCsr &a, const double *x, double *y, const int *skip, int timed)
{
    return spmv_t<double>(p, a, x, y, skip, timed);
}
int spmv32(amgh_problem *p, const DevCsr &a, const float *x, float *y, const int *skip, int timed)
{
    return spmv_t<float>(p, a, x, y, skip, timed);
}

int spmv2(amgh_problem *p, const DevCsr &a1, const double *x1, const DevCsr &a2, const double *x2,
          double c, double *y, const int *skip)
{
    if (a1.rows == 0) return AMGH_OK;
    k_spmv2<<<ceil_div(a1.rows, TPB), TPB, 0, p->stream>>>(a1.rows, a1.sl_ptr, a1.sl_ci, a1.sl_v, x1,
                                                           a2.sl_ptr, a2.sl_ci, a2.sl_v, x2, c, y, skip);
    LAUNCH_CHECK();
    return AMGH_OK;
}

template <typename T>
int cheb_first(amgh_problem *p, int n, const T *invd, const T *b, T *d, T *x, double c, const int *skip)
{
    if (n == 0) return AMGH_OK;
    k_cheb_first<T><<<ceil_div(n, TPB), TPB, 0, p->stream>>>(n, invd, b, d, x, (T)c, skip);
    LAUNCH_CHECK();
    return AMGH_OK;
}

template <typename T>
int cheb_step(amgh_problem *p, const DevCsr &a, const T *invd, const T *b, const T *x, T *d, T *xn,
              double cdv, double crv, const int *skip, int timed)
{
    if (a.rows == 0) return AMGH_OK;
    timer_begin(p, timed);
    k_cheb_step<T><<<ceil_div(a.rows, TPB), TPB, 0, p->stream>>>(a.rows, a.sl_ptr, a.sl_ci, h_sell_vals<T>(a),
                                                                 invd, b, x, d, xn, (T)cdv, (T)crv, skip);
    LAUNCH_CHECK();
    // algorithmic bytes: matrix + x gather + b, invd, d (read+write), xn
    timer_end(p, timed, spmv_bytes(a, sizeof(T)) + 4.0 * sizeof(T) * a.rows);
    return AMGH_OK;
}

template <typename T>
int residual(amgh_problem *p, const DevCsr &a, const T *b, const T *x, T *r, const int *skip, int timed)
{
    if (a.rows == 0) return AMGH_OK;
    timer_begin(p, timed);
    k_residual<T><<<ceil_div(a.rows, TPB), TPB, 0, p->stream>>>(a.rows, a.sl_ptr, a.sl_ci, h_sell_vals<T>(a), b,
                                                                x, r, skip);
    LAUNCH_CHECK();
    timer_end(p, timed, spmv_bytes(a, sizeof(T)) + sizeof(T) * (double)a.rows);
    return AMGH_OK;
}

template <typename T>
int restrict_first(amgh_problem *p, const DevCsr &st, const T *r, T *bc, const T *invd_c, T *d_c, T *x_c,
                   double c0, const int *skip)
{
    if (st.rows == 0) return AMGH_OK;
    k_restrict_first<T><<<ceil_div(st.rows, TPB), TPB, 0, p->stream>>>(st.rows, st.sl_ptr, st.sl_ci,
                                                                       h_sell_vals<T>(st), r, bc, invd_c, d_c, x_c,
                                                                       (T)c0, skip);
    LAUNCH_CHECK();
    return AMGH_OK;
}

template <typename T>
int prolong_add(amgh_problem *p, const DevCsr &s, const T *e, T *x, const int *skip)
{
    if (s.rows == 0) return AMGH_OK;
    k_prolong_add<T><<<ceil_div(s.rows, TPB), TPB, 0, p->stream>>>(s.rows, s.sl_ptr, s.sl_ci, h_sell_vals<T>(s), e,
                                                                   x, skip);
    LAUNCH_CHECK();
    return AMGH_OK;
}

template <typename T>
int dense_gemv(amgh_problem *p, int n, const double *inv, const T *b, T *x, const int *skip)
{
    if (n == 0) return AMGH_OK;
    k_dense_gemv<T><<<ceil_div((int64_t)n * 32, TPB), TPB, 0, p->stream>>>(n, inv, b, x, skip);
    LAUNCH_CHECK();
    return AMGH_OK;
}

#define INST(T)                                                                                       \
    template int cheb_first<T>(amgh_problem *, int, const T *, const T *, T *, T *, double, const int *); \
    template int cheb_step<T>(amgh_problem *, const DevCsr &, const T *, const T *, const T *, T *, T *,  \
                              double, double, const int *, int);                                      \
    template int residual<T>(amgh_problem *, const DevCsr &, const T *, const T *, T *, const int *, int); \
    template int prolong_add<T>(amgh_problem *, const DevCsr &, const T *, T *, const int *);            \
    template int restrict_first<T>(amgh_problem *, const DevCsr &, const T *, T *, const T *, T *, T *, double, \
                                   const int *);                                                         \
    template int dense_gemv<T>(amgh_problem *, int, const double *, const T *, T *, const int *);
INST(double)
INST(float)
