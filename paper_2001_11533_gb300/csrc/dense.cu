// dense.cu -- dense coarsest-level operators (at most 4096 rows):
//   * the explicit inverse of the coarsest AMG matrix A_{L-1} (the exact
//     coarse solve of the V-cycle), applied as one GEMV (an FP32 copy serves
//     the FP32 V-cycles);
//   * the dense coarsest Hessian H_c = M_yu^T A_c^-1 M_y A_c^-1 M_yu + beta M_u
//     on Hessian level l-1 and its explicit inverse -- the exact coarsest
//     inverse G_{l-1}^-1 assumed by the theory (Sec. 3.2).
// Both inverses come from a blocked right-looking Cholesky factorisation
// A = L L^T (INDEFINITE if a pivot is not positive) whose panel steps also
// form W = L^-1, then A^-1 = W^T W (upper triangle only, then mirrored).  All
// FP64 on the FMA pipe: on GB300 the FP64 tensor instruction is only about 4 %
// faster (amgh_fp64_peak measures both), and the products that carry the
// flops already keep the FP64 pipe busy almost all the time.
#include <math.h>

#include "internal.cuh"
#include "util.cuh"

__global__ void k_dense_from_csr(int rows, int cols, const int *__restrict__ rp, const int *__restrict__ ci,
                                 const double *__restrict__ v, double *__restrict__ g)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows) return;
    double *row = g + (int64_t)i * cols;
    for (int j = 0; j < cols; j++) row[j] = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; k++) row[ci[k]] = v[k];
}

int dense_from_csr(amgh_problem *p, const DevCsr &a, double *g)
{
    k_dense_from_csr<<<ceil_div(a.rows, 64), 64, 0, p->stream>>>(a.rows, a.cols, a.rp, a.ci, a.v, g);
    LAUNCH_CHECK();
    return AMGH_OK;
}

// Blocked right-looking Cholesky A = L L^T (lower triangle, row-major, NB-wide
// panels) fused with the forward sweep that forms W = L^-1, so that both share
// the panel steps.  With B = I at the start, panel k does
//   1. the factorisation of A_kk and D_k = L_kk^-1 (one block, in shared memory);
//   2. L_ik = A_ik D_k^T for the rows below the panel, and W_k. = D_k B_k.
//      for block row k of W (columns left of and on the diagonal block);
//   3. A_ij -= L_ik L_jk^T on the trailing lower triangle and
//      B_i. -= L_ik W_k. on the rows of W below the panel.
// Step 3 first updates the next panel's columns alone, then the rest, and the
// launch that does the rest also runs step 1 of the next panel in its block 0:
// the serial chain of the diagonal factorisation overlaps the K = NB products
// that carry the flops.
//
// FP64 on this GPU: every FP64 warp instruction holds its SM sub-partition's
// FP64 unit for the same time whatever the number of active lanes, so the
// kernels spread FP64 work over all four sub-partitions and over the elements
// that change, and keep the per-pivot chain to five dependent FP64 operations.
#define NB 32
#define DIAG_TRI (NB * (NB - 1) / 2)

// the single-precision estimate of 1 / sqrt(d) or 1 / d, for d > 0 with a
// binary exponent within +-120, as a double (exact bit moves, no FP64 work)
__device__ __forceinline__ double seed_from_float(double d, bool rsq)
{
    long long b = __double_as_longlong(d);
    int e = (int)((b >> 52) & 0x7ff) - 1023;
    float f = __int_as_float(((e + 127) << 23) | (int)((b >> 29) & 0x7fffff));
    float yf = rsq ? rsqrtf(f) : __fdividef(1.0f, f);
    int fb = __float_as_int(yf);
    return __longlong_as_double(((long long)(((fb >> 23) & 0xff) - 127 + 1023) << 52) |
                                ((long long)(fb & 0x7fffff) << 29));
}

__device__ __forceinline__ bool seed_range(double d)
{
    int e = (int)((__double_as_longlong(d) >> 52) & 0x7ff) - 1023;
    return e >= -120 && e <= 120;
}

// Newton-Raphson from the float estimate (relative error about 2^-22, squared
// by each step, so two steps reach rounding):
//   1 / d:        y <- y + y (1 - d y)
//   1 / sqrt(d):  y <- y (3 - d y^2) / 2
__device__ __forceinline__ double recip_newton(double d)
{
    if (!seed_range(d)) return 1.0 / d;
    double y = seed_from_float(d, false);
    y = fma(y, fma(-d, y, 1.0), y);
    return fma(y, fma(-d, y, 1.0), y);
}

__device__ __forceinline__ double rsqrt_newton(double d)
{
    if (!seed_range(d)) return 1.0 / sqrt(d);
    double y = seed_from_float(d, true), nh = -0.5 * d;
    y = y * fma(nh, y * y, 1.5);
    return y * fma(nh, y * y, 1.5);
}

// positive and finite, from the bits (no FP64 compare on the chain)
__device__ __forceinline__ bool pivot_ok(double d)
{
    long long b = __double_as_longlong(d);
    return b > 0 && b < 0x7ff0000000000000ll;
}

// Step 1 for the panel at k0, on a whole block (blockDim.x a multiple of 128).
// A_kk = L_u diag(p) L_u^T (L_u unit lower) in the right-looking order: pivot
// p_j, then a_ic -= (a_ij / p_j) a_cj for j < c <= i, one barrier per pivot.
// Thread 0 updates the next pivot and takes its reciprocal while the warps
// off its sub-partition update the rest (warps 4w share thread 0's FP64 unit
// and get no elements).  The columns are scaled to L_u afterwards.  Then
// X = L_u^-1 by recursive doubling over 2b x 2b diagonal blocks,
// b = 1, 2, 4, 8, 16: X_21 = -X_22 (L_21 X_11), and D = L^-1 = diag(p)^-1/2 X.
// Rows past the matrix are the identity, so the ragged last panel needs no
// special case.  A pivot that is not positive sets *info (1-based row) and is
// replaced by 1.
__device__ void diag_factor(int n, int k0, const double *__restrict__ g, double *__restrict__ dinv,
                            int *__restrict__ info)
{
    __shared__ double a[NB][NB + 1], x[NB][NB + 1], tmp[NB][NB + 1];
    __shared__ double piv[NB], rr[NB];
    __shared__ unsigned short tab[DIAG_TRI]; // row-major lower triangle (i, c <= i) of a 31 x 31 block
    int t = threadIdx.x, nt = blockDim.x;
    int nb = min(NB, n - k0);
    for (int e = t; e < NB * NB; e += nt) {
        int r = e / NB, c = e % NB;
        a[r][c] = r < nb && c < nb ? (c <= r ? g[(int64_t)(k0 + r) * n + k0 + c] : 0.0) : (r == c ? 1.0 : 0.0);
        x[r][c] = r == c ? 1.0 : 0.0;
    }
    for (int i = t; i < NB - 1; i += nt)
        for (int c = 0; c <= i; c++) tab[i * (i + 1) / 2 + c] = (unsigned short)((i << 8) | c);
    auto take_pivot = [&](int j, double p) {
        if (!pivot_ok(p)) {
            atomicCAS(info, 0, k0 + j + 1);
            p = 1.0;
        }
        piv[j] = p;
        rr[j] = recip_newton(p);
    };
    __syncthreads();
    if (t == 0) take_pivot(0, a[0][0]);
    int warp = t >> 5;
    bool worker = (warp & 3) != 0;
    int wk = (warp - (warp >> 2) - 1) * 32 + (t & 31), nwk = nt / 4 * 3;
    __syncthreads();
    for (int j = 0; j < nb; j++) {
        double r = rr[j];
        int m = nb - 1 - j, E = m * (m + 1) / 2;
        if (t == 0) {
            if (E > 0) {
                double u = a[j + 1][j];
                double p = fma(-(u * r), u, a[j + 1][j + 1]);
                a[j + 1][j + 1] = p;
                take_pivot(j + 1, p);
            }
        } else if (worker) {
            for (int e = 1 + wk; e < E; e += nwk) {
                int pk = tab[e], i = j + 1 + (pk >> 8), c = j + 1 + (pk & 255);
                a[i][c] = fma(-(a[i][j] * r), a[c][j], a[i][c]);
            }
        }
        __syncthreads();
    }
    for (int e = t; e < DIAG_TRI; e += nt) { // l_rq = a_rq / p_q below the diagonal
        int pk = tab[e], r = (pk >> 8) + 1, q = pk & 255;
        if (q < nb) a[r][q] *= rr[q];
    }
    __syncthreads();
    for (int lb = 0; lb < 5; lb++) { // b = 2^lb; 16 / b pairs of b x b blocks
        int b = 1 << lb, sh = 2 * lb;
        for (int e = t; e < 16 * b; e += nt) { // tmp = L_21 X_11
            int o = (e >> sh) * 2 * b, r = (e & (b * b - 1)) >> lb, c = e & (b - 1);
            double s0 = 0.0, s1 = 0.0;
            int q = c;
            for (; q + 1 < b; q += 2) {
                s0 = fma(a[o + b + r][o + q], x[o + q][o + c], s0);
                s1 = fma(a[o + b + r][o + q + 1], x[o + q + 1][o + c], s1);
            }
            if (q < b) s0 = fma(a[o + b + r][o + q], x[o + q][o + c], s0);
            tmp[o + b + r][o + c] = s0 + s1;
        }
        __syncthreads();
        for (int e = t; e < 16 * b; e += nt) { // X_21 = -X_22 tmp
            int o = (e >> sh) * 2 * b, r = (e & (b * b - 1)) >> lb, c = e & (b - 1);
            double s0 = 0.0, s1 = 0.0;
            int q = 0;
            for (; q + 1 <= r; q += 2) {
                s0 = fma(x[o + b + r][o + b + q], tmp[o + b + q][o + c], s0);
                s1 = fma(x[o + b + r][o + b + q + 1], tmp[o + b + q + 1][o + c], s1);
            }
            if (q <= r) s0 = fma(x[o + b + r][o + b + q], tmp[o + b + q][o + c], s0);
            x[o + b + r][o + c] = -(s0 + s1);
        }
        __syncthreads();
    }
    if (t < nb) rr[t] = rsqrt_newton(piv[t]);
    __syncthreads();
    double *d = dinv + (int64_t)(k0 / NB) * NB * NB;
    for (int e = t; e < NB * NB; e += nt) {
        int r = e / NB, c = e % NB;
        d[e] = c <= r ? (r < nb ? x[r][c] * rr[r] : x[r][c]) : 0.0;
    }
}

__global__ void __launch_bounds__(128) k_potrf_diag(int n, int k0, const double *__restrict__ g,
                                                    double *__restrict__ dinv, int *__restrict__ info)
{
    diag_factor(n, k0, g, dinv, info);
}

// step 2: blocks [0, rb) turn PANEL_WARPS rows each of the panel into L_ik;
// the next (k0/NB + 1) * NB/PANEL_WARPS blocks each form PANEL_WARPS rows of
// one 32-column strip of Y_k = D_k B_k. (one row per warp, so that no warp
// issues more than NB FP64 FMAs) into ybuf (NB x n, row-major).  B_k. stays in
// W until the next launch copies Y_k over it: a strip is read by all its
// blocks, so none of them may overwrite it.
#define PANEL_WARPS 4
__global__ void __launch_bounds__(32 * PANEL_WARPS) k_panel(int n, int k0, int rb, double *__restrict__ g,
                                                            const double *__restrict__ dinv,
                                                            const double *__restrict__ W, double *__restrict__ ybuf)
{
    __shared__ double d[NB][NB + 1], sb[NB][NB + 1];
    const double *dk = dinv + (int64_t)(k0 / NB) * NB * NB;
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) d[e / NB][e % NB] = dk[e];
    int nb = min(NB, n - k0);
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (blockIdx.x < rb) {
        __syncthreads();
        int i = k0 + nb + blockIdx.x * PANEL_WARPS + warp;
        if (i >= n) return; // warp-uniform, no block barrier follows
        double *row = g + (int64_t)i * n + k0;
        double gq = lane < nb ? row[lane] : 0.0;
        double acc0 = 0.0, acc1 = 0.0; // two chains: FP64 latency, not issue, bounds one warp
#pragma unroll
        for (int q = 0; q < NB; q += 2) {
            acc0 = fma(__shfl_sync(0xffffffffu, gq, q), d[lane][q], acc0);
            acc1 = fma(__shfl_sync(0xffffffffu, gq, q + 1), d[lane][q + 1], acc1);
        }
        if (lane < nb) row[lane] = acc0 + acc1;
        return;
    }
    int sblk = blockIdx.x - rb, strip = sblk / (NB / PANEL_WARPS), c0 = strip * NB, col = c0 + lane;
    int r = (sblk % (NB / PANEL_WARPS)) * PANEL_WARPS + warp;
    if (c0 == k0) { // the diagonal block: B_kk = I
        __syncthreads();
        if (r < nb && lane < nb) ybuf[(int64_t)r * n + col] = d[r][lane];
        return;
    }
    for (int q = warp; q < NB; q += PANEL_WARPS) sb[q][lane] = q < nb ? W[(int64_t)(k0 + q) * n + col] : 0.0;
    __syncthreads();
    if (r >= nb) return;
    double y0 = 0.0, y1 = 0.0;
#pragma unroll
    for (int q = 0; q < NB; q += 2) {
        y0 = fma(d[r][q], sb[q][lane], y0);
        y1 = fma(d[r][q + 1], sb[q + 1][lane], y1);
    }
    ybuf[(int64_t)r * n + col] = y0 + y1;
}

// step 3 tiles, 16 x 16 on 256 threads.  An A tile (ti, tj), tj <= ti, of the
// trailing matrix below and right of the panel at k0: A_ij -= sum_c L_ic L_jc
// on and below the diagonal.  A W tile: rows below the panel times the first
// k0 + nb columns, B_ij -= sum_c L_ic Y_cj (Y_k in ybuf).
__device__ __forceinline__ void trail_tile(int n, int k0, int ti, int tj, bool wtile, double *__restrict__ g,
                                           double *__restrict__ W, const double *__restrict__ ybuf)
{
    __shared__ double Li[16][NB + 1], Rj[NB][17];
    int nb = min(NB, n - k0), base = k0 + nb;
    int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    int r0 = base + ti * 16, j0 = wtile ? tj * 16 : base + tj * 16;
    for (int e = threadIdx.x; e < 16 * NB; e += 256) {
        int r = e / NB, c = e % NB;
        Li[r][c] = r0 + r < n && c < nb ? g[(int64_t)(r0 + r) * n + k0 + c] : 0.0;
        if (!wtile) Rj[c][r] = j0 + r < n && c < nb ? g[(int64_t)(j0 + r) * n + k0 + c] : 0.0;
    }
    if (wtile)
        for (int e = threadIdx.x; e < NB * 16; e += 256) {
            int c = e / 16, q = e % 16;
            Rj[c][q] = c < nb && j0 + q < base ? ybuf[(int64_t)c * n + j0 + q] : 0.0;
        }
    __syncthreads();
    int i = r0 + ty, j = j0 + tx;
    if (i >= n || (wtile ? j >= base : j > i)) return;
    double s0 = 0.0, s1 = 0.0;
#pragma unroll
    for (int c = 0; c < NB; c += 2) {
        s0 = fma(Li[ty][c], Rj[c][tx], s0);
        s1 = fma(Li[ty][c + 1], Rj[c + 1][tx], s1);
    }
    double *out = wtile ? W : g;
    out[(int64_t)i * n + j] -= s0 + s1;
}

__device__ __forceinline__ void tri_decode(int t, int &ti, int &tj)
{
    ti = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while ((ti + 1) * (ti + 2) / 2 <= t) ti++;
    while (ti * (ti + 1) / 2 > t) ti--;
    tj = t - ti * (ti + 1) / 2;
}

// the next panel's columns: A tiles (ti, 0) for ti < T and (ti, 1) for 1 <= ti < T
__global__ void __launch_bounds__(256) k_trail_next(int n, int k0, int T, double *__restrict__ g)
{
    int t = blockIdx.x;
    if (t < T) trail_tile(n, k0, t, 0, false, g, nullptr, nullptr);
    else trail_tile(n, k0, t - T + 1, 1, false, g, nullptr, nullptr);
}

// the rest: block 0 factors the next panel's diagonal block (updated by
// k_trail_next; none after the last panel), blocks [1, 1 + ta) the A tiles
// with 2 <= tj <= ti, the next T * tw the W tiles (T rows x tw columns of
// tiles), the last cb copy Y_k from ybuf into block row k of W (rows no other
// block of this launch reads or writes)
#define COPY_TPB 256
__global__ void __launch_bounds__(256) k_trail_rest(int n, int k0, int T, int ta, int tw, double *__restrict__ g,
                                                    double *__restrict__ W, const double *__restrict__ ybuf,
                                                    double *__restrict__ dinv, int *__restrict__ info)
{
    int t = blockIdx.x;
    if (t == 0) {
        if (k0 + NB < n) diag_factor(n, k0 + NB, g, dinv, info);
        return;
    }
    t -= 1;
    if (t < ta) {
        int ti, tj;
        tri_decode(t, ti, tj);
        trail_tile(n, k0, ti + 2, tj + 2, false, g, W, ybuf);
        return;
    }
    t -= ta;
    if (t < T * tw) {
        trail_tile(n, k0, t / tw, t % tw, true, g, W, ybuf);
        return;
    }
    t -= T * tw;
    int nb = min(NB, n - k0), width = k0 + nb;
    int64_t e = (int64_t)t * COPY_TPB + threadIdx.x;
    if (e < (int64_t)nb * width) {
        int r = (int)(e / width), c = (int)(e % width);
        W[(int64_t)(k0 + r) * n + c] = ybuf[(int64_t)r * n + c];
    }
}

// C = op(A) B (+ beta D), all row-major; transA: A is k x m and used as A^T
#define TILE 16
// lower != 0: only the tiles on and below the diagonal (C symmetric, and only
// its lower triangle is read afterwards)
__global__ void k_gemm(int m, int n, int kdim, const double *__restrict__ A, int transA,
                       const double *__restrict__ B, double beta, const double *__restrict__ D,
                       double *__restrict__ C, int lower)
{
    __shared__ double As[TILE][TILE + 1], Bs[TILE][TILE + 1];
    if (lower && blockIdx.x > blockIdx.y) return; // block-uniform
    int row = blockIdx.y * TILE + threadIdx.y, col = blockIdx.x * TILE + threadIdx.x;
    double acc = 0.0;
    for (int k0 = 0; k0 < kdim; k0 += TILE) {
        int ka = k0 + threadIdx.x, kb = k0 + threadIdx.y;
        double a = 0.0, b = 0.0;
        if (row < m && ka < kdim) a = transA ? A[(int64_t)ka * m + row] : A[(int64_t)row * kdim + ka];
        if (kb < kdim && col < n) b = B[(int64_t)kb * n + col];
        As[threadIdx.y][threadIdx.x] = a;
        Bs[threadIdx.y][threadIdx.x] = b;
        __syncthreads();
#pragma unroll
        for (int t = 0; t < TILE; t++) acc += As[threadIdx.y][t] * Bs[t][threadIdx.x];
        __syncthreads();
    }
    if (row < m && col < n) {
        if (D) acc += beta * D[(int64_t)row * n + col];
        C[(int64_t)row * n + col] = acc;
    }
}

static int gemm(amgh_problem *p, int m, int n, int k, const double *A, int transA, const double *B, double beta,
                const double *D, double *C, int lower)
{
    dim3 blk(TILE, TILE), grd(ceil_div(n, TILE), ceil_div(m, TILE));
    k_gemm<<<grd, blk, 0, p->stream>>>(m, n, k, A, transA, B, beta, D, C, lower);
    LAUNCH_CHECK();
    return AMGH_OK;
}

// C = W^T W for lower-triangular W (so C is symmetric): upper tiles only, the
// sum over k starting where both columns of W can be non-zero; then mirrored
__global__ void k_wtw_upper(int n, const double *__restrict__ W, double *__restrict__ C)
{
    __shared__ double As[TILE][TILE + 1], Bs[TILE][TILE + 1];
    if (blockIdx.y > blockIdx.x) return; // block-uniform: lower tiles come from the mirror
    int row = blockIdx.y * TILE + threadIdx.y, col = blockIdx.x * TILE + threadIdx.x;
    double acc = 0.0;
    // W[k][row] = 0 for k < row and W[k][col] = 0 for k < col
    for (int k0 = blockIdx.x * TILE; k0 < n; k0 += TILE) {
        int ka = k0 + threadIdx.x, kb = k0 + threadIdx.y;
        As[threadIdx.y][threadIdx.x] = row < n && ka < n ? W[(int64_t)ka * n + row] : 0.0;
        Bs[threadIdx.y][threadIdx.x] = kb < n && col < n ? W[(int64_t)kb * n + col] : 0.0;
        __syncthreads();
#pragma unroll
        for (int t = 0; t < TILE; t++) acc += As[threadIdx.y][t] * Bs[t][threadIdx.x];
        __syncthreads();
    }
    if (row < n && col < n && col >= row) C[(int64_t)row * n + col] = acc;
}

__global__ void k_mirror_lower(int n, double *__restrict__ C)
{
    int i = blockIdx.y * blockDim.y + threadIdx.y, j = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && j < i) C[(int64_t)i * n + j] = C[(int64_t)j * n + i];
}

// C = S op(D): S sparse (CSR, rows x inner), D dense row-major with leading
// dimension ld; transD = 0: D is inner x cols, 1: D is cols x inner (used as D^T)
__global__ void k_csr_dense(int rows, int cols, const int *__restrict__ rp, const int *__restrict__ ci,
                            const double *__restrict__ v, const double *__restrict__ D, int ld, int transD,
                            double *__restrict__ C)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
    if (j >= cols) return;
    double acc = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; k++) {
        int l = ci[k];
        acc += v[k] * (transD ? D[(int64_t)j * ld + l] : D[(int64_t)l * ld + j]);
    }
    C[(int64_t)i * cols + j] = acc;
}

static int csr_dense(amgh_problem *p, const DevCsr &a, const double *D, int ld, int cols, int transD, double *C)
{
    if (a.rows == 0 || cols == 0) return AMGH_OK;
    k_csr_dense<<<dim3(ceil_div(cols, 128), a.rows), 128, 0, p->stream>>>(a.rows, cols, a.rp, a.ci, a.v, D, ld,
                                                                          transD, C);
    LAUNCH_CHECK();
    return AMGH_OK;
}

// the inverse of the SPD matrix in g (n x n, lower triangle read, overwritten)
// into inv on stream s; *info_host (if given) gets the 1-based row of the
// first pivot that was not positive, 0 if none
static int spd_inverse_on(cudaStream_t s, double *g, int n, double *inv, int *info_dev, int *info_host)
{
    if (n <= 0) return AMGH_OK;
    Scratch sc;
    double *W = nullptr, *dinv = nullptr, *ybuf = nullptr;
    TRY(sc.alloc(&W, (int64_t)n * n));
    TRY(sc.alloc(&dinv, (int64_t)ceil_div(n, NB) * NB * NB));
    TRY(sc.alloc(&ybuf, (int64_t)NB * n));
    CU(cudaMemsetAsync(info_dev, 0, sizeof(int), s));
    CU(cudaMemsetAsync(W, 0, sizeof(double) * (size_t)n * n, s));
    k_potrf_diag<<<1, 128, 0, s>>>(n, 0, g, dinv, info_dev);
    LAUNCH_CHECK();
    for (int k0 = 0; k0 < n; k0 += NB) {
        int nb = n - k0 < NB ? n - k0 : NB, m = n - k0 - nb;
        int rb = ceil_div(m, PANEL_WARPS);
        k_panel<<<rb + (k0 / NB + 1) * (NB / PANEL_WARPS), 32 * PANEL_WARPS, 0, s>>>(n, k0, rb, g, dinv, W, ybuf);
        LAUNCH_CHECK();
        int T = ceil_div(m, 16), tw = ceil_div(k0 + nb, 16), ta = T > 2 ? (T - 2) * (T - 1) / 2 : 0;
        int cb = ceil_div((int64_t)nb * (k0 + nb), COPY_TPB);
        if (m > 0) {
            k_trail_next<<<T > 1 ? 2 * T - 1 : 1, 256, 0, s>>>(n, k0, T, g);
            LAUNCH_CHECK();
        }
        k_trail_rest<<<1 + ta + T * tw + cb, 256, 0, s>>>(n, k0, T, ta, tw, g, W, ybuf, dinv, info_dev);
        LAUNCH_CHECK();
    }
    // A^-1 = L^-T L^-1 = W^T W
    int tiles = ceil_div(n, TILE);
    k_wtw_upper<<<dim3(tiles, tiles), dim3(TILE, TILE), 0, s>>>(n, W, inv);
    LAUNCH_CHECK();
    k_mirror_lower<<<dim3(tiles, tiles), dim3(TILE, TILE), 0, s>>>(n, inv);
    LAUNCH_CHECK();
    int info = 0;
    CU(cudaMemcpyAsync(&info, info_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (info_host) *info_host = info;
    return info ? AMGH_ERR_INDEFINITE : AMGH_OK;
}

int dense_spd_inverse(amgh_problem *p, double *g, int n, double *inv, int *info_dev)
{
    return spd_inverse_on(p->stream, g, n, inv, info_dev, nullptr);
}

extern "C" int amgh_dense_spd_inverse(int n, const double *a_dev, double *inv_dev, void *stream, int *info)
{
    if (info) *info = 0;
    if (n <= 0 || n > AMGH_DENSE_MAX || !a_dev || !inv_dev) return AMGH_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    StreamScope ss(s);
    Scratch sc;
    double *g = nullptr;
    int *info_dev = nullptr;
    TRY(sc.alloc(&g, (int64_t)n * n));
    TRY(sc.alloc(&info_dev, 1));
    CU(cudaMemcpyAsync(g, a_dev, sizeof(double) * (size_t)n * n, cudaMemcpyDeviceToDevice, s));
    return spd_inverse_on(s, g, n, inv_dev, info_dev, info);
}

// H_c on Hessian level c and its inverse (hinv, n_c x n_c).  With W =
// M_yu^T A_c^-1 (sparse times dense) and U = M_y W^T (sparse times dense),
// H_c = W U + beta M_u: one dense product instead of four.
int dense_coarse_hessian(amgh_problem *p, int c, const double *ainv, double *hinv)
{
    StateLevel &S = p->sl[c];
    CtrlLevel &C = p->cl[c];
    int m = S.A.rows, n = C.Mu.rows;
    Scratch sc;
    double *W, *U, *Mu, *H;
    int *info;
    TRY(sc.alloc(&W, (int64_t)n * m));
    TRY(sc.alloc(&U, (int64_t)m * n));
    TRY(sc.alloc(&Mu, (int64_t)n * n));
    TRY(sc.alloc(&H, (int64_t)n * n));
    TRY(sc.alloc(&info, 1));
    TRY(dense_from_csr(p, C.Mu, Mu));
    TRY(csr_dense(p, C.Myut, ainv, m, m, 0, W)); // W = M_yu^T A^-1   (n x m)
    TRY(csr_dense(p, S.My, W, m, n, 1, U));      // U = M_y W^T       (m x n)
    TRY(gemm(p, n, n, m, W, 0, U, p->beta, Mu, H, 1)); // H = W U + beta M_u, lower triangle
    return dense_spd_inverse(p, H, n, hinv, info);
}
