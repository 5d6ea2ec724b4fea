// dense.cu -- dense coarsest-level operators (at most 4096 rows):
//   * the explicit inverse of the coarsest AMG matrix A_{L-1} (the exact
//     coarse solve of the V-cycle), applied as one GEMV (an FP32 copy serves
//     the FP32 V-cycles);
//   * the dense coarsest Hessian H_c = M_yu^T A_c^-1 M_y A_c^-1 M_yu + beta M_u
//     on Hessian level l-1 and its explicit inverse -- the exact coarsest
//     inverse G_{l-1}^-1 assumed by the theory (Sec. 3.2).
// Both inverses come from a blocked right-looking Cholesky factorisation
// A = L L^T (INDEFINITE if a pivot is not positive), the triangular inverse
// W = L^-1 computed column by column (one warp per column) and A^-1 = W^T W
// (upper triangle only, then mirrored).  All FP64 on CUDA cores.
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

// Blocked right-looking Cholesky with NB-wide panels (lower triangle, row-major):
// for each panel k: factor the NB x NB diagonal block in shared memory, solve
// the panel below it (L_ik L_kk^T = A_ik, one thread per row), and subtract
// L_ik L_jk^T from the trailing lower triangle.
#define NB 32

__global__ void k_potrf_diag(int n, int k0, double *__restrict__ g, int *__restrict__ info)
{
    __shared__ double a[NB][NB + 1];
    int nb = min(NB, n - k0);
    int t = threadIdx.x;
    for (int e = t; e < nb * nb; e += blockDim.x) a[e / nb][e % nb] = g[(int64_t)(k0 + e / nb) * n + k0 + e % nb];
    __syncthreads();
    for (int j = 0; j < nb; j++) {
        if (t == 0) {
            double d = a[j][j];
            if (!(d > 0.0)) {
                atomicCAS(info, 0, k0 + j + 1);
                d = 1.0;
            }
            a[j][j] = sqrt(d);
        }
        __syncthreads();
        double ljj = a[j][j];
        for (int i = j + 1 + t; i < nb; i += blockDim.x) a[i][j] /= ljj;
        __syncthreads();
        for (int e = t; e < (nb - j - 1) * (nb - j - 1); e += blockDim.x) {
            int i = j + 1 + e / (nb - j - 1), c = j + 1 + e % (nb - j - 1);
            if (c <= i) a[i][c] -= a[i][j] * a[c][j];
        }
        __syncthreads();
    }
    for (int e = t; e < nb * nb; e += blockDim.x) {
        int i = e / nb, c = e % nb;
        g[(int64_t)(k0 + i) * n + k0 + c] = c <= i ? a[i][c] : 0.0;
    }
}

// rows i >= k0 + NB: solve x L_kk^T = g[i, k0:k0+nb] by forward substitution,
// one warp per row: lane c holds x_c's running value and subtracts
// x_q l_cq for q = 0, 1, ... in order, x_q broadcast from lane q when final
#define TRSM_WARPS 8
__global__ void k_trsm_panel(int n, int k0, double *__restrict__ g)
{
    __shared__ double l[NB][NB + 1];
    int nb = min(NB, n - k0);
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) l[e / nb][e % nb] = g[(int64_t)(k0 + e / nb) * n + k0 + e % nb];
    __syncthreads();
    int lane = threadIdx.x & 31;
    int i = k0 + nb + blockIdx.x * TRSM_WARPS + (threadIdx.x >> 5);
    if (i >= n) return; // warp-uniform
    double *row = g + (int64_t)i * n + k0;
    double sc = lane < nb ? row[lane] : 0.0;
    for (int q = 0; q < nb; q++) {
        double xq = __shfl_sync(0xffffffffu, sc / l[q][q], q); // final on lane q
        if (lane == q) sc = xq;
        if (lane > q && lane < nb) sc -= xq * l[lane][q];
    }
    if (lane < nb) row[lane] = sc;
}

// trailing update g[i][j] -= sum_c L[i][k0+c] L[j][k0+c] for k0+nb <= j <= i (16x16 tiles)
__global__ void k_syrk_update(int n, int k0, double *__restrict__ g)
{
    __shared__ double Ai[16][NB + 1], Aj[16][NB + 1];
    int nb = min(NB, n - k0);
    int base = k0 + nb;
    int ti = blockIdx.y * 16, tj = blockIdx.x * 16;
    if (tj > ti) return; // upper tiles untouched (block-uniform)
    int t = threadIdx.y * 16 + threadIdx.x;
    for (int e = t; e < 16 * nb; e += 256) {
        int r = e / nb, c = e % nb;
        int gi = base + ti + r, gj = base + tj + r;
        Ai[r][c] = gi < n ? g[(int64_t)gi * n + k0 + c] : 0.0;
        Aj[r][c] = gj < n ? g[(int64_t)gj * n + k0 + c] : 0.0;
    }
    __syncthreads();
    int i = base + ti + threadIdx.y, j = base + tj + threadIdx.x;
    if (i >= n || j > i) return;
    double s = 0.0;
    for (int c = 0; c < nb; c++) s += Ai[threadIdx.y][c] * Aj[threadIdx.x][c];
    g[(int64_t)i * n + j] -= s;
}

// column k of W = L^-1 (one warp per column): w_k = 1 / l_kk and, for i > k,
// w_i = -(sum_{k <= j < i} l_ij w_j) / l_ii; the column is kept in shared memory
#define TRINV_WARPS 4
__global__ void k_trinv(int n, const double *__restrict__ L, double *__restrict__ W)
{
    extern __shared__ double wsh[];
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int k = blockIdx.x * TRINV_WARPS + warp;
    if (k >= n) return; // warp-uniform
    double *w = wsh + (int64_t)warp * n;
    if (lane == 0) w[k] = 1.0 / L[(int64_t)k * n + k];
    __syncwarp();
    for (int i = k + 1; i < n; i++) {
        const double *row = L + (int64_t)i * n;
        double s = 0.0;
        for (int j = k + lane; j < i; j += 32) s += row[j] * w[j];
        s = warp_sum(s);
        if (lane == 0) w[i] = -s / row[i];
        __syncwarp();
    }
    for (int i = lane; i < n; i += 32) W[(int64_t)i * n + k] = i >= k ? w[i] : 0.0;
}

// C = op(A) B (+ beta D), all row-major; transA: A is k x m and used as A^T
#define TILE 16
__global__ void k_gemm(int m, int n, int kdim, const double *__restrict__ A, int transA,
                       const double *__restrict__ B, double beta, const double *__restrict__ D,
                       double *__restrict__ C)
{
    __shared__ double As[TILE][TILE + 1], Bs[TILE][TILE + 1];
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
                const double *D, double *C)
{
    dim3 blk(TILE, TILE), grd(ceil_div(n, TILE), ceil_div(m, TILE));
    k_gemm<<<grd, blk, 0, p->stream>>>(m, n, k, A, transA, B, beta, D, C);
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

int dense_spd_inverse(amgh_problem *p, double *g, int n, double *inv, int *info_dev)
{
    cudaStream_t s = p->stream;
    CU(cudaMemsetAsync(info_dev, 0, sizeof(int), s));
    for (int k0 = 0; k0 < n; k0 += NB) {
        k_potrf_diag<<<1, 256, 0, s>>>(n, k0, g, info_dev);
        LAUNCH_CHECK();
        int rest = n - k0 - NB;
        if (rest > 0) {
            k_trsm_panel<<<ceil_div(rest, TRSM_WARPS), 32 * TRSM_WARPS, 0, s>>>(n, k0, g);
            LAUNCH_CHECK();
            int tiles = ceil_div(rest, 16);
            k_syrk_update<<<dim3(tiles, tiles), dim3(16, 16), 0, s>>>(n, k0, g);
            LAUNCH_CHECK();
        }
    }
    int info = 0;
    CU(cudaMemcpyAsync(&info, info_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (info) return AMGH_ERR_INDEFINITE;
    // A^-1 = L^-T L^-1 = W^T W
    Scratch sc;
    double *W = nullptr;
    TRY(sc.alloc(&W, (int64_t)n * n));
    size_t shm = sizeof(double) * (size_t)n * TRINV_WARPS;
    // per-function limit, set to the largest case (n <= AMGH_DENSE_MAX) so that
    // setups on several host threads never lower it under one another
    CU(cudaFuncSetAttribute(k_trinv, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)(sizeof(double) * (size_t)AMGH_DENSE_MAX * TRINV_WARPS)));
    k_trinv<<<ceil_div(n, TRINV_WARPS), 32 * TRINV_WARPS, shm, s>>>(n, g, W);
    LAUNCH_CHECK();
    int tiles = ceil_div(n, TILE);
    k_wtw_upper<<<dim3(tiles, tiles), dim3(TILE, TILE), 0, s>>>(n, W, inv);
    LAUNCH_CHECK();
    k_mirror_lower<<<dim3(tiles, tiles), dim3(TILE, TILE), 0, s>>>(n, inv);
    LAUNCH_CHECK();
    CU(cudaStreamSynchronize(s));
    return AMGH_OK;
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
    TRY(gemm(p, n, n, m, W, 0, U, p->beta, Mu, H)); // H = W U + beta M_u
    return dense_spd_inverse(p, H, n, hinv, info);
}
