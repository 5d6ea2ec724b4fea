// dense.cu -- dense coarsest-level operators (at most 4096 rows):
//   * the explicit inverse of the coarsest AMG matrix A_{L-1} (the exact
//     coarse solve of the V-cycle), applied as one GEMV;
//   * the dense coarsest Hessian H_c = M_yu^T A_c^-1 M_y A_c^-1 M_yu + beta M_u
//     on Hessian level l-1 and its explicit inverse -- the exact coarsest
//     inverse G_{l-1}^-1 assumed by the theory (Sec. 3.2).
// Both inverses come from a right-looking Cholesky factorisation A = L L^T
// (INDEFINITE if a pivot is not positive), the triangular inverse W = L^-1
// computed column by column (one block per column) and A^-1 = W^T W.
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

// column j: pivot and scaling (one block)
__global__ void k_chol_col(int n, int j, double *__restrict__ g, int *__restrict__ info)
{
    __shared__ double ljj;
    if (threadIdx.x == 0) {
        double s = g[(int64_t)j * n + j];
        if (!(s > 0.0)) {
            *info = j + 1;
            s = 1.0;
        }
        ljj = sqrt(s);
        g[(int64_t)j * n + j] = ljj;
    }
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) g[(int64_t)i * n + j] /= ljj;
}

// trailing update of the lower triangle: g_ik -= l_ij l_kj for j < k <= i
__global__ void k_chol_update(int n, int j, double *__restrict__ g)
{
    int64_t m = n - j - 1;
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m * m) return;
    int i = j + 1 + (int)(t / m), k = j + 1 + (int)(t % m);
    if (k > i) return;
    g[(int64_t)i * n + k] -= g[(int64_t)i * n + j] * g[(int64_t)k * n + j];
}

// column k of W = L^-1 (one block per column): w_k = 1 / l_kk and, for i > k,
// w_i = -(sum_{k <= j < i} l_ij w_j) / l_ii, the column kept in shared memory
__global__ void k_trinv(int n, const double *__restrict__ L, double *__restrict__ W)
{
    extern __shared__ double w[];
    __shared__ double sh32[32];
    int k = blockIdx.x;
    if (threadIdx.x == 0) w[k] = 1.0 / L[(int64_t)k * n + k];
    __syncthreads();
    for (int i = k + 1; i < n; i++) {
        const double *row = L + (int64_t)i * n;
        double s = 0.0;
        for (int j = k + threadIdx.x; j < i; j += blockDim.x) s += row[j] * w[j];
        s = block_sum(s, sh32);
        if (threadIdx.x == 0) w[i] = -s / row[i];
        __syncthreads();
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) W[(int64_t)i * n + k] = i >= k ? w[i] : 0.0;
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

int dense_spd_inverse(amgh_problem *p, double *g, int n, double *inv, int *info_dev)
{
    cudaStream_t s = p->stream;
    CU(cudaMemsetAsync(info_dev, 0, sizeof(int), s));
    for (int j = 0; j < n; j++) {
        k_chol_col<<<1, 256, 0, s>>>(n, j, g, info_dev);
        LAUNCH_CHECK();
        int64_t m = n - j - 1;
        if (m > 0) {
            k_chol_update<<<ceil_div(m * m, 256), 256, 0, s>>>(n, j, g);
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
    k_trinv<<<n, 256, sizeof(double) * n, s>>>(n, g, W);
    LAUNCH_CHECK();
    TRY(gemm(p, n, n, n, W, 1, W, 0.0, nullptr, inv));
    CU(cudaStreamSynchronize(s));
    return AMGH_OK;
}

// H_c on Hessian level c and its inverse (hinv, n_c x n_c)
int dense_coarse_hessian(amgh_problem *p, int c, const double *ainv, double *hinv)
{
    StateLevel &S = p->sl[c];
    CtrlLevel &C = p->cl[c];
    int m = S.A.rows, n = C.Mu.rows;
    Scratch sc;
    double *Myu, *My, *Mu, *X, *Y, *Z, *H;
    int *info;
    TRY(sc.alloc(&Myu, (int64_t)m * n));
    TRY(sc.alloc(&My, (int64_t)m * m));
    TRY(sc.alloc(&Mu, (int64_t)n * n));
    TRY(sc.alloc(&X, (int64_t)m * n));
    TRY(sc.alloc(&Y, (int64_t)m * n));
    TRY(sc.alloc(&Z, (int64_t)m * n));
    TRY(sc.alloc(&H, (int64_t)n * n));
    TRY(sc.alloc(&info, 1));
    TRY(dense_from_csr(p, C.Myu, Myu));
    TRY(dense_from_csr(p, S.My, My));
    TRY(dense_from_csr(p, C.Mu, Mu));
    TRY(gemm(p, m, n, m, ainv, 0, Myu, 0.0, nullptr, X));        // X = A^-1 M_yu
    TRY(gemm(p, m, n, m, My, 0, X, 0.0, nullptr, Y));            // Y = M_y X
    TRY(gemm(p, m, n, m, ainv, 0, Y, 0.0, nullptr, Z));          // Z = A^-1 Y
    TRY(gemm(p, n, n, m, Myu, 1, Z, p->beta, Mu, H));            // H = M_yu^T Z + beta M_u
    return dense_spd_inverse(p, H, n, hinv, info);
}
