// block.cu -- block (multi-column) solves: many desired states of one control
// problem, or many vectors of one operator, advanced together.
//
// K columns (K = 2, 4 or 8; a short last block is padded with zero columns)
// are stored interleaved -- entry i of column c at i*K + c -- so every row of
// a sparse operator is read once for all K columns and the K values gathered
// per column index are one contiguous 4K- or 8K-byte load: SpMM instead of K
// SpMVs, and one launch instead of K.
//
// Per column the method is the single-column one: the same single-reduction
// PCG for the state and adjoint solves (AMG V-cycle preconditioner) and for
// the mass solves (Jacobi), the same V-cycle, the multilevel preconditioner of
// Algorithm MLAS (Sec. 3.2, in the M_u-scaled form of Sec. 5.2) and the outer
// CG of Sec. 5.3.  Every column keeps its own CG scalars and stopping test; a
// column that has stopped is not updated again, and every launch of an inner
// CG loop returns at once when all its columns have stopped, so iterations
// are replayed from CUDA graphs in chunks as in the single-column solver.  A
// column that fails (indefinite, non-finite, cap reached) is marked failed and
// dropped; the other columns carry on.
//
// Precision: precision 0 runs FP64 V-cycles and an FP64 CG, as the
// single-column FP64 path; precisions 1 and 2 run FP32 V-cycles and a
// double-float CG as the single-column double-float path: vectors, updates,
// operator products A z and M z (from A = A_hi + A_lo) and reductions on the
// FP32 pipe, which on GB300 is about 64 times wider than the FP64 one (the
// refinement form of precision 1 has no block variant).  The control-side
// operators (M_yu, M_y, M_u, P and their transposes) and the outer CG are
// applied in FP64.
#include <math.h>
#include <string.h>

#include <functional>

#include "internal.cuh"
#include "spmv.cuh"
#include "util.cuh"

#define KB AMGH_BLOCK_MAX

static const int TPB = 256;
#define TPB_K 256 // threads per block of every block kernel that reduces

static inline int vblocks(int64_t n)
{
    int nb = ceil_div(n > 0 ? n : 1, TPB);
    return nb < 2432 ? nb : 2432; // 152 SMs x 16 blocks of 256 threads
}

// per-column CG scalars of one block loop
struct BScal {
    CgScal c[KB];
    int all; // every column has stopped
    int pad[3];
};

// ------------------------------------------------------------------ K-vectors
// K consecutive values of one row; the base is 4K- or 8K-byte aligned (block
// buffers come from the pool, 256-byte aligned, and rows are K values apart)
template <int K>
__device__ __forceinline__ void ldk(const float *p, float (&v)[K])
{
    if constexpr (K % 4 == 0) {
#pragma unroll
        for (int i = 0; i < K / 4; i++) {
            float4 w = reinterpret_cast<const float4 *>(p)[i];
            v[4 * i] = w.x;
            v[4 * i + 1] = w.y;
            v[4 * i + 2] = w.z;
            v[4 * i + 3] = w.w;
        }
    } else if constexpr (K % 2 == 0) {
#pragma unroll
        for (int i = 0; i < K / 2; i++) {
            float2 w = reinterpret_cast<const float2 *>(p)[i];
            v[2 * i] = w.x;
            v[2 * i + 1] = w.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < K; i++) v[i] = p[i];
    }
}

template <int K>
__device__ __forceinline__ void ldk(const double *p, double (&v)[K])
{
    if constexpr (K % 2 == 0) {
#pragma unroll
        for (int i = 0; i < K / 2; i++) {
            double2 w = reinterpret_cast<const double2 *>(p)[i];
            v[2 * i] = w.x;
            v[2 * i + 1] = w.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < K; i++) v[i] = p[i];
    }
}

// read-only gathers (the source is not written by the same kernel)
template <int K>
__device__ __forceinline__ void ldk_ro(const float *p, float (&v)[K])
{
    if constexpr (K % 4 == 0) {
#pragma unroll
        for (int i = 0; i < K / 4; i++) {
            float4 w = __ldg(reinterpret_cast<const float4 *>(p) + i);
            v[4 * i] = w.x;
            v[4 * i + 1] = w.y;
            v[4 * i + 2] = w.z;
            v[4 * i + 3] = w.w;
        }
    } else if constexpr (K % 2 == 0) {
#pragma unroll
        for (int i = 0; i < K / 2; i++) {
            float2 w = __ldg(reinterpret_cast<const float2 *>(p) + i);
            v[2 * i] = w.x;
            v[2 * i + 1] = w.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < K; i++) v[i] = __ldg(p + i);
    }
}

template <int K>
__device__ __forceinline__ void ldk_ro(const double *p, double (&v)[K])
{
    if constexpr (K % 2 == 0) {
#pragma unroll
        for (int i = 0; i < K / 2; i++) {
            double2 w = __ldg(reinterpret_cast<const double2 *>(p) + i);
            v[2 * i] = w.x;
            v[2 * i + 1] = w.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < K; i++) v[i] = __ldg(p + i);
    }
}

// loads through L2 (ld.global.cg): vectors that other blocks of the same
// launch have written (the persistent kernel; L1 is not coherent across SMs)
template <int K>
__device__ __forceinline__ void ldk_cg(const float *p, float (&v)[K])
{
    if constexpr (K % 4 == 0) {
#pragma unroll
        for (int i = 0; i < K / 4; i++) {
            float4 w = __ldcg(reinterpret_cast<const float4 *>(p) + i);
            v[4 * i] = w.x;
            v[4 * i + 1] = w.y;
            v[4 * i + 2] = w.z;
            v[4 * i + 3] = w.w;
        }
    } else if constexpr (K % 2 == 0) {
#pragma unroll
        for (int i = 0; i < K / 2; i++) {
            float2 w = __ldcg(reinterpret_cast<const float2 *>(p) + i);
            v[2 * i] = w.x;
            v[2 * i + 1] = w.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < K; i++) v[i] = __ldcg(p + i);
    }
}

template <int K>
__device__ __forceinline__ void stk(float *p, const float (&v)[K])
{
    if constexpr (K % 4 == 0) {
#pragma unroll
        for (int i = 0; i < K / 4; i++)
            reinterpret_cast<float4 *>(p)[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
    } else if constexpr (K % 2 == 0) {
#pragma unroll
        for (int i = 0; i < K / 2; i++) reinterpret_cast<float2 *>(p)[i] = make_float2(v[2 * i], v[2 * i + 1]);
    } else {
#pragma unroll
        for (int i = 0; i < K; i++) p[i] = v[i];
    }
}

template <int K>
__device__ __forceinline__ void stk(double *p, const double (&v)[K])
{
    if constexpr (K % 2 == 0) {
#pragma unroll
        for (int i = 0; i < K / 2; i++) reinterpret_cast<double2 *>(p)[i] = make_double2(v[2 * i], v[2 * i + 1]);
    } else {
#pragma unroll
        for (int i = 0; i < K; i++) p[i] = v[i];
    }
}

// Rows of at most ROW_UNROLL entries per lane: every value and index load is
// issued first, then the gathers in chunks of U entries (U * K values held
// at once), then the sums in entry order -- two or three memory round trips
// per row instead of one per entry.  Longer rows take the plain loop.
template <typename T, int K>
struct Chunk {
    static constexpr int U = (int)sizeof(T) * K <= 32 ? ROW_UNROLL : ROW_UNROLL / 2;
};

// row of A times K columns of x; every lane of the group returns the K sums
template <typename T, int TPR, int K>
__device__ __forceinline__ void row_sum_k(const MatView<T> &m, int row, const T *__restrict__ x, T (&acc)[K])
{
    constexpr int STEP = TPR == 1 ? 32 : TPR;
    constexpr int U = Chunk<T, K>::U;
#pragma unroll
    for (int c = 0; c < K; c++) acc[c] = (T)0;
    if (row < m.rows) {
        int k, end;
        lane_range<T, TPR>(m, row, k, end);
        if (m.wmax <= ROW_UNROLL) {
            T vv[ROW_UNROLL];
            int cc[ROW_UNROLL];
#pragma unroll
            for (int j = 0; j < ROW_UNROLL; j++) {
                bool ok = k + STEP * j < end;
                vv[j] = ok ? m.v[k + STEP * j] : (T)0;
                cc[j] = ok ? col_of(m, row, k + STEP * j) : -1;
            }
#pragma unroll
            for (int j0 = 0; j0 < ROW_UNROLL; j0 += U) {
                T xv[U][K];
#pragma unroll
                for (int j = 0; j < U; j++) {
                    if (cc[j0 + j] >= 0) ldk_ro<K>(x + (int64_t)cc[j0 + j] * K, xv[j]);
                    else {
#pragma unroll
                        for (int c = 0; c < K; c++) xv[j][c] = (T)0;
                    }
                }
#pragma unroll
                for (int j = 0; j < U; j++) {
                    if (cc[j0 + j] < 0) continue;
#pragma unroll
                    for (int c = 0; c < K; c++) acc[c] = rfma(vv[j0 + j], xv[j][c], acc[c]);
                }
            }
        } else {
#pragma unroll 2
            for (; k < end; k += STEP) {
                T a = m.v[k];
                T xv[K];
                ldk_ro<K>(x + (int64_t)col_of(m, row, k) * K, xv);
#pragma unroll
                for (int c = 0; c < K; c++) acc[c] = rfma(a, xv[c], acc[c]);
            }
        }
    }
    if (TPR > 1) {
#pragma unroll
        for (int c = 0; c < K; c++) {
#pragma unroll
            for (int o = TPR / 2; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o, TPR);
        }
    }
}

// row of (A_hi + A_lo) times K columns of z, accumulated in double-float;
// every lane of the group returns the K normalised sums
template <typename Z, int TPR, int K, bool CG = false>
__device__ __forceinline__ void row_sum_df_k(const MatView<float> &m, const float *__restrict__ lo, int row,
                                             const Z *__restrict__ z, DF (&out)[K])
{
    // CG: z is written by other blocks of the same launch: gathers through L2
    constexpr int STEP = TPR == 1 ? 32 : TPR;
    // K = 8 double-float accumulators already take 16 registers: gather in half chunks
    constexpr int U = K >= 8 ? ROW_UNROLL / 2 : Chunk<Z, K>::U;
    DF acc[K];
#pragma unroll
    for (int c = 0; c < K; c++) acc[c] = DF{0.f, 0.f};
    if (row < m.rows) {
        int k, end;
        lane_range<float, TPR>(m, row, k, end);
        if (m.wmax <= ROW_UNROLL) {
            float vh[ROW_UNROLL], vl[ROW_UNROLL];
            int cc[ROW_UNROLL];
#pragma unroll
            for (int j = 0; j < ROW_UNROLL; j++) {
                bool ok = k + STEP * j < end;
                vh[j] = ok ? m.v[k + STEP * j] : 0.f;
                vl[j] = ok ? lo[k + STEP * j] : 0.f;
                cc[j] = ok ? col_of(m, row, k + STEP * j) : -1;
            }
#pragma unroll
            for (int j0 = 0; j0 < ROW_UNROLL; j0 += U) {
                Z zv[U][K];
#pragma unroll
                for (int j = 0; j < U; j++) {
                    if (cc[j0 + j] >= 0) {
                        if constexpr (CG) ldk_cg<K>(z + (int64_t)cc[j0 + j] * K, zv[j]);
                        else ldk_ro<K>(z + (int64_t)cc[j0 + j] * K, zv[j]);
                    } else {
#pragma unroll
                        for (int c = 0; c < K; c++) zv[j][c] = (Z)0;
                    }
                }
#pragma unroll
                for (int j = 0; j < U; j++) {
                    if (cc[j0 + j] < 0) continue;
#pragma unroll
                    for (int c = 0; c < K; c++) df_term<Z>(acc[c], vh[j0 + j], vl[j0 + j], zv[j][c]);
                }
            }
        } else {
#pragma unroll 2
            for (; k < end; k += STEP) {
                float ah = m.v[k], al = lo[k];
                Z zv[K];
                if constexpr (CG) ldk_cg<K>(z + (int64_t)col_of(m, row, k) * K, zv);
                else ldk_ro<K>(z + (int64_t)col_of(m, row, k) * K, zv);
#pragma unroll
                for (int c = 0; c < K; c++) df_term<Z>(acc[c], ah, al, zv[c]);
            }
        }
    }
    if (TPR > 1) {
#pragma unroll
        for (int c = 0; c < K; c++) {
#pragma unroll
            for (int o = TPR / 2; o > 0; o >>= 1) {
                DF other = {__shfl_xor_sync(0xffffffffu, acc[c].hi, o, TPR),
                            __shfl_xor_sync(0xffffffffu, acc[c].lo, o, TPR)};
                df_merge(acc[c], other);
            }
        }
    }
#pragma unroll
    for (int c = 0; c < K; c++) quick_two_sum(acc[c].hi, acc[c].lo, out[c].hi, out[c].lo);
}

// ------------------------------------------------------------------ reductions
// Two-stage deterministic sum of NV values per thread over the grid (blocks of
// TPB threads).  Inside a block the values go through shared memory and warp
// w sums values w, w + 8, ... (fewer FP64 adds than NV butterflies); block
// partials ([NV][gridDim.x]) are summed in fixed order by the last block to
// finish, which issues all NV loads of a pass together.  Returns true in
// thread 0 of that block, with the sums in tot.
template <int NV>
__device__ bool reduce_k(const double (&val)[NV], double *partials, unsigned *ticket, double (&tot)[NV])
{
    __shared__ double sh[NV][TPB_K];
    __shared__ double stot[NV];
    __shared__ bool is_last;
    const int t = threadIdx.x, w = t >> 5, l = t & 31, nb = gridDim.x;
#pragma unroll
    for (int q = 0; q < NV; q++) sh[q][t] = val[q];
    __syncthreads();
    for (int q = w; q < NV; q += TPB_K / 32) {
        double s = 0.0;
#pragma unroll
        for (int j = l; j < TPB_K; j += 32) s += sh[q][j];
        s = warp_sum(s);
        if (l == 0) partials[q * nb + blockIdx.x] = s;
    }
    __threadfence();
    __syncthreads();
    if (t == 0) is_last = atomicAdd(ticket, 1u) == (unsigned)nb - 1;
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
    double s[NV];
#pragma unroll
    for (int q = 0; q < NV; q++) s[q] = 0.0;
    for (int b = t; b < nb; b += TPB_K) {
#pragma unroll
        for (int q = 0; q < NV; q++) s[q] += __ldcg(&partials[q * nb + b]);
    }
#pragma unroll
    for (int q = 0; q < NV; q++) sh[q][t] = s[q];
    __syncthreads();
    for (int q = w; q < NV; q += TPB_K / 32) {
        double u = 0.0;
#pragma unroll
        for (int j = l; j < TPB_K; j += 32) u += sh[q][j];
        u = warp_sum(u);
        if (l == 0) stot[q] = u;
    }
    __syncthreads();
    if (t != 0) return false;
#pragma unroll
    for (int q = 0; q < NV; q++) tot[q] = stot[q];
    *ticket = 0u;
    return true;
}

// The same in double-float for the double-float block CG: values transposed
// through shared memory as in reduce_k, warps summing columns of it, block
// partials as FP32 pairs ([NV][nb]), and the last block loading all NV
// partials of a block at once.
// shared staging of NV double-float values per thread (one buffer per kernel,
// passed to both helpers below)
template <int NV>
struct DfStage {
    float hi[NV][TPB_K], lo[NV][TPB_K];
    DF tot[NV];
};

template <int NV, int NVMAX = NV>
__device__ void block_df_partials(const DF (&val)[NV], float2 *part, int nb, int bid, DfStage<NVMAX> &st)
{
    static_assert(NV <= NVMAX, "staging buffer too small");
    float(&shh)[NVMAX][TPB_K] = st.hi;
    float(&shl)[NVMAX][TPB_K] = st.lo;
    const int t = threadIdx.x, w = t >> 5, l = t & 31;
#pragma unroll
    for (int q = 0; q < NV; q++) {
        shh[q][t] = val[q].hi;
        shl[q][t] = val[q].lo;
    }
    __syncthreads();
    for (int q = w; q < NV; q += TPB_K / 32) {
        DF s = {0.f, 0.f};
#pragma unroll
        for (int j = l; j < TPB_K; j += 32) s = df_add_fast(s, DF{shh[q][j], shl[q][j]});
        s = df_warp_sum(s);
        if (l == 0) part[q * nb + bid] = make_float2(s.hi, s.lo);
    }
}

// the NV sums over the nb block partials, in fixed order; thread 0 returns them
template <int NV, int NVMAX = NV>
__device__ void sum_df_partials(const float2 *part, int nb, double (&tot)[NV], DfStage<NVMAX> &st)
{
    static_assert(NV <= NVMAX, "staging buffer too small");
    float(&shh)[NVMAX][TPB_K] = st.hi;
    float(&shl)[NVMAX][TPB_K] = st.lo;
    DF(&stot)[NVMAX] = st.tot;
    const int t = threadIdx.x, w = t >> 5, l = t & 31;
    __syncthreads(); // the staging buffer may still be read by a previous step
    DF s[NV];
#pragma unroll
    for (int q = 0; q < NV; q++) s[q] = DF{0.f, 0.f};
    for (int b = t; b < nb; b += TPB_K) {
        float2 v[NV];
#pragma unroll
        for (int q = 0; q < NV; q++) v[q] = __ldcg(&part[q * nb + b]); // L2: written by other blocks
#pragma unroll
        for (int q = 0; q < NV; q++) s[q] = df_add_fast(s[q], DF{v[q].x, v[q].y});
    }
#pragma unroll
    for (int q = 0; q < NV; q++) {
        shh[q][t] = s[q].hi;
        shl[q][t] = s[q].lo;
    }
    __syncthreads();
    for (int q = w; q < NV; q += TPB_K / 32) {
        DF u = {0.f, 0.f};
#pragma unroll
        for (int j = l; j < TPB_K; j += 32) u = df_add_fast(u, DF{shh[q][j], shl[q][j]});
        u = df_warp_sum(u);
        if (l == 0) stot[q] = u;
    }
    __syncthreads();
    if (t == 0) {
#pragma unroll
        for (int q = 0; q < NV; q++) tot[q] = df_to_double(stot[q]);
    }
}

template <int NV>
__device__ bool reduce_dfk(const DF (&val)[NV], double *partials, unsigned *ticket, double (&tot)[NV])
{
    __shared__ bool is_last;
    __shared__ DfStage<NV> st;
    const int t = threadIdx.x, nb = gridDim.x;
    float2 *part = reinterpret_cast<float2 *>(partials);
    block_df_partials<NV>(val, part, nb, blockIdx.x, st);
    __threadfence();
    __syncthreads();
    if (t == 0) is_last = atomicAdd(ticket, 1u) == (unsigned)nb - 1;
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
    sum_df_partials<NV>(part, nb, tot, st);
    if (t != 0) return false;
    *ticket = 0u;
    return true;
}

// ------------------------------------------------------------------ finalisers
__device__ __forceinline__ bool nonfinite(double x) { return !(x == x) || isinf(x); }

template <int K>
__device__ void bs_all(BScal *bs)
{
    int a = 1;
#pragma unroll
    for (int c = 0; c < K; c++) a &= bs->c[c].done != 0;
    bs->all = a;
}

// f.f per column: stopping threshold tol^2 f.f; a zero column has converged
// df: the CG runs on the right side scaled by `scale` (double-float vectors),
// so r.r and the threshold are kept in scaled units
template <int K>
__device__ void fin_start(BScal *bs, const double (&t)[K], double tol2, int maxit, bool df = false)
{
    for (int c = 0; c < K; c++) {
        CgScal &s = bs->c[c];
        double ff = t[c];
        s.ff = ff;
        s.rr = ff;
        s.thr = tol2 * ff;
        s.maxit = maxit;
        s.iters = 0;
        s.k1 = 0;
        s.alpha = 0.0;
        s.beta = 0.0;
        s.rz = 0.0;
        s.status = CG_RUNNING;
        s.done = 0;
        // power of two nearest 1 / ||f||: the FP32 V-cycle sees r scaled by it
        // (exact, and PCG is invariant under a scalar multiple of the
        // preconditioner), which keeps tiny residuals inside FP32's range
        double nrm = sqrt(ff);
        s.scale = (nrm > 0.0 && !nonfinite(nrm)) ? exp2(-rint(log2(nrm))) : 1.0;
        s.ahi = s.alo = s.bhi = s.blo = 0.f;
        if (df) {
            double s2 = s.scale * s.scale; // a power of two: exact
            s.rr = ff * s2;
            s.thr = tol2 * ff * s2;
        }
        if (nonfinite(ff)) {
            s.status = CG_NUMERIC;
            s.done = 1;
        } else if (ff == 0.0) {
            s.status = CG_CONVERGED;
            s.done = 1;
        }
    }
    bs_all<K>(bs);
}

// single-reduction PCG: gamma = (r, z), delta = (z, A z) -> alpha, beta
template <int K>
__device__ void fin_cg2(BScal *bs, const double (&t)[2 * K])
{
    for (int c = 0; c < K; c++) {
        CgScal &s = bs->c[c];
        if (s.done) continue;
        double g = t[c], d = t[K + c];
        if (!(g > 0.0) || !(d > 0.0)) {
            s.status = (nonfinite(g) || nonfinite(d)) ? CG_NUMERIC : CG_INDEFINITE;
            s.done = 1;
            continue;
        }
        double beta = 0.0, alpha;
        if (s.k1 == 0) {
            alpha = g / d;
        } else {
            beta = g / s.rz;
            double den = d - beta * g / s.alpha;
            if (!(den > 0.0)) {
                s.status = nonfinite(den) ? CG_NUMERIC : CG_INDEFINITE;
                s.done = 1;
                continue;
            }
            alpha = g / den;
        }
        s.rz = g;
        s.alpha = alpha;
        s.beta = beta;
        s.ahi = (float)alpha;
        s.alo = (float)(alpha - (double)s.ahi);
        s.bhi = (float)beta;
        s.blo = (float)(beta - (double)s.bhi);
        s.k1 += 1;
    }
    bs_all<K>(bs);
}

// r.r per column -> iteration count and stopping test
template <int K>
__device__ void fin_rr(BScal *bs, const double (&t)[K])
{
    for (int c = 0; c < K; c++) {
        CgScal &s = bs->c[c];
        if (s.done) continue;
        double rr = t[c];
        s.rr = rr;
        s.iters += 1;
        s.total_iters += 1;
        if (nonfinite(rr)) {
            s.status = CG_NUMERIC;
            s.done = 1;
        } else if (rr <= s.thr) {
            s.status = CG_CONVERGED;
            s.done = 1;
        } else if (s.iters >= s.maxit) {
            s.status = CG_MAXIT;
            s.done = 1;
        }
    }
    bs_all<K>(bs);
}

// ------------------------------------------------------------------ CG kernels
// x = 0, r = f, optionally z = invd f (Jacobi, in the type Z of z); f.f per column
template <typename Z, int K>
__global__ void kb_cg_start(int n, const double *__restrict__ f, double *__restrict__ x, double *__restrict__ r,
                            Z *__restrict__ z, const double *__restrict__ invd, BScal *bs, double tol2,
                            int maxit, double *partials, unsigned *ticket)
{
    pdl_enter();
    double v[K], tot[K];
#pragma unroll
    for (int c = 0; c < K; c++) v[c] = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int64_t o = (int64_t)i * K;
        double fv[K], zero[K];
        ldk<K>(f + o, fv);
#pragma unroll
        for (int c = 0; c < K; c++) zero[c] = 0.0;
        stk<K>(x + o, zero);
        stk<K>(r + o, fv);
        if (z) {
            double iv = invd[i];
            Z zv[K];
#pragma unroll
            for (int c = 0; c < K; c++) zv[c] = (Z)(iv * fv[c]);
            stk<K>(z + o, zv);
        }
#pragma unroll
        for (int c = 0; c < K; c++) v[c] += fv[c] * fv[c];
    }
    if (reduce_k<K>(v, partials, ticket, tot)) fin_start<K>(bs, tot, tol2, maxit);
}

// s = A z with (r, z) and (z, s) per column -> alpha, beta, in FP64 (precision 0,
// as the single-column FP64 CG)
template <int TPR, int K>
__global__ void kb_cg_spmv64(MatView<double> A, const double *__restrict__ z, const double *__restrict__ r,
                             double *__restrict__ s, BScal *bs, double *partials, unsigned *ticket)
{
    pdl_enter();
    if (bs->all) return;
    int row = my_row<TPR>();
    double sv[K];
    row_sum_k<double, TPR, K>(A, row, z, sv);
    double a[2 * K], tot[2 * K];
#pragma unroll
    for (int q = 0; q < 2 * K; q++) a[q] = 0.0;
    if (row < A.rows && row_leader<TPR>()) {
        int64_t o = (int64_t)row * K;
        stk<K>(s + o, sv);
        double zr[K], rr[K];
        ldk_ro<K>(z + o, zr);
        ldk<K>(r + o, rr);
#pragma unroll
        for (int c = 0; c < K; c++) {
            a[c] = rr[c] * zr[c];
            a[K + c] = zr[c] * sv[c];
        }
    }
    if (reduce_k<2 * K>(a, partials, ticket, tot)) fin_cg2<K>(bs, tot);
}

// FP64 CG update (precision 0): p = z + beta p, q = s + beta q, x += alpha p,
// r -= alpha q per running column; for Jacobi z = invd r; r.r per column.
// For K = 8 two threads share a row, four columns each.
template <typename Z, int K>
__global__ void kb_cg_update(int n, Z *z, const double *__restrict__ s, double *__restrict__ pv,
                             double *__restrict__ q, double *__restrict__ x, double *__restrict__ r,
                             const double *__restrict__ invd, BScal *bs, double *partials,
                             unsigned *ticket)
{
    constexpr int H = K > 4 ? 2 : 1; // threads per row
    constexpr int KH = K / H;        // columns per thread
    pdl_enter();
    if (bs->all) return;
    double v[K], tot[K];
#pragma unroll
    for (int c = 0; c < K; c++) v[c] = 0.0;
    const int64_t items = (int64_t)n * H;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t it0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // the half a thread takes is fixed (stride is even), so are its scalars
    const int h = H == 1 ? 0 : (int)(it0 & 1);
    double al[KH], be[KH];
    bool run[KH], first[KH];
#pragma unroll
    for (int c = 0; c < KH; c++) {
        const CgScal &sc = bs->c[h * KH + c];
        al[c] = sc.alpha;
        be[c] = sc.beta;
        run[c] = !sc.done;
        first[c] = sc.beta == 0.0;
    }
    double vh[KH];
#pragma unroll
    for (int c = 0; c < KH; c++) vh[c] = 0.0;
    for (int64_t it = it0; it < items; it += stride) {
        int64_t i = it / H;
        int64_t o = i * K + h * KH;
        Z zv[KH];
        double sv[KH], pp[KH], qq[KH], xx[KH], rr[KH];
        ldk<KH>(z + o, zv);
        ldk<KH>(s + o, sv);
        ldk<KH>(pv + o, pp);
        ldk<KH>(q + o, qq);
        ldk<KH>(x + o, xx);
        ldk<KH>(r + o, rr);
#pragma unroll
        for (int c = 0; c < KH; c++) {
            if (!run[c]) continue;
            double zc = (double)zv[c];
            double pc = first[c] ? zc : zc + be[c] * pp[c];
            double qc = first[c] ? sv[c] : sv[c] + be[c] * qq[c];
            pp[c] = pc;
            qq[c] = qc;
            xx[c] = xx[c] + al[c] * pc;
            rr[c] = rr[c] - al[c] * qc;
        }
        stk<KH>(pv + o, pp);
        stk<KH>(q + o, qq);
        stk<KH>(x + o, xx);
        stk<KH>(r + o, rr);
        if (invd) {
            double iv = invd[i];
            Z zn[KH];
#pragma unroll
            for (int c = 0; c < KH; c++) zn[c] = (Z)(iv * rr[c]);
            stk<KH>(z + o, zn);
        }
#pragma unroll
        for (int c = 0; c < KH; c++) vh[c] += rr[c] * rr[c];
    }
#pragma unroll
    for (int c = 0; c < KH; c++) {
        if (H == 1 || h == 0) v[c] = vh[c];
        else v[KH + c] = vh[c];
    }
    if (reduce_k<K>(v, partials, ticket, tot)) fin_rr<K>(bs, tot);
}

// ------------------------------------------------------------------ double-float CG kernels
// CG of precisions 1 and 2 (FP32 V-cycles): x, r, p, q and s are double-float,
// each FP64-sized buffer of n*K doubles used as two FP32 arrays, hi = [0, nK)
// and lo = [nK, 2nK), interleaved by column like every block vector.  The
// CG solves for the right side scaled by an exact power of two per column
// (scale, from ||f||), so the FP32 halves stay far from FP32's exponent
// limits; the V-cycle reads r's hi half as its input.  Every per-element step
// and every reduction is on the FP32 pipe, as in the single-column
// double-float CG; only the conversions from f and to x, once per solve, use
// FP64.

// 1 / s for s an exact power of two in FP64's normal range, on the bits
__device__ __forceinline__ double inv_pow2(double s)
{
    long long e = (__double_as_longlong(s) >> 52) & 0x7ff;
    return __longlong_as_double((2046ll - e) << 52);
}

// f.f per column (FP64, once per solve) -> scale and the scaled threshold
template <int K>
__global__ void kbd_norm(int n, const double *__restrict__ f, BScal *bs, double tol2, int maxit,
                         double *partials, unsigned *ticket)
{
    pdl_enter();
    double v[K], tot[K];
#pragma unroll
    for (int c = 0; c < K; c++) v[c] = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double fv[K];
        ldk<K>(f + (int64_t)i * K, fv);
#pragma unroll
        for (int c = 0; c < K; c++) v[c] = fma(fv[c], fv[c], v[c]);
    }
    if (reduce_k<K>(v, partials, ticket, tot)) fin_start<K>(bs, tot, tol2, maxit, true);
}

// r = scale_c f (split into hi/lo), x = 0; for Jacobi also z = invd r_hi
template <int K>
__global__ void kbd_start(int64_t nk, const double *__restrict__ f, float *__restrict__ xh, float *__restrict__ xl,
                          float *__restrict__ rh, float *__restrict__ rl, float *__restrict__ z,
                          const float *__restrict__ invd32, const BScal *bs)
{
    pdl_enter();
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nk; e += (int64_t)gridDim.x * blockDim.x) {
        double v = f[e] * bs->c[e & (K - 1)].scale;
        float h = (float)v, l = (float)(v - (double)h);
        rh[e] = h;
        rl[e] = l;
        xh[e] = 0.f;
        xl[e] = 0.f;
        if (z) z[e] = invd32[e / K] * h;
    }
}

// s = A z in double-float (A = A_hi + A_lo, FP32 z) with (r, z) and (z, s)
// per column -> alpha, beta
template <int TPR, int K>
__global__ void __launch_bounds__(TPB_K, 3) kbd_spmv(MatView<float> A, const float *__restrict__ lo,
                                                     const float *__restrict__ z, const float *__restrict__ rh,
                                                     const float *__restrict__ rl, float *__restrict__ sh,
                                                     float *__restrict__ sl, BScal *bs, double *partials,
                                                     unsigned *ticket)
{
    pdl_enter();
    if (bs->all) return;
    int row = my_row<TPR>();
    DF sv[K];
    row_sum_df_k<float, TPR, K>(A, lo, row, z, sv);
    DF a[2 * K];
    double tot[2 * K];
#pragma unroll
    for (int q = 0; q < 2 * K; q++) a[q] = DF{0.f, 0.f};
    if (row < A.rows && row_leader<TPR>()) {
        int64_t o = (int64_t)row * K;
        float h[K], l[K], zr[K], rhv[K], rlv[K];
#pragma unroll
        for (int c = 0; c < K; c++) {
            h[c] = sv[c].hi;
            l[c] = sv[c].lo;
        }
        stk<K>(sh + o, h);
        stk<K>(sl + o, l);
        ldk_ro<K>(z + o, zr);
        ldk<K>(rh + o, rhv);
        ldk<K>(rl + o, rlv);
#pragma unroll
        for (int c = 0; c < K; c++) {
            a[c] = df_mulf(DF{rhv[c], rlv[c]}, zr[c]);
            a[K + c] = df_mulf(sv[c], zr[c]);
        }
    }
    if (reduce_dfk<2 * K>(a, partials, ticket, tot)) fin_cg2<K>(bs, tot);
}

// p = z + beta p, q = s + beta q, x += alpha p, r -= alpha q per running
// column in double-float; with invd32 (Jacobi) z = invd r_hi; r.r per column.
// For K = 8 two threads share a row, four columns each.
template <int K>
__global__ void kbd_update(int n, float *z, const float *__restrict__ sh, const float *__restrict__ sl,
                           float *__restrict__ ph, float *__restrict__ pl, float *__restrict__ qh,
                           float *__restrict__ ql, float *__restrict__ xh, float *__restrict__ xl,
                           float *__restrict__ rh, float *__restrict__ rl, const float *__restrict__ invd32,
                           BScal *bs, double *partials, unsigned *ticket)
{
    constexpr int H = K > 4 ? 2 : 1; // threads per row
    constexpr int KH = K / H;        // columns per thread
    pdl_enter();
    if (bs->all) return;
    const int64_t items = (int64_t)n * H;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t it0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int h = H == 1 ? 0 : (int)(it0 & 1); // fixed: the stride is even
    DF al[KH], nal[KH], be[KH];
    bool run[KH], first[KH];
#pragma unroll
    for (int c = 0; c < KH; c++) {
        const CgScal &sc = bs->c[h * KH + c];
        al[c] = DF{sc.ahi, sc.alo};
        nal[c] = DF{-sc.ahi, -sc.alo};
        be[c] = DF{sc.bhi, sc.blo};
        run[c] = !sc.done;
        first[c] = sc.bhi == 0.f && sc.blo == 0.f;
    }
    DF vh[KH];
#pragma unroll
    for (int c = 0; c < KH; c++) vh[c] = DF{0.f, 0.f};
    for (int64_t it = it0; it < items; it += stride) {
        int64_t i = it / H;
        int64_t o = i * K + h * KH;
        float zv[KH], s1[KH], s2[KH], p1[KH], p2[KH], q1[KH], q2[KH], x1[KH], x2[KH], r1[KH], r2[KH];
        ldk<KH>(z + o, zv);
        ldk<KH>(sh + o, s1);
        ldk<KH>(sl + o, s2);
        ldk<KH>(ph + o, p1);
        ldk<KH>(pl + o, p2);
        ldk<KH>(qh + o, q1);
        ldk<KH>(ql + o, q2);
        ldk<KH>(xh + o, x1);
        ldk<KH>(xl + o, x2);
        ldk<KH>(rh + o, r1);
        ldk<KH>(rl + o, r2);
#pragma unroll
        for (int c = 0; c < KH; c++) {
            if (!run[c]) continue;
            DF zi = {zv[c], 0.f}, si = {s1[c], s2[c]};
            DF pi = first[c] ? zi : df_add2(zi, df_mul2(be[c], DF{p1[c], p2[c]}));
            DF qi = first[c] ? si : df_add2(si, df_mul2(be[c], DF{q1[c], q2[c]}));
            DF xi = df_add2(DF{x1[c], x2[c]}, df_mul2(al[c], pi));
            DF ri = df_add2(DF{r1[c], r2[c]}, df_mul2(nal[c], qi));
            p1[c] = pi.hi;
            p2[c] = pi.lo;
            q1[c] = qi.hi;
            q2[c] = qi.lo;
            x1[c] = xi.hi;
            x2[c] = xi.lo;
            r1[c] = ri.hi;
            r2[c] = ri.lo;
            vh[c] = df_add_fast(vh[c], df_mul2(ri, ri)); // squares: no cancellation
        }
        stk<KH>(ph + o, p1);
        stk<KH>(pl + o, p2);
        stk<KH>(qh + o, q1);
        stk<KH>(ql + o, q2);
        stk<KH>(xh + o, x1);
        stk<KH>(xl + o, x2);
        stk<KH>(rh + o, r1);
        stk<KH>(rl + o, r2);
        if (invd32) {
            float iv = invd32[i], zn[KH];
#pragma unroll
            for (int c = 0; c < KH; c++) zn[c] = iv * r1[c];
            stk<KH>(z + o, zn);
        }
    }
    DF v[K];
    double tot[K];
#pragma unroll
    for (int c = 0; c < K; c++) v[c] = DF{0.f, 0.f};
#pragma unroll
    for (int q = 0; q < H; q++)
        if (q == h) {
#pragma unroll
            for (int c = 0; c < KH; c++) v[q * KH + c] = vh[c];
        }
    if (reduce_dfk<K>(v, partials, ticket, tot)) fin_rr<K>(bs, tot);
}

// x = (x_hi + x_lo) / scale_c (FP64, once per solve)
template <int K>
__global__ void kbd_out(int64_t nk, const float *__restrict__ xh, const float *__restrict__ xl, const BScal *bs,
                        double *__restrict__ y)
{
    pdl_enter();
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nk; e += (int64_t)gridDim.x * blockDim.x)
        y[e] = ((double)xh[e] + (double)xl[e]) * inv_pow2(bs->c[e & (K - 1)].scale);
}

// ------------------------------------------------------------------ persistent block mass CG
// The whole Jacobi-preconditioned double-float block CG of one mass solve as
// one cooperative launch (every block resident; rows and elements walked
// grid-stride).  Per iteration: s = M z with (r, z) and (z, s) per column,
// grid barrier; every block then sums the block partials in the same fixed
// order and takes the scalar step on its own shared copy of the per-column
// scalars, so all blocks reach the same alpha, beta and stopping decisions
// without another barrier; then p, q, x, r, z = D^-1 r_hi and r.r, grid
// barrier, and the stopping test the same way.  Block 0 writes the scalars
// back.  Row and element arithmetic are those of kbd_spmv and kbd_update; the
// sums are grouped by this launch's blocks.  Vectors written during the
// launch are read through L2.  A barrier that runs out makes every block
// leave at its next barrier (the call then returns AMGH_ERR_TIMEOUT).
#include "gridbar.cuh"

template <int TPR, int K>
__global__ void __launch_bounds__(TPB_K) kbp_mass_cg(MatView<float> A, const float *__restrict__ lo,
                                                    const float *__restrict__ invd32, float *z, float *sh,
                                                    float *sl, float *ph, float *pl, float *qh, float *ql, float *xh,
                                                    float *xl, float *rh, float *rl, BScal *bs, float2 *p1,
                                                    float2 *p2, GridBar *gb, int cap)
{
    constexpr int H = K > 4 ? 2 : 1; // threads per element in the update
    constexpr int KH = K / H;
    __shared__ BScal sb;
    __shared__ DfStage<2 * K> st;
    const int t = threadIdx.x, nb = gridDim.x, n = A.rows;
    if (t == 0) sb = *bs;
    __syncthreads();
    const int stride = nb * blockDim.x, slots = n * TPR;
    for (int it = 0; it <= cap && !sb.all; it++) {
        // ---- s = A z, (r, z), (z, s)
        DF a[2 * K];
        double tot[2 * K];
#pragma unroll
        for (int q = 0; q < 2 * K; q++) a[q] = DF{0.f, 0.f};
        for (int base = blockIdx.x * blockDim.x; base < slots; base += stride) {
            int row = (base + t) / TPR;
            DF sv[K];
            row_sum_df_k<float, TPR, K, true>(A, lo, row, z, sv);
            if (row < n && row_leader<TPR>()) {
                int64_t o = (int64_t)row * K;
                float hv[K], lv[K], zr[K], rhv[K], rlv[K];
#pragma unroll
                for (int c = 0; c < K; c++) {
                    hv[c] = sv[c].hi;
                    lv[c] = sv[c].lo;
                }
                stk<K>(sh + o, hv);
                stk<K>(sl + o, lv);
                ldk_cg<K>(z + o, zr);
                ldk_cg<K>(rh + o, rhv);
                ldk_cg<K>(rl + o, rlv);
#pragma unroll
                for (int c = 0; c < K; c++) {
                    a[c] = df_add_fast(a[c], df_mulf(DF{rhv[c], rlv[c]}, zr[c]));
                    a[K + c] = df_add_fast(a[K + c], df_mulf(sv[c], zr[c]));
                }
            }
        }
        block_df_partials<2 * K>(a, p1, nb, blockIdx.x, st);
        if (!grid_sync(gb, nb)) return;
        sum_df_partials<2 * K>(p1, nb, tot, st);
        if (t == 0) fin_cg2<K>(&sb, tot);
        __syncthreads();
        // ---- p = z + beta p, q = s + beta q, x += alpha p, r -= alpha q, z = D^-1 r_hi, r.r
        const int64_t items = (int64_t)n * H;
        int64_t it0 = (int64_t)blockIdx.x * blockDim.x + t;
        const int h = H == 1 ? 0 : (int)(it0 & 1); // fixed: the stride is even
        DF al[KH], nal[KH], be[KH], vh[KH];
        bool run[KH], first[KH];
#pragma unroll
        for (int c = 0; c < KH; c++) {
            const CgScal &sc = sb.c[h * KH + c];
            al[c] = DF{sc.ahi, sc.alo};
            nal[c] = DF{-sc.ahi, -sc.alo};
            be[c] = DF{sc.bhi, sc.blo};
            run[c] = !sc.done;
            first[c] = sc.bhi == 0.f && sc.blo == 0.f;
            vh[c] = DF{0.f, 0.f};
        }
        for (int64_t e = it0; e < items; e += stride) {
            int64_t i = e / H;
            int64_t o = i * K + h * KH;
            float zv[KH], s1[KH], s2[KH], q1[KH], q2[KH], x1[KH], x2[KH], r1[KH], r2[KH], pp1[KH], pp2[KH];
            ldk_cg<KH>(z + o, zv);
            ldk_cg<KH>(sh + o, s1);
            ldk_cg<KH>(sl + o, s2);
            ldk_cg<KH>(ph + o, pp1);
            ldk_cg<KH>(pl + o, pp2);
            ldk_cg<KH>(qh + o, q1);
            ldk_cg<KH>(ql + o, q2);
            ldk_cg<KH>(xh + o, x1);
            ldk_cg<KH>(xl + o, x2);
            ldk_cg<KH>(rh + o, r1);
            ldk_cg<KH>(rl + o, r2);
#pragma unroll
            for (int c = 0; c < KH; c++) {
                if (!run[c]) continue;
                DF zi = {zv[c], 0.f}, si = {s1[c], s2[c]};
                DF pi = first[c] ? zi : df_add2(zi, df_mul2(be[c], DF{pp1[c], pp2[c]}));
                DF qi = first[c] ? si : df_add2(si, df_mul2(be[c], DF{q1[c], q2[c]}));
                DF xi = df_add2(DF{x1[c], x2[c]}, df_mul2(al[c], pi));
                DF ri = df_add2(DF{r1[c], r2[c]}, df_mul2(nal[c], qi));
                pp1[c] = pi.hi;
                pp2[c] = pi.lo;
                q1[c] = qi.hi;
                q2[c] = qi.lo;
                x1[c] = xi.hi;
                x2[c] = xi.lo;
                r1[c] = ri.hi;
                r2[c] = ri.lo;
                vh[c] = df_add_fast(vh[c], df_mul2(ri, ri));
            }
            stk<KH>(ph + o, pp1);
            stk<KH>(pl + o, pp2);
            stk<KH>(qh + o, q1);
            stk<KH>(ql + o, q2);
            stk<KH>(xh + o, x1);
            stk<KH>(xl + o, x2);
            stk<KH>(rh + o, r1);
            stk<KH>(rl + o, r2);
            float iv = invd32[i], zn[KH];
#pragma unroll
            for (int c = 0; c < KH; c++) zn[c] = iv * r1[c];
            stk<KH>(z + o, zn);
        }
        DF v[K];
        double rr[K];
#pragma unroll
        for (int c = 0; c < K; c++) v[c] = DF{0.f, 0.f};
#pragma unroll
        for (int c = 0; c < KH; c++) {
            if (H == 1 || h == 0) v[c] = vh[c];
            else v[KH + c] = vh[c];
        }
        block_df_partials<K, 2 * K>(v, p2, nb, blockIdx.x, st);
        if (!grid_sync(gb, nb)) return;
        sum_df_partials<K, 2 * K>(p2, nb, rr, st);
        if (t == 0) fin_rr<K>(&sb, rr);
        __syncthreads();
    }
    if (blockIdx.x == 0 && t == 0) *bs = sb;
}

// ------------------------------------------------------------------ V-cycle kernels
// first smoother step from zero: d = x = c D^-1 b
template <typename T, int K>
__global__ void kb_cheb_first(int n, const T *__restrict__ invd, const T *__restrict__ b, T *__restrict__ d,
                              T *__restrict__ x, T cf, const BScal *bs)
{
    pdl_enter();
    if (bs && bs->all) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int64_t o = (int64_t)i * K;
        T bv[K], w[K];
        ldk<K>(b + o, bv);
        T ir = invd[i];
#pragma unroll
        for (int c = 0; c < K; c++) w[c] = cheb_first_point(bv[c], ir, cf);
        stk<K>(d + o, w);
        stk<K>(x + o, w);
    }
}

// Chebyshev step: d' = c_d d + c_r D^-1 (b - A x), x' = x + d'
template <typename T, int TPR, int K>
__global__ void kb_cheb_step(MatView<T> A, const T *__restrict__ invd, const T *__restrict__ b,
                             const T *__restrict__ x, T *__restrict__ d, T *__restrict__ xn, T cdv, T crv,
                             const BScal *bs)
{
    pdl_enter();
    if (bs && bs->all) return;
    int row = my_row<TPR>();
    T ax[K];
    row_sum_k<T, TPR, K>(A, row, x, ax);
    if (row < A.rows && row_leader<TPR>()) {
        int64_t o = (int64_t)row * K;
        T bv[K], dv[K], xv[K], dn[K], xo[K];
        ldk<K>(b + o, bv);
        ldk<K>(d + o, dv);
        ldk<K>(x + o, xv);
        T ir = invd[row];
#pragma unroll
        for (int c = 0; c < K; c++) cheb_point(bv[c], ax[c], ir, dv[c], xv[c], cdv, crv, dn[c], xo[c]);
        stk<K>(d + o, dn);
        stk<K>(xn + o, xo);
    }
}

// r = b - A x
template <typename T, int TPR, int K>
__global__ void kb_residual(MatView<T> A, const T *__restrict__ b, const T *__restrict__ x, T *__restrict__ r,
                            const BScal *bs)
{
    pdl_enter();
    if (bs && bs->all) return;
    int row = my_row<TPR>();
    T ax[K];
    row_sum_k<T, TPR, K>(A, row, x, ax);
    if (row < A.rows && row_leader<TPR>()) {
        int64_t o = (int64_t)row * K;
        T bv[K], w[K];
        ldk<K>(b + o, bv);
#pragma unroll
        for (int c = 0; c < K; c++) w[c] = rsub(bv[c], ax[c]);
        stk<K>(r + o, w);
    }
}

// y = A x (add = 0) or y += A x (add = 1): restriction and prolongation
template <typename T, int TPR, int K>
__global__ void kb_apply(MatView<T> A, const T *__restrict__ x, T *__restrict__ y, int add, const BScal *bs)
{
    pdl_enter();
    if (bs && bs->all) return;
    int row = my_row<TPR>();
    T ax[K];
    row_sum_k<T, TPR, K>(A, row, x, ax);
    if (row < A.rows && row_leader<TPR>()) {
        int64_t o = (int64_t)row * K;
        if (add) {
            T yv[K];
            ldk<K>(y + o, yv);
#pragma unroll
            for (int c = 0; c < K; c++) ax[c] = radd(yv[c], ax[c]);
        }
        stk<K>(y + o, ax);
    }
}

// x = inv b for a dense row-major inverse with leading dimension ld: one warp
// per row
template <typename T, int K>
__global__ void kb_dense(int n, const T *__restrict__ inv, int ld, const T *__restrict__ b, T *__restrict__ x,
                         const BScal *bs)
{
    pdl_enter();
    if (bs && bs->all) return;
    int row = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    int lane = threadIdx.x & 31;
    if (row >= n) return; // whole warps
    const T *a = inv + (int64_t)row * ld;
    T acc[K];
#pragma unroll
    for (int c = 0; c < K; c++) acc[c] = (T)0;
    for (int j = lane; j < n; j += 32) {
        T aj = a[j], bv[K];
        ldk_ro<K>(b + (int64_t)j * K, bv);
#pragma unroll
        for (int c = 0; c < K; c++) acc[c] = rfma(aj, bv[c], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < K; c++) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
    }
    if (lane == 0) stk<K>(x + (int64_t)row * K, acc);
}

template <typename T>
__global__ void kb_copy(int64_t nk, const T *__restrict__ a, T *__restrict__ b, const BScal *bs)
{
    pdl_enter();
    if (bs && bs->all) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nk; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = a[i];
}

// ------------------------------------------------------------------ FP64 operators and vectors
// y = alpha A x + beta y (beta = 0: y is not read)
template <int TPR, int K>
__global__ void kb_spmm(MatView<double> A, const double *__restrict__ x, double *__restrict__ y, double alpha,
                        double beta)
{
    pdl_enter();
    int row = my_row<TPR>();
    double ax[K];
    row_sum_k<double, TPR, K>(A, row, x, ax);
    if (row < A.rows && row_leader<TPR>()) {
        int64_t o = (int64_t)row * K;
        double w[K];
        if (beta != 0.0) {
            double yv[K];
            ldk<K>(y + o, yv);
#pragma unroll
            for (int c = 0; c < K; c++) w[c] = alpha * ax[c] + beta * yv[c];
        } else {
#pragma unroll
            for (int c = 0; c < K; c++) w[c] = alpha * ax[c];
        }
        stk<K>(y + o, w);
    }
}

struct Coef {
    double a[KB], b[KB];
};

// out = a_c x + b_c y per column (y may be null)
template <int K>
__global__ void kb_axpby(int n, Coef cf, const double *__restrict__ x, const double *__restrict__ y, double *out)
{
    pdl_enter();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int64_t o = (int64_t)i * K;
        double xv[K], w[K];
        ldk<K>(x + o, xv);
        if (y) {
            double yv[K];
            ldk<K>(y + o, yv);
#pragma unroll
            for (int c = 0; c < K; c++) w[c] = cf.a[c] * xv[c] + cf.b[c] * yv[c];
        } else {
#pragma unroll
            for (int c = 0; c < K; c++) w[c] = cf.a[c] * xv[c];
        }
        stk<K>(out + o, w);
    }
}

// out = ta + (w1 - tb) / beta (the two-grid combination of Eq.
// twogridinmultiactual, all columns)
__global__ void kb_rcomb(int64_t nk, const double *__restrict__ ta, const double *__restrict__ w1,
                         const double *__restrict__ tb, double beta, double *__restrict__ out)
{
    pdl_enter();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nk; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = ta[i] + (w1[i] - tb[i]) / beta;
}

// out[c] = (x_c, y_c)
template <int K>
__global__ void kb_dot(int n, const double *__restrict__ x, const double *__restrict__ y, double *out,
                       double *partials, unsigned *ticket)
{
    pdl_enter();
    double v[K], tot[K];
#pragma unroll
    for (int c = 0; c < K; c++) v[c] = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int64_t o = (int64_t)i * K;
        double xv[K], yv[K];
        ldk<K>(x + o, xv);
        ldk<K>(y + o, yv);
#pragma unroll
        for (int c = 0; c < K; c++) v[c] += xv[c] * yv[c];
    }
    if (reduce_k<K>(v, partials, ticket, tot)) {
#pragma unroll
        for (int c = 0; c < K; c++) out[c] = tot[c];
    }
}

// column-major (leading dimension ld, nc columns) -> interleaved K columns,
// padding columns zero
template <int K>
__global__ void kb_pack(int n, int nc, const double *__restrict__ src, int64_t ld, double *__restrict__ dst)
{
    pdl_enter();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double w[K];
#pragma unroll
        for (int c = 0; c < K; c++) w[c] = c < nc ? src[(int64_t)c * ld + i] : 0.0;
        stk<K>(dst + (int64_t)i * K, w);
    }
}

template <int K>
__global__ void kb_unpack(int n, int nc, const double *__restrict__ src, double *__restrict__ dst, int64_t ld)
{
    pdl_enter();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double w[K];
        ldk<K>(src + (int64_t)i * K, w);
#pragma unroll
        for (int c = 0; c < K; c++)
            if (c < nc) dst[(int64_t)c * ld + i] = w[c];
    }
}

// desired states at the state dofs: dst[s][c] = yd[c][vertex_of_state[s]]
template <int K>
__global__ void kb_gather_state(int m, int nc, const double *__restrict__ yd, int64_t nv,
                                const int *__restrict__ vos, double *__restrict__ dst)
{
    pdl_enter();
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < m; s += gridDim.x * blockDim.x) {
        int64_t v = vos[s];
        double w[K];
#pragma unroll
        for (int c = 0; c < K; c++) w[c] = c < nc ? yd[(int64_t)c * nv + v] : 0.0;
        stk<K>(dst + (int64_t)s * K, w);
    }
}

// ------------------------------------------------------------------ work space
struct BGraph {
    cudaGraphExec_t start = nullptr, iter = nullptr;
    int ns = 0, ni = 0;
};

struct BState {
    double *x = nullptr, *r = nullptr, *pv = nullptr, *q = nullptr, *s = nullptr;
    void *z = nullptr;     // V-cycle output (FP32 or FP64)
    void *vb = nullptr, *vx = nullptr, *vx2 = nullptr, *vd = nullptr, *vr = nullptr;
    BScal *bs = nullptr;
    RedSlot red;
    BGraph g;
    int hint = 0;
};

struct BCtrl {
    double *mx = nullptr, *mr = nullptr, *mz = nullptr, *mp = nullptr, *mq = nullptr, *ms = nullptr;
    BScal *mbs = nullptr;
    RedSlot red;
    BGraph mg;
    int mhint = 0;
    double *bc = nullptr, *qc = nullptr, *wc = nullptr, *w1 = nullptr, *ta = nullptr, *tb = nullptr;
    double *hu = nullptr, *rq = nullptr, *du = nullptr;
    double *t1 = nullptr, *ys = nullptr, *t2 = nullptr, *ps = nullptr; // state-sized
};

struct BlockWork {
    int K = 0, f32 = 1;
    Arena ar;
    BState sl[AMGH_MAXL];
    BCtrl cl[AMGH_MAXL];
    double *ob = nullptr, *ou = nullptr, *orr = nullptr, *oz = nullptr, *op = nullptr, *oq = nullptr;
    double *oyd = nullptr, *dots = nullptr;
    RedSlot ored;
    BScal *h_bs = nullptr;
    double *h_dots = nullptr;
    // persistent mass CG (persistent_cg): barrier and block partials of its
    // cooperative launch, up to PERSIST_MAX_BLOCKS blocks
    GridBar *pbar = nullptr;
    float2 *pp1 = nullptr, *pp2 = nullptr;
    int fail[KB]; // sticky per-column status of the current call
};
#define PERSIST_MAX_BLOCKS (152 * 8)

static void free_bgraph(BGraph &g)
{
    if (g.start) cudaGraphExecDestroy(g.start);
    if (g.iter) cudaGraphExecDestroy(g.iter);
    g = BGraph();
}

void block_free(amgh_problem *p)
{
    BlockWork *W = p->blk;
    if (!W) return;
    for (int l = 0; l < AMGH_MAXL; l++) {
        free_bgraph(W->sl[l].g);
        free_bgraph(W->cl[l].mg);
    }
    W->ar.free_all();
    if (W->h_bs) cudaFreeHost(W->h_bs);
    if (W->h_dots) cudaFreeHost(W->h_dots);
    delete W;
    p->blk = nullptr;
}

// partial sums of nv values for up to `blocks` blocks
static int bred_alloc(Arena &ar, RedSlot &slot, int blocks, int nv)
{
    slot.capacity = blocks + 8;
    TRY(ar.alloc(&slot.partials, (int64_t)slot.capacity * nv));
    TRY(ar.alloc(&slot.ticket, 1));
    CU(cudaMemsetAsync(slot.ticket, 0, sizeof(unsigned), g_alloc_stream));
    return AMGH_OK;
}

// most blocks of a reducing launch on a's rows (the CG update runs up to two
// threads per row)
static int red_blocks(const DevCsr &a)
{
    int g = rows_grid(a.rows, a.tpr < 1 ? 1 : a.tpr);
    int v = vblocks(2 * (int64_t)a.rows);
    return g > v ? g : v;
}

// grid of kb_cg_update<., K>
template <int K>
static inline int update_blocks(int n)
{
    return vblocks((int64_t)n * (K > 4 ? 2 : 1));
}

static int block_alloc_into(amgh_problem *p, BlockWork *W, int K);

// work space for blocks of K columns (kept while K and the V-cycle precision
// stay the same); on failure nothing is left allocated
static int block_alloc(amgh_problem *p, int K)
{
    int f32 = p->aopts.precision != 0;
    if (p->blk && p->blk->K == K && p->blk->f32 == f32) return AMGH_OK;
    block_free(p);
    BlockWork *W = new (std::nothrow) BlockWork();
    if (!W) return AMGH_ERR_OOM;
    p->blk = W;
    W->f32 = f32;
    int st = block_alloc_into(p, W, K);
    if (st != AMGH_OK) {
        block_free(p);
        return st;
    }
    W->K = K;
    return AMGH_OK;
}

static int block_alloc_into(amgh_problem *p, BlockWork *W, int K)
{
    int f32 = W->f32;
    Arena &ar = W->ar;
    size_t vs = f32 ? sizeof(float) : sizeof(double);
    for (int l = 0; l < p->Ls; l++) {
        BState &B = W->sl[l];
        int64_t n = (int64_t)p->sl[l].A.rows * K;
        TRY(ar.alloc(&B.x, n));
        TRY(ar.alloc(&B.r, n));
        TRY(ar.alloc(&B.pv, n));
        TRY(ar.alloc(&B.q, n));
        TRY(ar.alloc(&B.s, n));
        char *v = nullptr;
        TRY(ar.alloc(&v, (int64_t)(6 * n * vs)));
        void **dst[6] = {&B.z, &B.vb, &B.vx, &B.vx2, &B.vd, &B.vr};
        for (int k = 0; k < 6; k++) *dst[k] = v + k * n * vs;
        TRY(ar.alloc(&B.bs, 1));
        CU(cudaMemsetAsync(B.bs, 0, sizeof(BScal), g_alloc_stream));
        TRY(bred_alloc(ar, B.red, red_blocks(p->sl[l].A), 2 * K));
    }
    for (int l = 0; l < p->Lc; l++) {
        BCtrl &D = W->cl[l];
        int64_t n = (int64_t)p->cl[l].Mu.rows * K;
        int64_t m = (int64_t)p->sl[l < p->Ls ? l : 0].A.rows * K;
        double **vec[15] = {&D.mx, &D.mr, &D.mz, &D.mp, &D.mq, &D.ms, &D.bc, &D.qc,
                            &D.wc, &D.w1, &D.ta, &D.tb, &D.hu, &D.rq, &D.du};
        for (auto d : vec) TRY(ar.alloc(d, n));
        if (l < p->Ls) {
            TRY(ar.alloc(&D.t1, m));
            TRY(ar.alloc(&D.ys, m));
            TRY(ar.alloc(&D.t2, m));
            TRY(ar.alloc(&D.ps, m));
        }
        TRY(ar.alloc(&D.mbs, 1));
        CU(cudaMemsetAsync(D.mbs, 0, sizeof(BScal), g_alloc_stream));
        TRY(bred_alloc(ar, D.red, red_blocks(p->cl[l].Mu), 2 * K));
    }
    int64_t n = (int64_t)p->n * K;
    double **vec[6] = {&W->ob, &W->ou, &W->orr, &W->oz, &W->op, &W->oq};
    for (auto d : vec) TRY(ar.alloc(d, n));
    TRY(ar.alloc(&W->oyd, (int64_t)p->m * K));
    TRY(ar.alloc(&W->dots, KB));
    TRY(bred_alloc(ar, W->ored, vblocks(p->n > p->m ? p->n : p->m), K));
    CU(cudaHostAlloc((void **)&W->h_bs, sizeof(BScal), cudaHostAllocDefault));
    CU(cudaHostAlloc((void **)&W->h_dots, sizeof(double) * KB, cudaHostAllocDefault));
    if (f32 && p->aopts.persistent_cg && !p->parent && !p->in_batch) {
        TRY(ar.alloc(&W->pbar, 1));
        CU(cudaMemsetAsync(W->pbar, 0, sizeof(GridBar), g_alloc_stream));
        TRY(ar.alloc(&W->pp1, (int64_t)PERSIST_MAX_BLOCKS * 2 * K));
        TRY(ar.alloc(&W->pp2, (int64_t)PERSIST_MAX_BLOCKS * K));
    }
    return AMGH_OK;
}

// ------------------------------------------------------------------ launch helpers
template <int V>
struct IntC {
    static constexpr int value = V;
};

// f(IntC<tpr>) for the lane counts the operators use; false for any other
template <typename F>
static bool with_tpr(int tpr, F &&f)
{
    switch (tpr) {
    case 1: f(IntC<1>()); return true;
    case 2: f(IntC<2>()); return true;
    case 4: f(IntC<4>()); return true;
    case 8: f(IntC<8>()); return true;
    case 16: f(IntC<16>()); return true;
    case 32: f(IntC<32>()); return true;
    }
    return false;
}

template <typename T>
static inline MatView<T> bview(const DevCsr &a)
{
    MatView<T> m = view<T>(a);
    if (m.tpr < 1) m.tpr = 1;
    return m;
}

static int read_bscal(amgh_problem *p, const BScal *dev, BScal *out)
{
    CU(cudaMemcpyAsync(p->blk->h_bs, dev, sizeof(BScal), cudaMemcpyDeviceToHost, p->stream));
    TRY(sync_stream(p));
    *out = *p->blk->h_bs;
    return AMGH_OK;
}

static int col_status(const CgScal &s)
{
    if (!s.done) return AMGH_ERR_NOT_CONVERGED;
    switch (s.status) {
    case CG_CONVERGED: return AMGH_OK;
    case CG_INDEFINITE: return AMGH_ERR_INDEFINITE;
    case CG_NUMERIC: return AMGH_ERR_NUMERIC;
    }
    return AMGH_ERR_NOT_CONVERGED;
}

// keep the first failure of each column
static void note_fail(BlockWork &W, int c, int st)
{
    if (st != AMGH_OK && W.fail[c] == AMGH_OK) W.fail[c] = st;
}

// ------------------------------------------------------------------ the block solver
template <typename T, int K>
struct Blk {
    static int spmm(amgh_problem *p, const DevCsr &a, const double *x, double *y, double alpha, double beta)
    {
        MatView<double> A = bview<double>(a);
        if (!with_tpr(A.tpr, [&](auto t) {
                constexpr int TPR = decltype(t)::value;
                pdl_launch(kb_spmm<TPR, K>, dim3(rows_grid(A.rows, TPR)), dim3(TPB), 0, p->stream, A, x, y, alpha,
                           beta);
            }))
            return AMGH_ERR_INVALID_ARG;
        LAUNCH_CHECK();
        return AMGH_OK;
    }

    static int axpby(amgh_problem *p, int n, const Coef &cf, const double *x, const double *y, double *out)
    {
        pdl_launch(kb_axpby<K>, dim3(vblocks(n)), dim3(TPB), 0, p->stream, n, cf, x, y, out);
        LAUNCH_CHECK();
        return AMGH_OK;
    }

    static int copy(amgh_problem *p, int64_t nk, const double *a, double *b)
    {
        pdl_launch(kb_copy<double>, dim3(vblocks(nk)), dim3(TPB), 0, p->stream, nk, a, b, (const BScal *)nullptr);
        LAUNCH_CHECK();
        return AMGH_OK;
    }

    // (x_c, y_c) for every column, on the host
    static int dots(amgh_problem *p, int n, const double *x, const double *y, double *out)
    {
        BlockWork &W = *p->blk;
        pdl_launch(kb_dot<K>, dim3(vblocks(n)), dim3(TPB), 0, p->stream, n, x, y, W.dots, W.ored.partials,
                   W.ored.ticket);
        LAUNCH_CHECK();
        CU(cudaMemcpyAsync(W.h_dots, W.dots, sizeof(double) * K, cudaMemcpyDeviceToHost, p->stream));
        TRY(sync_stream(p));
        for (int c = 0; c < K; c++) out[c] = W.h_dots[c];
        return AMGH_OK;
    }

    // ---- V-cycle on level l (x = V_l b from zero), K columns
    static int vcyc(amgh_problem *p, int l, const T *b, T *x, const BScal *bs)
    {
        BlockWork &W = *p->blk;
        StateLevel &S = p->sl[l];
        BState &B = W.sl[l];
        int n = S.A.rows;
        if (l == p->Ls - 1) {
            const T *inv;
            int ld;
            if (sizeof(T) == sizeof(float)) {
                inv = (const T *)p->Acoarse.inv32;
                ld = p->Acoarse.ld32;
            } else {
                inv = (const T *)p->Acoarse.inv;
                ld = n;
            }
            pdl_launch(kb_dense<T, K>, dim3(ceil_div((int64_t)n * 32, TPB)), dim3(TPB), 0, p->stream, n, inv, ld,
                       b, x, bs);
            LAUNCH_CHECK();
            return AMGH_OK;
        }
        const T *invd = sizeof(T) == sizeof(float) ? (const T *)S.invd32 : (const T *)S.invd;
        T *tmp = (x == (T *)B.vx) ? (T *)B.vx2 : (T *)B.vx;
        T *d = (T *)B.vd, *r = (T *)B.vr;
        T *cur = tmp, *nxt = x;
        MatView<T> A = bview<T>(S.A);
        pdl_launch(kb_cheb_first<T, K>, dim3(vblocks(n)), dim3(TPB), 0, p->stream, n, invd, b, d, cur,
                   (T)p->cr[0], bs);
        LAUNCH_CHECK();
        auto step = [&](double cdv, double crv) -> int {
            if (!with_tpr(A.tpr, [&](auto t) {
                    constexpr int TPR = decltype(t)::value;
                    pdl_launch(kb_cheb_step<T, TPR, K>, dim3(rows_grid(n, TPR)), dim3(TPB), 0, p->stream, A, invd,
                               b, (const T *)cur, d, nxt, (T)cdv, (T)crv, bs);
                }))
                return AMGH_ERR_INVALID_ARG;
            LAUNCH_CHECK();
            T *t = cur;
            cur = nxt;
            nxt = t;
            return AMGH_OK;
        };
        for (int s = 1; s < p->nsteps; s++) TRY(step(p->cd[s], p->cr[s]));
        // coarse-grid correction
        if (!with_tpr(A.tpr, [&](auto t) {
                constexpr int TPR = decltype(t)::value;
                pdl_launch(kb_residual<T, TPR, K>, dim3(rows_grid(n, TPR)), dim3(TPB), 0, p->stream, A, b,
                           (const T *)cur, r, bs);
            }))
            return AMGH_ERR_INVALID_ARG;
        LAUNCH_CHECK();
        BState &Bc = W.sl[l + 1];
        T *bc = (T *)Bc.vb, *xc = (T *)Bc.vx;
        TRY(apply(p, S.St, r, bc, 0, bs));
        TRY(vcyc(p, l + 1, bc, xc, bs));
        TRY(apply(p, S.S, xc, cur, 1, bs));
        for (int s = 0; s < p->nsteps; s++) TRY(step(s == 0 ? 0.0 : p->cd[s], p->cr[s]));
        if (cur != x) {
            pdl_launch(kb_copy<T>, dim3(vblocks((int64_t)n * K)), dim3(TPB), 0, p->stream, (int64_t)n * K,
                       (const T *)cur, x, bs);
            LAUNCH_CHECK();
        }
        return AMGH_OK;
    }

    static int apply(amgh_problem *p, const DevCsr &a, const T *x, T *y, int add, const BScal *bs)
    {
        MatView<T> A = bview<T>(a);
        if (!with_tpr(A.tpr, [&](auto t) {
                constexpr int TPR = decltype(t)::value;
                pdl_launch(kb_apply<T, TPR, K>, dim3(rows_grid(A.rows, TPR)), dim3(TPB), 0, p->stream, A, x, y, add,
                           bs);
            }))
            return AMGH_ERR_INVALID_ARG;
        LAUNCH_CHECK();
        return AMGH_OK;
    }

    // s = A z with (r, z), (z, s) -> alpha, beta in FP64 (precision 0)
    template <typename Z>
    static int cg_spmv(amgh_problem *p, const DevCsr &a, const Z *z, const double *r, double *s, BScal *bs,
                       RedSlot &red)
    {
        MatView<double> A = bview<double>(a);
        if (!with_tpr(A.tpr, [&](auto t) {
                constexpr int TPR = decltype(t)::value;
                pdl_launch(kb_cg_spmv64<TPR, K>, dim3(rows_grid(A.rows, TPR)), dim3(TPB), 0, p->stream, A,
                           (const double *)z, r, s, bs, red.partials, red.ticket);
            }))
            return AMGH_ERR_INVALID_ARG;
        LAUNCH_CHECK();
        return AMGH_OK;
    }

    // ---- double-float CG pieces (FP32 V-cycles): v is an FP64-sized buffer of
    // n*K doubles holding hi = [0, nK) and lo = [nK, 2nK)
    static float *hi(double *v) { return (float *)v; }
    static float *lo(double *v, int n) { return (float *)v + (int64_t)n * K; }

    static int df_start(amgh_problem *p, int n, const double *f, double *x, double *r, float *z, const float *invd32,
                        BScal *bs, RedSlot &red, double tol, int maxit)
    {
        pdl_launch(kbd_norm<K>, dim3(vblocks(n)), dim3(TPB), 0, p->stream, n, f, bs, tol * tol, maxit, red.partials,
                   red.ticket);
        LAUNCH_CHECK();
        int64_t nk = (int64_t)n * K;
        pdl_launch(kbd_start<K>, dim3(vblocks(nk)), dim3(TPB), 0, p->stream, nk, f, hi(x), lo(x, n), hi(r), lo(r, n),
                   z, invd32, (const BScal *)bs);
        LAUNCH_CHECK();
        return AMGH_OK;
    }

    static int df_iter(amgh_problem *p, const DevCsr &a, float *z, double *r, double *s, double *pv, double *q,
                       double *x, const float *invd32, BScal *bs, RedSlot &red)
    {
        int n = a.rows;
        MatView<float> A = bview<float>(a);
        if (!a.lo32) return AMGH_ERR_INVALID_ARG;
        if (!with_tpr(A.tpr, [&](auto t) {
                constexpr int TPR = decltype(t)::value;
                pdl_launch(kbd_spmv<TPR, K>, dim3(rows_grid(A.rows, TPR)), dim3(TPB), 0, p->stream, A,
                           (const float *)a.lo32, (const float *)z, (const float *)hi(r), (const float *)lo(r, n),
                           hi(s), lo(s, n), bs, red.partials, red.ticket);
            }))
            return AMGH_ERR_INVALID_ARG;
        LAUNCH_CHECK();
        pdl_launch(kbd_update<K>, dim3(update_blocks<K>(n)), dim3(TPB), 0, p->stream, n, z, (const float *)hi(s),
                   (const float *)lo(s, n), hi(pv), lo(pv, n), hi(q), lo(q, n), hi(x), lo(x, n), hi(r), lo(r, n),
                   invd32, bs, red.partials, red.ticket);
        LAUNCH_CHECK();
        return AMGH_OK;
    }

    // the mass CG's iterations as one cooperative launch (persistent_cg)
    static int persistent_mass(amgh_problem *p, const DevCsr &a, BCtrl &D, const float *invd32, int maxit)
    {
        BlockWork &W = *p->blk;
        int n = a.rows, dev = 0, sms = 0;
        MatView<float> A = bview<float>(a);
        if (!a.lo32 || !W.pbar) return AMGH_ERR_INVALID_ARG;
        CU(cudaGetDevice(&dev));
        CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        cudaError_t err = cudaSuccess;
        if (!with_tpr(A.tpr, [&](auto t) {
                constexpr int TPR = decltype(t)::value;
                auto kern = kbp_mass_cg<TPR, K>;
                int per_sm = 0;
                err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TPB, 0);
                if (err != cudaSuccess) return;
                int64_t want = ceil_div((int64_t)n * (TPR > 2 ? TPR : 2), TPB);
                int64_t grid = (int64_t)per_sm * sms;
                if (grid > PERSIST_MAX_BLOCKS) grid = PERSIST_MAX_BLOCKS;
                if (grid > want) grid = want;
                if (grid < 1 || per_sm < 1) {
                    err = cudaErrorInvalidConfiguration;
                    return;
                }
                cudaLaunchConfig_t cfg = {};
                cudaLaunchAttribute attr[1];
                attr[0].id = cudaLaunchAttributeCooperative;
                attr[0].val.cooperative = 1;
                cfg.gridDim = dim3((unsigned)grid, 1, 1);
                cfg.blockDim = dim3(TPB, 1, 1);
                cfg.stream = p->stream;
                cfg.attrs = attr;
                cfg.numAttrs = 1;
                err = cudaLaunchKernelEx(&cfg, kern, A, (const float *)a.lo32, invd32, (float *)D.mz, hi(D.ms),
                                         lo(D.ms, n), hi(D.mp), lo(D.mp, n), hi(D.mq), lo(D.mq, n), hi(D.mx),
                                         lo(D.mx, n), hi(D.mr), lo(D.mr, n), D.mbs, W.pp1, W.pp2, (GridBar *)W.pbar,
                                         maxit + 2);
                amgh_count_launch();
            }))
            return AMGH_ERR_INVALID_ARG;
        if (err != cudaSuccess) {
            cudaGetLastError();
            amgh_note_error((int)err, __FILE__, __LINE__);
            return AMGH_ERR_CUDA;
        }
        return AMGH_OK;
    }

    static int df_out(amgh_problem *p, int n, double *x, const BScal *bs, double *y)
    {
        int64_t nk = (int64_t)n * K;
        pdl_launch(kbd_out<K>, dim3(vblocks(nk)), dim3(TPB), 0, p->stream, nk, (const float *)hi(x),
                   (const float *)lo(x, n), bs, y);
        LAUNCH_CHECK();
        return AMGH_OK;
    }

    // replay one inner CG loop (start body once, iteration body in chunks)
    // until every column has stopped or the cap is passed
    static int run_loop(amgh_problem *p, BGraph &g, const std::function<int()> &start,
                        const std::function<int()> &iter, BScal *bs, int maxit, int *hint, BScal *out)
    {
        bool gr = graphs_enabled(p);
        if (gr && !g.iter) {
            if (start) TRY(graph_capture(p, start, &g.start, &g.ns));
            TRY(graph_capture(p, iter, &g.iter, &g.ni));
        }
        if (start) {
            if (gr) TRY(graph_replay(p, g.start, g.ns));
            else TRY(start());
        }
        int chunk = *hint > 1 ? (*hint * 7) / 8 : 1;
        int enq = 0;
        BScal h;
        for (;;) {
            for (int c = 0; c < chunk; c++) {
                if (gr) TRY(graph_replay(p, g.iter, g.ni));
                else TRY(iter());
            }
            enq += chunk;
            TRY(read_bscal(p, bs, &h));
            if (h.all || enq > maxit + 2) break;
            int most = 0;
            for (int c = 0; c < K; c++) most = h.c[c].iters > most ? h.c[c].iters : most;
            chunk = most / 8 > 1 ? most / 8 : 1;
        }
        int most = 0;
        for (int c = 0; c < K; c++) most = h.c[c].iters > most ? h.c[c].iters : most;
        if (most > 0) *hint = most;
        *out = h;
        return AMGH_OK;
    }

    // ---- A_l y = f to relative residual tol per column
    static int state_solve(amgh_problem *p, int l, const double *f, double *y, double tol)
    {
        BlockWork &W = *p->blk;
        StateLevel &S = p->sl[l];
        BState &B = W.sl[l];
        int n = S.A.rows;
        int maxit = p->sopts.inner_max_iter;
        const bool f32 = sizeof(T) == sizeof(float);
        T *z = (T *)B.z;
        std::function<int()> start, iter;
        if constexpr (sizeof(T) == sizeof(float)) {
            // double-float CG; the FP32 V-cycle reads r's hi half
            TRY(df_start(p, n, f, B.x, B.r, (float *)nullptr, (const float *)nullptr, B.bs, B.red, tol, maxit));
            const T *vin = (const T *)hi(B.r);
            start = [&]() { return vcyc(p, l, vin, z, B.bs); };
            iter = [&]() {
                TRY(df_iter(p, S.A, (float *)z, B.r, B.s, B.pv, B.q, B.x, (const float *)nullptr, B.bs, B.red));
                return vcyc(p, l, vin, z, B.bs);
            };
        } else {
            pdl_launch(kb_cg_start<double, K>, dim3(vblocks(n)), dim3(TPB), 0, p->stream, n, f, B.x, B.r,
                       (double *)nullptr, (const double *)nullptr, B.bs, tol * tol, maxit, B.red.partials,
                       B.red.ticket);
            LAUNCH_CHECK();
            const T *vin = (const T *)B.r;
            start = [&]() { return vcyc(p, l, vin, z, B.bs); };
            iter = [&]() {
                TRY(cg_spmv<T>(p, S.A, z, B.r, B.s, B.bs, B.red));
                pdl_launch(kb_cg_update<T, K>, dim3(update_blocks<K>(n)), dim3(TPB), 0, p->stream, n, z,
                           (const double *)B.s, B.pv, B.q, B.x, B.r, (const double *)nullptr, B.bs,
                           B.red.partials, B.red.ticket);
                LAUNCH_CHECK();
                return vcyc(p, l, vin, z, B.bs);
            };
        }
        BScal h;
        TRY(run_loop(p, B.g, start, iter, B.bs, maxit, &B.hint, &h));
        for (int c = 0; c < K; c++) {
            p->c_inner += h.c[c].iters;
            p->c_inner_lvl[l] += h.c[c].iters;
            note_fail(W, c, col_status(h.c[c]));
        }
        if (f32) return df_out(p, n, B.x, B.bs, y);
        return copy(p, (int64_t)n * K, B.x, y);
    }

    // ---- M_{u,l} x = b (Jacobi-preconditioned CG) per column
    static int mass_solve(amgh_problem *p, int l, const double *b, double *x)
    {
        BlockWork &W = *p->blk;
        CtrlLevel &C = p->cl[l];
        BCtrl &D = W.cl[l];
        int n = C.Mu.rows;
        int maxit = p->sopts.mass_max_iter;
        double tol = p->sopts.mass_tol;
        // with FP32 V-cycles the mass CG is double-float with the Jacobi
        // direction z in FP32, as the single-column double-float mass CG
        const bool z32 = W.f32 != 0;
        std::function<int()> iter;
        const bool persist = z32 && W.pbar != nullptr;
        if (z32) {
            TRY(df_start(p, n, b, D.mx, D.mr, (float *)D.mz, (const float *)C.mu_invdiag32, D.mbs, D.red, tol,
                         maxit));
            iter = [&]() {
                return df_iter(p, C.Mu, (float *)D.mz, D.mr, D.ms, D.mp, D.mq, D.mx, (const float *)C.mu_invdiag32,
                               D.mbs, D.red);
            };
        } else {
            pdl_launch(kb_cg_start<double, K>, dim3(vblocks(n)), dim3(TPB), 0, p->stream, n, b, D.mx, D.mr, D.mz,
                       (const double *)C.mu_invdiag, D.mbs, tol * tol, maxit, D.red.partials, D.red.ticket);
            LAUNCH_CHECK();
            iter = [&]() {
                TRY(cg_spmv<double>(p, C.Mu, D.mz, D.mr, D.ms, D.mbs, D.red));
                pdl_launch(kb_cg_update<double, K>, dim3(update_blocks<K>(n)), dim3(TPB), 0, p->stream, n, D.mz,
                           (const double *)D.ms, D.mp, D.mq, D.mx, D.mr, (const double *)C.mu_invdiag, D.mbs,
                           D.red.partials, D.red.ticket);
                LAUNCH_CHECK();
                return AMGH_OK;
            };
        }
        BScal h;
        if (persist) {
            TRY(persistent_mass(p, C.Mu, D, (const float *)C.mu_invdiag32, maxit));
            TRY(read_bscal(p, D.mbs, &h));
        } else {
            TRY(run_loop(p, D.mg, std::function<int()>(), iter, D.mbs, maxit, &D.mhint, &h));
        }
        for (int c = 0; c < K; c++) {
            p->c_mass += h.c[c].iters;
            p->c_mass_lvl[l] += h.c[c].iters;
            note_fail(W, c, col_status(h.c[c]));
        }
        if (z32) return df_out(p, n, D.mx, D.mbs, x);
        return copy(p, (int64_t)n * K, D.mx, x);
    }

    // ---- H_l v (Eq. firstorderpractice on level l), K columns
    static int hessian(amgh_problem *p, int l, const double *v, double *hv)
    {
        BlockWork &W = *p->blk;
        StateLevel &S = p->sl[l];
        CtrlLevel &C = p->cl[l];
        BCtrl &D = W.cl[l];
        double tol = l == 0 ? p->sopts.inner_tol : p->sopts.precond_tol;
        TRY(spmm(p, C.Myu, v, D.t1, 1.0, 0.0));
        TRY(state_solve(p, l, D.t1, D.ys, tol));
        TRY(spmm(p, S.My, D.ys, D.t2, 1.0, 0.0));
        TRY(state_solve(p, l, D.t2, D.ps, tol));
        TRY(spmm(p, C.Myut, D.ps, hv, 1.0, 0.0));
        TRY(spmm(p, C.Mu, v, hv, p->beta, 1.0));
        return AMGH_OK;
    }

    // ---- R_j b (Eq. twogridinmultiactual in M-form)
    static int mlas_R(amgh_problem *p, int j, const double *b, double *out)
    {
        BlockWork &W = *p->blk;
        CtrlLevel &C = p->cl[j];
        BCtrl &D = W.cl[j], &Dc = W.cl[j + 1];
        int n = C.Mu.rows;
        TRY(spmm(p, C.Pt, b, Dc.bc, 1.0, 0.0));
        TRY(mlas_Q(p, j + 1, Dc.bc, Dc.qc));
        TRY(mass_solve(p, j, b, D.w1));
        TRY(mass_solve(p, j + 1, Dc.bc, Dc.wc));
        TRY(spmm(p, C.P, Dc.qc, D.ta, 1.0, 0.0));
        TRY(spmm(p, C.P, Dc.wc, D.tb, 1.0, 0.0));
        int64_t nk = (int64_t)n * K;
        pdl_launch(kb_rcomb, dim3(vblocks(nk)), dim3(TPB), 0, p->stream, nk, (const double *)D.ta,
                   (const double *)D.w1, (const double *)D.tb, p->beta, out);
        LAUNCH_CHECK();
        return AMGH_OK;
    }

    // ---- Q_{ell-1} b by CG on H_{ell-1} from zero, per column, stopping at
    // ||r_k|| <= coarse_tol ||b||; the iterate at the cap is used as it stands
    static int coarse_cg(amgh_problem *p, int j, const double *b, double *u)
    {
        BlockWork &W = *p->blk;
        BCtrl &D = W.cl[j];
        int n = p->cl[j].Mu.rows;
        double *r = D.rq, *pv = D.du, *q = D.hu;
        CU(cudaMemsetAsync(u, 0, sizeof(double) * n * K, p->stream));
        TRY(copy(p, (int64_t)n * K, b, r));
        TRY(copy(p, (int64_t)n * K, b, pv));
        double ff[K], rz[K], nf[K];
        bool run[K];
        TRY(dots(p, n, b, b, ff));
        bool any = false;
        for (int c = 0; c < K; c++) {
            if (!(ff[c] == ff[c])) note_fail(W, c, AMGH_ERR_NUMERIC);
            run[c] = ff[c] > 0.0 && W.fail[c] == AMGH_OK;
            nf[c] = sqrt(ff[c]);
            rz[c] = ff[c];
            any = any || run[c];
        }
        Coef cf;
        if (any) {
            // columns that do not run get p = 0 (their inner solves then stop at once)
            for (int c = 0; c < K; c++) {
                cf.a[c] = run[c] ? 1.0 : 0.0;
                cf.b[c] = 0.0;
            }
            TRY(axpby(p, n, cf, b, nullptr, pv));
        }
        double tol = p->sopts.coarse_tol;
        for (int k = 1; any && k <= p->sopts.coarse_max_iter; k++) {
            TRY(hessian(p, j, pv, q));
            for (int c = 0; c < K; c++) {
                if (run[c]) p->c_coarse += 1;
                if (W.fail[c] != AMGH_OK) run[c] = false;
            }
            double pq[K], alpha[K];
            TRY(dots(p, n, pv, q, pq));
            for (int c = 0; c < K; c++) {
                alpha[c] = 0.0;
                if (!run[c]) continue;
                if (!(pq[c] > 0.0)) {
                    note_fail(W, c, pq[c] == pq[c] ? AMGH_ERR_INDEFINITE : AMGH_ERR_NUMERIC);
                    run[c] = false;
                    continue;
                }
                alpha[c] = rz[c] / pq[c];
            }
            for (int c = 0; c < K; c++) {
                cf.a[c] = 1.0;
                cf.b[c] = alpha[c];
            }
            TRY(axpby(p, n, cf, u, pv, u));
            for (int c = 0; c < K; c++) cf.b[c] = -alpha[c];
            TRY(axpby(p, n, cf, r, q, r));
            double rr[K], beta[K];
            TRY(dots(p, n, r, r, rr));
            any = false;
            for (int c = 0; c < K; c++) {
                beta[c] = 0.0;
                if (!run[c]) continue;
                if (!(rr[c] == rr[c])) {
                    note_fail(W, c, AMGH_ERR_NUMERIC);
                    run[c] = false;
                } else if (sqrt(rr[c]) <= tol * nf[c]) {
                    run[c] = false;
                } else if (!(rr[c] > 0.0)) {
                    note_fail(W, c, AMGH_ERR_INDEFINITE);
                    run[c] = false;
                } else {
                    beta[c] = rr[c] / rz[c];
                    rz[c] = rr[c];
                }
                any = any || run[c];
            }
            for (int c = 0; c < K; c++) {
                cf.a[c] = run[c] ? 1.0 : 0.0;
                cf.b[c] = run[c] ? beta[c] : 0.0;
            }
            TRY(axpby(p, n, cf, r, pv, pv));
        }
        return AMGH_OK;
    }

    // ---- Q_j b (Algorithm MLAS)
    static int mlas_Q(amgh_problem *p, int j, const double *b, double *u)
    {
        BlockWork &W = *p->blk;
        CtrlLevel &C = p->cl[j];
        BCtrl &D = W.cl[j];
        int n = C.Mu.rows;
        if (j == p->ell - 1) {
            if (p->coarse_cg) return coarse_cg(p, j, b, u);
            pdl_launch(kb_dense<double, K>, dim3(ceil_div((int64_t)n * 32, TPB)), dim3(TPB), 0, p->stream, n,
                       (const double *)p->Hcoarse.inv, n, b, u, (const BScal *)nullptr);
            LAUNCH_CHECK();
            return AMGH_OK;
        }
        TRY(mlas_R(p, j, b, u));
        if (j == 0) return AMGH_OK;
        TRY(hessian(p, j, u, D.hu));
        Coef cf;
        for (int c = 0; c < K; c++) {
            cf.a[c] = 1.0;
            cf.b[c] = -1.0;
        }
        TRY(axpby(p, n, cf, b, D.hu, D.rq));
        TRY(mlas_R(p, j, D.rq, D.du));
        for (int c = 0; c < K; c++) cf.b[c] = 1.0;
        TRY(axpby(p, n, cf, u, D.du, u));
        return AMGH_OK;
    }

    // ---- outer CG on H u = b per column (Sec. 5.3); columns [nact, K) are
    // padding.  u (block) receives the controls.
    static int outer(amgh_problem *p, int nact, const amgh_solve_opts &o, double *u, double *relres, int *iters)
    {
        BlockWork &W = *p->blk;
        int n = p->n;
        double *b = W.ob, *r = W.orr, *z = W.oz, *pv = W.op, *q = W.oq;
        // b = M_yu^T A^-1 M_y y_d per column
        {
            BCtrl &D0 = W.cl[0];
            TRY(spmm(p, p->sl[0].My, W.oyd, D0.t2, 1.0, 0.0));
            TRY(state_solve(p, 0, D0.t2, D0.ps, p->sopts.inner_tol));
            TRY(spmm(p, p->cl[0].Myut, D0.ps, b, 1.0, 0.0));
        }
        double bb[K];
        TRY(dots(p, n, b, b, bb));
        bool run[K];
        bool any = false;
        Coef cf;
        for (int c = 0; c < K; c++) {
            iters[c] = 0;
            relres[c] = 0.0;
            if (c < nact && !(bb[c] == bb[c])) note_fail(W, c, AMGH_ERR_NUMERIC);
            run[c] = c < nact && bb[c] > 0.0 && W.fail[c] == AMGH_OK;
            any = any || run[c];
            cf.a[c] = run[c] ? 1.0 : 0.0;
            cf.b[c] = 0.0;
        }
        CU(cudaMemsetAsync(u, 0, sizeof(double) * n * K, p->stream));
        // r = b on running columns, 0 elsewhere (stopped columns cost nothing below)
        TRY(axpby(p, n, cf, b, nullptr, r));
        double rz[K];
        auto precond = [&]() -> int {
            if (o.precond) return mlas_Q(p, 0, r, z);
            return copy(p, (int64_t)n * K, r, z);
        };
        auto drop_failed = [&]() {
            for (int c = 0; c < K; c++)
                if (W.fail[c] != AMGH_OK) run[c] = false;
        };
        if (any) {
            TRY(precond());
            drop_failed();
            TRY(dots(p, n, r, z, rz));
            for (int c = 0; c < K; c++) {
                if (run[c] && !(rz[c] > 0.0)) {
                    note_fail(W, c, rz[c] == rz[c] ? AMGH_ERR_INDEFINITE : AMGH_ERR_NUMERIC);
                    run[c] = false;
                }
                cf.a[c] = run[c] ? 1.0 : 0.0;
            }
            TRY(axpby(p, n, cf, z, nullptr, pv));
        }
        for (;;) {
            any = false;
            for (int c = 0; c < K; c++) any = any || run[c];
            if (!any) break;
            TRY(hessian(p, 0, pv, q));
            for (int c = 0; c < K; c++)
                if (run[c]) p->c_happ += 1;
            drop_failed();
            double pq[K], alpha[K];
            TRY(dots(p, n, pv, q, pq));
            for (int c = 0; c < K; c++) {
                alpha[c] = 0.0;
                if (!run[c]) continue;
                if (!(pq[c] > 0.0)) {
                    note_fail(W, c, pq[c] == pq[c] ? AMGH_ERR_INDEFINITE : AMGH_ERR_NUMERIC);
                    run[c] = false;
                    continue;
                }
                alpha[c] = rz[c] / pq[c];
            }
            for (int c = 0; c < K; c++) {
                cf.a[c] = 1.0;
                cf.b[c] = alpha[c];
            }
            TRY(axpby(p, n, cf, u, pv, u));
            for (int c = 0; c < K; c++) cf.b[c] = -alpha[c];
            TRY(axpby(p, n, cf, r, q, r));
            double rr[K];
            TRY(dots(p, n, r, r, rr));
            bool stop[K];
            for (int c = 0; c < K; c++) {
                stop[c] = false;
                if (!run[c]) continue;
                iters[c] += 1;
                if (!(rr[c] == rr[c])) {
                    note_fail(W, c, AMGH_ERR_NUMERIC);
                    stop[c] = true;
                } else if (rr[c] <= o.tol * o.tol * bb[c]) {
                    stop[c] = true;
                } else if (iters[c] >= o.max_iter) {
                    note_fail(W, c, AMGH_ERR_NOT_CONVERGED);
                    stop[c] = true;
                }
            }
            any = false;
            for (int c = 0; c < K; c++) {
                if (stop[c]) run[c] = false;
                any = any || run[c];
            }
            if (!any) break;
            // stopped columns: r = 0, so the preconditioner does no work for them
            for (int c = 0; c < K; c++) {
                cf.a[c] = run[c] ? 1.0 : 0.0;
                cf.b[c] = 0.0;
            }
            TRY(axpby(p, n, cf, r, nullptr, r));
            TRY(precond());
            drop_failed();
            double rzn[K], beta[K];
            TRY(dots(p, n, r, z, rzn));
            for (int c = 0; c < K; c++) {
                beta[c] = 0.0;
                if (!run[c]) continue;
                if (!(rzn[c] > 0.0)) {
                    note_fail(W, c, rzn[c] == rzn[c] ? AMGH_ERR_INDEFINITE : AMGH_ERR_NUMERIC);
                    run[c] = false;
                    continue;
                }
                beta[c] = rzn[c] / rz[c];
                rz[c] = rzn[c];
            }
            for (int c = 0; c < K; c++) {
                cf.a[c] = run[c] ? 1.0 : 0.0;
                cf.b[c] = run[c] ? beta[c] : 0.0;
            }
            TRY(axpby(p, n, cf, z, pv, pv));
        }
        // true relative residual ||b - H u|| / ||b|| of every converged column
        bool want = false;
        for (int c = 0; c < K; c++) {
            cf.a[c] = (c < nact && W.fail[c] == AMGH_OK) ? 1.0 : 0.0;
            cf.b[c] = 0.0;
            want = want || cf.a[c] != 0.0;
        }
        if (want) {
            TRY(axpby(p, n, cf, u, nullptr, pv));
            TRY(hessian(p, 0, pv, q));
            for (int c = 0; c < K; c++)
                if (cf.a[c] != 0.0) p->c_happ += 1;
            for (int c = 0; c < K; c++) cf.b[c] = -cf.a[c];
            TRY(axpby(p, n, cf, b, q, r));
            double rr[K];
            TRY(dots(p, n, r, r, rr));
            for (int c = 0; c < K; c++)
                if (cf.a[c] != 0.0) relres[c] = bb[c] > 0.0 ? sqrt(rr[c] / bb[c]) : 0.0;
        }
        return AMGH_OK;
    }
};

// ------------------------------------------------------------------ entry points
static int block_width(int ncols) { return ncols <= 2 ? 2 : ncols <= 4 ? 4 : 8; }

template <int K>
static int pack(amgh_problem *p, int n, int nc, const double *src, int64_t ld, double *dst)
{
    pdl_launch(kb_pack<K>, dim3(vblocks(n)), dim3(TPB), 0, p->stream, n, nc, src, ld, dst);
    LAUNCH_CHECK();
    return AMGH_OK;
}

template <int K>
static int unpack(amgh_problem *p, int n, int nc, const double *src, double *dst, int64_t ld)
{
    pdl_launch(kb_unpack<K>, dim3(vblocks(n)), dim3(TPB), 0, p->stream, n, nc, src, dst, ld);
    LAUNCH_CHECK();
    return AMGH_OK;
}

// first failure over the columns, in column order
static int first_fail(const BlockWork &W, int nc)
{
    for (int c = 0; c < nc; c++)
        if (W.fail[c] != AMGH_OK) return W.fail[c];
    return AMGH_OK;
}

enum { OP_HESSIAN = 0, OP_PRECOND = 1 };

template <typename T, int K>
static int apply_blocks(amgh_problem *p, int op, const double *in, double *out, int ncols)
{
    BlockWork &W = *p->blk;
    int n = p->n;
    for (int c0 = 0; c0 < ncols; c0 += K) {
        int nc = ncols - c0 < K ? ncols - c0 : K;
        for (int c = 0; c < KB; c++) W.fail[c] = AMGH_OK;
        TRY(pack<K>(p, n, nc, in + (int64_t)c0 * n, n, W.orr));
        if (op == OP_HESSIAN) {
            TRY((Blk<T, K>::hessian(p, 0, W.orr, W.oq)));
            p->c_happ += nc;
        } else {
            TRY((Blk<T, K>::mlas_Q(p, 0, W.orr, W.oq)));
        }
        TRY(unpack<K>(p, n, nc, W.oq, out + (int64_t)c0 * n, n));
        TRY(first_fail(W, nc));
    }
    return AMGH_OK;
}

template <typename T, int K>
static int solve_blocks(amgh_problem *p, const double *yd, int ncols, double *u, const amgh_solve_opts &o,
                        amgh_solve_info *info, int *first_status)
{
    BlockWork &W = *p->blk;
    int n = p->n, m = p->m;
    for (int c0 = 0; c0 < ncols; c0 += K) {
        int nc = ncols - c0 < K ? ncols - c0 : K;
        for (int c = 0; c < KB; c++) W.fail[c] = AMGH_OK;
        pdl_launch(kb_gather_state<K>, dim3(vblocks(m)), dim3(TPB), 0, p->stream, m, nc,
                   yd + (int64_t)c0 * p->nv, (int64_t)p->nv, (const int *)p->vertex_of_state, W.oyd);
        LAUNCH_CHECK();
        double relres[K];
        int it[K];
        TRY((Blk<T, K>::outer(p, nc, o, W.ou, relres, it)));
        TRY(unpack<K>(p, n, nc, W.ou, u + (int64_t)c0 * n, n));
        for (int c = 0; c < nc; c++) {
            info->outer_iters += it[c];
            if (W.fail[c] == AMGH_OK && relres[c] > info->final_relres) info->final_relres = relres[c];
        }
        int st = first_fail(W, nc);
        if (st != AMGH_OK && *first_status == AMGH_OK) *first_status = st;
    }
    return AMGH_OK;
}

template <typename T>
static int dispatch_apply(amgh_problem *p, int K, int op, const double *in, double *out, int ncols)
{
    switch (K) {
    case 2: return apply_blocks<T, 2>(p, op, in, out, ncols);
    case 4: return apply_blocks<T, 4>(p, op, in, out, ncols);
    default: return apply_blocks<T, 8>(p, op, in, out, ncols);
    }
}

template <typename T>
static int dispatch_solve(amgh_problem *p, int K, const double *yd, int ncols, double *u, const amgh_solve_opts &o,
                          amgh_solve_info *info, int *first_status)
{
    switch (K) {
    case 2: return solve_blocks<T, 2>(p, yd, ncols, u, o, info, first_status);
    case 4: return solve_blocks<T, 4>(p, yd, ncols, u, o, info, first_status);
    default: return solve_blocks<T, 8>(p, yd, ncols, u, o, info, first_status);
    }
}

int block_apply(amgh_problem *p, int op, const double *in, double *out, int ncols)
{
    int K = block_width(ncols);
    TRY(block_alloc(p, K));
    if (p->blk->f32) return dispatch_apply<float>(p, K, op, in, out, ncols);
    return dispatch_apply<double>(p, K, op, in, out, ncols);
}

int block_hessian_apply(amgh_problem *p, const double *u, double *hu, int ncols)
{
    return block_apply(p, OP_HESSIAN, u, hu, ncols);
}

int block_precond_apply(amgh_problem *p, const double *r, double *z, int ncols)
{
    return block_apply(p, OP_PRECOND, r, z, ncols);
}

int block_solve(amgh_problem *p, const double *yd, int ncols, double *u, const amgh_solve_opts &o,
                amgh_solve_info *info)
{
    int K = block_width(ncols);
    TRY(block_alloc(p, K));
    int first = AMGH_OK;
    int st;
    if (p->blk->f32) st = dispatch_solve<float>(p, K, yd, ncols, u, o, info, &first);
    else st = dispatch_solve<double>(p, K, yd, ncols, u, o, info, &first);
    if (st != AMGH_OK) return st;
    return first;
}

// poll limit of this file's grid barrier waits (-1: default)
int block_set_grid_polls(int polls)
{
    int v = polls < 0 ? GRIDBAR_POLLS : polls;
    CU(cudaMemcpyToSymbol(g_gridbar_polls, &v, sizeof(int)));
    return AMGH_OK;
}

// AMGH_ERR_TIMEOUT (and the flag and barrier reset) if a persistent block CG
// of this problem gave up at a barrier
int block_grid_timeout_check(amgh_problem *p)
{
    int h = 0;
    CU(cudaMemcpyFromSymbolAsync(&h, g_gridbar_timeout, sizeof(int), 0, cudaMemcpyDeviceToHost, p->stream));
    CU(cudaStreamSynchronize(p->stream));
    if (!h) return AMGH_OK;
    int zero = 0;
    CU(cudaMemcpyToSymbolAsync(g_gridbar_timeout, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, p->stream));
    if (p->blk && p->blk->pbar) CU(cudaMemsetAsync(p->blk->pbar, 0, sizeof(GridBar), p->stream));
    if (p->pm_bar) CU(cudaMemsetAsync(p->pm_bar, 0, sizeof(GridBar), p->stream));
    CU(cudaStreamSynchronize(p->stream));
    return AMGH_ERR_TIMEOUT;
}

// The single-column double-float mass CG of precision 2 (persistent_cg) with
// the K = 1 kernels of the block solver: norm and start, all iterations in
// one cooperative launch, and the output.  Same method as the graph-replayed
// double-float mass CG (scaled right side, Jacobi direction in FP32); sums
// grouped by this launch's blocks.
int persistent_mass_single(amgh_problem *p, int l, const double *b, double *x, int64_t *iters)
{
    CtrlLevel &C = p->cl[l];
    const DevCsr &a = C.Mu;
    int n = a.rows, maxit = p->sopts.mass_max_iter, dev = 0, sms = 0;
    if (n == 0) return AMGH_OK;
    if (!a.lo32 || !C.mu_invdiag32) return AMGH_ERR_INVALID_ARG;
    Arena &ar = p->harena;
    if (!p->pm_bs) {
        BScal *bs = nullptr;
        float2 *p1 = nullptr, *p2 = nullptr;
        GridBar *bar = nullptr;
        TRY(ar.alloc(&bs, 1));
        TRY(ar.alloc(&p1, (int64_t)PERSIST_MAX_BLOCKS * 2));
        TRY(ar.alloc(&p2, (int64_t)PERSIST_MAX_BLOCKS));
        TRY(ar.alloc(&bar, 1));
        CU(cudaMemsetAsync(bs, 0, sizeof(BScal), p->stream));
        CU(cudaMemsetAsync(bar, 0, sizeof(GridBar), p->stream));
        p->pm_bs = bs;
        p->pm_p1 = p1;
        p->pm_p2 = p2;
        p->pm_bar = bar;
    }
    BScal *bs = (BScal *)p->pm_bs;
    auto hi = [&](double *v) { return (float *)v; };
    auto lo = [&](double *v) { return (float *)v + n; };
    double tol = p->sopts.mass_tol;
    pdl_launch(kbd_norm<1>, dim3(vblocks(n)), dim3(TPB), 0, p->stream, n, b, bs, tol * tol, maxit, C.red.partials,
               C.red.ticket);
    LAUNCH_CHECK();
    pdl_launch(kbd_start<1>, dim3(vblocks(n)), dim3(TPB), 0, p->stream, (int64_t)n, b, hi(C.mx), lo(C.mx), hi(C.mr),
               lo(C.mr), (float *)C.mz, (const float *)C.mu_invdiag32, (const BScal *)bs);
    LAUNCH_CHECK();
    CU(cudaGetDevice(&dev));
    CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    MatView<float> A = bview<float>(a);
    cudaError_t err = cudaSuccess;
    if (!with_tpr(A.tpr, [&](auto t) {
            constexpr int TPR = decltype(t)::value;
            auto kern = kbp_mass_cg<TPR, 1>;
            int per_sm = 0;
            err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TPB, 0);
            if (err != cudaSuccess) return;
            int64_t want = ceil_div((int64_t)n * TPR, TPB), grid = (int64_t)per_sm * sms;
            if (grid > PERSIST_MAX_BLOCKS) grid = PERSIST_MAX_BLOCKS;
            if (grid > want) grid = want;
            if (grid < 1 || per_sm < 1) {
                err = cudaErrorInvalidConfiguration;
                return;
            }
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeCooperative;
            attr[0].val.cooperative = 1;
            cfg.gridDim = dim3((unsigned)grid, 1, 1);
            cfg.blockDim = dim3(TPB, 1, 1);
            cfg.stream = p->stream;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            err = cudaLaunchKernelEx(&cfg, kern, A, (const float *)a.lo32, (const float *)C.mu_invdiag32,
                                     (float *)C.mz, hi(C.ms), lo(C.ms), hi(C.mp), lo(C.mp), hi(C.mq), lo(C.mq),
                                     hi(C.mx), lo(C.mx), hi(C.mr), lo(C.mr), bs, (float2 *)p->pm_p1,
                                     (float2 *)p->pm_p2, (GridBar *)p->pm_bar, maxit + 2);
            amgh_count_launch();
        }))
        return AMGH_ERR_INVALID_ARG;
    if (err != cudaSuccess) {
        cudaGetLastError();
        amgh_note_error((int)err, __FILE__, __LINE__);
        return AMGH_ERR_CUDA;
    }
    pdl_launch(kbd_out<1>, dim3(vblocks(n)), dim3(TPB), 0, p->stream, (int64_t)n, (const float *)hi(C.mx),
               (const float *)lo(C.mx), (const BScal *)bs, x);
    LAUNCH_CHECK();
    CgScal h;
    CU(cudaMemcpyAsync(&h, &bs->c[0], sizeof(CgScal), cudaMemcpyDeviceToHost, p->stream));
    TRY(sync_stream(p));
    // algorithmic bytes: per iteration those of the graph-replayed pair (the
    // double-float SpMV with its dots, the update with the Jacobi direction)
    count_bytes((double)h.iters * (spmv_bytes(a, 4) + 4.0 * a.nnz + 12.0 * n + 84.0 * n) + 48.0 * n);
    p->c_mass_lvl[l] += h.iters;
    p->c_mass += h.iters;
    if (iters) *iters = h.iters;
    return AMGH_OK;
}
