// blas.cu -- conjugate-gradient building blocks with device-resident scalars.
//
// Every CG loop keeps its scalars (r.z, alpha, beta, ||r||^2, the stopping
// threshold, an iteration count and a `done` flag) in a CgScal in device
// memory.  Each kernel below fuses a vector update with the next inner
// product; its reduction is two-stage and deterministic (block partials
// summed in fixed order by the last block to finish), and that last block
// also computes the new alpha / beta or the stopping decision.  Every kernel
// returns at once when `done` is set, so the host can enqueue several
// iterations ahead and only read the flag back now and then.
//
// The inner (state and mass) solves use the single-reduction form of
// preconditioned CG (Chronopoulos & Gear, J. Comput. Appl. Math. 25, 1989):
// with z = M r and s = A z computed together,
//   gamma = (r, z), delta = (z, s), beta = gamma / gamma_old,
//   alpha = gamma / (delta - beta gamma / alpha_old),
//   p = z + beta p, q = s + beta q, x += alpha p, r -= alpha q,
// which equals standard PCG in exact arithmetic and needs one SpMV (one
// gather of z) and one reduction point per iteration.
#include <math.h>

#include <algorithm>

#include "internal.cuh"
#include "spmv.cuh"
#include "util.cuh"

static const int TPB = 256;

static inline int vec_blocks(int64_t n)
{
    int nb = ceil_div(n > 0 ? n : 1, TPB);
    return nb < 2432 ? nb : 2432; // 152 SMs x 16 blocks of 256 threads
}

int red_alloc(Arena &ar, RedSlot &slot, int capacity_rows)
{
    // SpMV-class kernels launch up to 32 threads per row
    int cap = ceil_div((int64_t)(capacity_rows > 0 ? capacity_rows : 1) * 32, TPB) + 8;
    slot.capacity = cap;
    TRY(ar.alloc(&slot.partials, (int64_t)cap * 2));
    TRY(ar.alloc(&slot.ticket, 1));
    CU(cudaMemsetAsync(slot.ticket, 0, sizeof(unsigned), g_alloc_stream));
    return AMGH_OK;
}

enum {
    F_START = 0,     // t0 = f.f -> ff, thr, done if zero
    F_RZ_FIRST,      // t0 = r.z -> rz
    F_PQ,            // t0 = p.q -> alpha
    F_RR,            // t0 = r.r -> iteration count, stop test
    F_RZ_NEXT,       // t0 = r.z -> beta, rz
    F_MASS_START,    // t0 = f.f, t1 = r.z
    F_MASS_UPDATE,   // t0 = r.r, t1 = r.z
    F_REF_START,     // t0 = f.f -> scale, thr
    F_REF_UPDATE,    // t0 = r.r -> refinement stop test, scale
    F_STORE,         // t0 -> *out
    F_CG2,           // t0 = (r,z), t1 = (z,Az) -> alpha, beta (single-reduction CG)
    F_SCALE,         // t0 = f.f -> scale = power of two nearest 1 / ||f||
};

__device__ __forceinline__ bool bad(double x) { return !(x == x) || isinf(x); }

__device__ void cg_finalize(int mode, const double *t, CgScal *sc, double *out)
{
    switch (mode) {
    case F_START:
    case F_MASS_START: {
        double ff = t[0];
        sc->ff = ff;
        sc->rr = ff;
        sc->thr = sc->thr * ff; // host stored tol^2 in thr
        sc->iters = 0;
        sc->status = CG_RUNNING;
        sc->done = 0;
        if (bad(ff)) {
            sc->status = CG_NUMERIC;
            sc->done = 1;
        } else if (ff == 0.0) {
            sc->status = CG_CONVERGED;
            sc->done = 1;
        }
        if (mode == F_MASS_START && !sc->done) {
            sc->rz = t[1];
            sc->beta = 0.0;
            if (!(t[1] > 0.0)) {
                sc->status = bad(t[1]) ? CG_NUMERIC : CG_INDEFINITE;
                sc->done = 1;
            }
        }
        break;
    }
    case F_RZ_FIRST:
        sc->rz = t[0];
        sc->beta = 0.0;
        if (!(t[0] > 0.0)) {
            sc->status = bad(t[0]) ? CG_NUMERIC : CG_INDEFINITE;
            sc->done = 1;
        }
        break;
    case F_PQ:
        sc->pq = t[0];
        if (!(t[0] > 0.0)) {
            sc->status = bad(t[0]) ? CG_NUMERIC : CG_INDEFINITE;
            sc->alpha = 0.0;
            sc->done = 1;
        } else {
            sc->alpha = sc->rz / t[0];
        }
        break;
    case F_RR:
    case F_MASS_UPDATE:
        sc->rr = t[0];
        sc->iters += 1;
        sc->total_iters += 1;
        if (bad(t[0])) {
            sc->status = CG_NUMERIC;
            sc->done = 1;
        } else if (t[0] <= sc->thr) {
            sc->status = CG_CONVERGED;
            sc->done = 1;
        } else if (sc->iters >= sc->maxit) {
            sc->status = CG_MAXIT;
            sc->done = 1;
        }
        if (mode == F_MASS_UPDATE && !sc->done) {
            double rzn = t[1];
            if (!(rzn > 0.0)) {
                sc->status = bad(rzn) ? CG_NUMERIC : CG_INDEFINITE;
                sc->done = 1;
            } else {
                sc->beta = rzn / sc->rz;
                sc->rz = rzn;
            }
        }
        break;
    case F_RZ_NEXT:
        if (!(t[0] > 0.0)) {
            sc->status = bad(t[0]) ? CG_NUMERIC : CG_INDEFINITE;
            sc->done = 1;
        } else {
            sc->beta = t[0] / sc->rz;
            sc->rz = t[0];
        }
        break;
    case F_REF_START: {
        double ff = t[0];
        sc->ff = ff;
        sc->rr = ff;
        sc->thr = sc->thr * ff;
        sc->iters = 0;
        sc->status = CG_RUNNING;
        sc->done = 0;
        sc->scale = sqrt(ff);
        if (bad(ff)) {
            sc->status = CG_NUMERIC;
            sc->done = 1;
        } else if (ff == 0.0) {
            sc->status = CG_CONVERGED;
            sc->done = 1;
        }
        break;
    }
    case F_REF_UPDATE:
        sc->rr = t[0];
        sc->iters += 1;
        sc->total_iters += 1;
        sc->scale = sqrt(t[0]);
        if (bad(t[0])) {
            sc->status = CG_NUMERIC;
            sc->done = 1;
        } else if (t[0] <= sc->thr) {
            sc->status = CG_CONVERGED;
            sc->done = 1;
        } else if (sc->iters >= sc->maxit) {
            sc->status = CG_MAXIT;
            sc->done = 1;
        }
        break;
    case F_STORE:
        *out = t[0];
        break;
    case F_SCALE: {
        double nrm = sqrt(t[0]);
        sc->scale = (nrm > 0.0 && !bad(nrm)) ? exp2(-rint(log2(nrm))) : 1.0;
        break;
    }
    case F_CG2: {
        double g = t[0], d = t[1];
        if (!(g > 0.0) || !(d > 0.0)) {
            sc->status = (bad(g) || bad(d)) ? CG_NUMERIC : CG_INDEFINITE;
            sc->done = 1;
            break;
        }
        double beta = 0.0, alpha;
        if (sc->k1 == 0) {
            alpha = g / d;
        } else {
            beta = g / sc->rz;
            double den = d - beta * g / sc->alpha;
            if (!(den > 0.0)) {
                sc->status = bad(den) ? CG_NUMERIC : CG_INDEFINITE;
                sc->done = 1;
                break;
            }
            alpha = g / den;
        }
        sc->rz = g;
        sc->alpha = alpha;
        sc->beta = beta;
        sc->k1 += 1;
        sc->ahi = (float)alpha;
        sc->alo = (float)(alpha - (double)sc->ahi);
        sc->bhi = (float)beta;
        sc->blo = (float)(beta - (double)sc->bhi);
        break;
    }
    }
}

#define SKIP_DONE() \
    if (sc->done) return

// x = 0 (optional), r = f, reduce f.f ; host put tol^2 in sc->thr and maxit
template <typename T>
__global__ void k_cg_start(int n, const T *__restrict__ f, T *__restrict__ x, T *__restrict__ r, CgScal *sc,
                           int zero_x, double *partials, unsigned *ticket, int mode)
{
    pdl_enter();
    double v[1] = {0.0}, tot[1];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        T fi = f[i];
        r[i] = fi;
        if (zero_x) x[i] = (T)0;
        v[0] += (double)fi * (double)fi;
    }
    if (reduce_last_block<1>(v, partials, ticket, tot)) cg_finalize(mode, tot, sc, nullptr);
}

// mass CG start: x = 0, r = f, z = invd r; reduce f.f
__global__ void k_mass_start(int n, const double *__restrict__ f, double *__restrict__ x, double *__restrict__ r,
                             double *__restrict__ z, const double *__restrict__ invd, CgScal *sc, double *partials,
                             unsigned *ticket)
{
    pdl_enter();
    double v[1] = {0.0}, tot[1];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double fi = f[i];
        r[i] = fi;
        x[i] = 0.0;
        z[i] = invd[i] * fi;
        v[0] += fi * fi;
    }
    if (reduce_last_block<1>(v, partials, ticket, tot)) cg_finalize(F_START, tot, sc, nullptr);
}

// K1: s = A z, reduce (r, z) and (z, s) -> alpha, beta.  z may be FP32 (the
// output of an FP32 V-cycle) while A, r and s are FP64.
template <typename T, typename Z, int TPR>
__global__ void k_cg2_spmv(MatView<T> A, const Z *__restrict__ z, const T *__restrict__ r, T *__restrict__ s,
                           CgScal *sc, double *partials, unsigned *ticket)
{
    pdl_enter();
    SKIP_DONE();
    int row = my_row<TPR>();
    T v = row_sum<T, TPR>(A, row, [&](int c) { return (T)__ldg(&z[c]); });
    double a[2] = {0.0, 0.0}, tot[2];
    if (row < A.rows && row_leader<TPR>()) {
        s[row] = v;
        double zr = (double)z[row];
        a[0] = (double)r[row] * zr;
        a[1] = zr * (double)v;
    }
    if (reduce_last_block<2>(a, partials, ticket, tot)) cg_finalize(F_CG2, tot, sc, nullptr);
}

// K1 with the products on the FP32 pipe: s = (A_hi + A_lo) z accumulated in
// double-float (about 2^-48 relative), converted to FP64 per row
template <typename Z, int TPR>
__global__ void k_cg2_spmv_df(MatView<float> A, const float *__restrict__ lo, const Z *__restrict__ z,
                              const double *__restrict__ r, double *__restrict__ s, CgScal *sc, double *partials,
                              unsigned *ticket)
{
    pdl_enter();
    SKIP_DONE();
    int row = my_row<TPR>();
    double v = row_sum_df<Z, TPR>(A, lo, row, z);
    double a[2] = {0.0, 0.0}, tot[2];
    if (row < A.rows && row_leader<TPR>()) {
        s[row] = v;
        double zr = (double)z[row];
        a[0] = r[row] * zr;
        a[1] = zr * v;
    }
    if (reduce_last_block<2>(a, partials, ticket, tot)) cg_finalize(F_CG2, tot, sc, nullptr);
}

// K2: p = z + beta p, q = s + beta q, x += alpha p, r -= alpha q, reduce r.r;
// optionally r32 = r (input of an FP32 V-cycle) or, for the Jacobi-
// preconditioned mass CG, z = invd r for the next K1.
template <typename T, typename Z>
__global__ void k_cg2_update(int n, Z *__restrict__ z, const T *__restrict__ s, T *__restrict__ pv,
                             T *__restrict__ q, T *__restrict__ x, T *__restrict__ r, float *__restrict__ r32,
                             const double *__restrict__ invd, T *__restrict__ vd, T *__restrict__ vx,
                             const T *__restrict__ vinvd, T c0, CgScal *sc, double *partials, unsigned *ticket)
{
    pdl_enter();
    SKIP_DONE();
    T a = (T)sc->alpha, b = (T)sc->beta;
    bool first = sc->beta == 0.0;
    double v[1] = {0.0}, tot[1];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        T zi = (T)z[i];
        T pi = first ? zi : zi + b * pv[i];
        T qi = first ? s[i] : s[i] + b * q[i];
        pv[i] = pi;
        q[i] = qi;
        x[i] = x[i] + a * pi;
        T ri = r[i] - a * qi;
        r[i] = ri;
        if (r32) r32[i] = (float)ri;
        if (invd) z[i] = (Z)(invd[i] * (double)ri);
        if (vd) { // the V-cycle's first smoother step on the new residual
            T v0 = cheb_first_point(ri, vinvd[i], c0);
            vd[i] = v0;
            vx[i] = v0;
        }
        v[0] += (double)ri * (double)ri;
    }
    if (reduce_last_block<1>(v, partials, ticket, tot)) cg_finalize(F_RR, tot, sc, nullptr);
}

// rz = r.z and p = z (first iteration) or beta from rz (later)
template <typename T>
__global__ void k_rz(int n, const T *__restrict__ r, const T *__restrict__ z, T *__restrict__ pv, CgScal *sc,
                     int first, double *partials, unsigned *ticket)
{
    pdl_enter();
    SKIP_DONE();
    double v[1] = {0.0}, tot[1];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        T zi = z[i];
        if (first) pv[i] = zi;
        v[0] += (double)r[i] * (double)zi;
    }
    if (reduce_last_block<1>(v, partials, ticket, tot)) cg_finalize(first ? F_RZ_FIRST : F_RZ_NEXT, tot, sc, nullptr);
}

// p = z + beta p
template <typename T>
__global__ void k_xpay(int n, const T *__restrict__ z, T *__restrict__ pv, const CgScal *sc)
{
    pdl_enter();
    SKIP_DONE();
    T b = (T)sc->beta;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) pv[i] = z[i] + b * pv[i];
}

// outer CG: x += alpha p, r -= alpha q, reduce r.r -> stop test
__global__ void k_update(int n, double *__restrict__ x, double *__restrict__ r, const double *__restrict__ pv,
                         const double *__restrict__ q, CgScal *sc, double *partials, unsigned *ticket)
{
    pdl_enter();
    SKIP_DONE();
    double a = sc->alpha;
    double v[1] = {0.0}, tot[1];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        x[i] = x[i] + a * pv[i];
        double ri = r[i] - a * q[i];
        r[i] = ri;
        v[0] += ri * ri;
    }
    if (reduce_last_block<1>(v, partials, ticket, tot)) cg_finalize(F_RR, tot, sc, nullptr);
}

// generic dot with finaliser (outer CG: p.Hp; r.z)
__global__ void k_dot(int n, const double *__restrict__ x, const double *__restrict__ y, CgScal *sc, int mode,
                      double *out, double *partials, unsigned *ticket)
{
    pdl_enter();
    if (sc && mode != F_STORE && sc->done) return;
    double v[1] = {0.0}, tot[1];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v[0] += x[i] * y[i];
    if (reduce_last_block<1>(v, partials, ticket, tot)) cg_finalize(mode, tot, sc, out);
}

// refinement: r32 = r / scale
__global__ void k_ref_to32(int n, const double *__restrict__ r, float *__restrict__ r32, const CgScal *rs)
{
    pdl_enter();
    if (rs->done) return;
    double inv = 1.0 / rs->scale;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        r32[i] = (float)(r[i] * inv);
}

// refinement: y += scale * e
__global__ void k_ref_add(int n, double *__restrict__ y, const float *__restrict__ e, const CgScal *rs)
{
    pdl_enter();
    if (rs->done) return;
    double s = rs->scale;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        y[i] = y[i] + s * (double)e[i];
}

// refinement: r = f - A y (FP64), reduce r.r -> stop test
template <typename T, int TPR>
__global__ void k_ref_resid(MatView<T> A, const T *__restrict__ f, const T *__restrict__ y, T *__restrict__ r,
                            CgScal *rs, double *partials, unsigned *ticket)
{
    pdl_enter();
    if (rs->done) return;
    int i = my_row<TPR>();
    T ay = row_sum<T, TPR>(A, i, [&](int c) { return __ldg(&y[c]); });
    double v[1] = {0.0}, tot[1];
    if (i < A.rows && row_leader<TPR>()) {
        T ri = f[i] - ay;
        r[i] = ri;
        v[0] = (double)ri * (double)ri;
    }
    if (reduce_last_block<1>(v, partials, ticket, tot)) cg_finalize(F_REF_UPDATE, tot, rs, nullptr);
}

__global__ void k_set_scal(CgScal *sc, double tol2, int maxit)
{
    pdl_enter();
    sc->thr = tol2;
    sc->maxit = maxit;
    sc->done = 0;
    sc->iters = 0;
    sc->k1 = 0;
    sc->beta = 0.0;
    sc->status = CG_RUNNING;
}

__global__ void k_axpby(int n, double a, const double *__restrict__ x, double b, const double *__restrict__ y,
                        double *__restrict__ out)
{
    pdl_enter();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = a * x[i] + b * (y ? y[i] : 0.0);
}

__global__ void k_fill(int n, double v, double *__restrict__ x)
{
    pdl_enter();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] = v;
}

// ------------------------------------------------------------------ host side
static int set_scal(amgh_problem *p, CgScal *sc, double tol, int maxit)
{
    pdl_launch(k_set_scal, dim3(1), dim3(1), 0, p->stream, sc, tol * tol, maxit);
    LAUNCH_CHECK();
    return AMGH_OK;
}

// single-reduction CG pieces (templated on the vector type T and the type Z of z)
template <typename Z>
static int cg2_spmv_df(amgh_problem *p, RedSlot &red, const DevCsr &a, const Z *z, const double *r, double *s,
                       CgScal *sc)
{
    MatView<float> A = view<float>(a);
    const float *lo = a.lo32;
    const int cls = fine_cls(p, a.rows, KC_CGSPMV0, KC_CGSPMV);
    timer_begin(p, cls);
    switch (A.tpr) {
    case 2: pdl_launch(k_cg2_spmv_df<Z, 2>, dim3(rows_grid(A.rows, 2)), dim3(TPB), 0, p->stream, A, lo, z, r, s, sc, red.partials, red.ticket); break;
    case 4: pdl_launch(k_cg2_spmv_df<Z, 4>, dim3(rows_grid(A.rows, 4)), dim3(TPB), 0, p->stream, A, lo, z, r, s, sc, red.partials, red.ticket); break;
    case 8: pdl_launch(k_cg2_spmv_df<Z, 8>, dim3(rows_grid(A.rows, 8)), dim3(TPB), 0, p->stream, A, lo, z, r, s, sc, red.partials, red.ticket); break;
    case 16: pdl_launch(k_cg2_spmv_df<Z, 16>, dim3(rows_grid(A.rows, 16)), dim3(TPB), 0, p->stream, A, lo, z, r, s, sc, red.partials, red.ticket); break;
    case 32: pdl_launch(k_cg2_spmv_df<Z, 32>, dim3(rows_grid(A.rows, 32)), dim3(TPB), 0, p->stream, A, lo, z, r, s, sc, red.partials, red.ticket); break;
    default: pdl_launch(k_cg2_spmv_df<Z, 1>, dim3(rows_grid(A.rows, 1)), dim3(TPB), 0, p->stream, A, lo, z, r, s, sc, red.partials, red.ticket); break;
    }
    LAUNCH_CHECK();
    // FP32 hi and lo values, indices, z gathered; FP64 r read and s written
    timer_end(p, cls, spmv_bytes(a, 4) + 4.0 * a.nnz + (16.0 - 4.0) * a.rows);
    return AMGH_OK;
}

template <typename T, typename Z>
int cg2_spmv(amgh_problem *p, RedSlot &red, const DevCsr &a, const Z *z, const T *r, T *s, CgScal *sc, int timed)
{
    // FP64 CG operator applied to an FP32 z with the hi/lo split available:
    // products on the FP32 pipe
    if (sizeof(T) == 8 && sizeof(Z) == 4 && a.lo32 && p->df_spmv)
        return cg2_spmv_df<Z>(p, red, a, z, (const double *)r, (double *)s, sc);
    (void)timed;
    MatView<T> A = view<T>(a);
    const int cls = fine_cls(p, a.rows, KC_CGSPMV0, KC_CGSPMV);
    timer_begin(p, cls);
    switch (A.tpr) {
    case 2: pdl_launch(k_cg2_spmv<T, Z, 2>, dim3(rows_grid(A.rows, 2)), dim3(TPB), 0, p->stream, A, z, r, s, sc, red.partials, red.ticket); break;
    case 4: pdl_launch(k_cg2_spmv<T, Z, 4>, dim3(rows_grid(A.rows, 4)), dim3(TPB), 0, p->stream, A, z, r, s, sc, red.partials, red.ticket); break;
    case 8: pdl_launch(k_cg2_spmv<T, Z, 8>, dim3(rows_grid(A.rows, 8)), dim3(TPB), 0, p->stream, A, z, r, s, sc, red.partials, red.ticket); break;
    case 16: pdl_launch(k_cg2_spmv<T, Z, 16>, dim3(rows_grid(A.rows, 16)), dim3(TPB), 0, p->stream, A, z, r, s, sc, red.partials, red.ticket); break;
    case 32: pdl_launch(k_cg2_spmv<T, Z, 32>, dim3(rows_grid(A.rows, 32)), dim3(TPB), 0, p->stream, A, z, r, s, sc, red.partials, red.ticket); break;
    default: pdl_launch(k_cg2_spmv<T, Z, 1>, dim3(rows_grid(A.rows, 1)), dim3(TPB), 0, p->stream, A, z, r, s, sc, red.partials, red.ticket); break;
    }
    LAUNCH_CHECK();
    // matrix + gather of z + reads of r, z + write of s
    timer_end(p, cls, spmv_bytes(a, sizeof(T)) - (double)sizeof(T) * a.cols + (double)sizeof(Z) * a.cols +
                            (double)(sizeof(T) + sizeof(Z)) * a.rows);
    return AMGH_OK;
}

template <typename T, typename Z>
int cg2_update(amgh_problem *p, RedSlot &red, int n, Z *z, const T *s, T *pv, T *q, T *x, T *r, float *r32,
               const double *invd, CgScal *sc, T *vd, T *vx, const T *vinvd, double c0)
{
    const int cls = fine_cls(p, n, KC_CGUPD0, KC_CGUPD);
    timer_begin(p, cls);
    pdl_launch(k_cg2_update<T, Z>, dim3(vec_blocks(n)), dim3(TPB), 0, p->stream, n, z, s, pv, q, x, r, r32, invd,
               vd, vx, vinvd, (T)c0, sc, red.partials, red.ticket);
    LAUNCH_CHECK();
    // z, s, p, q, x, r read; p, q, x, r written; the optional FP32 copy of r,
    // Jacobi z and the V-cycle's first step
    const double tb = sizeof(T);
    timer_end(p, cls, n * (sizeof(Z) + 9.0 * tb + (r32 ? 4.0 : 0.0) + (invd ? 8.0 + sizeof(Z) : 0.0) +
                           (vd ? 3.0 * tb : 0.0)));
    return AMGH_OK;
}

template int cg2_spmv<double, double>(amgh_problem *, RedSlot &, const DevCsr &, const double *, const double *,
                                      double *, CgScal *, int);
template int cg2_spmv<double, float>(amgh_problem *, RedSlot &, const DevCsr &, const float *, const double *,
                                     double *, CgScal *, int);
template int cg2_spmv<float, float>(amgh_problem *, RedSlot &, const DevCsr &, const float *, const float *, float *,
                                    CgScal *, int);
template int cg2_update<double, double>(amgh_problem *, RedSlot &, int, double *, const double *, double *, double *,
                                        double *, double *, float *, const double *, CgScal *, double *, double *,
                                        const double *, double);
template int cg2_update<double, float>(amgh_problem *, RedSlot &, int, float *, const double *, double *, double *,
                                       double *, double *, float *, const double *, CgScal *, double *, double *,
                                       const double *, double);
template int cg2_update<float, float>(amgh_problem *, RedSlot &, int, float *, const float *, float *, float *,
                                      float *, float *, float *, const double *, CgScal *, float *, float *,
                                      const float *, double);

template <typename T>
int cg_start(amgh_problem *p, RedSlot &red, int n, const T *f, T *x, T *r, CgScal *sc, double tol, int maxit,
             int zero_x)
{
    TRY(set_scal(p, sc, tol, maxit));
    timer_begin(p, KC_VEC);
    pdl_launch(k_cg_start<T>, dim3(vec_blocks(n)), dim3(TPB), 0, p->stream, n, f, x, r, sc, zero_x, red.partials, red.ticket, F_START);
    LAUNCH_CHECK();
    timer_end(p, KC_VEC, 3.0 * sizeof(T) * n);
    return AMGH_OK;
}
template int cg_start<double>(amgh_problem *, RedSlot &, int, const double *, double *, double *, CgScal *, double,
                              int, int);
template int cg_start<float>(amgh_problem *, RedSlot &, int, const float *, float *, float *, CgScal *, double, int,
                             int);

int cg_update_outer(amgh_problem *p, RedSlot &red, int n, double *x, double *r, const double *pv, const double *q,
                    CgScal *sc)
{
    timer_begin(p, KC_VEC);
    pdl_launch(k_update, dim3(vec_blocks(n)), dim3(TPB), 0, p->stream, n, x, r, pv, q, sc, red.partials, red.ticket);
    LAUNCH_CHECK();
    timer_end(p, KC_VEC, 48.0 * n);
    return AMGH_OK;
}

// mass CG pieces
int mass_start(amgh_problem *p, RedSlot &red, int n, const double *f, double *x, double *r, double *z,
               const double *invd, CgScal *sc, double tol, int maxit)
{
    TRY(set_scal(p, sc, tol, maxit));
    timer_begin(p, KC_VEC);
    pdl_launch(k_mass_start, dim3(vec_blocks(n)), dim3(TPB), 0, p->stream, n, f, x, r, z, invd, sc, red.partials, red.ticket);
    LAUNCH_CHECK();
    timer_end(p, KC_VEC, 40.0 * n);
    return AMGH_OK;
}

// outer CG pieces (operator applied by the host between them)
int outer_dot(amgh_problem *p, RedSlot &red, int n, const double *x, const double *y, CgScal *sc, int mode)
{
    timer_begin(p, KC_VEC);
    pdl_launch(k_dot, dim3(vec_blocks(n)), dim3(TPB), 0, p->stream, n, x, y, sc, mode, nullptr, red.partials, red.ticket);
    LAUNCH_CHECK();
    timer_end(p, KC_VEC, 16.0 * n);
    return AMGH_OK;
}

int outer_pq(amgh_problem *p, RedSlot &red, int n, const double *pv, const double *q, CgScal *sc)
{
    return outer_dot(p, red, n, pv, q, sc, F_PQ);
}

int outer_rz(amgh_problem *p, RedSlot &red, int n, const double *r, const double *z, double *pv, CgScal *sc,
             int first)
{
    timer_begin(p, KC_VEC);
    pdl_launch(k_rz<double>, dim3(vec_blocks(n)), dim3(TPB), 0, p->stream, n, r, z, pv, sc, first, red.partials, red.ticket);
    LAUNCH_CHECK();
    timer_end(p, KC_VEC, (first ? 24.0 : 16.0) * n);
    if (!first) {
        timer_begin(p, KC_VEC);
        pdl_launch(k_xpay<double>, dim3(vec_blocks(n)), dim3(TPB), 0, p->stream, n, z, pv, sc);
        LAUNCH_CHECK();
        timer_end(p, KC_VEC, 24.0 * n);
    }
    return AMGH_OK;
}

int vec_dot(amgh_problem *p, RedSlot &red, int n, const double *x, const double *y, double *out_dev)
{
    timer_begin(p, KC_VEC);
    pdl_launch(k_dot, dim3(vec_blocks(n)), dim3(TPB), 0, p->stream, n, x, y, nullptr, F_STORE, out_dev, red.partials, red.ticket);
    LAUNCH_CHECK();
    timer_end(p, KC_VEC, 16.0 * n);
    return AMGH_OK;
}

// refinement pieces
int ref_start(amgh_problem *p, RedSlot &red, int n, const double *f, double *y, double *r, CgScal *rs, double tol,
              int maxit)
{
    TRY(set_scal(p, rs, tol, maxit));
    timer_begin(p, KC_VEC);
    pdl_launch(k_cg_start<double>, dim3(vec_blocks(n)), dim3(TPB), 0, p->stream, n, f, y, r, rs, 1, red.partials, red.ticket,
                                                             F_REF_START);
    LAUNCH_CHECK();
    timer_end(p, KC_VEC, 24.0 * n);
    return AMGH_OK;
}

int ref_to32(amgh_problem *p, RedSlot & /*red*/, int n, const double *r, float *r32, CgScal *rs)
{
    timer_begin(p, KC_VEC);
    pdl_launch(k_ref_to32, dim3(vec_blocks(n)), dim3(TPB), 0, p->stream, n, r, r32, rs);
    LAUNCH_CHECK();
    timer_end(p, KC_VEC, 12.0 * n);
    return AMGH_OK;
}

int ref_update(amgh_problem *p, RedSlot &red, const DevCsr &a, const double *f, double *y, const float *e32,
               double *r, CgScal *rs)
{
    int n = a.rows;
    timer_begin(p, KC_VEC);
    pdl_launch(k_ref_add, dim3(vec_blocks(n)), dim3(TPB), 0, p->stream, n, y, e32, rs);
    LAUNCH_CHECK();
    timer_end(p, KC_VEC, 20.0 * n);
    MatView<double> A = view<double>(a);
    timer_begin(p, KC_SPMV);
    switch (A.tpr) {
    case 2: pdl_launch(k_ref_resid<double, 2>, dim3(rows_grid(n, 2)), dim3(TPB), 0, p->stream, A, f, y, r, rs, red.partials, red.ticket); break;
    case 4: pdl_launch(k_ref_resid<double, 4>, dim3(rows_grid(n, 4)), dim3(TPB), 0, p->stream, A, f, y, r, rs, red.partials, red.ticket); break;
    case 8: pdl_launch(k_ref_resid<double, 8>, dim3(rows_grid(n, 8)), dim3(TPB), 0, p->stream, A, f, y, r, rs, red.partials, red.ticket); break;
    case 16: pdl_launch(k_ref_resid<double, 16>, dim3(rows_grid(n, 16)), dim3(TPB), 0, p->stream, A, f, y, r, rs, red.partials, red.ticket); break;
    case 32: pdl_launch(k_ref_resid<double, 32>, dim3(rows_grid(n, 32)), dim3(TPB), 0, p->stream, A, f, y, r, rs, red.partials, red.ticket); break;
    default: pdl_launch(k_ref_resid<double, 1>, dim3(rows_grid(n, 1)), dim3(TPB), 0, p->stream, A, f, y, r, rs, red.partials, red.ticket); break;
    }
    LAUNCH_CHECK();
    timer_end(p, KC_SPMV, spmv_bytes(a, 8) + 8.0 * n);
    return AMGH_OK;
}

int vec_axpby(amgh_problem *p, int n, double a, const double *x, double b, const double *y, double *out)
{
    if (n == 0) return AMGH_OK;
    timer_begin(p, KC_VEC);
    pdl_launch(k_axpby, dim3(vec_blocks(n)), dim3(TPB), 0, p->stream, n, a, x, b, y, out);
    LAUNCH_CHECK();
    timer_end(p, KC_VEC, (y ? 24.0 : 16.0) * n);
    return AMGH_OK;
}

int vec_fill(amgh_problem *p, int n, double v, double *x)
{
    if (n == 0) return AMGH_OK;
    timer_begin(p, KC_VEC);
    pdl_launch(k_fill, dim3(vec_blocks(n)), dim3(TPB), 0, p->stream, n, v, x);
    LAUNCH_CHECK();
    timer_end(p, KC_VEC, 8.0 * n);
    return AMGH_OK;
}

// ------------------------------------------------------------------ double-float CG
// Inner CG of precision mode 2 with every vector (x, r, p, q, s) held as
// double-float: the FP64-sized buffer of n doubles is used as two FP32 arrays,
// hi = [0, n) and lo = [n, 2n).  All per-element arithmetic stays on the FP32
// pipe; the FP32 V-cycle reads r's hi half directly.  Reductions stay in
// double-float across lanes, warps and blocks; only the final sums become FP64
// for the CG scalars.

// ||f||^2 -> sc->scale, the power of two nearest 1 / ||f||.  The double-float
// CG solves for the scaled right side (an exact scaling) so that its FP32
// halves stay far from the FP32 exponent limits whatever the size of f.
__global__ void k_df_norm(int n, const double *__restrict__ f, CgScal *sc, double *partials, unsigned *ticket)
{
    pdl_enter();
    double v[1] = {0.0}, tot[1];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v[0] += f[i] * f[i];
    if (reduce_last_block<1>(v, partials, ticket, tot)) cg_finalize(F_SCALE, tot, sc, nullptr);
}

// r = scale f (split into hi/lo), x = 0, reduce (scale f).(scale f)
__global__ void k_df_start(int n, const double *__restrict__ f, float *__restrict__ xh, float *__restrict__ xl,
                           float *__restrict__ rh, float *__restrict__ rl, CgScal *sc, double *partials,
                           unsigned *ticket)
{
    pdl_enter();
    DF acc = {0.f, 0.f}, tot_df[1];
    double tot[1];
    double scale = sc->scale;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        DF fi = df_from_double(scale * f[i]);
        rh[i] = fi.hi;
        rl[i] = fi.lo;
        xh[i] = 0.f;
        xl[i] = 0.f;
        acc = df_add_fast(acc, df_mul2(fi, fi));
    }
    tot_df[0] = acc;
    if (reduce_df_last_block<1>(tot_df, partials, ticket, tot)) cg_finalize(F_START, tot, sc, nullptr);
}

// K1: s = A z (FP32 z), reduce (r, z) and (z, s) -> alpha, beta
template <int TPR>
__global__ void k_df_spmv(MatView<float> A, const float *__restrict__ lo, const float *__restrict__ z,
                          const float *__restrict__ rh, const float *__restrict__ rl, float *__restrict__ sh,
                          float *__restrict__ sl, CgScal *sc, double *partials, unsigned *ticket)
{
    pdl_enter();
    SKIP_DONE();
    // a grid that fits on the GPU at once walks the rows, so each block pays
    // its reduction tail once for several rows per thread
    DF a[2] = {{0.f, 0.f}, {0.f, 0.f}};
    double tot[2];
    const int stride = gridDim.x * blockDim.x, slots = A.rows * TPR;
    for (int base = blockIdx.x * blockDim.x; base < slots; base += stride) {
        int row = (base + (int)threadIdx.x) / TPR;
        bool lead = row < A.rows && row_leader<TPR>();
        float zr = 0.f, rhr = 0.f, rlr = 0.f;
        if (lead) {
            zr = z[row];
            rhr = rh[row];
            rlr = rl[row];
        }
        DF v = row_sum_dfv<float, TPR>(A, lo, row, z);
        if (lead) {
            sh[row] = v.hi;
            sl[row] = v.lo;
            a[0] = df_add_fast(a[0], df_mulf(DF{rhr, rlr}, zr));
            a[1] = df_add_fast(a[1], df_mulf(v, zr));
        }
    }
    if (reduce_df_last_block<2>(a, partials, ticket, tot)) cg_finalize(F_CG2, tot, sc, nullptr);
}

// K2: p = z + beta p, q = s + beta q, x += alpha p, r -= alpha q, reduce r.r
// With invd32 the preconditioner is Jacobi and the new z = D^-1 r (FP32, from
// r's hi half) is written over z in the same pass (element i is read before it
// is written, by the same thread).
__global__ void k_df_update(int n, const float *z, const float *__restrict__ sh, const float *__restrict__ sl,
                            float *__restrict__ ph, float *__restrict__ pl, float *__restrict__ qh,
                            float *__restrict__ ql, float *__restrict__ xh, float *__restrict__ xl,
                            float *__restrict__ rh, float *__restrict__ rl, const float *__restrict__ invd32,
                            float *znew, float *__restrict__ vd, float *__restrict__ vx, float c0, CgScal *sc,
                            double *partials, unsigned *ticket)
{
    pdl_enter();
    SKIP_DONE();
    DF al = {sc->ahi, sc->alo}, be = {sc->bhi, sc->blo};
    DF nal = {-al.hi, -al.lo};
    bool first = sc->beta == 0.0;
    DF acc = {0.f, 0.f}, tot_df[1];
    double tot[1];
    // operands of one element: z, s, p, q, x, r (hi/lo) and D^-1
    struct In {
        float z, s1, s2, p1, p2, q1, q2, x1, x2, r1, r2, iv;
    };
    auto load = [&](int i, In &e) {
        e.z = z[i];
        e.s1 = sh[i];
        e.s2 = sl[i];
        e.p1 = ph[i];
        e.p2 = pl[i];
        e.q1 = qh[i];
        e.q2 = ql[i];
        e.x1 = xh[i];
        e.x2 = xl[i];
        e.r1 = rh[i];
        e.r2 = rl[i];
        e.iv = invd32 ? invd32[i] : 0.f;
    };
    auto step = [&](int i, const In &e) {
        DF zi = {e.z, 0.f};
        DF si = {e.s1, e.s2};
        DF pi = first ? zi : df_add2(zi, df_mul2(be, DF{e.p1, e.p2}));
        DF qi = first ? si : df_add2(si, df_mul2(be, DF{e.q1, e.q2}));
        DF xi = df_add2(DF{e.x1, e.x2}, df_mul2(al, pi));
        DF ri = df_add2(DF{e.r1, e.r2}, df_mul2(nal, qi));
        ph[i] = pi.hi;
        pl[i] = pi.lo;
        qh[i] = qi.hi;
        ql[i] = qi.lo;
        xh[i] = xi.hi;
        xl[i] = xi.lo;
        rh[i] = ri.hi;
        rl[i] = ri.lo;
        if (vd) {
            // the V-cycle's first smoother step from zero on the new residual
            float v = cheb_first_point(ri.hi, e.iv, c0);
            vd[i] = v;
            vx[i] = v;
        } else if (invd32) {
            znew[i] = ri.hi * e.iv;
        }
        acc = df_add_fast(acc, df_mul2(ri, ri)); // squares: no cancellation
    };
    // two elements (one stride apart) per pass with all their loads issued
    // first; r.r takes them in the order one element per pass would
    const int stride = gridDim.x * blockDim.x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += 2 * stride) {
        const int j = i + stride;
        In e0, e1;
        load(i, e0);
        if (j < n) load(j, e1);
        step(i, e0);
        if (j < n) step(j, e1);
    }
    tot_df[0] = acc;
    if (reduce_df_last_block<1>(tot_df, partials, ticket, tot)) cg_finalize(F_RR, tot, sc, nullptr);
}

// y = x / scale (exact: scale is a power of two)
__global__ void k_df_to_double(int n, const float *__restrict__ xh, const float *__restrict__ xl,
                               const CgScal *sc, double *__restrict__ y)
{
    pdl_enter();
    double inv = 1.0 / sc->scale;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        y[i] = ((double)xh[i] + (double)xl[i]) * inv;
}

static inline float *hi_of(double *b) { return (float *)b; }
static inline float *lo_of(double *b, int n) { return (float *)b + n; }
static inline const float *hi_of(const double *b) { return (const float *)b; }
static inline const float *lo_of(const double *b, int n) { return (const float *)b + n; }

int dfcg_start(amgh_problem *p, RedSlot &red, int n, const double *f, double *x, double *r, CgScal *sc, double tol,
               int maxit)
{
    TRY(set_scal(p, sc, tol, maxit));
    timer_begin(p, KC_VEC);
    pdl_launch(k_df_norm, dim3(vec_blocks(n)), dim3(TPB), 0, p->stream, n, f, sc, red.partials, red.ticket);
    LAUNCH_CHECK();
    timer_end(p, KC_VEC, 8.0 * n);
    timer_begin(p, KC_VEC);
    pdl_launch(k_df_start, dim3(std::min(vec_blocks(n), resident_grid((const void *)k_df_start, TPB))), dim3(TPB), 0, p->stream, n, f, hi_of(x), lo_of(x, n), hi_of(r), lo_of(r, n), sc,
                                                    red.partials, red.ticket);
    LAUNCH_CHECK();
    timer_end(p, KC_VEC, 24.0 * n);
    return AMGH_OK;
}

int dfcg_spmv(amgh_problem *p, RedSlot &red, const DevCsr &a, const float *z, const double *r, double *s,
              CgScal *sc, int timed)
{
    (void)timed;
    MatView<float> A = view<float>(a);
    int n = a.rows;
    const float *lo = a.lo32;
    const int cls = fine_cls(p, n, KC_CGSPMV0, KC_CGSPMV);
    timer_begin(p, cls);
#define DFSPMV(TPR)                                                                                            \
    pdl_launch(k_df_spmv<TPR>,                                                                                 \
               dim3(std::min(rows_grid(n, TPR), resident_grid((const void *)k_df_spmv<TPR>, TPB))), dim3(TPB), \
               0, p->stream, A, lo, z, hi_of(r), lo_of(r, n), hi_of(s), lo_of(s, n), sc, red.partials, red.ticket)
    switch (A.tpr) {
    case 2: DFSPMV(2); break;
    case 4: DFSPMV(4); break;
    case 8: DFSPMV(8); break;
    case 16: DFSPMV(16); break;
    case 32: DFSPMV(32); break;
    default: DFSPMV(1); break;
    }
#undef DFSPMV
    LAUNCH_CHECK();
    // FP32 hi and lo values, indices, z gathered; r read and s written as hi + lo
    timer_end(p, cls, spmv_bytes(a, 4) + 4.0 * a.nnz + (16.0 - 4.0) * n);
    return AMGH_OK;
}

int dfcg_update(amgh_problem *p, RedSlot &red, int n, const float *z, const double *s, double *pv, double *q,
                double *x, double *r, CgScal *sc, const float *invd32, float *vd, float *vx, double c0)
{
    const int cls = fine_cls(p, n, KC_CGUPD0, KC_CGUPD);
    timer_begin(p, cls);
    pdl_launch(k_df_update, dim3(std::min(vec_blocks(n), resident_grid((const void *)k_df_update, TPB))), dim3(TPB), 0, p->stream, n, z, hi_of(s), lo_of(s, n), hi_of(pv), lo_of(pv, n),
                                                     hi_of(q), lo_of(q, n), hi_of(x), lo_of(x, n), hi_of(r),
                                                     lo_of(r, n), invd32, (float *)z, vd, vx, (float)c0, sc, red.partials, red.ticket);
    LAUNCH_CHECK();
    // z (FP32), s, p, q, x, r (hi + lo) read; p, q, x, r written; D^-1 read
    // and either z (Jacobi) or the V-cycle's d and x written
    timer_end(p, cls, n * (4.0 + 9.0 * 8.0 + (invd32 ? 4.0 + (vd ? 8.0 : 4.0) : 0.0)));
    return AMGH_OK;
}

// z = D^-1 r from r's hi half (Jacobi start of the double-float mass CG)
__global__ void k_df_jacobi(int n, const float *__restrict__ rh, const float *__restrict__ invd32,
                            float *__restrict__ z)
{
    pdl_enter();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) z[i] = rh[i] * invd32[i];
}

int dfcg_jacobi(amgh_problem *p, int n, const double *r, const float *invd32, float *z)
{
    timer_begin(p, KC_VEC);
    pdl_launch(k_df_jacobi, dim3(std::min(vec_blocks(n), resident_grid((const void *)k_df_jacobi, TPB))), dim3(TPB), 0, p->stream, n, hi_of(r), invd32, z);
    LAUNCH_CHECK();
    timer_end(p, KC_VEC, 12.0 * n);
    return AMGH_OK;
}

int df_to_double(amgh_problem *p, int n, const double *x, const CgScal *sc, double *y)
{
    timer_begin(p, KC_VEC);
    pdl_launch(k_df_to_double, dim3(std::min(vec_blocks(n), resident_grid((const void *)k_df_to_double, TPB))), dim3(TPB), 0, p->stream, n, hi_of(x), lo_of(x, n), sc, y);
    LAUNCH_CHECK();
    timer_end(p, KC_VEC, 16.0 * n);
    return AMGH_OK;
}
