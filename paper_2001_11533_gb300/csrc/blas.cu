// blas.cu -- conjugate-gradient building blocks with device-resident scalars.
//
// Every CG loop keeps its scalars (r.z, p.q, alpha, beta, ||r||^2, the
// stopping threshold, an iteration count and a `done` flag) in a CgScal in
// device memory.  Each kernel below fuses a vector update with the next
// inner product; its reduction is two-stage and deterministic (block
// partials summed in fixed order by the last block to finish), and that last
// block also computes the new alpha / beta or the stopping decision.  Every
// kernel returns at once when `done` is set, so the host can enqueue several
// iterations ahead and only read the flag back now and then.
#include <math.h>

#include "internal.cuh"
#include "util.cuh"

static const int TPB = 256;

static inline int vec_blocks(int64_t n)
{
    int nb = ceil_div(n > 0 ? n : 1, TPB);
    return nb < 2432 ? nb : 2432; // 152 SMs x 16 blocks of 256 threads
}

int red_alloc(Arena &ar, RedSlot &slot, int capacity_rows)
{
    int cap = ceil_div(capacity_rows > 0 ? capacity_rows : 1, TPB) + 8;
    slot.capacity = cap;
    TRY(ar.alloc(&slot.partials, (int64_t)cap * 2));
    TRY(ar.alloc(&slot.ticket, 1));
    CU(cudaMemset(slot.ticket, 0, sizeof(unsigned)));
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
    }
}

#define SKIP_DONE() \
    if (sc->done) return

// x = 0 (optional), r = f, reduce f.f ; host put tol^2 in sc->thr and maxit
template <typename T>
__global__ void k_cg_start(int n, const T *__restrict__ f, T *__restrict__ x, T *__restrict__ r, CgScal *sc,
                           int zero_x, double *partials, unsigned *ticket, int mode)
{
    double v[1] = {0.0}, tot[1];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        T fi = f[i];
        r[i] = fi;
        if (zero_x) x[i] = (T)0;
        v[0] += (double)fi * (double)fi;
    }
    if (reduce_last_block<1>(v, partials, ticket, tot)) cg_finalize(mode, tot, sc, nullptr);
}

// mass CG start: x = 0, r = f, z = invd r; reduce f.f and r.z (beta = 0)
__global__ void k_mass_start(int n, const double *__restrict__ f, double *__restrict__ x, double *__restrict__ r,
                             double *__restrict__ z, const double *__restrict__ invd, CgScal *sc, double *partials,
                             unsigned *ticket)
{
    double v[2] = {0.0, 0.0}, tot[2];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double fi = f[i];
        double zi = invd[i] * fi;
        r[i] = fi;
        x[i] = 0.0;
        z[i] = zi;
        v[0] += fi * fi;
        v[1] += fi * zi;
    }
    if (reduce_last_block<2>(v, partials, ticket, tot)) cg_finalize(F_MASS_START, tot, sc, nullptr);
}

// inner CG r.z without touching p (the p update is fused into the next SpMV)
template <typename T>
__global__ void k_rz_only(int n, const T *__restrict__ r, const T *__restrict__ z, CgScal *sc, int mode,
                          double *partials, unsigned *ticket)
{
    SKIP_DONE();
    double v[1] = {0.0}, tot[1];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        v[0] += (double)r[i] * (double)z[i];
    if (reduce_last_block<1>(v, partials, ticket, tot)) cg_finalize(mode, tot, sc, nullptr);
}

// z64 = z32 and r.z (FP32 V-cycle inside FP64 CG)
__global__ void k_f2d_rz(int n, const float *__restrict__ z32, double *__restrict__ z, const double *__restrict__ r,
                         CgScal *sc, int mode, double *partials, unsigned *ticket)
{
    SKIP_DONE();
    double v[1] = {0.0}, tot[1];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double zi = (double)z32[i];
        z[i] = zi;
        v[0] += r[i] * zi;
    }
    if (reduce_last_block<1>(v, partials, ticket, tot)) cg_finalize(mode, tot, sc, nullptr);
}

// p_out = z + beta p_in (p_out = z when beta = 0) and q = A p_out, reduce p.q -> alpha
template <typename T>
__global__ void k_spmv_pq_xpay(int rows, const int *__restrict__ slp, const int *__restrict__ sci,
                               const T *__restrict__ sv, const T *__restrict__ z, const T *__restrict__ pin,
                               T *__restrict__ pout, T *__restrict__ q, CgScal *sc, double *partials,
                               unsigned *ticket)
{
    SKIP_DONE();
    T b = (T)sc->beta;
    bool first = sc->beta == 0.0;
    double v[1] = {0.0}, tot[1];
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < rows) {
        int s = r >> 5, lane = r & 31;
        T acc = (T)0;
        if (first) {
            for (int k = slp[s] + lane; k < slp[s + 1]; k += 32) acc += sv[k] * __ldg(&z[sci[k]]);
        } else {
            for (int k = slp[s] + lane; k < slp[s + 1]; k += 32) {
                int c = sci[k];
                acc += sv[k] * (__ldg(&z[c]) + b * __ldg(&pin[c]));
            }
        }
        T pr = first ? z[r] : z[r] + b * pin[r];
        pout[r] = pr;
        q[r] = acc;
        v[0] = (double)pr * (double)acc;
    }
    if (reduce_last_block<1>(v, partials, ticket, tot)) cg_finalize(F_PQ, tot, sc, nullptr);
}

// rz = r.z and p = z (first iteration) or beta from rz (later)
template <typename T>
__global__ void k_rz(int n, const T *__restrict__ r, const T *__restrict__ z, T *__restrict__ pv, CgScal *sc,
                     int first, double *partials, unsigned *ticket)
{
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
    SKIP_DONE();
    T b = (T)sc->beta;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) pv[i] = z[i] + b * pv[i];
}

// x += alpha p, r -= alpha q (and r32 = r when given), reduce r.r -> stop test
template <typename T>
__global__ void k_update(int n, T *__restrict__ x, T *__restrict__ r, const T *__restrict__ pv,
                         const T *__restrict__ q, CgScal *sc, float *__restrict__ r32, double *partials,
                         unsigned *ticket)
{
    SKIP_DONE();
    T a = (T)sc->alpha;
    double v[1] = {0.0}, tot[1];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        x[i] = x[i] + a * pv[i];
        T ri = r[i] - a * q[i];
        r[i] = ri;
        if (r32) r32[i] = (float)ri;
        v[0] += (double)ri * (double)ri;
    }
    if (reduce_last_block<1>(v, partials, ticket, tot)) cg_finalize(F_RR, tot, sc, nullptr);
}

// mass CG: x += alpha p, r -= alpha q, z = invd r; reduce r.r, r.z
__global__ void k_mass_update(int n, double *__restrict__ x, double *__restrict__ r, double *__restrict__ z,
                              const double *__restrict__ pv, const double *__restrict__ q,
                              const double *__restrict__ invd, CgScal *sc, double *partials, unsigned *ticket)
{
    SKIP_DONE();
    double a = sc->alpha;
    double v[2] = {0.0, 0.0}, tot[2];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        x[i] = x[i] + a * pv[i];
        double ri = r[i] - a * q[i];
        r[i] = ri;
        double zi = invd[i] * ri;
        z[i] = zi;
        v[0] += ri * ri;
        v[1] += ri * zi;
    }
    if (reduce_last_block<2>(v, partials, ticket, tot)) cg_finalize(F_MASS_UPDATE, tot, sc, nullptr);
}

// generic dot with finaliser (outer CG: p.Hp; r.z)
__global__ void k_dot(int n, const double *__restrict__ x, const double *__restrict__ y, CgScal *sc, int mode,
                      double *out, double *partials, unsigned *ticket)
{
    if (sc && mode != F_STORE && sc->done) return;
    double v[1] = {0.0}, tot[1];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v[0] += x[i] * y[i];
    if (reduce_last_block<1>(v, partials, ticket, tot)) cg_finalize(mode, tot, sc, out);
}

// refinement: r32 = r / scale
__global__ void k_ref_to32(int n, const double *__restrict__ r, float *__restrict__ r32, const CgScal *rs)
{
    if (rs->done) return;
    double inv = 1.0 / rs->scale;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        r32[i] = (float)(r[i] * inv);
}

// refinement: y += scale * e
__global__ void k_ref_add(int n, double *__restrict__ y, const float *__restrict__ e, const CgScal *rs)
{
    if (rs->done) return;
    double s = rs->scale;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        y[i] = y[i] + s * (double)e[i];
}

// refinement: r = f - A y (FP64), reduce r.r -> stop test
__global__ void k_ref_resid(int rows, const int *__restrict__ slp, const int *__restrict__ sci,
                            const double *__restrict__ sv, const double *__restrict__ f,
                            const double *__restrict__ y, double *__restrict__ r, CgScal *rs, double *partials,
                            unsigned *ticket)
{
    if (rs->done) return;
    double v[1] = {0.0}, tot[1];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < rows) {
        int s = i >> 5, lane = i & 31;
        double acc = 0.0;
        for (int k = slp[s] + lane; k < slp[s + 1]; k += 32) acc += sv[k] * __ldg(&y[sci[k]]);
        double ri = f[i] - acc;
        r[i] = ri;
        v[0] = ri * ri;
    }
    if (reduce_last_block<1>(v, partials, ticket, tot)) cg_finalize(F_REF_UPDATE, tot, rs, nullptr);
}

__global__ void k_set_scal(CgScal *sc, double tol2, int maxit)
{
    sc->thr = tol2;
    sc->maxit = maxit;
    sc->done = 0;
    sc->iters = 0;
    sc->status = CG_RUNNING;
}

__global__ void k_axpby(int n, double a, const double *__restrict__ x, double b, const double *__restrict__ y,
                        double *__restrict__ out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = a * x[i] + b * (y ? y[i] : 0.0);
}

__global__ void k_fill(int n, double v, double *__restrict__ x)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] = v;
}

// ------------------------------------------------------------------ host side
static int set_scal(amgh_problem *p, CgScal *sc, double tol, int maxit)
{
    k_set_scal<<<1, 1, 0, p->stream>>>(sc, tol * tol, maxit);
    LAUNCH_CHECK();
    return AMGH_OK;
}

template <typename T>
int cg_start(amgh_problem *p, RedSlot &red, int n, const T *f, T *x, T *r, CgScal *sc, double tol, int maxit,
             int zero_x)
{
    TRY(set_scal(p, sc, tol, maxit));
    k_cg_start<T><<<vec_blocks(n), TPB, 0, p->stream>>>(n, f, x, r, sc, zero_x, red.partials, red.ticket,
                                                        F_START);
    LAUNCH_CHECK();
    return AMGH_OK;
}

template <typename T>
int cg_rz_first(amgh_problem *p, RedSlot &red, int n, const T *r, const T *z, CgScal *sc)
{
    k_rz_only<T><<<vec_blocks(n), TPB, 0, p->stream>>>(n, r, z, sc, F_RZ_FIRST, red.partials, red.ticket);
    LAUNCH_CHECK();
    return AMGH_OK;
}

template <typename T>
int cg_spmv_pq_xpay(amgh_problem *p, RedSlot &red, const DevCsr &a, const T *z, const T *pin, T *pout, T *q,
                    CgScal *sc, int timed)
{
    const T *sv;
    if (sizeof(T) == 8) sv = (const T *)a.sl_v;
    else sv = (const T *)a.sl_v32;
    timer_begin(p, timed);
    k_spmv_pq_xpay<T><<<ceil_div(a.rows, TPB), TPB, 0, p->stream>>>(a.rows, a.sl_ptr, a.sl_ci, sv, z, pin, pout, q,
                                                                    sc, red.partials, red.ticket);
    LAUNCH_CHECK();
    // matrix + gathers of z and p_in + writes of p_out and q
    timer_end(p, timed,
              (double)a.nnz * (sizeof(T) + 4) + 4.0 * (a.rows + 1) + (double)sizeof(T) * (2.0 * a.cols + 2.0 * a.rows));
    return AMGH_OK;
}

template <typename T>
int cg_update(amgh_problem *p, RedSlot &red, int n, T *x, T *r, const T *pv, const T *q, CgScal *sc, float *r32)
{
    k_update<T><<<vec_blocks(n), TPB, 0, p->stream>>>(n, x, r, pv, q, sc, r32, red.partials, red.ticket);
    LAUNCH_CHECK();
    return AMGH_OK;
}

template <typename T>
int cg_rz_next(amgh_problem *p, RedSlot &red, int n, const T *r, const T *z, CgScal *sc)
{
    k_rz_only<T><<<vec_blocks(n), TPB, 0, p->stream>>>(n, r, z, sc, F_RZ_NEXT, red.partials, red.ticket);
    LAUNCH_CHECK();
    return AMGH_OK;
}

int cg_f2d_rz(amgh_problem *p, RedSlot &red, int n, const float *z32, double *z, const double *r, CgScal *sc,
              int first)
{
    k_f2d_rz<<<vec_blocks(n), TPB, 0, p->stream>>>(n, z32, z, r, sc, first ? F_RZ_FIRST : F_RZ_NEXT, red.partials,
                                                    red.ticket);
    LAUNCH_CHECK();
    return AMGH_OK;
}

#define INST(T)                                                                                              \
    template int cg_start<T>(amgh_problem *, RedSlot &, int, const T *, T *, T *, CgScal *, double, int, int); \
    template int cg_rz_first<T>(amgh_problem *, RedSlot &, int, const T *, const T *, CgScal *);              \
    template int cg_spmv_pq_xpay<T>(amgh_problem *, RedSlot &, const DevCsr &, const T *, const T *, T *, T *,  \
                                    CgScal *, int);                                                          \
    template int cg_update<T>(amgh_problem *, RedSlot &, int, T *, T *, const T *, const T *, CgScal *, float *); \
    template int cg_rz_next<T>(amgh_problem *, RedSlot &, int, const T *, const T *, CgScal *);
INST(double)
INST(float)

// mass CG pieces
int mass_start(amgh_problem *p, RedSlot &red, int n, const double *f, double *x, double *r, double *z,
               const double *invd, CgScal *sc, double tol, int maxit)
{
    TRY(set_scal(p, sc, tol, maxit));
    k_mass_start<<<vec_blocks(n), TPB, 0, p->stream>>>(n, f, x, r, z, invd, sc, red.partials, red.ticket);
    LAUNCH_CHECK();
    return AMGH_OK;
}

int mass_iter(amgh_problem *p, RedSlot &red, const DevCsr &M, double *x, double *r, double *z, const double *pin,
              double *pout, double *q, const double *invd, CgScal *sc)
{
    int n = M.rows;
    TRY(cg_spmv_pq_xpay<double>(p, red, M, z, pin, pout, q, sc, 0));
    k_mass_update<<<vec_blocks(n), TPB, 0, p->stream>>>(n, x, r, z, pout, q, invd, sc, red.partials, red.ticket);
    LAUNCH_CHECK();
    return AMGH_OK;
}

// outer CG pieces (operator applied by the host between them)
int outer_dot(amgh_problem *p, RedSlot &red, int n, const double *x, const double *y, CgScal *sc, int mode)
{
    k_dot<<<vec_blocks(n), TPB, 0, p->stream>>>(n, x, y, sc, mode, nullptr, red.partials, red.ticket);
    LAUNCH_CHECK();
    return AMGH_OK;
}

int outer_pq(amgh_problem *p, RedSlot &red, int n, const double *pv, const double *q, CgScal *sc)
{
    return outer_dot(p, red, n, pv, q, sc, F_PQ);
}

int outer_rz(amgh_problem *p, RedSlot &red, int n, const double *r, const double *z, double *pv, CgScal *sc,
             int first)
{
    k_rz<double><<<vec_blocks(n), TPB, 0, p->stream>>>(n, r, z, pv, sc, first, red.partials, red.ticket);
    LAUNCH_CHECK();
    if (!first) {
        k_xpay<double><<<vec_blocks(n), TPB, 0, p->stream>>>(n, z, pv, sc);
        LAUNCH_CHECK();
    }
    return AMGH_OK;
}

int vec_dot(amgh_problem *p, RedSlot &red, int n, const double *x, const double *y, double *out_dev)
{
    k_dot<<<vec_blocks(n), TPB, 0, p->stream>>>(n, x, y, nullptr, F_STORE, out_dev, red.partials, red.ticket);
    LAUNCH_CHECK();
    return AMGH_OK;
}

// refinement pieces
int ref_start(amgh_problem *p, RedSlot &red, int n, const double *f, double *y, double *r, CgScal *rs, double tol,
              int maxit)
{
    TRY(set_scal(p, rs, tol, maxit));
    k_cg_start<double><<<vec_blocks(n), TPB, 0, p->stream>>>(n, f, y, r, rs, 1, red.partials, red.ticket,
                                                             F_REF_START);
    LAUNCH_CHECK();
    return AMGH_OK;
}

int ref_to32(amgh_problem *p, RedSlot & /*red*/, int n, const double *r, float *r32, CgScal *rs)
{
    k_ref_to32<<<vec_blocks(n), TPB, 0, p->stream>>>(n, r, r32, rs);
    LAUNCH_CHECK();
    return AMGH_OK;
}

int ref_update(amgh_problem *p, RedSlot &red, const DevCsr &a, const double *f, double *y, const float *e32,
               double *r, CgScal *rs)
{
    int n = a.rows;
    k_ref_add<<<vec_blocks(n), TPB, 0, p->stream>>>(n, y, e32, rs);
    LAUNCH_CHECK();
    k_ref_resid<<<ceil_div(n, TPB), TPB, 0, p->stream>>>(n, a.sl_ptr, a.sl_ci, a.sl_v, f, y, r, rs, red.partials,
                                                          red.ticket);
    LAUNCH_CHECK();
    return AMGH_OK;
}

int vec_axpby(amgh_problem *p, int n, double a, const double *x, double b, const double *y, double *out)
{
    if (n == 0) return AMGH_OK;
    k_axpby<<<vec_blocks(n), TPB, 0, p->stream>>>(n, a, x, b, y, out);
    LAUNCH_CHECK();
    return AMGH_OK;
}

int vec_fill(amgh_problem *p, int n, double v, double *x)
{
    if (n == 0) return AMGH_OK;
    k_fill<<<vec_blocks(n), TPB, 0, p->stream>>>(n, v, x);
    LAUNCH_CHECK();
    return AMGH_OK;
}
