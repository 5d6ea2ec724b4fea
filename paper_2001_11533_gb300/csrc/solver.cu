// solver.cu -- the solve layer of the hot path, orchestrated from the host:
//   V-cycle (Sec. 5.2's AMG preconditioner for A, levels l..L-1),
//   AMG-preconditioned CG for A_l y = f (Sec. 5.2, inner solves) in FP64, or
//     FP32 CG/V-cycle wrapped in FP64 iterative refinement,
//   Jacobi-preconditioned CG for the mass solves M_{u,l} x = b (Sec. 5.2),
//   H_l v = M_yu^T A^-1 M_y A^-1 M_yu v + beta M_u v (Eq. firstorderpractice),
//   Algorithm MLAS in the M_u-scaled form (Sec. 3.2, Sec. 5.2):
//     R_j b = P_j Q_{j+1} P_j^T b + beta^-1 (M_{u,j}^-1 b - P_j M_{u,j+1}^-1 P_j^T b)
//     Q_{l-1} = H_{l-1}^-1,  Q_j b = R_j b + R_j (b - H_j R_j b) (0 < j < l-1),  Q_0 = R_0,
//   outer CG on H u = b (Sec. 5.3).
// CG loops run on device scalars (blas.cu); the host enqueues a chunk of
// iterations, then reads the `done` flag once.
#include <math.h>
#include <string.h>

#include <chrono>

#include "internal.cuh"
#include "util.cuh"

// pieces from blas.cu without a template
int mass_start(amgh_problem *p, RedSlot &red, int n, const double *f, double *x, double *r, double *z, double *pv,
               const double *invd, CgScal *sc, double tol, int maxit);
int mass_iter(amgh_problem *p, RedSlot &red, const DevCsr &M, double *x, double *r, double *z, double *pv,
              double *q, const double *invd, CgScal *sc);
int outer_pq(amgh_problem *p, RedSlot &red, int n, const double *pv, const double *q, CgScal *sc);
int outer_rz(amgh_problem *p, RedSlot &red, int n, const double *r, const double *z, double *pv, CgScal *sc,
             int first);

int sync_stream(amgh_problem *p)
{
    CU(cudaStreamSynchronize(p->stream));
    return AMGH_OK;
}

static int read_scal(amgh_problem *p, const CgScal *sc, CgScal *out)
{
    CU(cudaMemcpyAsync(p->h_scal, sc, sizeof(CgScal), cudaMemcpyDeviceToHost, p->stream));
    CU(cudaStreamSynchronize(p->stream));
    *out = *p->h_scal;
    return AMGH_OK;
}

static int cg_status(const CgScal &h)
{
    switch (h.status) {
    case CG_CONVERGED: return AMGH_OK;
    case CG_INDEFINITE: return AMGH_ERR_INDEFINITE;
    case CG_NUMERIC: return AMGH_ERR_NUMERIC;
    case CG_MAXIT: return AMGH_ERR_NOT_CONVERGED;
    }
    return AMGH_ERR_NOT_CONVERGED;
}

// ------------------------------------------------------------------ allocation
int solver_alloc(amgh_problem *p)
{
    Arena &ar = p->harena;
    for (int l = 0; l < p->Ls; l++) {
        StateLevel &S = p->sl[l];
        int m = S.A.rows;
        TRY(ar.alloc(&S.vb, m));
        TRY(ar.alloc(&S.vx, m));
        TRY(ar.alloc(&S.vx2, m));
        TRY(ar.alloc(&S.vd, m));
        TRY(ar.alloc(&S.vr, m));
        TRY(ar.alloc(&S.fb, m));
        TRY(ar.alloc(&S.fx, m));
        TRY(ar.alloc(&S.fx2, m));
        TRY(ar.alloc(&S.fd, m));
        TRY(ar.alloc(&S.fr, m));
        TRY(ar.alloc(&S.cx, m));
        TRY(ar.alloc(&S.cr, m));
        TRY(ar.alloc(&S.cz, m));
        TRY(ar.alloc(&S.cp, m));
        TRY(ar.alloc(&S.cq, m));
        TRY(ar.alloc(&S.gx, m));
        TRY(ar.alloc(&S.gr, m));
        TRY(ar.alloc(&S.gz, m));
        TRY(ar.alloc(&S.gp, m));
        TRY(ar.alloc(&S.gq, m));
        TRY(ar.alloc(&S.ry, m));
        TRY(ar.alloc(&S.scal, 1));
        TRY(ar.alloc(&S.scal32, 1));
        TRY(ar.alloc(&S.rscal, 1));
        CU(cudaMemset(S.scal, 0, sizeof(CgScal)));
        CU(cudaMemset(S.scal32, 0, sizeof(CgScal)));
        CU(cudaMemset(S.rscal, 0, sizeof(CgScal)));
        TRY(red_alloc(ar, S.red, m));
        p->chunk_hint[l] = 8;
    }
    for (int l = 0; l < p->Lc; l++) {
        CtrlLevel &C = p->cl[l];
        int n = C.Mu.rows;
        int m = l < p->Ls ? p->sl[l].A.rows : 1;
        double **vn[] = {&C.mx, &C.mr, &C.mz, &C.mp, &C.mq, &C.bc, &C.qc, &C.wc,
                         &C.w1, &C.ta, &C.tb, &C.hu, &C.rq, &C.du};
        for (double **q : vn) TRY(ar.alloc(q, n));
        double **vm[] = {&C.t1, &C.ys, &C.t2, &C.ps};
        for (double **q : vm) TRY(ar.alloc(q, m));
        TRY(ar.alloc(&C.mscal, 1));
        CU(cudaMemset(C.mscal, 0, sizeof(CgScal)));
        int cap = n > m ? n : m;
        TRY(red_alloc(ar, C.red, cap));
        p->mchunk_hint[l] = 8;
    }
    int n = p->n;
    double **vo[] = {&p->ou, &p->or_, &p->oz, &p->op, &p->oq, &p->ob};
    for (double **q : vo) TRY(ar.alloc(q, n));
    TRY(ar.alloc(&p->oscal, 1));
    CU(cudaMemset(p->oscal, 0, sizeof(CgScal)));
    TRY(red_alloc(ar, p->ored, n > p->m ? n : p->m));
    TRY(ar.alloc(&p->dscratch, 4));
    return AMGH_OK;
}

// ------------------------------------------------------------------ V-cycle
template <typename T>
struct VBuf;
template <>
struct VBuf<double> {
    static double *b(StateLevel &s) { return s.vb; }
    static double *x(StateLevel &s) { return s.vx; }
    static double *x2(StateLevel &s) { return s.vx2; }
    static double *d(StateLevel &s) { return s.vd; }
    static double *r(StateLevel &s) { return s.vr; }
    static const double *invd(StateLevel &s) { return s.invd; }
};
template <>
struct VBuf<float> {
    static float *b(StateLevel &s) { return s.fb; }
    static float *x(StateLevel &s) { return s.fx; }
    static float *x2(StateLevel &s) { return s.fx2; }
    static float *d(StateLevel &s) { return s.fd; }
    static float *r(StateLevel &s) { return s.fr; }
    static const float *invd(StateLevel &s) { return s.invd32; }
};

template <typename T>
__global__ void k_copy(int n, const T *__restrict__ a, T *__restrict__ b, const int *skip)
{
    if (skip && *skip) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = a[i];
}

// x = V_l b from x = 0; x and b must not alias level-l internal buffers
template <typename T>
static int vcyc(amgh_problem *p, int l, const T *b, T *x, const int *skip)
{
    StateLevel &S = p->sl[l];
    int n = S.A.rows;
    if (l == p->Ls - 1) return dense_gemv<T>(p, n, p->Acoarse.inv, b, x, skip);
    int timed = (l == 0);
    T *tmp = (x == VBuf<T>::x(S)) ? VBuf<T>::x2(S) : VBuf<T>::x(S);
    T *d = VBuf<T>::d(S), *r = VBuf<T>::r(S);
    const T *invd = VBuf<T>::invd(S);
    T *cur = tmp, *nxt = x;
    // pre-smoothing from zero
    TRY(cheb_first<T>(p, n, invd, b, d, cur, p->cr[0], skip));
    for (int s = 1; s < p->nsteps; s++) {
        TRY(cheb_step<T>(p, S.A, invd, b, cur, d, nxt, p->cd[s], p->cr[s], skip, timed));
        T *t = cur;
        cur = nxt;
        nxt = t;
    }
    // coarse-grid correction
    TRY(residual<T>(p, S.A, b, cur, r, skip, timed));
    StateLevel &Sc = p->sl[l + 1];
    T *bc = VBuf<T>::b(Sc), *xc = VBuf<T>::x(Sc);
    TRY(spmv_t<T>(p, S.St, r, bc, skip, 0));
    TRY(vcyc<T>(p, l + 1, bc, xc, skip));
    TRY(prolong_add<T>(p, S.S, xc, cur, skip));
    // post-smoothing with the same polynomial
    for (int s = 0; s < p->nsteps; s++) {
        TRY(cheb_step<T>(p, S.A, invd, b, cur, d, nxt, s == 0 ? 0.0 : p->cd[s], p->cr[s], skip, timed));
        T *t = cur;
        cur = nxt;
        nxt = t;
    }
    if (cur != x) {
        k_copy<T><<<ceil_div(n, 256), 256, 0, p->stream>>>(n, cur, x, skip);
        LAUNCH_CHECK();
    }
    return AMGH_OK;
}

int vcycle_run(amgh_problem *p, int l0, int prec32, const void *b, void *x, const int *skip)
{
    if (prec32) return vcyc<float>(p, l0, (const float *)b, (float *)x, skip);
    return vcyc<double>(p, l0, (const double *)b, (double *)x, skip);
}

// ------------------------------------------------------------------ AMG-CG
// PCG for A_l x = f (x, r, z, p, q of type T), preconditioned by V_l
template <typename T>
static int pcg_amg(amgh_problem *p, int l, const T *f, T *x, T *r, T *z, T *pv, T *q, CgScal *sc, double tol,
                   int maxit, int64_t *iters)
{
    StateLevel &S = p->sl[l];
    int n = S.A.rows;
    const int *skip = &sc->done;
    TRY(cg_start<T>(p, S.red, n, f, x, r, sc, tol, maxit, 1));
    TRY(vcyc<T>(p, l, r, z, skip));
    TRY(cg_rz_first<T>(p, S.red, n, r, z, pv, sc));
    int chunk = p->chunk_hint[l] > 0 ? p->chunk_hint[l] : 4;
    int enq = 0;
    CgScal h;
    for (;;) {
        for (int c = 0; c < chunk; c++) {
            TRY(cg_spmv_pq<T>(p, S.red, S.A, pv, q, sc, l == 0));
            TRY(cg_update<T>(p, S.red, n, x, r, pv, q, sc));
            TRY(vcyc<T>(p, l, r, z, skip));
            TRY(cg_rz_next<T>(p, S.red, n, r, z, pv, sc));
        }
        enq += chunk;
        TRY(read_scal(p, sc, &h));
        if (h.done || enq > maxit + 2) break;
        chunk = h.iters / 4 > 1 ? h.iters / 4 : 1;
    }
    if (h.iters > 0) p->chunk_hint[l] = h.iters;
    if (iters) *iters = h.iters;
    p->c_inner += h.iters;
    if (!h.done) return AMGH_ERR_NOT_CONVERGED;
    return cg_status(h);
}

// A_l y = f to relative residual tol (FP64 CG, or FP32 CG inside FP64 refinement)
int state_solve(amgh_problem *p, int l, const double *f, double *y, double tol, int64_t *iters)
{
    StateLevel &S = p->sl[l];
    int maxit = p->sopts.inner_max_iter;
    if (!p->aopts.precision) return pcg_amg<double>(p, l, f, y, S.cr, S.cz, S.cp, S.cq, S.scal, tol, maxit, iters);
    // mixed: r = f - A y in FP64, FP32 PCG on A e = r / ||r||, y += ||r|| e
    int n = S.A.rows;
    TRY(ref_start(p, S.red, n, f, y, S.ry, S.rscal, tol, 50));
    CgScal h;
    TRY(read_scal(p, S.rscal, &h));
    int64_t it_total = 0;
    double inner = 1e-4;
    while (!h.done) {
        TRY(ref_to32(p, S.red, n, S.ry, S.gq, S.rscal));
        int64_t it = 0;
        int st = pcg_amg<float>(p, l, S.gq, S.gx, S.gr, S.gz, S.gp, S.gq, S.scal32, inner, maxit, &it);
        it_total += it;
        // FP32 CG stops at its own accuracy floor; refinement continues from there
        if (st != AMGH_OK && st != AMGH_ERR_NOT_CONVERGED) return st;
        TRY(ref_update(p, S.red, S.A, f, y, S.gx, S.ry, S.rscal));
        TRY(read_scal(p, S.rscal, &h));
        p->c_refine += 1;
    }
    if (iters) *iters = it_total;
    return cg_status(h);
}

// ------------------------------------------------------------------ mass solves
int mass_solve(amgh_problem *p, int l, const double *b, double *x, int64_t *iters)
{
    CtrlLevel &C = p->cl[l];
    int n = C.Mu.rows;
    TRY(mass_start(p, C.red, n, b, x, C.mr, C.mz, C.mp, C.mu_invdiag, C.mscal, p->sopts.mass_tol,
                   p->sopts.mass_max_iter));
    int chunk = p->mchunk_hint[l] > 0 ? p->mchunk_hint[l] : 4;
    int enq = 0;
    CgScal h;
    for (;;) {
        for (int c = 0; c < chunk; c++) TRY(mass_iter(p, C.red, C.Mu, x, C.mr, C.mz, C.mp, C.mq, C.mu_invdiag, C.mscal));
        enq += chunk;
        TRY(read_scal(p, C.mscal, &h));
        if (h.done || enq > p->sopts.mass_max_iter + 2) break;
        chunk = h.iters / 4 > 1 ? h.iters / 4 : 1;
    }
    if (h.iters > 0) p->mchunk_hint[l] = h.iters;
    if (iters) *iters = h.iters;
    p->c_mass += h.iters;
    if (!h.done) return AMGH_ERR_NOT_CONVERGED;
    return cg_status(h);
}

// ------------------------------------------------------------------ Hessian
int hessian_level(amgh_problem *p, int l, const double *v, double *hv)
{
    StateLevel &S = p->sl[l];
    CtrlLevel &C = p->cl[l];
    double tol = p->sopts.inner_tol;
    TRY(spmv(p, C.Myu, v, C.t1, nullptr, 0));
    TRY(state_solve(p, l, C.t1, C.ys, tol, nullptr));
    TRY(spmv(p, S.My, C.ys, C.t2, nullptr, 0));
    TRY(state_solve(p, l, C.t2, C.ps, tol, nullptr));
    TRY(spmv2(p, C.Myut, C.ps, C.Mu, v, p->beta, hv, nullptr));
    if (l == 0) p->c_happ += 1;
    return AMGH_OK;
}

// ------------------------------------------------------------------ MLAS
__global__ void k_r_combine(int n, const double *__restrict__ ta, const double *__restrict__ w1,
                            const double *__restrict__ tb, double beta, double *__restrict__ out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = ta[i] + (w1[i] - tb[i]) / beta;
}

int mlas_R(amgh_problem *p, int j, const double *b, double *out)
{
    CtrlLevel &C = p->cl[j], &Cc = p->cl[j + 1];
    int n = C.Mu.rows;
    TRY(spmv(p, C.Pt, b, Cc.bc, nullptr, 0));
    TRY(mlas_Q(p, j + 1, Cc.bc, Cc.qc));
    TRY(mass_solve(p, j, b, C.w1, nullptr));
    TRY(mass_solve(p, j + 1, Cc.bc, Cc.wc, nullptr));
    TRY(spmv(p, C.P, Cc.qc, C.ta, nullptr, 0));
    TRY(spmv(p, C.P, Cc.wc, C.tb, nullptr, 0));
    k_r_combine<<<ceil_div(n, 256), 256, 0, p->stream>>>(n, C.ta, C.w1, C.tb, p->beta, out);
    LAUNCH_CHECK();
    return AMGH_OK;
}

int mlas_Q(amgh_problem *p, int j, const double *b, double *u)
{
    CtrlLevel &C = p->cl[j];
    int n = C.Mu.rows;
    if (j == p->ell - 1) return dense_gemv<double>(p, n, p->Hcoarse.inv, b, u, nullptr);
    TRY(mlas_R(p, j, b, u));
    if (j == 0) return AMGH_OK;
    TRY(hessian_level(p, j, u, C.hu));
    TRY(vec_axpby(p, n, 1.0, b, -1.0, C.hu, C.rq));
    TRY(mlas_R(p, j, C.rq, C.du));
    TRY(vec_axpby(p, n, 1.0, u, 1.0, C.du, u));
    return AMGH_OK;
}

// ------------------------------------------------------------------ right side
int rhs_apply(amgh_problem *p, double *b)
{
    StateLevel &S = p->sl[0];
    CtrlLevel &C = p->cl[0];
    TRY(spmv(p, S.My, p->yd_state, C.t2, nullptr, 0));
    TRY(state_solve(p, 0, C.t2, C.ps, p->sopts.inner_tol, nullptr));
    TRY(spmv(p, C.Myut, C.ps, b, nullptr, 0));
    return AMGH_OK;
}

// ------------------------------------------------------------------ outer CG
static double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

static int dot_host(amgh_problem *p, RedSlot &red, int n, const double *x, const double *y, double *out)
{
    TRY(vec_dot(p, red, n, x, y, p->dscratch));
    CU(cudaMemcpyAsync(out, p->dscratch, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    CU(cudaStreamSynchronize(p->stream));
    return AMGH_OK;
}

int outer_solve(amgh_problem *p, const double *u0, double *u, const amgh_solve_opts *o, amgh_solve_info *info)
{
    double t0 = now_s();
    int n = p->n;
    double *b = p->ob, *r = p->or_, *z = p->oz, *pv = p->op, *q = p->oq;
    TRY(rhs_apply(p, b));
    double bb = 0.0;
    TRY(dot_host(p, p->ored, n, b, b, &bb));
    double tol = o->tol;
    const double *f = b;
    if (u0) {
        // solve H d = b - H u0 for the correction, stopping on ||b - H u|| <= tol ||b||
        TRY(hessian_level(p, 0, u0, q));
        TRY(vec_axpby(p, n, 1.0, b, -1.0, q, p->ou));
        double rr0 = 0.0;
        TRY(dot_host(p, p->ored, n, p->ou, p->ou, &rr0));
        tol = rr0 > 0.0 ? tol * sqrt(bb / rr0) : tol;
        f = p->ou;
    }
    CgScal *sc = p->oscal;
    const int *skip = &sc->done;
    (void)skip;
    TRY(cg_start<double>(p, p->ored, n, f, u, r, sc, tol, o->max_iter, 1));
    CgScal h;
    TRY(read_scal(p, sc, &h));
    int st = AMGH_OK;
    int outer = 0;
    if (!h.done) {
        if (o->precond) TRY(mlas_Q(p, 0, r, z));
        else CU(cudaMemcpyAsync(z, r, sizeof(double) * n, cudaMemcpyDeviceToDevice, p->stream));
        TRY(outer_rz(p, p->ored, n, r, z, pv, sc, 1));
        for (;;) {
            TRY(read_scal(p, sc, &h));
            if (h.done) break;
            TRY(hessian_level(p, 0, pv, q));
            TRY(outer_pq(p, p->ored, n, pv, q, sc));
            TRY(cg_update<double>(p, p->ored, n, u, r, pv, q, sc));
            TRY(read_scal(p, sc, &h));
            if (h.done) break;
            if (o->precond) TRY(mlas_Q(p, 0, r, z));
            else CU(cudaMemcpyAsync(z, r, sizeof(double) * n, cudaMemcpyDeviceToDevice, p->stream));
            TRY(outer_rz(p, p->ored, n, r, z, pv, sc, 0));
        }
        st = cg_status(h);
        outer = h.iters;
    }
    if (u0) TRY(vec_axpby(p, n, 1.0, u, 1.0, u0, u));
    // true relative residual ||b - H u|| / ||b||
    double relres = 0.0;
    if (bb > 0.0 && (st == AMGH_OK || st == AMGH_ERR_NOT_CONVERGED)) {
        TRY(hessian_level(p, 0, u, q));
        TRY(vec_axpby(p, n, 1.0, b, -1.0, q, r));
        double rr = 0.0;
        TRY(dot_host(p, p->ored, n, r, r, &rr));
        relres = sqrt(rr / bb);
    }
    if (info) {
        info->status = st;
        info->outer_iters = outer;
        info->final_relres = relres;
        info->t_solve_s = now_s() - t0;
    }
    return st;
}
