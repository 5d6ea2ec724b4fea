// diag.cu -- the two-level approximation numbers of the multilevel analysis
// (Sec. 4 and Sec. 5.1), estimated on the GPU by the power method.
//
// With K_j = A_j^-1 M_yu,j the control-to-state map on level j, S_j and P_j
// the state and control interpolations and Pi_j = M_u,j+1^-1 P_j^T M_u,j the
// L2 projection onto the coarse control space,
//   D_j = K_j - S_j K_j+1 Pi_j,
//   a~_j = ||D_j||_2                                  (Eq. aj-tilde)
//   a_j  = ||M_y,j^1/2 D_j M_u,j^-1/2||_2             (Eq. ajnumerical)
// a~_j is the square root of the largest eigenvalue of D^T D (power method
// in the Euclidean inner product); a_j that of M_u^-1 D^T M_y D, which is
// self-adjoint in the M_u inner product (power method in that inner
// product).  Every application of D or D^T is two AMG-CG state solves, one
// mass solve and sparse products, at the problem's solve tolerances.
#include <math.h>

#include "internal.cuh"

static int dot_to_host(amgh_problem *p, RedSlot &red, int n, const double *x, const double *y, double *out)
{
    TRY(vec_dot(p, red, n, x, y, p->dscratch));
    CU(cudaMemcpyAsync(out, p->dscratch, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    TRY(sync_stream(p));
    return AMGH_OK;
}

struct DiagWork {
    double *t1, *y, *u1, *c1, *w, *t2, *y2, *s2; // D v
    double *z, *r1, *sx, *z2, *k2, *q, *pq, *r2; // D^T x
};

// out = D_j v (m_j)
static int apply_D(amgh_problem *p, int j, DiagWork &W, const double *v, double *out)
{
    StateLevel &S = p->sl[j];
    CtrlLevel &C = p->cl[j], &C1 = p->cl[j + 1];
    const double tol = p->sopts.inner_tol;
    TRY(spmv(p, C.Myu, v, W.t1, nullptr, KC_SPMV));
    TRY(state_solve(p, j, W.t1, W.y, tol, nullptr));
    TRY(spmv(p, C.Mu, v, W.u1, nullptr, KC_SPMV));
    TRY(spmv(p, C.Pt, W.u1, W.c1, nullptr, KC_SPMV));
    TRY(mass_solve(p, j + 1, W.c1, W.w, nullptr)); // Pi_j v
    TRY(spmv(p, C1.Myu, W.w, W.t2, nullptr, KC_SPMV));
    TRY(state_solve(p, j + 1, W.t2, W.y2, tol, nullptr));
    TRY(spmv(p, S.S, W.y2, W.s2, nullptr, KC_SPMV));
    return vec_axpby(p, S.A.rows, 1.0, W.y, -1.0, W.s2, out);
}

// out = D_j^T x (n_j); A_j is symmetric, so K_j^T x = M_yu,j^T A_j^-1 x
static int apply_Dt(amgh_problem *p, int j, DiagWork &W, const double *x, double *out)
{
    StateLevel &S = p->sl[j];
    CtrlLevel &C = p->cl[j], &C1 = p->cl[j + 1];
    const double tol = p->sopts.inner_tol;
    TRY(state_solve(p, j, x, W.z, tol, nullptr));
    TRY(spmv(p, C.Myut, W.z, W.r1, nullptr, KC_SPMV));
    TRY(spmv(p, S.St, x, W.sx, nullptr, KC_SPMV));
    TRY(state_solve(p, j + 1, W.sx, W.z2, tol, nullptr));
    TRY(spmv(p, C1.Myut, W.z2, W.k2, nullptr, KC_SPMV));
    TRY(mass_solve(p, j + 1, W.k2, W.q, nullptr));
    TRY(spmv(p, C.P, W.q, W.pq, nullptr, KC_SPMV));
    TRY(spmv(p, C.Mu, W.pq, W.r2, nullptr, KC_SPMV)); // Pi_j^T = M_u,j P_j M_u,j+1^-1
    return vec_axpby(p, C.Mu.rows, 1.0, W.r1, -1.0, W.r2, out);
}

int aj_estimate(amgh_problem *p, int j, int weighted, int iters, const double *v0, double *est)
{
    const int m = p->sl[j].A.rows, n = p->cl[j].Mu.rows;
    const int m1 = p->sl[j + 1].A.rows, n1 = p->cl[j + 1].Mu.rows;
    Scratch sc;
    DiagWork W;
    double **vm[] = {&W.t1, &W.y, &W.s2, &W.z};
    double **vn[] = {&W.u1, &W.r1, &W.pq, &W.r2};
    double **vm1[] = {&W.t2, &W.y2, &W.sx, &W.z2};
    double **vn1[] = {&W.c1, &W.w, &W.k2, &W.q};
    for (double **q : vm) TRY(sc.alloc(q, m));
    for (double **q : vn) TRY(sc.alloc(q, n));
    for (double **q : vm1) TRY(sc.alloc(q, m1));
    for (double **q : vn1) TRY(sc.alloc(q, n1));
    double *v = nullptr, *x = nullptr, *mx = nullptr, *g = nullptr, *mv = nullptr;
    TRY(sc.alloc(&v, n));
    TRY(sc.alloc(&x, m));
    TRY(sc.alloc(&mx, m));
    TRY(sc.alloc(&g, n));
    TRY(sc.alloc(&mv, n));
    RedSlot &red = p->ored;
    CtrlLevel &C = p->cl[j];
    StateLevel &S = p->sl[j];
    // v = v0 / ||v0|| (Euclidean, or in the M_u,j inner product)
    CU(cudaMemcpyAsync(v, v0, sizeof(double) * n, cudaMemcpyDeviceToDevice, p->stream));
    double nv = 0.0;
    if (weighted) {
        TRY(spmv(p, C.Mu, v, mv, nullptr, KC_SPMV));
        TRY(dot_to_host(p, red, n, v, mv, &nv));
    } else {
        TRY(dot_to_host(p, red, n, v, v, &nv));
    }
    if (!(nv > 0.0) || !isfinite(nv)) return AMGH_ERR_INVALID_ARG;
    TRY(vec_axpby(p, n, 1.0 / sqrt(nv), v, 0.0, nullptr, v));
    double lam = 0.0;
    for (int k = 0; k < iters; k++) {
        TRY(apply_D(p, j, W, v, x));
        const double *xr = x;
        if (weighted) {
            TRY(spmv(p, S.My, x, mx, nullptr, KC_SPMV));
            TRY(dot_to_host(p, red, m, x, mx, &lam)); // (Dv)^T M_y (Dv), v of unit M_u norm
            xr = mx;
        } else {
            TRY(dot_to_host(p, red, m, x, x, &lam));
        }
        if (!isfinite(lam)) return AMGH_ERR_NUMERIC;
        if (k + 1 == iters || lam == 0.0) break;
        TRY(apply_Dt(p, j, W, xr, g));
        if (weighted) {
            TRY(mass_solve(p, j, g, v, nullptr)); // M_u,j^-1 D^T M_y D v
            TRY(spmv(p, C.Mu, v, mv, nullptr, KC_SPMV));
            TRY(dot_to_host(p, red, n, v, mv, &nv));
        } else {
            CU(cudaMemcpyAsync(v, g, sizeof(double) * n, cudaMemcpyDeviceToDevice, p->stream));
            TRY(dot_to_host(p, red, n, v, v, &nv));
        }
        if (nv == 0.0) break; // D^T D v = 0: lam is the answer
        if (!(nv > 0.0) || !isfinite(nv)) return AMGH_ERR_NUMERIC;
        TRY(vec_axpby(p, n, 1.0 / sqrt(nv), v, 0.0, nullptr, v));
    }
    *est = sqrt(lam);
    return AMGH_OK;
}
