/*
 * amgh_oracle.c -- plain, slow FP64 CPU oracle for AMG preconditioning of the
 * reduced Hessian (Barker & Draganescu, "Algebraic multigrid preconditioning
 * of the Hessian in PDE-constrained optimization").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file's library.  It shares no
 * code with the CUDA path: every routine below is written from the paper's
 * definitions (cited per function) and from the stated readings of the
 * points the paper leaves open.  Everything is sequential, in FP64, with
 * sums taken in ascending index order.  Compile with -ffp-contract=off so
 * that no multiply-add is fused: the assembly, the strength test and the
 * Galerkin products must reproduce bit-for-bit on any host.
 *
 * What it computes (Sec. 2 and Sec. 5.2):
 *   A, M_y, M_u, M_yu        P1 stiffness / mass matrices (Sec. 2)
 *   H u = M_yu^T A^-1 M_y A^-1 M_yu u + beta M_u u     (Eq. firstorderpractice)
 *   b   = M_yu^T A^-1 M_y y_d
 *   smoothed-aggregation prolongators S_j (state) and P_j (control) (Sec. 3.1)
 *   Galerkin coarse matrices (Eq. coarsestiffness, coarsemass)
 *   the multilevel preconditioner of Sec. 3.2 (Eq. twogridinmulti,
 *   twogridinmultiactual, Algorithm MLAS) in the M_u-scaled form of Sec. 5.2:
 *     R_j b = P_j Q_{j+1} P_j^T b + beta^-1 (M_{u,j}^-1 b - P_j M_{u,j+1}^-1 P_j^T b)
 *     Q_{l-1} = H_{l-1}^-1 (dense inverse, or CG on H_{l-1} to a relative
 *               tolerance, chosen by the coarse-solve mode; Sec. 5.5-5.6),
 *     Q_j = 2R_j - R_j H_j R_j (0<j<l-1),  Q_0 = R_0
 *   outer CG on H u = b (Sec. 5.3).
 *
 * Pins (tests/test_oracle_*.py): assembly against exact integrals, an
 * independent assembly and harmonic linear functions; aggregation against a
 * greedy sequential MIS(2) and a golden 5x5 grid; Galerkin products and the
 * prolongator against their definitions; the smoother's error propagator
 * against the closed-form Chebyshev residual polynomial (and (1-t)^k for
 * l1-Jacobi) of D^-1 A; the V-cycle by symmetry, positivity and contraction; H against the dense formula, a KKT direct solve and a
 * closed form; MLAS against its closed two-grid formula and the coarse CG
 * against a dense solve of H_{l-1}.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_INVALID -1
#define ORC_NOT_SETUP -2
#define ORC_OOM -4
#define ORC_NOT_CONVERGED -5
#define ORC_INDEFINITE -6
#define ORC_NUMERIC -7

#define MAXL 32
#define DENSE_MAX 4096

/* Row loops of the solve phase may be split over threads when the file is
 * compiled with -fopenmp (the multi-core CPU timing of the benchmark).  Each
 * row is still computed by one thread in the same order and every dot
 * product stays sequential, so the results are bit-identical to the plain
 * sequential build used by the tests. */
#ifdef _OPENMP
#include <omp.h>
/* the loop's trip count must be a variable named n */
#define ORC_ROWS _Pragma("omp parallel for schedule(static) if(n > 16384)")
#else
#define ORC_ROWS
#endif

typedef struct {
    int rows, cols;
    int *rp, *ci;
    double *v;
} csr_t;

typedef struct {
    int dim;
    long nv, ne;
    double *coords;
    int *elems;
    unsigned char *dir;
    double *kappa;
    double beta;
    double *yd_state; /* y_d at interior vertices, length m */
    int m, n;
    int *state_of_vertex; /* -1 for Dirichlet */
    csr_t Kfull, Mfull;
    /* options */
    int max_levels, hess_levels, coarse_max, smoother, degree, smooth_p;
    int aggressive; /* level 0 aggregated twice (aggregates of aggregates) */
    int geometric;  /* nested structured-grid interpolation instead of AMG */
    double theta;
    int setup_done;
    /* state hierarchy */
    int Ls;
    csr_t A[MAXL], My[MAXL], S[MAXL], St[MAXL];
    int *sagg[MAXL];
    int snagg[MAXL];
    double *dl1[MAXL];
    double *Ac_chol; /* dense Cholesky factor of A[Ls-1] */
    /* control hierarchy */
    int Lc;
    csr_t KN[MAXL], Mu[MAXL], P[MAXL], Pt[MAXL];
    int *cagg[MAXL];
    int cnagg[MAXL];
    /* cross matrices, levels 0 .. min(Ls,Lc)-1 */
    csr_t Myu[MAXL], Myut[MAXL];
    int ell;
    double *Hc_chol; /* dense Cholesky factor of H_{ell-1} */
    double *Aell_chol; /* dense Cholesky of A[ell-1] when ell-1 != Ls-1 */
    /* smoother coefficients */
    int nsteps;
    double cd[16], cr[16];
    /* solve parameters used by the preconditioner */
    double inner_tol, mass_tol;
    double pc_inner_tol; /* inner solves of the coarse Hessians inside the preconditioner */
    int inner_maxit, mass_maxit;
    long inner_iters, mass_iters, happlies;
    /* coarsest Hessian level: 0 = dense Cholesky of H_{ell-1}, 1 = plain CG,
     * 2 = dense up to 4096 control dofs there, else CG */
    int coarse_solve, coarse_maxit;
    double coarse_tol;
    long coarse_iters;
} orc_t;

/* ------------------------------------------------------------------ utils */

static void *xcalloc(size_t n, size_t s)
{
    if (n == 0) n = 1;
    return calloc(n, s);
}

static void csr_free(csr_t *a)
{
    free(a->rp);
    free(a->ci);
    free(a->v);
    memset(a, 0, sizeof(*a));
}

static int cmp_int(const void *a, const void *b)
{
    int x = *(const int *)a, y = *(const int *)b;
    return (x > y) - (x < y);
}

/* position of column c in row r of a (sorted columns), or -1 */
static long csr_find(const csr_t *a, int r, int c)
{
    int lo = a->rp[r], hi = a->rp[r + 1] - 1;
    while (lo <= hi) {
        int mid = lo + (hi - lo) / 2;
        if (a->ci[mid] == c) return mid;
        if (a->ci[mid] < c) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

/* y = a x  (row by row, ascending columns) */
static void spmv(const csr_t *a, const double *x, double *y)
{
    int n = a->rows;
    ORC_ROWS
    for (int i = 0; i < n; i++) {
        double s = 0.0;
        for (int k = a->rp[i]; k < a->rp[i + 1]; k++) s += a->v[k] * x[a->ci[k]];
        y[i] = s;
    }
}

static double dot(int n, const double *x, const double *y)
{
    double s = 0.0;
    for (int i = 0; i < n; i++) s += x[i] * y[i];
    return s;
}

static double nrm2(int n, const double *x) { return sqrt(dot(n, x, x)); }

/* transpose with ascending columns in every row */
static int csr_transpose(const csr_t *a, csr_t *t)
{
    t->rows = a->cols;
    t->cols = a->rows;
    int nnz = a->rp[a->rows];
    t->rp = xcalloc((size_t)t->rows + 1, sizeof(int));
    t->ci = xcalloc((size_t)nnz, sizeof(int));
    t->v = xcalloc((size_t)nnz, sizeof(double));
    int *fill = xcalloc((size_t)t->rows + 1, sizeof(int));
    if (!t->rp || !t->ci || !t->v || !fill) return ORC_OOM;
    for (int k = 0; k < nnz; k++) t->rp[a->ci[k] + 1]++;
    for (int r = 0; r < t->rows; r++) t->rp[r + 1] += t->rp[r];
    for (int r = 0; r < t->rows; r++) fill[r] = t->rp[r];
    for (int i = 0; i < a->rows; i++)
        for (int k = a->rp[i]; k < a->rp[i + 1]; k++) {
            int pos = fill[a->ci[k]]++;
            t->ci[pos] = i;
            t->v[pos] = a->v[k];
        }
    free(fill);
    return ORC_OK;
}

/*
 * C = A B.  Entry C_iJ is the sum over the columns j of row i of A, taken in
 * ascending j, of A_ij * B_jJ (each product rounded, then added in that
 * order).  Output columns are sorted; every structurally reachable (i,J) is
 * kept even if its value cancels to zero.
 */
static int spgemm(const csr_t *a, const csr_t *b, csr_t *c)
{
    int n = a->rows, nc = b->cols;
    int *mark = malloc(sizeof(int) * (size_t)(nc > 0 ? nc : 1));
    double *acc = xcalloc((size_t)nc, sizeof(double));
    int *list = malloc(sizeof(int) * (size_t)(nc > 0 ? nc : 1));
    if (!mark || !acc || !list) return ORC_OOM;
    for (int j = 0; j < nc; j++) mark[j] = -1;
    c->rows = n;
    c->cols = nc;
    c->rp = xcalloc((size_t)n + 1, sizeof(int));
    /* symbolic */
    long total = 0;
    for (int i = 0; i < n; i++) {
        int cnt = 0;
        for (int k = a->rp[i]; k < a->rp[i + 1]; k++) {
            int j = a->ci[k];
            for (int q = b->rp[j]; q < b->rp[j + 1]; q++) {
                int J = b->ci[q];
                if (mark[J] != i) { mark[J] = i; cnt++; }
            }
        }
        total += cnt;
        if (total > 2147483647L) return ORC_OOM;
        c->rp[i + 1] = (int)total;
    }
    c->ci = xcalloc((size_t)total, sizeof(int));
    c->v = xcalloc((size_t)total, sizeof(double));
    if (!c->ci || !c->v) return ORC_OOM;
    for (int j = 0; j < nc; j++) mark[j] = -1;
    /* numeric */
    for (int i = 0; i < n; i++) {
        int cnt = 0;
        for (int k = a->rp[i]; k < a->rp[i + 1]; k++) {
            int j = a->ci[k];
            double aij = a->v[k];
            for (int q = b->rp[j]; q < b->rp[j + 1]; q++) {
                int J = b->ci[q];
                double prod = aij * b->v[q];
                if (mark[J] != i) {
                    mark[J] = i;
                    acc[J] = 0.0;
                    list[cnt++] = J;
                }
                acc[J] = acc[J] + prod;
            }
        }
        qsort(list, (size_t)cnt, sizeof(int), cmp_int);
        int base = c->rp[i];
        for (int t = 0; t < cnt; t++) {
            c->ci[base + t] = list[t];
            c->v[base + t] = acc[list[t]];
        }
    }
    free(mark);
    free(acc);
    free(list);
    return ORC_OK;
}

/*
 * Make a matrix with symmetric pattern exactly symmetric: every entry below
 * the diagonal takes the value of its mirror above the diagonal.  (Reading:
 * Galerkin products S^T A S are symmetric in exact arithmetic; the upper
 * triangle is taken as the computed value so that the strength graph of the
 * next level is symmetric.)
 */
static int symmetrize_upper(csr_t *a)
{
    for (int i = 0; i < a->rows; i++)
        for (int k = a->rp[i]; k < a->rp[i + 1]; k++) {
            int j = a->ci[k];
            if (j < i) {
                long q = csr_find(a, j, i);
                if (q < 0) return ORC_INVALID;
                a->v[k] = a->v[q];
            }
        }
    return ORC_OK;
}

/* RAP product C = Rt (A Pm), Rt = transpose of the left prolongator */
static int galerkin(const csr_t *rt, const csr_t *a, const csr_t *pm, int symmetric, csr_t *c)
{
    csr_t ap = {0};
    int st = spgemm(a, pm, &ap);
    if (st) return st;
    st = spgemm(rt, &ap, c);
    csr_free(&ap);
    if (st) return st;
    if (symmetric) st = symmetrize_upper(c);
    return st;
}

/* ------------------------------------------------------------- assembly */

/*
 * P1 element matrices (Sec. 2: [A]_ij = a(phi_j, phi_i) with
 * a(y, v) = int kappa grad y . grad v, [M]_ij = (phi_j, phi_i)).
 * With e_k = p_k - p_0 and D = det[e_1 .. e_d], the barycentric gradients are
 * grad(lambda_k) = c_k / D where, in 2D, c_1 = (e2y, -e2x), c_2 = (-e1y, e1x),
 * and in 3D c_1 = e2 x e3, c_2 = e3 x e1, c_3 = e1 x e2; c_0 = -(c_1+c_2+c_3).
 * Then K_ab = kappa |T| c_a.c_b / D^2 = kappa c_a.c_b / (d! |D|), and the
 * consistent mass is M_ab = |T| (1 + delta_ab) / ((d+1)(d+2)), i.e.
 * |D|/12, |D|/24 in 2D and |D|/60, |D|/120 in 3D.
 */
static void element_matrices(int dim, const double *coords, const int *ev, double kappa,
                             double K[4][4], double M[4][4])
{
    double c[4][3];
    double absdet;
    if (dim == 2) {
        const double *p0 = coords + 2 * (long)ev[0], *p1 = coords + 2 * (long)ev[1],
                     *p2 = coords + 2 * (long)ev[2];
        double e1x = p1[0] - p0[0], e1y = p1[1] - p0[1];
        double e2x = p2[0] - p0[0], e2y = p2[1] - p0[1];
        double det = e1x * e2y - e1y * e2x;
        c[1][0] = e2y;
        c[1][1] = -e2x;
        c[2][0] = -e1y;
        c[2][1] = e1x;
        c[0][0] = -(c[1][0] + c[2][0]);
        c[0][1] = -(c[1][1] + c[2][1]);
        absdet = fabs(det);
        double coef = kappa / (2.0 * absdet);
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) {
                double d = c[a][0] * c[b][0] + c[a][1] * c[b][1];
                K[a][b] = coef * d;
                M[a][b] = (a == b) ? absdet / 12.0 : absdet / 24.0;
            }
    } else {
        const double *p0 = coords + 3 * (long)ev[0], *p1 = coords + 3 * (long)ev[1],
                     *p2 = coords + 3 * (long)ev[2], *p3 = coords + 3 * (long)ev[3];
        double e1[3], e2[3], e3[3];
        for (int k = 0; k < 3; k++) {
            e1[k] = p1[k] - p0[k];
            e2[k] = p2[k] - p0[k];
            e3[k] = p3[k] - p0[k];
        }
        /* c1 = e2 x e3, c2 = e3 x e1, c3 = e1 x e2 */
        c[1][0] = e2[1] * e3[2] - e2[2] * e3[1];
        c[1][1] = e2[2] * e3[0] - e2[0] * e3[2];
        c[1][2] = e2[0] * e3[1] - e2[1] * e3[0];
        c[2][0] = e3[1] * e1[2] - e3[2] * e1[1];
        c[2][1] = e3[2] * e1[0] - e3[0] * e1[2];
        c[2][2] = e3[0] * e1[1] - e3[1] * e1[0];
        c[3][0] = e1[1] * e2[2] - e1[2] * e2[1];
        c[3][1] = e1[2] * e2[0] - e1[0] * e2[2];
        c[3][2] = e1[0] * e2[1] - e1[1] * e2[0];
        for (int k = 0; k < 3; k++) c[0][k] = -((c[1][k] + c[2][k]) + c[3][k]);
        double det = e1[0] * c[1][0] + e1[1] * c[1][1] + e1[2] * c[1][2];
        absdet = fabs(det);
        double coef = kappa / (6.0 * absdet);
        for (int a = 0; a < 4; a++)
            for (int b = 0; b < 4; b++) {
                double d = c[a][0] * c[b][0] + c[a][1] * c[b][1] + c[a][2] * c[b][2];
                K[a][b] = coef * d;
                M[a][b] = (a == b) ? absdet / 60.0 : absdet / 120.0;
            }
    }
}

/* Assemble the all-vertex stiffness K and mass M; per entry, element
 * contributions are added in ascending element order. */
static int assemble(orc_t *o)
{
    int nv = (int)o->nv, d1 = o->dim + 1;
    /* vertex -> element incidence */
    int *vcnt = xcalloc((size_t)nv + 1, sizeof(int));
    if (!vcnt) return ORC_OOM;
    for (long e = 0; e < o->ne; e++)
        for (int a = 0; a < d1; a++) vcnt[o->elems[e * d1 + a] + 1]++;
    for (int v = 0; v < nv; v++) vcnt[v + 1] += vcnt[v];
    int *vel = xcalloc((size_t)vcnt[nv], sizeof(int));
    int *fill = xcalloc((size_t)nv, sizeof(int));
    if (!vel || !fill) return ORC_OOM;
    for (long e = 0; e < o->ne; e++)
        for (int a = 0; a < d1; a++) {
            int v = o->elems[e * d1 + a];
            vel[vcnt[v] + fill[v]++] = (int)e;
        }
    /* sparsity: neighbours through shared elements */
    int *rp = xcalloc((size_t)nv + 1, sizeof(int));
    int *tmp = malloc(sizeof(int) * 4096);
    if (!rp || !tmp) return ORC_OOM;
    for (int pass = 0; pass < 2; pass++) {
        int *ci = NULL;
        if (pass == 1) {
            o->Kfull.ci = xcalloc((size_t)rp[nv], sizeof(int));
            o->Mfull.ci = xcalloc((size_t)rp[nv], sizeof(int));
            if (!o->Kfull.ci || !o->Mfull.ci) return ORC_OOM;
            ci = o->Kfull.ci;
        }
        for (int v = 0; v < nv; v++) {
            int cnt = 0;
            for (int q = vcnt[v]; q < vcnt[v + 1]; q++) {
                long e = vel[q];
                for (int a = 0; a < d1; a++) {
                    if (cnt >= 4096) return ORC_INVALID;
                    tmp[cnt++] = o->elems[e * d1 + a];
                }
            }
            qsort(tmp, (size_t)cnt, sizeof(int), cmp_int);
            int u = 0;
            for (int t = 0; t < cnt; t++)
                if (u == 0 || tmp[t] != tmp[u - 1]) tmp[u++] = tmp[t];
            if (pass == 0) rp[v + 1] = rp[v] + u;
            else memcpy(ci + rp[v], tmp, sizeof(int) * (size_t)u);
        }
    }
    int nnz = rp[nv];
    o->Kfull.rows = o->Kfull.cols = nv;
    o->Mfull.rows = o->Mfull.cols = nv;
    o->Kfull.rp = rp;
    o->Mfull.rp = xcalloc((size_t)nv + 1, sizeof(int));
    memcpy(o->Mfull.rp, rp, sizeof(int) * ((size_t)nv + 1));
    memcpy(o->Mfull.ci, o->Kfull.ci, sizeof(int) * (size_t)nnz);
    o->Kfull.v = xcalloc((size_t)nnz, sizeof(double));
    o->Mfull.v = xcalloc((size_t)nnz, sizeof(double));
    if (!o->Kfull.v || !o->Mfull.v) return ORC_OOM;
    for (long e = 0; e < o->ne; e++) {
        double K[4][4], M[4][4];
        const int *ev = o->elems + e * d1;
        element_matrices(o->dim, o->coords, ev, o->kappa[e], K, M);
        for (int a = 0; a < d1; a++)
            for (int b = 0; b < d1; b++) {
                long q = csr_find(&o->Kfull, ev[a], ev[b]);
                o->Kfull.v[q] = o->Kfull.v[q] + K[a][b];
                o->Mfull.v[q] = o->Mfull.v[q] + M[a][b];
            }
    }
    free(vcnt);
    free(vel);
    free(fill);
    free(tmp);
    return ORC_OK;
}

/* submatrix of rows with rmap[r] >= 0 and columns with cmap[c] >= 0, renumbered */
static int extract(const csr_t *a, const int *rmap, int nr, const int *cmap, int nc, csr_t *o)
{
    o->rows = nr;
    o->cols = nc;
    o->rp = xcalloc((size_t)nr + 1, sizeof(int));
    long cnt = 0;
    for (int i = 0; i < a->rows; i++) {
        if (rmap[i] < 0) continue;
        int c = 0;
        for (int k = a->rp[i]; k < a->rp[i + 1]; k++) c += cmap[a->ci[k]] >= 0;
        o->rp[rmap[i] + 1] = c;
        cnt += c;
    }
    for (int r = 0; r < nr; r++) o->rp[r + 1] += o->rp[r];
    o->ci = xcalloc((size_t)cnt, sizeof(int));
    o->v = xcalloc((size_t)cnt, sizeof(double));
    if (!o->ci || !o->v) return ORC_OOM;
    for (int i = 0; i < a->rows; i++) {
        if (rmap[i] < 0) continue;
        int pos = o->rp[rmap[i]];
        for (int k = a->rp[i]; k < a->rp[i + 1]; k++) {
            int c = cmap[a->ci[k]];
            if (c < 0) continue;
            o->ci[pos] = c;
            o->v[pos] = a->v[k];
            pos++;
        }
    }
    return ORC_OK;
}

/* --------------------------------------------------------- aggregation */

/*
 * Vertex priority for the distance-2 maximal independent set: the splitmix64
 * output function (Steele, Lea & Flood 2014; Vigna's splitmix64) applied to
 * (seed XOR i).  It is a bijection of 64-bit words, so priorities never tie.
 */
#define PRIO_SEED 0x9E3779B97F4A7C15ULL
uint64_t orc_priority(uint64_t i)
{
    uint64_t z = PRIO_SEED ^ i;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/*
 * Strong connections (smoothed aggregation, Sec. 3.1 reading): j != i is a
 * strong neighbour of i iff a_ij^2 >= theta^2 a_ii a_jj, evaluated as
 * (a_ij*a_ij) >= (theta2 * (a_ii*a_jj)) with theta2 = theta*theta.
 */
static int strength(const csr_t *a, double theta2, csr_t *s)
{
    int n = a->rows;
    double *diag = xcalloc((size_t)n, sizeof(double));
    if (!diag) return ORC_OOM;
    for (int i = 0; i < n; i++) {
        long q = csr_find(a, i, i);
        diag[i] = q >= 0 ? a->v[q] : 0.0;
    }
    s->rows = s->cols = n;
    s->rp = xcalloc((size_t)n + 1, sizeof(int));
    for (int pass = 0; pass < 2; pass++) {
        for (int i = 0; i < n; i++) {
            int cnt = 0;
            int pos = pass ? s->rp[i] : 0;
            for (int k = a->rp[i]; k < a->rp[i + 1]; k++) {
                int j = a->ci[k];
                if (j == i) continue;
                double aij = a->v[k];
                if (aij * aij >= theta2 * (diag[i] * diag[j])) {
                    if (pass) {
                        s->ci[pos] = j;
                        s->v[pos] = aij;
                        pos++;
                    }
                    cnt++;
                }
            }
            if (!pass) s->rp[i + 1] = s->rp[i] + cnt;
        }
        if (!pass) {
            s->ci = xcalloc((size_t)s->rp[n], sizeof(int));
            s->v = xcalloc((size_t)s->rp[n], sizeof(double));
            if (!s->ci || !s->v) return ORC_OOM;
        }
    }
    free(diag);
    return ORC_OK;
}

typedef struct {
    uint64_t p;
    int i;
} prio_t;

static int cmp_prio_desc(const void *a, const void *b)
{
    const prio_t *x = a, *y = b;
    if (x->p != y->p) return x->p < y->p ? 1 : -1;
    return (x->i > y->i) - (x->i < y->i);
}

/*
 * Distance-2 maximal independent set of the strong graph by the sequential
 * greedy rule: visit vertices in decreasing priority; a vertex not yet within
 * distance 2 of a chosen root becomes a root.
 */
static int mis2_greedy(const csr_t *s, unsigned char *root)
{
    int n = s->rows;
    prio_t *order = malloc(sizeof(prio_t) * (size_t)(n > 0 ? n : 1));
    unsigned char *covered = xcalloc((size_t)n, 1);
    if (!order || !covered) return ORC_OOM;
    for (int i = 0; i < n; i++) {
        order[i].p = orc_priority((uint64_t)i);
        order[i].i = i;
        root[i] = 0;
    }
    qsort(order, (size_t)n, sizeof(prio_t), cmp_prio_desc);
    for (int t = 0; t < n; t++) {
        int v = order[t].i;
        if (covered[v]) continue;
        root[v] = 1;
        covered[v] = 1;
        for (int k = s->rp[v]; k < s->rp[v + 1]; k++) {
            int w = s->ci[k];
            covered[w] = 1;
            for (int q = s->rp[w]; q < s->rp[w + 1]; q++) covered[s->ci[q]] = 1;
        }
    }
    free(order);
    free(covered);
    return ORC_OK;
}

/*
 * Aggregation (reading of Sec. 3.1's smoothed aggregation with a deterministic
 * rule):
 *   phase 1  each MIS-2 root and its strong neighbours form an aggregate; the
 *            aggregate id is the rank of the root in ascending vertex order;
 *   phase 2  each vertex not yet aggregated joins the phase-1 aggregate of the
 *            strong neighbour with the largest |a_ij| (ties: smallest id);
 *            only phase-1 assignments are read;
 *   phase 3  any vertex still free becomes a singleton, ids appended in
 *            ascending vertex order.
 */
static int aggregate(const csr_t *a, double theta2, int *agg, int *nagg_out, unsigned char *root_out)
{
    int n = a->rows;
    csr_t s = {0};
    int st = strength(a, theta2, &s);
    if (st) return st;
    unsigned char *root = root_out ? root_out : xcalloc((size_t)n, 1);
    if (!root) return ORC_OOM;
    st = mis2_greedy(&s, root);
    if (st) return st;
    for (int i = 0; i < n; i++) agg[i] = -1;
    int nagg = 0;
    for (int i = 0; i < n; i++)
        if (root[i]) agg[i] = nagg++;
    for (int i = 0; i < n; i++)
        if (root[i])
            for (int k = s.rp[i]; k < s.rp[i + 1]; k++) agg[s.ci[k]] = agg[i];
    int *phase2 = malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    if (!phase2) return ORC_OOM;
    for (int i = 0; i < n; i++) {
        phase2[i] = agg[i];
        if (agg[i] >= 0) continue;
        double best = -1.0;
        int bid = -1;
        for (int k = s.rp[i]; k < s.rp[i + 1]; k++) {
            int j = s.ci[k];
            if (agg[j] < 0) continue;
            double w = fabs(s.v[k]);
            if (w > best || (w == best && agg[j] < bid)) {
                best = w;
                bid = agg[j];
            }
        }
        phase2[i] = bid;
    }
    for (int i = 0; i < n; i++) {
        agg[i] = phase2[i];
        if (agg[i] < 0) agg[i] = nagg++;
    }
    free(phase2);
    if (!root_out) free(root);
    csr_free(&s);
    *nagg_out = nagg;
    return ORC_OK;
}

/*
 * Smoothed prolongator S = (I - omega D^-1 A) S_hat (Vanek-Mandel-Brezina):
 * S_hat is the unnormalised piecewise-constant aggregate indicator;
 * omega = 4 / (3 rho) with rho = max_i sum_j |a_ij| / a_ii (Gershgorin bound
 * of D^-1 A).  Row i has the columns {agg(j) : a_ij in pattern}; its value for
 * column J is [agg(i)==J] - (omega/a_ii) * sum_{j ascending, agg(j)=J} a_ij.
 */
static int prolongator(const csr_t *a, const int *agg, int nagg, int smooth, csr_t *p)
{
    int n = a->rows;
    p->rows = n;
    p->cols = nagg;
    p->rp = xcalloc((size_t)n + 1, sizeof(int));
    if (!smooth) {
        p->ci = xcalloc((size_t)n, sizeof(int));
        p->v = xcalloc((size_t)n, sizeof(double));
        for (int i = 0; i < n; i++) {
            p->rp[i + 1] = i + 1;
            p->ci[i] = agg[i];
            p->v[i] = 1.0;
        }
        return ORC_OK;
    }
    double rho = 0.0;
    for (int i = 0; i < n; i++) {
        double s = 0.0, aii = 0.0;
        for (int k = a->rp[i]; k < a->rp[i + 1]; k++) {
            s += fabs(a->v[k]);
            if (a->ci[k] == i) aii = a->v[k];
        }
        double r = s / aii;
        if (r > rho) rho = r;
    }
    double omega = 4.0 / (3.0 * rho);
    int *mark = malloc(sizeof(int) * (size_t)(nagg > 0 ? nagg : 1));
    double *acc = xcalloc((size_t)nagg, sizeof(double));
    int *list = malloc(sizeof(int) * 4096);
    if (!mark || !acc || !list) return ORC_OOM;
    for (int J = 0; J < nagg; J++) mark[J] = -1;
    for (int i = 0; i < n; i++) {
        int cnt = 0;
        for (int k = a->rp[i]; k < a->rp[i + 1]; k++) {
            int J = agg[a->ci[k]];
            if (mark[J] != i) { mark[J] = i; cnt++; }
        }
        p->rp[i + 1] = p->rp[i] + cnt;
    }
    p->ci = xcalloc((size_t)p->rp[n], sizeof(int));
    p->v = xcalloc((size_t)p->rp[n], sizeof(double));
    if (!p->ci || !p->v) return ORC_OOM;
    for (int J = 0; J < nagg; J++) mark[J] = -1;
    for (int i = 0; i < n; i++) {
        int cnt = 0;
        double aii = 0.0;
        for (int k = a->rp[i]; k < a->rp[i + 1]; k++) {
            int J = agg[a->ci[k]];
            if (a->ci[k] == i) aii = a->v[k];
            if (mark[J] != i) {
                mark[J] = i;
                acc[J] = 0.0;
                if (cnt >= 4096) return ORC_INVALID;
                list[cnt++] = J;
            }
            acc[J] = acc[J] + a->v[k];
        }
        double wi = omega / aii;
        qsort(list, (size_t)cnt, sizeof(int), cmp_int);
        int base = p->rp[i];
        for (int t = 0; t < cnt; t++) {
            int J = list[t];
            double delta = (J == agg[i]) ? 1.0 : 0.0;
            double tv = wi * acc[J];
            p->ci[base + t] = J;
            p->v[base + t] = delta - tv;
        }
    }
    free(mark);
    free(acc);
    free(list);
    return ORC_OK;
}

/*
 * Aggressive first-level coarsening (Sec. 5.1 uses it for the first level
 * of BoomerAMG; reading for smoothed aggregation): aggregate A, form the
 * tentative (unsmoothed) Galerkin matrix S_hat^T A S_hat of those aggregates,
 * aggregate that matrix with the next level's threshold, and give every
 * vertex the aggregate of its aggregate.
 */
static int aggregate_aggressive(const csr_t *a, double theta2, int *agg, int *nagg_out)
{
    int n = a->rows, n1 = 0, n2 = 0;
    int *agg1 = malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    if (!agg1) return ORC_OOM;
    int st = aggregate(a, theta2, agg1, &n1, NULL);
    if (st) return st;
    csr_t sh = {0}, sht = {0}, t = {0};
    if ((st = prolongator(a, agg1, n1, 0, &sh))) return st;
    if ((st = csr_transpose(&sh, &sht))) return st;
    if ((st = galerkin(&sht, a, &sh, 1, &t))) return st;
    int *agg2 = malloc(sizeof(int) * (size_t)(n1 > 0 ? n1 : 1));
    if (!agg2) return ORC_OOM;
    if ((st = aggregate(&t, theta2 * 0.25, agg2, &n2, NULL))) return st;
    for (int i = 0; i < n; i++) agg[i] = agg2[agg1[i]];
    *nagg_out = n2;
    free(agg1);
    free(agg2);
    csr_free(&sh);
    csr_free(&sht);
    csr_free(&t);
    return ORC_OK;
}

/*
 * Geometric hierarchy of the structured N x N square grid (vertex i + N j,
 * squares split along the (i,j)-(i+1,j+1) diagonal; the setting of the
 * geometric comparison of Sec. 5.4): the coarse grid takes every other
 * vertex, Nc = (N+1)/2, and the P1 interpolation from it is
 *   (2I, 2J)           <- coarse (I, J)                         weight 1
 *   (2I+1, 2J)         <- (I, J), (I+1, J)                      weights 1/2
 *   (2I, 2J+1)         <- (I, J), (I, J+1)                      weights 1/2
 *   (2I+1, 2J+1)       <- (I, J), (I+1, J+1) (the diagonal)     weights 1/2.
 * The state interpolation is its restriction to interior rows and columns.
 */
static int geometric_interp(int N, csr_t *p)
{
    int Nc = (N + 1) / 2, n = N * N;
    p->rows = n;
    p->cols = Nc * Nc;
    p->rp = xcalloc((size_t)n + 1, sizeof(int));
    p->ci = xcalloc((size_t)2 * n, sizeof(int));
    p->v = xcalloc((size_t)2 * n, sizeof(double));
    if (!p->rp || !p->ci || !p->v) return ORC_OOM;
    int k = 0;
    for (int j = 0; j < N; j++)
        for (int i = 0; i < N; i++) {
            int I = i / 2, J = j / 2;
            if (i % 2 == 0 && j % 2 == 0) {
                p->ci[k] = I + Nc * J;
                p->v[k++] = 1.0;
            } else {
                int I2 = I + (i % 2), J2 = J + (j % 2);
                p->ci[k] = I + Nc * J;
                p->v[k++] = 0.5;
                p->ci[k] = I2 + Nc * J2;
                p->v[k++] = 0.5;
            }
            p->rp[i + N * j + 1] = k;
        }
    return ORC_OK;
}

/* map of the N x N grid's vertices to interior numbering (-1 on the boundary) */
static int *grid_interior(int N)
{
    int *map = malloc(sizeof(int) * (size_t)N * N), m = 0;
    if (!map) return NULL;
    for (int j = 0; j < N; j++)
        for (int i = 0; i < N; i++)
            map[i + N * j] = (i > 0 && j > 0 && i < N - 1 && j < N - 1) ? m++ : -1;
    return map;
}

/* ---------------------------------------------------------------- dense */

/* lower Cholesky factor of the n x n matrix g (row-major); INDEFINITE on a
 * non-positive pivot */
static int chol(double *g, int n)
{
    for (int j = 0; j < n; j++) {
        double s = g[(long)j * n + j];
        for (int k = 0; k < j; k++) s -= g[(long)j * n + k] * g[(long)j * n + k];
        if (!(s > 0.0)) return ORC_INDEFINITE;
        double ljj = sqrt(s);
        g[(long)j * n + j] = ljj;
        for (int i = j + 1; i < n; i++) {
            double t = g[(long)i * n + j];
            for (int k = 0; k < j; k++) t -= g[(long)i * n + k] * g[(long)j * n + k];
            g[(long)i * n + j] = t / ljj;
        }
    }
    for (int i = 0; i < n; i++)
        for (int j = i + 1; j < n; j++) g[(long)i * n + j] = 0.0;
    return ORC_OK;
}

static void chol_solve(const double *l, int n, const double *b, double *x)
{
    for (int i = 0; i < n; i++) {
        double s = b[i];
        for (int k = 0; k < i; k++) s -= l[(long)i * n + k] * x[k];
        x[i] = s / l[(long)i * n + i];
    }
    for (int i = n - 1; i >= 0; i--) {
        double s = x[i];
        for (int k = i + 1; k < n; k++) s -= l[(long)k * n + i] * x[k];
        x[i] = s / l[(long)i * n + i];
    }
}

static double *dense_of(const csr_t *a)
{
    double *g = xcalloc((size_t)a->rows * (size_t)a->cols, sizeof(double));
    if (!g) return NULL;
    for (int i = 0; i < a->rows; i++)
        for (int k = a->rp[i]; k < a->rp[i + 1]; k++) g[(long)i * a->cols + a->ci[k]] = a->v[k];
    return g;
}

/* ---------------------------------------------------------- smoothing */

/*
 * Polynomial smoother on D^-1 A with D = l1 row sums (d_i = sum_j |a_ij|, so
 * the spectrum of D^-1 A lies in (0, 1]).  Each step:
 *   d <- cd[s] d + cr[s] D^-1 (b - A x);  x <- x + d.
 * Chebyshev of degree k on [1/30, 1] (Saad, Iterative Methods, Alg. 12.1):
 *   theta = (hi+lo)/2, delta = (hi-lo)/2, sigma = theta/delta, rho_0 = 1/sigma,
 *   d_0 = r_0 / theta,  rho_s = 1/(2 sigma - rho_{s-1}),
 *   d_s = rho_s rho_{s-1} d_{s-1} + (2 rho_s / delta) r_s.
 * l1-Jacobi with nu sweeps is cd = 0, cr = 1 for every step.
 */
static void smoother_coeffs(orc_t *o)
{
    if (o->smoother == 0) {
        o->nsteps = o->degree;
        for (int s = 0; s < o->nsteps; s++) {
            o->cd[s] = 0.0;
            o->cr[s] = 1.0;
        }
        return;
    }
    double lo = 1.0 / 30.0, hi = 1.0;
    double theta = (hi + lo) / 2.0, delta = (hi - lo) / 2.0, sigma = theta / delta;
    double rho = 1.0 / sigma;
    o->nsteps = o->degree;
    o->cd[0] = 0.0;
    o->cr[0] = 1.0 / theta;
    for (int s = 1; s < o->nsteps; s++) {
        double rn = 1.0 / (2.0 * sigma - rho);
        o->cd[s] = rn * rho;
        o->cr[s] = 2.0 * rn / delta;
        rho = rn;
    }
}

static void smooth(orc_t *o, int l, const double *b, double *x, int zero_init, double *d, double *r)
{
    const csr_t *A = &o->A[l];
    int n = A->rows;
    for (int s = 0; s < o->nsteps; s++) {
        if (s == 0 && zero_init) {
            ORC_ROWS
            for (int i = 0; i < n; i++) r[i] = b[i];
        } else {
            spmv(A, x, r);
            ORC_ROWS
            for (int i = 0; i < n; i++) r[i] = b[i] - r[i];
        }
        ORC_ROWS
        for (int i = 0; i < n; i++) {
            double ri = r[i] / o->dl1[l][i];
            double prev = (s == 0) ? 0.0 : d[i];
            d[i] = o->cd[s] * prev + o->cr[s] * ri;
            x[i] = (s == 0 && zero_init) ? d[i] : x[i] + d[i];
        }
    }
}

/* --------------------------------------------------------------- V-cycle */

/*
 * One symmetric V-cycle for A_l x = b starting from x = 0 (the AMG
 * preconditioner of the state/adjoint solves, Sec. 5.2): pre-smooth,
 * restrict the residual with S^T, recurse, prolongate with S, post-smooth
 * with the same polynomial; dense Cholesky on the coarsest level.
 */
static int vcycle(orc_t *o, int l, const double *b, double *x)
{
    int n = o->A[l].rows;
    if (l == o->Ls - 1) {
        chol_solve(o->Ac_chol, n, b, x);
        return ORC_OK;
    }
    int nc = o->A[l + 1].rows;
    double *d = xcalloc((size_t)n, sizeof(double)), *r = xcalloc((size_t)n, sizeof(double));
    double *bc = xcalloc((size_t)nc, sizeof(double)), *ec = xcalloc((size_t)nc, sizeof(double));
    double *t = xcalloc((size_t)n, sizeof(double));
    if (!d || !r || !bc || !ec || !t) return ORC_OOM;
    smooth(o, l, b, x, 1, d, r);
    spmv(&o->A[l], x, r);
    ORC_ROWS
    for (int i = 0; i < n; i++) r[i] = b[i] - r[i];
    spmv(&o->St[l], r, bc);
    int st = vcycle(o, l + 1, bc, ec);
    spmv(&o->S[l], ec, t);
    ORC_ROWS
    for (int i = 0; i < n; i++) x[i] = x[i] + t[i];
    smooth(o, l, b, x, 0, d, r);
    free(d);
    free(r);
    free(bc);
    free(ec);
    free(t);
    return st;
}

/* ------------------------------------------------------------------- CG */

typedef int (*apply_fn)(orc_t *o, int level, const double *x, double *y);

/*
 * Preconditioned conjugate gradients from x = 0, stopping when
 * ||r_k||_2 <= tol ||f||_2 (recursively updated residual).  Returns
 * INDEFINITE if p.Ap <= 0 or r.z <= 0, NOT_CONVERGED after maxit.
 */
static int pcg(orc_t *o, int level, int n, apply_fn op, apply_fn prec, const double *f, double *x,
               double tol, int maxit, long *iters, double *relres)
{
    double *r = xcalloc((size_t)n, sizeof(double)), *z = xcalloc((size_t)n, sizeof(double));
    double *p = xcalloc((size_t)n, sizeof(double)), *q = xcalloc((size_t)n, sizeof(double));
    if (!r || !z || !p || !q) return ORC_OOM;
    int st = ORC_OK;
    long k = 0;
    for (int i = 0; i < n; i++) {
        x[i] = 0.0;
        r[i] = f[i];
    }
    double nf = nrm2(n, f), nr = nf;
    if (!(nf == nf)) { st = ORC_NUMERIC; goto done; }
    if (nf == 0.0) goto done;
    if ((st = prec(o, level, r, z))) goto done;
    memcpy(p, z, sizeof(double) * (size_t)n);
    double rz = dot(n, r, z);
    if (!(rz > 0.0)) { st = (rz == rz) ? ORC_INDEFINITE : ORC_NUMERIC; goto done; }
    for (k = 1; k <= maxit; k++) {
        if ((st = op(o, level, p, q))) goto done;
        double pq = dot(n, p, q);
        if (!(pq > 0.0)) { st = (pq == pq) ? ORC_INDEFINITE : ORC_NUMERIC; goto done; }
        double alpha = rz / pq;
        ORC_ROWS
        for (int i = 0; i < n; i++) {
            x[i] = x[i] + alpha * p[i];
            r[i] = r[i] - alpha * q[i];
        }
        nr = nrm2(n, r);
        if (!(nr == nr)) { st = ORC_NUMERIC; goto done; }
        if (nr <= tol * nf) break;
        if ((st = prec(o, level, r, z))) goto done;
        double rzn = dot(n, r, z);
        if (!(rzn > 0.0)) { st = (rzn == rzn) ? ORC_INDEFINITE : ORC_NUMERIC; goto done; }
        double beta = rzn / rz;
        rz = rzn;
        ORC_ROWS
        for (int i = 0; i < n; i++) p[i] = z[i] + beta * p[i];
    }
    if (k > maxit) { k = maxit; st = ORC_NOT_CONVERGED; }
done:
    if (iters) *iters = k;
    if (relres) *relres = nf > 0.0 ? nr / nf : 0.0;
    free(r);
    free(z);
    free(p);
    free(q);
    return st;
}

static int op_A(orc_t *o, int l, const double *x, double *y)
{
    spmv(&o->A[l], x, y);
    return ORC_OK;
}
static int prec_V(orc_t *o, int l, const double *x, double *y) { return vcycle(o, l, x, y); }
static int op_Mu(orc_t *o, int l, const double *x, double *y)
{
    spmv(&o->Mu[l], x, y);
    return ORC_OK;
}
static int prec_Jmu(orc_t *o, int l, const double *x, double *y)
{
    const csr_t *M = &o->Mu[l];
    int n = M->rows;
    ORC_ROWS
    for (int i = 0; i < n; i++) y[i] = x[i] / M->v[csr_find(M, i, i)];
    return ORC_OK;
}

/* A_l^-1 f by AMG-preconditioned CG (Sec. 5.2: inner state/adjoint solves) */
static int state_solve(orc_t *o, int l, const double *f, double *y, double tol)
{
    long it = 0;
    int st = pcg(o, l, o->A[l].rows, op_A, prec_V, f, y, tol, o->inner_maxit, &it, NULL);
    o->inner_iters += it;
    return st;
}

/* M_{u,l}^-1 b by Jacobi-preconditioned CG (Sec. 5.2: mass solves) */
static int mass_solve(orc_t *o, int l, const double *b, double *x)
{
    long it = 0;
    int st = pcg(o, l, o->Mu[l].rows, op_Mu, prec_Jmu, b, x, o->mass_tol, o->mass_maxit, &it, NULL);
    o->mass_iters += it;
    return st;
}

/* ------------------------------------------------------------- Hessian */

/* H_l v = M_yu^T A^-1 M_y A^-1 M_yu v + beta M_u v (Eq. firstorderpractice,
 * on level l with the Galerkin matrices of Eq. coarsestiffness/coarsemass) */
static int hessian(orc_t *o, int l, const double *v, double *hv)
{
    int m = o->A[l].rows, n = o->Mu[l].rows;
    double *t1 = xcalloc((size_t)m, sizeof(double)), *y = xcalloc((size_t)m, sizeof(double));
    double *t2 = xcalloc((size_t)m, sizeof(double)), *p = xcalloc((size_t)m, sizeof(double));
    double *w = xcalloc((size_t)n, sizeof(double));
    if (!t1 || !y || !t2 || !p || !w) return ORC_OOM;
    int st;
    /* level 0: the operator of the outer CG; levels >= 1 occur only inside
     * the preconditioner (Algorithm MLAS) and use the preconditioner tolerance */
    double tol = l == 0 ? o->inner_tol : o->pc_inner_tol;
    spmv(&o->Myu[l], v, t1);
    if ((st = state_solve(o, l, t1, y, tol))) goto done;
    spmv(&o->My[l], y, t2);
    if ((st = state_solve(o, l, t2, p, tol))) goto done;
    spmv(&o->Myut[l], p, hv);
    spmv(&o->Mu[l], v, w);
    ORC_ROWS
    for (int i = 0; i < n; i++) hv[i] = hv[i] + o->beta * w[i];
    o->happlies += (l == 0);
done:
    free(t1);
    free(y);
    free(t2);
    free(p);
    free(w);
    return st;
}

/* ------------------------------------------------------------- MLAS */

static int mlas_Q(orc_t *o, int j, const double *b, double *u);

/* R_j b = P_j Q_{j+1} P_j^T b + beta^-1 (M_{u,j}^-1 b - P_j M_{u,j+1}^-1 P_j^T b)
 * (Eq. twogridinmulti in the M_u-scaled form of Sec. 5.2) */
static int mlas_R(orc_t *o, int j, const double *b, double *out)
{
    int n = o->Mu[j].rows, nc = o->Mu[j + 1].rows;
    double *bc = xcalloc((size_t)nc, sizeof(double)), *qc = xcalloc((size_t)nc, sizeof(double));
    double *wc = xcalloc((size_t)nc, sizeof(double)), *w1 = xcalloc((size_t)n, sizeof(double));
    double *ta = xcalloc((size_t)n, sizeof(double)), *tb = xcalloc((size_t)n, sizeof(double));
    if (!bc || !qc || !wc || !w1 || !ta || !tb) return ORC_OOM;
    int st;
    spmv(&o->Pt[j], b, bc);
    if ((st = mlas_Q(o, j + 1, bc, qc))) goto done;
    if ((st = mass_solve(o, j, b, w1))) goto done;
    if ((st = mass_solve(o, j + 1, bc, wc))) goto done;
    spmv(&o->P[j], qc, ta);
    spmv(&o->P[j], wc, tb);
    ORC_ROWS
    for (int i = 0; i < n; i++) out[i] = ta[i] + (w1[i] - tb[i]) / o->beta;
done:
    free(bc);
    free(qc);
    free(wc);
    free(w1);
    free(ta);
    free(tb);
    return st;
}

static int op_H(orc_t *o, int l, const double *x, double *y) { return hessian(o, l, x, y); }
static int prec_none(orc_t *o, int l, const double *x, double *y)
{
    memcpy(y, x, sizeof(double) * (size_t)o->Mu[l].rows);
    return ORC_OK;
}

/* Algorithm MLAS (Sec. 3.2), M_u-scaled: Q_j approximates H_j^-1.  On the
 * coarsest level Q is H^-1 itself (dense Cholesky, the assumption of the
 * analysis), or unpreconditioned CG on H to a loose tolerance as in the
 * implementation of Sec. 5.2 (the iterate at the cap is used as it stands). */
static int mlas_Q(orc_t *o, int j, const double *b, double *u)
{
    int n = o->Mu[j].rows;
    if (j == o->ell - 1) {
        if (o->coarse_solve == 1 || (o->coarse_solve == 2 && n > 4096)) {
            long it = 0;
            int st = pcg(o, j, n, op_H, prec_none, b, u, o->coarse_tol, o->coarse_maxit, &it, NULL);
            o->coarse_iters += it;
            return st == ORC_NOT_CONVERGED ? ORC_OK : st;
        }
        chol_solve(o->Hc_chol, n, b, u);
        return ORC_OK;
    }
    int st = mlas_R(o, j, b, u);
    if (st || j == 0) return st;
    double *hu = xcalloc((size_t)n, sizeof(double)), *du = xcalloc((size_t)n, sizeof(double));
    if (!hu || !du) return ORC_OOM;
    if ((st = hessian(o, j, u, hu))) goto done;
    for (int i = 0; i < n; i++) hu[i] = b[i] - hu[i];
    if ((st = mlas_R(o, j, hu, du))) goto done;
    for (int i = 0; i < n; i++) u[i] = u[i] + du[i];
done:
    free(hu);
    free(du);
    return st;
}

/* ------------------------------------------------------------- setup */

static int dense_chol_of(const csr_t *a, double **out)
{
    if (a->rows > DENSE_MAX) return ORC_INVALID;
    double *g = dense_of(a);
    if (!g) return ORC_OOM;
    int st = chol(g, a->rows);
    if (st) { free(g); return st; }
    *out = g;
    return ORC_OK;
}

/*
 * Dense coarsest Hessian H_c = M_yu^T A^-1 M_y A^-1 M_yu + beta M_u on level c
 * (the exact coarsest inverse assumed by the theory, Sec. 3.2) and its
 * Cholesky factor.
 */
static int build_coarse_hessian(orc_t *o)
{
    int c = o->ell - 1;
    int m = o->A[c].rows, n = o->Mu[c].rows;
    if (n > DENSE_MAX || m > DENSE_MAX) return ORC_INVALID;
    const double *la = o->Ac_chol;
    if (c != o->Ls - 1) {
        int st = dense_chol_of(&o->A[c], &o->Aell_chol);
        if (st) return st;
        la = o->Aell_chol;
    }
    double *H = xcalloc((size_t)n * (size_t)n, sizeof(double));
    double *e = xcalloc((size_t)n, sizeof(double)), *t1 = xcalloc((size_t)m, sizeof(double));
    double *y = xcalloc((size_t)m, sizeof(double)), *t2 = xcalloc((size_t)m, sizeof(double));
    double *p = xcalloc((size_t)m, sizeof(double)), *col = xcalloc((size_t)n, sizeof(double));
    double *w = xcalloc((size_t)n, sizeof(double));
    if (!H || !e || !t1 || !y || !t2 || !p || !col || !w) return ORC_OOM;
    for (int k = 0; k < n; k++) {
        memset(e, 0, sizeof(double) * (size_t)n);
        e[k] = 1.0;
        spmv(&o->Myu[c], e, t1);
        chol_solve(la, m, t1, y);
        spmv(&o->My[c], y, t2);
        chol_solve(la, m, t2, p);
        spmv(&o->Myut[c], p, col);
        spmv(&o->Mu[c], e, w);
        for (int i = 0; i < n; i++) H[(long)i * n + k] = col[i] + o->beta * w[i];
    }
    free(e);
    free(t1);
    free(y);
    free(t2);
    free(p);
    free(col);
    free(w);
    int st = chol(H, n);
    if (st) { free(H); return st; }
    o->Hc_chol = H;
    return ORC_OK;
}

static void free_hierarchy(orc_t *o)
{
    for (int l = 0; l < MAXL; l++) {
        csr_free(&o->A[l]);
        csr_free(&o->My[l]);
        csr_free(&o->S[l]);
        csr_free(&o->St[l]);
        csr_free(&o->KN[l]);
        csr_free(&o->Mu[l]);
        csr_free(&o->P[l]);
        csr_free(&o->Pt[l]);
        csr_free(&o->Myu[l]);
        csr_free(&o->Myut[l]);
        free(o->sagg[l]);
        free(o->cagg[l]);
        free(o->dl1[l]);
        o->sagg[l] = o->cagg[l] = NULL;
        o->dl1[l] = NULL;
    }
    free(o->Ac_chol);
    free(o->Hc_chol);
    free(o->Aell_chol);
    o->Ac_chol = o->Hc_chol = o->Aell_chol = NULL;
    o->Ls = o->Lc = o->ell = 0;
    o->setup_done = 0;
}

/* ------------------------------------------------------------ public API */

void orc_destroy(void *h);

int orc_create(int dim, long nv, const double *coords, long ne, const int *elems,
               const unsigned char *dirichlet, const double *kappa, double beta, const double *yd,
               void **out)
{
    if (!out || (dim != 2 && dim != 3) || nv <= 0 || ne <= 0 || !(beta > 0.0)) return ORC_INVALID;
    orc_t *o = xcalloc(1, sizeof(orc_t));
    if (!o) return ORC_OOM;
    o->dim = dim;
    o->nv = nv;
    o->ne = ne;
    o->beta = beta;
    o->coords = malloc(sizeof(double) * (size_t)nv * dim);
    o->elems = malloc(sizeof(int) * (size_t)ne * (dim + 1));
    o->dir = malloc((size_t)nv);
    o->kappa = malloc(sizeof(double) * (size_t)ne);
    if (!o->coords || !o->elems || !o->dir || !o->kappa) return ORC_OOM;
    memcpy(o->coords, coords, sizeof(double) * (size_t)nv * dim);
    memcpy(o->elems, elems, sizeof(int) * (size_t)ne * (dim + 1));
    memcpy(o->dir, dirichlet, (size_t)nv);
    memcpy(o->kappa, kappa, sizeof(double) * (size_t)ne);
    for (long q = 0; q < ne * (dim + 1); q++)
        if (elems[q] < 0 || elems[q] >= nv) return ORC_INVALID;
    o->state_of_vertex = malloc(sizeof(int) * (size_t)nv);
    int m = 0;
    for (long v = 0; v < nv; v++) o->state_of_vertex[v] = dirichlet[v] ? -1 : m++;
    if (m == 0) { /* no vertex off the Dirichlet boundary: empty state space (Sec. 2) */
        orc_destroy(o);
        return ORC_INVALID;
    }
    o->m = m;
    o->n = (int)nv;
    o->yd_state = xcalloc((size_t)m, sizeof(double));
    for (long v = 0; v < nv; v++)
        if (!dirichlet[v]) o->yd_state[o->state_of_vertex[v]] = yd ? yd[v] : 0.0;
    int st = assemble(o);
    if (st) return st;
    *out = o;
    return ORC_OK;
}

int orc_set_yd(void *h, const double *yd)
{
    orc_t *o = h;
    for (long v = 0; v < o->nv; v++)
        if (!o->dir[v]) o->yd_state[o->state_of_vertex[v]] = yd[v];
    return ORC_OK;
}

int orc_setup(void *h, int max_levels, int hessian_levels, double theta, int coarse_max,
              int smoother, int degree, int smooth_p)
{
    orc_t *o = h;
    if (!o || max_levels < 1 || max_levels > MAXL || degree < 1 || degree > 16 || coarse_max < 1)
        return ORC_INVALID;
    free_hierarchy(o);
    o->max_levels = max_levels;
    o->hess_levels = hessian_levels;
    o->theta = theta;
    o->coarse_max = coarse_max;
    o->smoother = smoother;
    o->degree = degree;
    o->smooth_p = smooth_p;
    smoother_coeffs(o);
    int st;
    /* level 0: state dofs are the non-Dirichlet vertices, control dofs all vertices */
    int *all = malloc(sizeof(int) * (size_t)o->n);
    for (int v = 0; v < o->n; v++) all[v] = v;
    if ((st = extract(&o->Kfull, o->state_of_vertex, o->m, o->state_of_vertex, o->m, &o->A[0]))) return st;
    if ((st = extract(&o->Mfull, o->state_of_vertex, o->m, o->state_of_vertex, o->m, &o->My[0]))) return st;
    if ((st = extract(&o->Mfull, o->state_of_vertex, o->m, all, o->n, &o->Myu[0]))) return st;
    if ((st = extract(&o->Kfull, all, o->n, all, o->n, &o->KN[0]))) return st;
    if ((st = extract(&o->Mfull, all, o->n, all, o->n, &o->Mu[0]))) return st;
    free(all);
    if (o->geometric) {
        /* the mesh must be the structured square grid with its whole boundary Dirichlet */
        int N = (int)lround(sqrt((double)o->n));
        if (o->dim != 2 || N * N != o->n || N < 3) return ORC_INVALID;
        int *bmap = grid_interior(N);
        for (int v = 0; v < o->n; v++)
            if ((bmap[v] >= 0) != (o->state_of_vertex[v] >= 0)) return ORC_INVALID;
        free(bmap);
        o->Ls = o->Lc = 1;
        for (int l = 0; l + 1 < max_levels && N >= 5 && N % 2 == 1 && o->KN[l].rows > coarse_max; l++) {
            int Nc = (N + 1) / 2;
            int *fi = grid_interior(N), *ci = grid_interior(Nc);
            int *allc = malloc(sizeof(int) * (size_t)Nc * Nc);
            for (int v = 0; v < Nc * Nc; v++) allc[v] = v;
            csr_t pg = {0};
            if ((st = geometric_interp(N, &pg))) return st;
            if ((st = extract(&pg, fi, (N - 2) * (N - 2), ci, (Nc - 2) * (Nc - 2), &o->S[l]))) return st;
            int *allf = malloc(sizeof(int) * (size_t)N * N);
            for (int v = 0; v < N * N; v++) allf[v] = v;
            if ((st = extract(&pg, allf, N * N, allc, Nc * Nc, &o->P[l]))) return st;
            free(allf);
            free(allc);
            free(fi);
            free(ci);
            csr_free(&pg);
            if ((st = csr_transpose(&o->S[l], &o->St[l]))) return st;
            if ((st = galerkin(&o->St[l], &o->A[l], &o->S[l], 1, &o->A[l + 1]))) return st;
            if ((st = galerkin(&o->St[l], &o->My[l], &o->S[l], 1, &o->My[l + 1]))) return st;
            if ((st = csr_transpose(&o->P[l], &o->Pt[l]))) return st;
            if ((st = galerkin(&o->Pt[l], &o->KN[l], &o->P[l], 1, &o->KN[l + 1]))) return st;
            if ((st = galerkin(&o->Pt[l], &o->Mu[l], &o->P[l], 1, &o->Mu[l + 1]))) return st;
            o->Ls = o->Lc = l + 2;
            N = Nc;
        }
        goto hierarchies_done;
    }
    /* coarsen: strength threshold theta at level 0, halved per level */
    double th = theta;
    o->Ls = 1;
    for (int l = 0; l + 1 < max_levels && o->A[l].rows > coarse_max; l++) {
        int n = o->A[l].rows;
        int *agg = malloc(sizeof(int) * (size_t)n);
        int nagg = 0;
        if (l == 0 && o->aggressive) st = aggregate_aggressive(&o->A[l], th * th, agg, &nagg);
        else st = aggregate(&o->A[l], th * th, agg, &nagg, NULL);
        if (st) return st;
        if ((double)n < 1.2 * (double)nagg) { free(agg); break; }
        o->sagg[l] = agg;
        o->snagg[l] = nagg;
        if ((st = prolongator(&o->A[l], agg, nagg, smooth_p, &o->S[l]))) return st;
        if ((st = csr_transpose(&o->S[l], &o->St[l]))) return st;
        if ((st = galerkin(&o->St[l], &o->A[l], &o->S[l], 1, &o->A[l + 1]))) return st;
        if ((st = galerkin(&o->St[l], &o->My[l], &o->S[l], 1, &o->My[l + 1]))) return st;
        o->Ls = l + 2;
        th = th * 0.5;
    }
    th = theta;
    o->Lc = 1;
    for (int l = 0; l + 1 < max_levels && o->KN[l].rows > coarse_max; l++) {
        int n = o->KN[l].rows;
        int *agg = malloc(sizeof(int) * (size_t)n);
        int nagg = 0;
        if (l == 0 && o->aggressive) st = aggregate_aggressive(&o->KN[l], th * th, agg, &nagg);
        else st = aggregate(&o->KN[l], th * th, agg, &nagg, NULL);
        if (st) return st;
        if ((double)n < 1.2 * (double)nagg) { free(agg); break; }
        o->cagg[l] = agg;
        o->cnagg[l] = nagg;
        if ((st = prolongator(&o->KN[l], agg, nagg, smooth_p, &o->P[l]))) return st;
        if ((st = csr_transpose(&o->P[l], &o->Pt[l]))) return st;
        if ((st = galerkin(&o->Pt[l], &o->KN[l], &o->P[l], 1, &o->KN[l + 1]))) return st;
        if ((st = galerkin(&o->Pt[l], &o->Mu[l], &o->P[l], 1, &o->Mu[l + 1]))) return st;
        o->Lc = l + 2;
        th = th * 0.5;
    }
hierarchies_done:;
    int lmin = o->Ls < o->Lc ? o->Ls : o->Lc;
    for (int l = 0; l + 1 < lmin; l++)
        if ((st = galerkin(&o->St[l], &o->Myu[l], &o->P[l], 0, &o->Myu[l + 1]))) return st;
    for (int l = 0; l < lmin; l++)
        if ((st = csr_transpose(&o->Myu[l], &o->Myut[l]))) return st;
    /* l1 smoother diagonals */
    for (int l = 0; l < o->Ls; l++) {
        const csr_t *a = &o->A[l];
        o->dl1[l] = xcalloc((size_t)a->rows, sizeof(double));
        for (int i = 0; i < a->rows; i++) {
            double s = 0.0;
            for (int k = a->rp[i]; k < a->rp[i + 1]; k++) s += fabs(a->v[k]);
            o->dl1[l][i] = s;
        }
    }
    if ((st = dense_chol_of(&o->A[o->Ls - 1], &o->Ac_chol))) return st;
    o->ell = lmin;
    if (hessian_levels > 0 && hessian_levels < o->ell) o->ell = hessian_levels;
    o->inner_tol = 1e-10;
    o->mass_tol = 1e-10;
    o->pc_inner_tol = 1e-10;
    o->inner_maxit = 1000;
    o->mass_maxit = 1000;
    if ((st = build_coarse_hessian(o))) return st;
    o->setup_done = 1;
    return ORC_OK;
}

/* hierarchy kind for the next orc_setup: aggressive first-level coarsening,
 * or the geometric hierarchy of a structured square grid */
int orc_set_hierarchy(void *h, int aggressive, int geometric)
{
    orc_t *o = h;
    if (aggressive < 0 || aggressive > 1 || geometric < 0 || geometric > 1) return ORC_INVALID;
    o->aggressive = aggressive;
    o->geometric = geometric;
    return ORC_OK;
}

int orc_set_tols(void *h, double inner_tol, double mass_tol, int inner_maxit, int mass_maxit)
{
    orc_t *o = h;
    o->inner_tol = inner_tol;
    o->pc_inner_tol = inner_tol;
    o->mass_tol = mass_tol;
    o->inner_maxit = inner_maxit;
    o->mass_maxit = mass_maxit;
    return ORC_OK;
}

int orc_set_coarse_solve(void *h, int mode, double tol, int maxit, long *iters)
{
    orc_t *o = h;
    if (mode < 0 || mode > 2 || !(tol > 0.0) || maxit < 1) return ORC_INVALID;
    o->coarse_solve = mode;
    o->coarse_tol = tol;
    o->coarse_maxit = maxit;
    if (iters) *iters = o->coarse_iters;
    o->coarse_iters = 0;
    return ORC_OK;
}

int orc_set_precond_tol(void *h, double pc_inner_tol)
{
    orc_t *o = h;
    o->pc_inner_tol = pc_inner_tol;
    return ORC_OK;
}

int orc_sizes(void *h, long *m, long *n, int *Ls, int *Lc, int *ell, long *ssz, long *csz)
{
    orc_t *o = h;
    *m = o->m;
    *n = o->n;
    *Ls = o->Ls;
    *Lc = o->Lc;
    *ell = o->ell;
    for (int l = 0; l < o->Ls; l++) ssz[l] = o->A[l].rows;
    for (int l = 0; l < o->Lc; l++) csz[l] = o->KN[l].rows;
    return ORC_OK;
}

/* which: 0 A, 1 M_y, 2 M_yu, 3 S, 4 K_N, 5 M_u, 6 P, 7 K_full, 8 M_full */
static const csr_t *pick(orc_t *o, int which, int l)
{
    if (l < 0 || l >= MAXL) return NULL;
    switch (which) {
    case 0: return l < o->Ls ? &o->A[l] : NULL;
    case 1: return l < o->Ls ? &o->My[l] : NULL;
    case 2: return l < (o->Ls < o->Lc ? o->Ls : o->Lc) ? &o->Myu[l] : NULL;
    case 3: return l + 1 < o->Ls ? &o->S[l] : NULL;
    case 4: return l < o->Lc ? &o->KN[l] : NULL;
    case 5: return l < o->Lc ? &o->Mu[l] : NULL;
    case 6: return l + 1 < o->Lc ? &o->P[l] : NULL;
    case 7: return &o->Kfull;
    case 8: return &o->Mfull;
    }
    return NULL;
}

int orc_matrix_info(void *h, int which, int l, long *rows, long *cols, long *nnz)
{
    const csr_t *a = pick(h, which, l);
    if (!a || !a->rp) return ORC_INVALID;
    *rows = a->rows;
    *cols = a->cols;
    *nnz = a->rp[a->rows];
    return ORC_OK;
}

int orc_matrix_copy(void *h, int which, int l, int *rp, int *ci, double *v)
{
    const csr_t *a = pick(h, which, l);
    if (!a || !a->rp) return ORC_INVALID;
    memcpy(rp, a->rp, sizeof(int) * ((size_t)a->rows + 1));
    memcpy(ci, a->ci, sizeof(int) * (size_t)a->rp[a->rows]);
    memcpy(v, a->v, sizeof(double) * (size_t)a->rp[a->rows]);
    return ORC_OK;
}

int orc_aggregates(void *h, int hier, int l, int *agg, int *nagg)
{
    orc_t *o = h;
    int L = hier ? o->Lc : o->Ls;
    if (l < 0 || l + 1 >= L || o->geometric) return ORC_INVALID;
    int n = hier ? o->KN[l].rows : o->A[l].rows;
    memcpy(agg, hier ? o->cagg[l] : o->sagg[l], sizeof(int) * (size_t)n);
    *nagg = hier ? o->cnagg[l] : o->snagg[l];
    return ORC_OK;
}

/* standalone aggregation of an arbitrary symmetric CSR matrix (for pins) */
int orc_aggregate_csr(int n, const int *rp, const int *ci, const double *v, double theta, int *agg,
                      unsigned char *roots, int *nagg)
{
    csr_t a = {n, n, (int *)rp, (int *)ci, (double *)v};
    return aggregate(&a, theta * theta, agg, nagg, roots);
}

int orc_vcycle(void *h, int l, const double *b, double *x)
{
    orc_t *o = h;
    if (!o->setup_done || l < 0 || l >= o->Ls) return ORC_NOT_SETUP;
    return vcycle(o, l, b, x);
}

/* the level-l smoother alone: x <- x after the nsteps polynomial steps for
 * A_l x = b (zero_init: start from x = 0, else from the x passed in) */
int orc_smooth(void *h, int l, const double *b, double *x, int zero_init)
{
    orc_t *o = h;
    if (!o->setup_done || l < 0 || l >= o->Ls) return ORC_NOT_SETUP;
    int n = o->A[l].rows;
    double *d = xcalloc((size_t)n, sizeof(double)), *r = xcalloc((size_t)n, sizeof(double));
    if (!d || !r) return ORC_OOM;
    smooth(o, l, b, x, zero_init, d, r);
    free(d);
    free(r);
    return ORC_OK;
}

int orc_state_solve(void *h, int l, double tol, const double *f, double *y, long *iters)
{
    orc_t *o = h;
    if (!o->setup_done || l < 0 || l >= o->Ls) return ORC_NOT_SETUP;
    long before = o->inner_iters;
    int st = state_solve(o, l, f, y, tol);
    if (iters) *iters = o->inner_iters - before;
    return st;
}

int orc_mass_solve(void *h, int l, const double *b, double *x, long *iters)
{
    orc_t *o = h;
    if (!o->setup_done || l < 0 || l >= o->Lc) return ORC_NOT_SETUP;
    long before = o->mass_iters;
    int st = mass_solve(o, l, b, x);
    if (iters) *iters = o->mass_iters - before;
    return st;
}

int orc_hessian(void *h, int l, const double *u, double *hu)
{
    orc_t *o = h;
    if (!o->setup_done || l < 0 || l >= o->ell) return ORC_NOT_SETUP;
    return hessian(o, l, u, hu);
}

int orc_mlas(void *h, int which, int l, const double *b, double *u)
{
    orc_t *o = h;
    if (!o->setup_done || l < 0 || l >= o->ell) return ORC_NOT_SETUP;
    if (which == 0) return mlas_Q(o, l, b, u);
    if (l >= o->ell - 1) return ORC_INVALID;
    return mlas_R(o, l, b, u);
}

/* b = M_yu^T A^-1 M_y y_d (right side of Eq. firstorderpractice) */
int orc_rhs(void *h, double *b)
{
    orc_t *o = h;
    if (!o->setup_done) return ORC_NOT_SETUP;
    int m = o->m;
    double *t = xcalloc((size_t)m, sizeof(double)), *p = xcalloc((size_t)m, sizeof(double));
    spmv(&o->My[0], o->yd_state, t);
    int st = state_solve(o, 0, t, p, o->inner_tol);
    if (!st) spmv(&o->Myut[0], p, b);
    free(t);
    free(p);
    return st;
}

/* state y = A^-1 M_yu u and reduced cost J(u) = 1/2 (y-y_d)^T M_y (y-y_d)
 * + beta/2 u^T M_u u (Eq. functional); gradient M_yu^T A^-1 M_y (y - y_d)
 * + beta M_u u */
int orc_objective(void *h, const double *u, double *y, double *J, double *grad)
{
    orc_t *o = h;
    if (!o->setup_done) return ORC_NOT_SETUP;
    int m = o->m, n = o->n;
    double *t = xcalloc((size_t)m, sizeof(double)), *e = xcalloc((size_t)m, sizeof(double));
    double *me = xcalloc((size_t)m, sizeof(double)), *p = xcalloc((size_t)m, sizeof(double));
    double *mu = xcalloc((size_t)n, sizeof(double));
    spmv(&o->Myu[0], u, t);
    int st = state_solve(o, 0, t, y, o->inner_tol);
    if (st) goto done;
    for (int i = 0; i < m; i++) e[i] = y[i] - o->yd_state[i];
    spmv(&o->My[0], e, me);
    spmv(&o->Mu[0], u, mu);
    *J = 0.5 * dot(m, e, me) + 0.5 * o->beta * dot(n, u, mu);
    if (grad) {
        if ((st = state_solve(o, 0, me, p, o->inner_tol))) goto done;
        spmv(&o->Myut[0], p, grad);
        for (int i = 0; i < n; i++) grad[i] = grad[i] + o->beta * mu[i];
    }
done:
    free(t);
    free(e);
    free(me);
    free(p);
    free(mu);
    return st;
}

static int op_H0(orc_t *o, int l, const double *x, double *y) { return hessian(o, l, x, y); }
static int prec_Q0(orc_t *o, int l, const double *x, double *y) { return mlas_Q(o, l, x, y); }
static int prec_I(orc_t *o, int l, const double *x, double *y)
{
    memcpy(y, x, sizeof(double) * (size_t)o->Mu[l].rows);
    return ORC_OK;
}

/*
 * Outer CG on (K^T M_y K + beta M_u) u = K^T M_y y_d (Eq. firstorderpractice),
 * preconditioned by Q_0 (precond = 1) or the identity (precond = 0), to
 * ||b - H u_k|| <= tol ||b|| (Sec. 5.3).  u0 is not supported (start at 0).
 */
int orc_solve(void *h, int precond, double tol, int maxit, double *u, double *y, int *outer,
              double *relres, long *happlies)
{
    orc_t *o = h;
    if (!o->setup_done) return ORC_NOT_SETUP;
    int n = o->n;
    double *b = xcalloc((size_t)n, sizeof(double));
    int st = orc_rhs(o, b);
    if (st) { free(b); return st; }
    o->happlies = 0;
    long it = 0;
    st = pcg(o, 0, n, op_H0, precond ? prec_Q0 : prec_I, b, u, tol, maxit, &it, relres);
    if (outer) *outer = (int)it;
    if (happlies) *happlies = o->happlies;
    if (!st && y) {
        double *t = xcalloc((size_t)o->m, sizeof(double));
        spmv(&o->Myu[0], u, t);
        st = state_solve(o, 0, t, y, o->inner_tol);
        free(t);
    }
    free(b);
    return st;
}

/* threads the row loops use (1 in the sequential build) */
int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* set the threads of the row loops (no effect in the sequential build) */
int orc_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
    return ORC_OK;
}

int orc_counters(void *h, long *inner, long *mass, long *happ)
{
    orc_t *o = h;
    *inner = o->inner_iters;
    *mass = o->mass_iters;
    *happ = o->happlies;
    return ORC_OK;
}

void orc_destroy(void *h)
{
    orc_t *o = h;
    if (!o) return;
    free_hierarchy(o);
    csr_free(&o->Kfull);
    csr_free(&o->Mfull);
    free(o->coords);
    free(o->elems);
    free(o->dir);
    free(o->kappa);
    free(o->yd_state);
    free(o->state_of_vertex);
    free(o);
}
