// api.cu -- the C ABI declared in include/amgh.h.
#include <math.h>
#include <string.h>

#include <chrono>
#include <new>

#include "internal.cuh"
#include "util.cuh"

static void zero_counters(amgh_problem *p);

static double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

extern "C" void amgh_amg_opts_default(amgh_amg_opts *o)
{
    if (!o) return;
    o->max_levels = 25;
    o->hessian_levels = 0;
    o->theta = 0.08;
    o->coarse_max = 256;
    o->smoother = 1;
    o->smooth_degree = 2;
    o->precision = 0;
    o->smooth_prolongator = 1;
    o->coarse_solve = 0;
    o->fuse_coarse = 0;
    o->autotune = 0;
    o->aggressive = 0;
    o->geometric = 0;
    o->matrix_free = 0;
    o->persistent_cg = 0;
}

extern "C" void amgh_solve_opts_default(amgh_solve_opts *o)
{
    if (!o) return;
    o->tol = 1e-8;
    o->max_iter = 200;
    o->inner_tol = 1e-10;
    o->mass_tol = 1e-10;
    o->precond = 1;
    o->ncols = 1;
    o->inner_max_iter = 1000;
    o->mass_max_iter = 1000;
    o->precond_tol = 0.0;
    o->coarse_tol = 1e-4;
    o->coarse_max_iter = 1000;
    o->level_fallback = 0;
}

extern "C" const char *amgh_status_string(int s)
{
    switch (s) {
    case AMGH_OK: return "ok";
    case AMGH_ERR_INVALID_ARG: return "invalid argument";
    case AMGH_ERR_NOT_SETUP: return "amg setup has not run";
    case AMGH_ERR_CUDA: return "CUDA error";
    case AMGH_ERR_OOM: return "out of memory";
    case AMGH_ERR_NOT_CONVERGED: return "not converged";
    case AMGH_ERR_INDEFINITE: return "indefinite operator or preconditioner";
    case AMGH_ERR_NUMERIC: return "NaN or Inf in a residual";
    case AMGH_ERR_TIMEOUT: return "bounded wait ran out";
    }
    return "unknown status";
}

static int copy_in(void *dst, const void *src, size_t bytes, int on_device, cudaStream_t s)
{
    CU(cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    return AMGH_OK;
}

__global__ void k_gather_state(int m, const int *__restrict__ vos, const double *__restrict__ full,
                               double *__restrict__ st)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) st[i] = full[vos[i]];
}

static int load_yd(amgh_problem *p, const double *y_d, int on_device)
{
    Scratch sc;
    double *full = nullptr;
    TRY(sc.alloc(&full, p->nv));
    if (y_d) TRY(copy_in(full, y_d, sizeof(double) * p->nv, on_device, p->stream));
    else CU(cudaMemsetAsync(full, 0, sizeof(double) * p->nv, p->stream));
    if (p->m > 0) {
        k_gather_state<<<ceil_div(p->m, 256), 256, 0, p->stream>>>(p->m, p->vertex_of_state, full, p->yd_state);
        LAUNCH_CHECK();
    }
    CU(cudaStreamSynchronize(p->stream));
    return AMGH_OK;
}

static int create_impl(const amgh_mesh *mesh, const double *kappa, double beta, const double *y_d, int yd_dev,
                       amgh_problem *p)
{
    p->dim = mesh->dim;
    p->nv = mesh->n_vertices;
    p->ne = mesh->n_elements;
    p->beta = beta;
    amgh_amg_opts_default(&p->aopts);
    amgh_solve_opts_default(&p->sopts);
    p->sopts.precond_tol = p->sopts.inner_tol;
    CU(cudaHostAlloc((void **)&p->h_scal, sizeof(CgScal), cudaHostAllocDefault));
    CU(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
    int d1 = p->dim + 1;
    Arena &ar = p->arena;
    TRY(ar.alloc(&p->coords, p->nv * p->dim));
    TRY(ar.alloc(&p->elems, p->ne * d1));
    TRY(ar.alloc(&p->dir, p->nv));
    TRY(ar.alloc(&p->kappa, p->ne));
    int od = mesh->on_device;
    TRY(copy_in(p->coords, mesh->coords, sizeof(double) * p->nv * p->dim, od, p->stream));
    TRY(copy_in(p->elems, mesh->elements, sizeof(int) * p->ne * d1, od, p->stream));
    TRY(copy_in(p->dir, mesh->dirichlet, p->nv, od, p->stream));
    TRY(copy_in(p->kappa, kappa, sizeof(double) * p->ne, od, p->stream));
    CU(cudaStreamSynchronize(p->stream));
    TRY(assemble_full(p));
    TRY(ar.alloc(&p->yd_state, p->m));
    TRY(load_yd(p, y_d, yd_dev));
    return AMGH_OK;
}

extern "C" int amgh_problem_create(const amgh_mesh *mesh, const double *kappa, double beta, const double *y_d,
                                   int y_d_on_device, amgh_problem **out)
{
    if (!out) return AMGH_ERR_INVALID_ARG;
    *out = nullptr;
    if (!mesh || !kappa || !mesh->coords || !mesh->elements || !mesh->dirichlet) return AMGH_ERR_INVALID_ARG;
    if ((mesh->dim != 2 && mesh->dim != 3) || mesh->n_vertices <= 0 || mesh->n_elements <= 0) return AMGH_ERR_INVALID_ARG;
    if (mesh->n_vertices >= (int64_t)1 << 31 || mesh->n_elements * (mesh->dim + 1) >= ((int64_t)1 << 31))
        return AMGH_ERR_INVALID_ARG;
    if (!(beta > 0.0) || isinf(beta)) return AMGH_ERR_INVALID_ARG;
    amgh_problem *p = new (std::nothrow) amgh_problem();
    if (!p) return AMGH_ERR_OOM;
    zero_counters(p);
    int st = create_impl(mesh, kappa, beta, y_d, y_d_on_device, p);
    if (st) {
        amgh_problem_destroy(p);
        return st;
    }
    *out = p;
    return AMGH_OK;
}

extern "C" int amgh_problem_share(amgh_problem *parent, amgh_problem **out)
{
    if (!out) return AMGH_ERR_INVALID_ARG;
    *out = nullptr;
    if (!parent) return AMGH_ERR_INVALID_ARG;
    if (!parent->setup_done) return AMGH_ERR_NOT_SETUP;
    if (parent->parent) parent = (amgh_problem *)parent->parent;
    amgh_problem *p = new (std::nothrow) amgh_problem();
    if (!p) return AMGH_ERR_OOM;
    zero_counters(p);
    p->parent = parent;
    p->dim = parent->dim;
    p->nv = parent->nv;
    p->ne = parent->ne;
    p->beta = parent->beta;
    p->m = parent->m;
    p->n = parent->n;
    p->stream = parent->stream;
    p->df_spmv = parent->df_spmv;
    p->coords = parent->coords;
    p->kappa = parent->kappa;
    p->elems = parent->elems;
    p->dir = parent->dir;
    p->state_of_vertex = parent->state_of_vertex;
    p->vertex_of_state = parent->vertex_of_state;
    p->Kfull = parent->Kfull;
    p->Mfull = parent->Mfull;
    p->aopts = parent->aopts;
    p->sopts = parent->sopts;
    p->Ls = parent->Ls;
    p->Lc = parent->Lc;
    p->ell = parent->ell;
    p->coarse_cg = parent->coarse_cg;
    for (int l = 0; l < AMGH_MAXL; l++) {
        p->sl[l] = parent->sl[l];
        p->cl[l] = parent->cl[l];
        for (CgGraph &g : p->sl[l].graph) g = CgGraph();
        p->cl[l].mgraph = CgGraph();
        p->chunk_hint[l] = parent->chunk_hint[l];
        p->chunk_hint32[l] = parent->chunk_hint32[l];
        p->mchunk_hint[l] = parent->mchunk_hint[l];
    }
    p->Acoarse = parent->Acoarse;
    p->Aell = parent->Aell;
    p->Hcoarse = parent->Hcoarse;
    p->nsteps = parent->nsteps;
    for (int k = 0; k < 16; k++) {
        p->cd[k] = parent->cd[k];
        p->cr[k] = parent->cr[k];
    }
    p->t_setup = parent->t_setup;
    p->kuhn_checked = parent->kuhn_checked;
    p->kuhn_N = parent->kuhn_N;
    p->kappa32 = parent->kappa32;
    int st = AMGH_OK;
    {
        StreamScope ss_(p->stream);
        if (cudaHostAlloc((void **)&p->h_scal, sizeof(CgScal), cudaHostAllocDefault) != cudaSuccess ||
            cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
            st = AMGH_ERR_CUDA;
        if (!st) st = p->arena.alloc(&p->yd_state, p->m);
        if (!st && p->m > 0 &&
            cudaMemcpyAsync(p->yd_state, parent->yd_state, sizeof(double) * p->m, cudaMemcpyDeviceToDevice,
                            p->stream) != cudaSuccess)
            st = AMGH_ERR_CUDA;
        if (!st) st = solver_alloc(p);
        if (!st) st = fused_setup(p); // its own table: it names this handle's vectors
        if (!st && cudaStreamSynchronize(p->stream) != cudaSuccess) st = AMGH_ERR_CUDA;
    }
    if (st) {
        amgh_problem_destroy(p);
        return st;
    }
    p->setup_done = 1;
    *out = p;
    return AMGH_OK;
}

extern "C" int amgh_set_yd(amgh_problem *p, const double *y_d, int on_device)
{
    if (!p || !y_d) return AMGH_ERR_INVALID_ARG;
    StreamScope ss_(p->stream);
    return load_yd(p, y_d, on_device);
}

extern "C" int amgh_set_stream(amgh_problem *p, void *stream)
{
    if (!p) return AMGH_ERR_INVALID_ARG;
    p->stream = (cudaStream_t)stream;
    return AMGH_OK;
}

extern "C" int amgh_set_solve_opts(amgh_problem *p, const amgh_solve_opts *o)
{
    if (!p || !o) return AMGH_ERR_INVALID_ARG;
    if (!(o->inner_tol > 0.0) || !(o->mass_tol > 0.0) || o->inner_max_iter < 1 || o->mass_max_iter < 1 ||
        !(o->precond_tol >= 0.0) || !(o->coarse_tol > 0.0) || o->coarse_max_iter < 1)
        return AMGH_ERR_INVALID_ARG;
    p->sopts.inner_tol = o->inner_tol;
    p->sopts.precond_tol = o->precond_tol > 0.0 ? o->precond_tol : o->inner_tol;
    p->sopts.mass_tol = o->mass_tol;
    p->sopts.inner_max_iter = o->inner_max_iter;
    p->sopts.mass_max_iter = o->mass_max_iter;
    p->sopts.coarse_tol = o->coarse_tol;
    p->sopts.coarse_max_iter = o->coarse_max_iter;
    return AMGH_OK;
}

// ------------------------------------------------------------------ setup
static void reset_hierarchy(amgh_problem *p)
{
    block_free(p);
    solver_free_graphs(p);
    p->harena.free_all();
    for (int l = 0; l < AMGH_MAXL; l++) {
        p->sl[l] = StateLevel();
        p->cl[l] = CtrlLevel();
    }
    p->Acoarse = Dense();
    p->Aell = Dense();
    p->Hcoarse = Dense();
    p->Ls = p->Lc = p->ell = 0;
    p->setup_done = 0;
}

static void smoother_coeffs(amgh_problem *p)
{
    const amgh_amg_opts &o = p->aopts;
    p->nsteps = o.smooth_degree;
    if (o.smoother == 0) {
        for (int s = 0; s < p->nsteps; s++) {
            p->cd[s] = 0.0;
            p->cr[s] = 1.0;
        }
        return;
    }
    // Chebyshev on [1/30, 1] for D_l1^-1 A (Saad, Iterative Methods, Alg. 12.1)
    double lo = 1.0 / 30.0, hi = 1.0;
    double theta = (hi + lo) / 2.0, delta = (hi - lo) / 2.0, sigma = theta / delta;
    double rho = 1.0 / sigma;
    p->cd[0] = 0.0;
    p->cr[0] = 1.0 / theta;
    for (int s = 1; s < p->nsteps; s++) {
        double rn = 1.0 / (2.0 * sigma - rho);
        p->cd[s] = rn * rho;
        p->cr[s] = 2.0 * rn / delta;
        rho = rn;
    }
}

static int dense_inverse_of(amgh_problem *p, const DevCsr &a, Dense &out)
{
    if (a.rows > AMGH_DENSE_MAX) {
        amgh_note_msg("coarsest AMG level has more than 4096 rows (coarsening stalled): no dense inverse");
        return AMGH_ERR_INVALID_ARG;
    }
    int n = a.rows;
    Scratch sc;
    double *g = nullptr;
    int *info = nullptr;
    TRY(sc.alloc(&g, (int64_t)n * n));
    TRY(sc.alloc(&info, 1));
    TRY(p->harena.alloc(&out.inv, (int64_t)n * n));
    out.n = n;
    TRY(dense_from_csr(p, a, g));
    return dense_spd_inverse(p, g, n, out.inv, info);
}

// Make level ell-1 the coarsest level of the Hessian preconditioner: with the
// exact coarse solve, H_{ell-1} is formed densely (Eq. firstorderpractice on
// that level) and inverted.  Memory of an earlier coarse level stays in the
// arena until the next setup.
static int coarse_hessian_setup(amgh_problem *p, int ell)
{
    int c = ell - 1;
    p->Hcoarse = Dense();
    int mode = p->aopts.coarse_solve;
    if (mode == 2) mode = p->cl[c].Mu.rows <= AMGH_DENSE_MAX ? 0 : 1;
    p->coarse_cg = mode == 1;
    if (mode == 0) {
        if (p->cl[c].Mu.rows > AMGH_DENSE_MAX) {
            amgh_note_msg("coarsest Hessian level has more than 4096 controls: use coarse_solve 1 or 2");
            return AMGH_ERR_INVALID_ARG;
        }
        const double *ainv = p->Acoarse.inv;
        if (c != p->Ls - 1) {
            TRY(dense_inverse_of(p, p->sl[c].A, p->Aell));
            ainv = p->Aell.inv;
        }
        int nc = p->cl[c].Mu.rows;
        TRY(p->harena.alloc(&p->Hcoarse.inv, (int64_t)nc * nc));
        p->Hcoarse.n = nc;
        TRY(dense_coarse_hessian(p, c, ainv, p->Hcoarse.inv));
    }
    p->ell = ell;
    return AMGH_OK;
}

static int setup_impl(amgh_problem *p)
{
    cudaStream_t s = p->stream;
    Arena &ar = p->harena;
    const amgh_amg_opts &o = p->aopts;
    if (o.matrix_free) {
        TRY(kuhn_detect(p));
        if (!p->kuhn_N) {
            amgh_note_msg("matrix_free: the mesh is not the structured Kuhn cube");
            return AMGH_ERR_INVALID_ARG;
        }
    }
    // level 0: state dofs = non-Dirichlet vertices, control dofs = all vertices
    StateLevel &S0 = p->sl[0];
    CtrlLevel &C0 = p->cl[0];
    TRY(extract_sub(ar, p->Kfull, p->state_of_vertex, p->m, p->state_of_vertex, p->m, S0.A, s));
    TRY(extract_sub(ar, p->Mfull, p->state_of_vertex, p->m, p->state_of_vertex, p->m, S0.My, s));
    TRY(extract_sub(ar, p->Mfull, p->state_of_vertex, p->m, nullptr, p->n, C0.Myu, s));
    TRY(extract_sub(ar, p->Kfull, nullptr, p->n, nullptr, p->n, C0.KN, s));
    TRY(extract_sub(ar, p->Mfull, nullptr, p->n, nullptr, p->n, C0.Mu, s));
    if (o.geometric) {
        TRY(geometric_hierarchy(p));
        goto hierarchies_done;
    }
    {
    // state hierarchy on A (theta halved per level)
    double th = o.theta;
    p->Ls = 1;
    for (int l = 0; l + 1 < o.max_levels && p->sl[l].A.rows > o.coarse_max; l++) {
        StateLevel &S = p->sl[l];
        int n = S.A.rows;
        TRY(ar.alloc(&S.agg, n));
        int nagg = 0;
        if (l == 0 && o.aggressive) TRY(amg_aggregate_aggressive(p, S.A, th * th, S.agg, &nagg));
        else TRY(amg_aggregate(p, S.A, th * th, S.agg, &nagg));
        if ((double)n < 1.2 * (double)nagg) break;
        S.nagg = nagg;
        TRY(amg_prolongator(p, ar, S.A, S.agg, nagg, o.smooth_prolongator, S.S));
        TRY(csr_transpose(ar, S.S, S.St, s));
        TRY(galerkin_pair(p, ar, S.St, S.A, S.My, S.S, p->sl[l + 1].A, p->sl[l + 1].My));
        p->Ls = l + 2;
        th = th * 0.5;
    }
    // control hierarchy on the all-vertex stiffness K_N
    th = o.theta;
    p->Lc = 1;
    for (int l = 0; l + 1 < o.max_levels && p->cl[l].KN.rows > o.coarse_max; l++) {
        CtrlLevel &C = p->cl[l];
        int n = C.KN.rows;
        TRY(ar.alloc(&C.agg, n));
        int nagg = 0;
        if (l == 0 && o.aggressive) TRY(amg_aggregate_aggressive(p, C.KN, th * th, C.agg, &nagg));
        else TRY(amg_aggregate(p, C.KN, th * th, C.agg, &nagg));
        if ((double)n < 1.2 * (double)nagg) break;
        C.nagg = nagg;
        TRY(amg_prolongator(p, ar, C.KN, C.agg, nagg, o.smooth_prolongator, C.P));
        TRY(csr_transpose(ar, C.P, C.Pt, s));
        TRY(galerkin_pair(p, ar, C.Pt, C.KN, C.Mu, C.P, p->cl[l + 1].KN, p->cl[l + 1].Mu));
        p->Lc = l + 2;
        th = th * 0.5;
    }
    }
hierarchies_done:
    int lmin = p->Ls < p->Lc ? p->Ls : p->Lc;
    for (int l = 0; l + 1 < lmin; l++)
        TRY(galerkin(p, ar, p->sl[l].St, p->cl[l].Myu, p->cl[l].P, 0, p->cl[l + 1].Myu));
    for (int l = 0; l < lmin; l++) TRY(csr_transpose(ar, p->cl[l].Myu, p->cl[l].Myut, s));
    // SELL copies of the operators applied in the solve phase, smoother and mass diagonals
    for (int l = 0; l < p->Ls; l++) {
        StateLevel &S = p->sl[l];
        TRY(prepare_tuned(p, ar, S.A, 1));
        TRY(build_lo_parts(ar, S.A, s));
        TRY(prepare_operator(ar, S.My, s));
        if (l + 1 < p->Ls) {
            TRY(prepare_operator(ar, S.S, s));
            TRY(prepare_operator(ar, S.St, s));
        }
        TRY(ar.alloc(&S.invd, S.A.rows));
        TRY(ar.alloc(&S.invd32, S.A.rows));
        TRY(l1_invdiag(p, S.A, S.invd, S.invd32));
    }
    for (int l = 0; l < p->Lc; l++) {
        CtrlLevel &C = p->cl[l];
        TRY(prepare_operator(ar, C.Mu, s));
        TRY(build_lo_parts(ar, C.Mu, s));
        if (l + 1 < p->Lc) {
            TRY(prepare_operator(ar, C.P, s));
            TRY(prepare_operator(ar, C.Pt, s));
        }
        if (l < lmin) {
            TRY(prepare_operator(ar, C.Myu, s));
            TRY(prepare_operator(ar, C.Myut, s));
        }
        TRY(ar.alloc(&C.mu_invdiag, C.Mu.rows));
        TRY(diag_inv(p, C.Mu, C.mu_invdiag));
        TRY(ar.alloc(&C.mu_invdiag32, C.Mu.rows));
        TRY(to_f32(p, C.mu_invdiag, C.Mu.rows, C.mu_invdiag32));
    }
    // exact coarsest state solve, then the coarsest Hessian level
    TRY(dense_inverse_of(p, p->sl[p->Ls - 1].A, p->Acoarse));
    TRY(dense_make32(p, p->harena, p->Acoarse));
    int ell = lmin;
    if (o.hessian_levels > 0 && o.hessian_levels < ell) ell = o.hessian_levels;
    TRY(coarse_hessian_setup(p, ell));
    smoother_coeffs(p);
    TRY(solver_alloc(p));
    TRY(fused_setup(p));
    CU(cudaStreamSynchronize(s));
    return AMGH_OK;
}

extern "C" int amgh_amg_setup(amgh_problem *p, const amgh_amg_opts *opts)
{
    if (!p || p->parent) return AMGH_ERR_INVALID_ARG;
    amgh_amg_opts o;
    if (opts) o = *opts;
    else amgh_amg_opts_default(&o);
    if (o.max_levels < 1 || o.max_levels > AMGH_MAXL || o.smooth_degree < 1 || o.smooth_degree > 16 ||
        o.coarse_max < 1 || !(o.theta >= 0.0) || (o.smoother != 0 && o.smoother != 1) ||
        o.precision < 0 || o.precision > 2 || o.hessian_levels < 0 || o.coarse_solve < 0 || o.coarse_solve > 2 || (o.fuse_coarse < 0 || o.fuse_coarse > 2) ||
        (o.autotune != 0 && o.autotune != 1) || (o.aggressive != 0 && o.aggressive != 1) ||
        (o.geometric != 0 && o.geometric != 1) || (o.matrix_free != 0 && o.matrix_free != 1) ||
        (o.persistent_cg != 0 && o.persistent_cg != 1))
        return AMGH_ERR_INVALID_ARG;
    double t0 = now_s();
    StreamScope ss_(p->stream);
    amgh_note_msg("");
    reset_hierarchy(p);
    p->aopts = o;
    int st = setup_impl(p);
    if (st) {
        reset_hierarchy(p);
        return st;
    }
    p->setup_done = 1;
    p->t_setup = now_s() - t0;
    return AMGH_OK;
}

// ------------------------------------------------------------------ applies
// Every solve-phase entry point works on the problem's stream and counts its
// kernels' algorithmic bytes into the problem's counter.
struct CallScope {
    StreamScope ss;
    ByteSink bs;
    explicit CallScope(amgh_problem *p) : ss(p->stream), bs(&p->c_bytes) {}
};

#define NEED_SETUP(p)                          \
    do {                                       \
        if (!(p)) return AMGH_ERR_INVALID_ARG; \
        if (!(p)->setup_done) return AMGH_ERR_NOT_SETUP; \
    } while (0)

// End of a solve-phase entry point: wait for the stream, then report a staged
// copy that timed out in place of any other status, since it invalidates every
// value the call produced.
static int finish_call(amgh_problem *p, int st)
{
    int s2 = sync_stream(p);
    int s3 = s2 == AMGH_OK ? bulk_timeout_check(p->stream) : s2;
    int s4 = s2 == AMGH_OK ? grid_timeout_check(p) : s2;
    int s5 = s2 == AMGH_OK ? block_grid_timeout_check(p) : s2;
    if (s3 == AMGH_ERR_TIMEOUT || s4 == AMGH_ERR_TIMEOUT || s5 == AMGH_ERR_TIMEOUT) return AMGH_ERR_TIMEOUT;
    if (s4 == AMGH_OK) s4 = s5;
    if (s3 == AMGH_OK) s3 = s4;
    return st != AMGH_OK ? st : s3;
}

extern "C" int amgh_hessian_apply(amgh_problem *p, const double *u, double *hu, int ncols)
{
    NEED_SETUP(p);
    CallScope cs_(p);
    if (!u || !hu || ncols < 1) return AMGH_ERR_INVALID_ARG;
    int st = ncols > 1 ? block_hessian_apply(p, u, hu, ncols) : hessian_level(p, 0, u, hu);
    if (st == AMGH_OK) st = timer_collect(p);
    return finish_call(p, st);
}

extern "C" int amgh_precond_apply(amgh_problem *p, const double *r, double *z, int ncols)
{
    NEED_SETUP(p);
    CallScope cs_(p);
    if (!r || !z || ncols < 1) return AMGH_ERR_INVALID_ARG;
    int st = ncols > 1 ? block_precond_apply(p, r, z, ncols) : mlas_Q(p, 0, r, z);
    if (st == AMGH_OK) st = timer_collect(p);
    return finish_call(p, st);
}

extern "C" int amgh_rhs(amgh_problem *p, double *b)
{
    NEED_SETUP(p);
    CallScope cs_(p);
    if (!b) return AMGH_ERR_INVALID_ARG;
    return finish_call(p, rhs_apply(p, b));
}

static void fill_info(amgh_problem *p, amgh_solve_info *info)
{
    info->hessian_applies = p->c_happ;
    info->inner_iters = p->c_inner;
    info->mass_iters = p->c_mass;
    info->refinements = p->c_refine;
    info->t_setup_s = p->t_setup;
    info->hessian_levels = p->ell;
    info->coarse_iters = p->c_coarse;
    info->alg_bytes = p->c_bytes;
}

extern "C" int amgh_solve(amgh_problem *p, const double *u0, double *u, double *y, const amgh_solve_opts *opts,
                          amgh_solve_info *info)
{
    NEED_SETUP(p);
    CallScope cs_(p);
    if (!u) return AMGH_ERR_INVALID_ARG;
    amgh_solve_opts o;
    if (opts) o = *opts;
    else amgh_solve_opts_default(&o);
    if (!(o.tol > 0.0) || o.max_iter < 1 || o.ncols != 1) return AMGH_ERR_INVALID_ARG;
    TRY(amgh_set_solve_opts(p, &o));
    zero_counters(p);
    amgh_solve_info loc;
    memset(&loc, 0, sizeof(loc));
    int st = outer_solve(p, u0, u, &o, &loc);
    int fallbacks = 0;
    // an indefinite multilevel preconditioner: one Hessian level fewer, restart
    while (st == AMGH_ERR_INDEFINITE && o.level_fallback && o.precond && p->ell > 2) {
        if (p->aopts.coarse_solve == 0 && p->cl[p->ell - 2].Mu.rows > AMGH_DENSE_MAX) break;
        int s2 = coarse_hessian_setup(p, p->ell - 1);
        if (s2) {
            st = s2;
            break;
        }
        fallbacks++;
        st = outer_solve(p, u0, u, &o, &loc);
    }
    if (st == AMGH_OK && y) {
        CtrlLevel &C = p->cl[0];
        int s2 = spmv(p, C.Myu, u, C.t1, nullptr, KC_SPMV);
        if (s2 == AMGH_OK) s2 = state_solve(p, 0, C.t1, y, p->sopts.inner_tol, nullptr);
        st = s2;
    }
    fill_info(p, &loc);
    loc.status = st;
    loc.fallbacks = fallbacks;
    if (info) *info = loc;
    int st2 = timer_collect(p);
    if (st == AMGH_OK) st = st2;
    return finish_call(p, st);
}

extern "C" int amgh_solve_block(amgh_problem *p, const double *yd, int ncols, double *u,
                                const amgh_solve_opts *opts, amgh_solve_info *info)
{
    NEED_SETUP(p);
    CallScope cs_(p);
    if (!yd || !u || ncols < 1) return AMGH_ERR_INVALID_ARG;
    amgh_solve_opts o;
    if (opts) o = *opts;
    else amgh_solve_opts_default(&o);
    if (!(o.tol > 0.0) || o.max_iter < 1 || o.ncols != 1) return AMGH_ERR_INVALID_ARG;
    TRY(amgh_set_solve_opts(p, &o));
    zero_counters(p);
    double t0 = now_s();
    amgh_solve_info loc;
    memset(&loc, 0, sizeof(loc));
    int st = block_solve(p, yd, ncols, u, o, &loc);
    int fallbacks = 0;
    // as amgh_solve: an indefinite preconditioner drops the coarsest Hessian
    // level and the whole block restarts from u = 0
    while (st == AMGH_ERR_INDEFINITE && o.level_fallback && o.precond && p->ell > 2) {
        if (p->aopts.coarse_solve == 0 && p->cl[p->ell - 2].Mu.rows > AMGH_DENSE_MAX) break;
        int s2 = coarse_hessian_setup(p, p->ell - 1);
        if (s2) {
            st = s2;
            break;
        }
        fallbacks++;
        memset(&loc, 0, sizeof(loc));
        st = block_solve(p, yd, ncols, u, o, &loc);
    }
    fill_info(p, &loc);
    loc.status = st;
    loc.fallbacks = fallbacks;
    loc.t_solve_s = now_s() - t0;
    if (info) *info = loc;
    return finish_call(p, st);
}

extern "C" int amgh_solve_host(amgh_problem *p, const double *u0_host, double *u_host, double *y_host,
                               const amgh_solve_opts *opts, amgh_solve_info *info)
{
    NEED_SETUP(p);
    CallScope cs_(p);
    if (!u_host) return AMGH_ERR_INVALID_ARG;
    Scratch sc;
    double *u0 = nullptr, *u = nullptr, *y = nullptr;
    TRY(sc.alloc(&u, p->n));
    if (u0_host) {
        TRY(sc.alloc(&u0, p->n));
        CU(cudaMemcpyAsync(u0, u0_host, sizeof(double) * p->n, cudaMemcpyHostToDevice, p->stream));
    }
    if (y_host) TRY(sc.alloc(&y, p->m));
    int st = amgh_solve(p, u0, u, y, opts, info);
    if (st) return st;
    CU(cudaMemcpyAsync(u_host, u, sizeof(double) * p->n, cudaMemcpyDeviceToHost, p->stream));
    if (y_host) CU(cudaMemcpyAsync(y_host, y, sizeof(double) * p->m, cudaMemcpyDeviceToHost, p->stream));
    return sync_stream(p);
}

__global__ void k_sub(int n, const double *__restrict__ a, const double *__restrict__ b, double *__restrict__ c)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) c[i] = a[i] - b[i];
}

extern "C" int amgh_state_solve(amgh_problem *p, const double *u, double *y, double *J)
{
    NEED_SETUP(p);
    CallScope cs_(p);
    if (!u || !y) return AMGH_ERR_INVALID_ARG;
    CtrlLevel &C = p->cl[0];
    StateLevel &S = p->sl[0];
    TRY(spmv(p, C.Myu, u, C.t1, nullptr, KC_SPMV));
    int st = state_solve(p, 0, C.t1, y, p->sopts.inner_tol, nullptr);
    if (st != AMGH_OK) return finish_call(p, st);
    if (J) {
        int m = p->m, n = p->n;
        k_sub<<<ceil_div(m, 256), 256, 0, p->stream>>>(m, y, p->yd_state, C.t1);
        LAUNCH_CHECK();
        TRY(spmv(p, S.My, C.t1, C.t2, nullptr, KC_SPMV));
        TRY(spmv(p, C.Mu, u, p->oq, nullptr, KC_SPMV));
        TRY(vec_dot(p, p->ored, m, C.t1, C.t2, p->dscratch));
        TRY(vec_dot(p, p->ored, n, u, p->oq, p->dscratch + 1));
        double h[2];
        CU(cudaMemcpyAsync(h, p->dscratch, 2 * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
        CU(cudaStreamSynchronize(p->stream));
        *J = 0.5 * h[0] + 0.5 * p->beta * h[1];
    }
    return finish_call(p, AMGH_OK);
}

extern "C" int amgh_gradient(amgh_problem *p, const double *u, const double *y, double *g)
{
    NEED_SETUP(p);
    CallScope cs_(p);
    if (!u || !y || !g) return AMGH_ERR_INVALID_ARG;
    CtrlLevel &C = p->cl[0];
    StateLevel &S = p->sl[0];
    int m = p->m;
    k_sub<<<ceil_div(m, 256), 256, 0, p->stream>>>(m, y, p->yd_state, C.t1);
    LAUNCH_CHECK();
    TRY(spmv(p, S.My, C.t1, C.t2, nullptr, KC_SPMV));
    int st = state_solve(p, 0, C.t2, C.ps, p->sopts.inner_tol, nullptr);
    if (st == AMGH_OK) st = spmv2(p, C.Myut, C.ps, C.Mu, u, p->beta, g, nullptr);
    return finish_call(p, st);
}

extern "C" int amgh_state_adjoint(amgh_problem *p, const double *w, double *g)
{
    NEED_SETUP(p);
    CallScope cs_(p);
    if (!w || !g) return AMGH_ERR_INVALID_ARG;
    CtrlLevel &C = p->cl[0];
    // A is symmetric, so A^-T w is one more AMG-CG solve
    int st = state_solve(p, 0, w, C.ps, p->sopts.inner_tol, nullptr);
    if (st == AMGH_OK) st = spmv(p, C.Myut, C.ps, g, nullptr, KC_SPMV);
    return finish_call(p, st);
}

// ------------------------------------------------------------------ level-wise
extern "C" int amgh_vcycle(amgh_problem *p, int level, const double *b, double *x)
{
    NEED_SETUP(p);
    CallScope cs_(p);
    if (level < 0 || level >= p->Ls || !b || !x) return AMGH_ERR_INVALID_ARG;
    return finish_call(p, vcycle_run(p, level, 0, b, x, nullptr));
}

extern "C" int amgh_state_solve_level(amgh_problem *p, int level, const double *f, double *y, double tol,
                                      int64_t *iters)
{
    NEED_SETUP(p);
    CallScope cs_(p);
    if (level < 0 || level >= p->Ls || !f || !y || !(tol > 0.0)) return AMGH_ERR_INVALID_ARG;
    return finish_call(p, state_solve(p, level, f, y, tol, iters));
}

extern "C" int amgh_mass_solve(amgh_problem *p, int level, const double *b, double *x, int64_t *iters)
{
    NEED_SETUP(p);
    CallScope cs_(p);
    if (level < 0 || level >= p->Lc || !b || !x) return AMGH_ERR_INVALID_ARG;
    TRY(mass_solve(p, level, b, x, iters));
    return sync_stream(p);
}

extern "C" int amgh_hessian_apply_level(amgh_problem *p, int level, const double *v, double *hv)
{
    NEED_SETUP(p);
    CallScope cs_(p);
    if (level < 0 || level >= p->ell || !v || !hv) return AMGH_ERR_INVALID_ARG;
    return finish_call(p, hessian_level(p, level, v, hv));
}

extern "C" int amgh_precond_apply_level(amgh_problem *p, int which, int level, const double *b, double *z)
{
    NEED_SETUP(p);
    CallScope cs_(p);
    if (level < 0 || level >= p->ell || !b || !z) return AMGH_ERR_INVALID_ARG;
    if (which != 0 && level >= p->ell - 1) return AMGH_ERR_INVALID_ARG;
    return finish_call(p, which == 0 ? mlas_Q(p, level, b, z) : mlas_R(p, level, b, z));
}

// ------------------------------------------------------------------ matrix-free
extern "C" int amgh_kuhn_apply(amgh_problem *p, int prec32, const void *x, void *y)
{
    if (!p || !x || !y || (prec32 != 0 && prec32 != 1)) return AMGH_ERR_INVALID_ARG;
    CallScope cs_(p);
    TRY(kuhn_detect(p));
    if (!p->kuhn_N) {
        amgh_note_msg("amgh_kuhn_apply: the mesh is not the structured Kuhn cube");
        return AMGH_ERR_INVALID_ARG;
    }
    return finish_call(p, kuhn_apply(p, prec32, x, y));
}

// ------------------------------------------------------------------ diagnostics
extern "C" int amgh_aj_estimate(amgh_problem *p, int level, int weighted, int iters, const double *v0,
                                double *est)
{
    NEED_SETUP(p);
    CallScope cs_(p);
    int lmin = p->Ls < p->Lc ? p->Ls : p->Lc;
    if (level < 0 || level + 1 >= lmin || iters < 1 || !v0 || !est || (weighted != 0 && weighted != 1))
        return AMGH_ERR_INVALID_ARG;
    return finish_call(p, aj_estimate(p, level, weighted, iters, v0, est));
}

// ------------------------------------------------------------------ queries
extern "C" int amgh_query_sizes(const amgh_problem *p, int64_t *m, int64_t *n, int *Ls, int *Lc, int *ell,
                                int64_t *ssz, int64_t *csz)
{
    if (!p) return AMGH_ERR_INVALID_ARG;
    if (m) *m = p->m;
    if (n) *n = p->n;
    if (Ls) *Ls = p->Ls;
    if (Lc) *Lc = p->Lc;
    if (ell) *ell = p->ell;
    for (int l = 0; l < p->Ls && ssz; l++) ssz[l] = p->sl[l].A.rows;
    for (int l = 0; l < p->Lc && csz; l++) csz[l] = p->cl[l].Mu.rows;
    return AMGH_OK;
}

extern "C" int amgh_get_aggregates(const amgh_problem *p, int hier, int level, int32_t *agg, int32_t *nagg)
{
    if (!p || !agg) return AMGH_ERR_INVALID_ARG;
    if (!p->setup_done) return AMGH_ERR_NOT_SETUP;
    int L = hier ? p->Lc : p->Ls;
    if (level < 0 || level + 1 >= L || p->aopts.geometric) return AMGH_ERR_INVALID_ARG;
    const int *src = hier ? p->cl[level].agg : p->sl[level].agg;
    int rows = hier ? p->cl[level].Mu.rows : p->sl[level].A.rows;
    CU(cudaMemcpyAsync(agg, src, sizeof(int) * rows, cudaMemcpyDeviceToHost, p->stream));
    CU(cudaStreamSynchronize(p->stream));
    if (nagg) *nagg = hier ? p->cl[level].nagg : p->sl[level].nagg;
    return AMGH_OK;
}

static const DevCsr *pick(const amgh_problem *p, int which, int l)
{
    int lmin = p->Ls < p->Lc ? p->Ls : p->Lc;
    if (which == 7) return &p->Kfull;
    if (which == 8) return &p->Mfull;
    if (!p->setup_done || l < 0 || l >= AMGH_MAXL) return nullptr;
    switch (which) {
    case 0: return l < p->Ls ? &p->sl[l].A : nullptr;
    case 1: return l < p->Ls ? &p->sl[l].My : nullptr;
    case 2: return l < lmin ? &p->cl[l].Myu : nullptr;
    case 3: return l + 1 < p->Ls ? &p->sl[l].S : nullptr;
    case 4: return l < p->Lc ? &p->cl[l].KN : nullptr;
    case 5: return l < p->Lc ? &p->cl[l].Mu : nullptr;
    case 6: return l + 1 < p->Lc ? &p->cl[l].P : nullptr;
    }
    return nullptr;
}

extern "C" int amgh_get_matrix_info(const amgh_problem *p, int which, int level, int64_t *rows, int64_t *cols,
                                    int64_t *nnz)
{
    if (!p) return AMGH_ERR_INVALID_ARG;
    const DevCsr *a = pick(p, which, level);
    if (!a || !a->rp) return AMGH_ERR_INVALID_ARG;
    if (rows) *rows = a->rows;
    if (cols) *cols = a->cols;
    if (nnz) *nnz = a->nnz;
    return AMGH_OK;
}

extern "C" int amgh_get_matrix(const amgh_problem *p, int which, int level, int32_t *rp, int32_t *ci, double *v)
{
    if (!p || !rp || !ci || !v) return AMGH_ERR_INVALID_ARG;
    const DevCsr *a = pick(p, which, level);
    if (!a || !a->rp) return AMGH_ERR_INVALID_ARG;
    CU(cudaMemcpyAsync(rp, a->rp, sizeof(int) * (a->rows + 1), cudaMemcpyDeviceToHost, p->stream));
    CU(cudaMemcpyAsync(ci, a->ci, sizeof(int) * a->nnz, cudaMemcpyDeviceToHost, p->stream));
    CU(cudaMemcpyAsync(v, a->v, sizeof(double) * a->nnz, cudaMemcpyDeviceToHost, p->stream));
    CU(cudaStreamSynchronize(p->stream));
    return AMGH_OK;
}

extern "C" int amgh_get_counters(const amgh_problem *p, amgh_solve_info *info)
{
    if (!p || !info) return AMGH_ERR_INVALID_ARG;
    memset(info, 0, sizeof(*info));
    fill_info((amgh_problem *)p, info);
    return AMGH_OK;
}

static void zero_counters(amgh_problem *p)
{
    p->c_inner = p->c_mass = p->c_happ = p->c_refine = p->c_coarse = 0;
    p->c_bytes = 0.0;
    for (int l = 0; l < AMGH_MAXL; l++) p->c_inner_lvl[l] = p->c_mass_lvl[l] = 0;
}

extern "C" int amgh_reset_counters(amgh_problem *p)
{
    if (!p) return AMGH_ERR_INVALID_ARG;
    zero_counters(p);
    return AMGH_OK;
}

extern "C" int amgh_get_level_counters(const amgh_problem *p, int64_t *inner, int64_t *mass)
{
    if (!p) return AMGH_ERR_INVALID_ARG;
    for (int l = 0; l < AMGH_MAXL; l++) {
        if (inner) inner[l] = p->c_inner_lvl[l];
        if (mass) mass[l] = p->c_mass_lvl[l];
    }
    return AMGH_OK;
}

extern "C" int amgh_debug_limits(int bulk_first_polls, int mis_round_cap, int prol_row_cap)
{
    if (bulk_first_polls < -1 || mis_round_cap < -1 || prol_row_cap < -1) return AMGH_ERR_INVALID_ARG;
    mis_set_round_cap(mis_round_cap);
    prol_set_row_cap(prol_row_cap);
    return bulk_set_first_polls(bulk_first_polls);
}

extern "C" int amgh_debug_grid_polls(int polls)
{
    if (polls < -1) return AMGH_ERR_INVALID_ARG;
    TRY(fused_set_grid_polls(polls));
    return block_set_grid_polls(polls);
}

extern "C" int amgh_kernel_timing_mask(amgh_problem *p, unsigned mask)
{
    if (!p) return AMGH_ERR_INVALID_ARG;
    TRY(timer_collect(p));
    p->timer.mask = mask & ((1u << KC_N) - 1u);
    p->timer.enabled = p->timer.mask ? 1 : 0;
    for (int c = 0; c < KC_N; c++) {
        p->timer.launches[c] = 0;
        p->timer.ms[c] = 0.0;
        p->timer.bytes[c] = 0.0;
    }
    return AMGH_OK;
}

extern "C" int amgh_kernel_timing(amgh_problem *p, int enable)
{
    return amgh_kernel_timing_mask(p, enable ? (1u << KC_N) - 1u : 0u);
}

extern "C" int amgh_kernel_class_stats(amgh_problem *p, int cls, int64_t *launches, double *ms, double *bytes,
                                       const char **name)
{
    if (!p || cls < 0 || cls >= KC_N) return AMGH_ERR_INVALID_ARG;
    TRY(timer_collect(p));
    if (launches) *launches = p->timer.launches[cls];
    if (ms) *ms = p->timer.ms[cls];
    if (bytes) *bytes = p->timer.bytes[cls];
    if (name) *name = kclass_name(cls);
    return AMGH_OK;
}

extern "C" int amgh_kernel_stats(amgh_problem *p, int64_t *launches, double *ms, double *bytes)
{
    return amgh_kernel_class_stats(p, KC_CHEB0, launches, ms, bytes, nullptr);
}

extern "C" void amgh_problem_destroy(amgh_problem *p)
{
    if (!p) return;
    StreamScope ss_(p->stream);
    if (p->stream) cudaStreamSynchronize(p->stream);
    else cudaDeviceSynchronize();
    for (auto e : p->timer.ev) cudaEventDestroy(e);
    for (auto e : p->timer.pool) cudaEventDestroy(e);
    block_free(p);
    solver_free_graphs(p);
    p->harena.free_all();
    p->arena.free_all();
    if (p->stream) cudaStreamSynchronize(p->stream);
    else cudaDeviceSynchronize();
    if (p->h_scal) cudaFreeHost(p->h_scal);
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    if (p->wait_ev) cudaEventDestroy(p->wait_ev);
    delete p;
}
