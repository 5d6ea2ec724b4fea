// solver.cu -- the solve layer of the hot path, orchestrated from the host:
//   V-cycle (Sec. 5.2's AMG preconditioner for A, levels l..L-1),
//   AMG-preconditioned CG for A_l y = f (Sec. 5.2, inner solves) in FP64,
//     in double-float with FP32 V-cycles (precision 2), or as FP32 CG and
//     V-cycle wrapped in FP64 iterative refinement (precision 1),
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

#include <algorithm>
#include <chrono>
#include <vector>

#include "internal.cuh"
#include "util.cuh"

// pieces from blas.cu without a template
int mass_start(amgh_problem *p, RedSlot &red, int n, const double *f, double *x, double *r, double *z,
               const double *invd, CgScal *sc, double tol, int maxit);
int outer_pq(amgh_problem *p, RedSlot &red, int n, const double *pv, const double *q, CgScal *sc);
int outer_rz(amgh_problem *p, RedSlot &red, int n, const double *r, const double *z, double *pv, CgScal *sc,
             int first);

// Wait for the problem's stream: a spin in cudaStreamSynchronize, or a sleep
// on a blocking-sync event when many host threads share few cores.
int sync_stream(amgh_problem *p)
{
    if (p->wait_ev) {
        CU(cudaEventRecord(p->wait_ev, p->stream));
        CU(cudaEventSynchronize(p->wait_ev));
        return AMGH_OK;
    }
    CU(cudaStreamSynchronize(p->stream));
    return AMGH_OK;
}

static int read_scal(amgh_problem *p, const CgScal *sc, CgScal *out)
{
    CU(cudaMemcpyAsync(p->h_scal, sc, sizeof(CgScal), cudaMemcpyDeviceToHost, p->stream));
    TRY(sync_stream(p));
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
        TRY(ar.alloc(&S.cs, m));
        TRY(ar.alloc(&S.gs, m));
        TRY(ar.alloc(&S.gx, m));
        TRY(ar.alloc(&S.gr, m));
        TRY(ar.alloc(&S.gz, m));
        TRY(ar.alloc(&S.gp, m));
        TRY(ar.alloc(&S.gq, m));
        TRY(ar.alloc(&S.ry, m));
        TRY(ar.alloc(&S.scal, 1));
        TRY(ar.alloc(&S.scal32, 1));
        TRY(ar.alloc(&S.rscal, 1));
        CU(cudaMemsetAsync(S.scal, 0, sizeof(CgScal), g_alloc_stream));
        CU(cudaMemsetAsync(S.scal32, 0, sizeof(CgScal), g_alloc_stream));
        CU(cudaMemsetAsync(S.rscal, 0, sizeof(CgScal), g_alloc_stream));
        TRY(red_alloc(ar, S.red, m));
        p->chunk_hint[l] = 8;
        p->chunk_hint32[l] = 8;
    }
    for (int l = 0; l < p->Lc; l++) {
        CtrlLevel &C = p->cl[l];
        int n = C.Mu.rows;
        int m = l < p->Ls ? p->sl[l].A.rows : 1;
        double **vn[] = {&C.mx, &C.mr, &C.mz, &C.mp, &C.mq, &C.ms, &C.bc, &C.qc, &C.wc,
                         &C.w1, &C.ta, &C.tb, &C.hu, &C.rq, &C.du};
        for (double **q : vn) TRY(ar.alloc(q, n));
        double **vm[] = {&C.t1, &C.ys, &C.t2, &C.ps};
        for (double **q : vm) TRY(ar.alloc(q, m));
        TRY(ar.alloc(&C.mscal, 1));
        CU(cudaMemsetAsync(C.mscal, 0, sizeof(CgScal), g_alloc_stream));
        int cap = n > m ? n : m;
        TRY(red_alloc(ar, C.red, cap));
        p->mchunk_hint[l] = 8;
    }
    int n = p->n;
    double **vo[] = {&p->ou, &p->or_, &p->oz, &p->op, &p->oq, &p->ob};
    for (double **q : vo) TRY(ar.alloc(q, n));
    TRY(ar.alloc(&p->oscal, 1));
    CU(cudaMemsetAsync(p->oscal, 0, sizeof(CgScal), g_alloc_stream));
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
    pdl_enter();
    if (skip && *skip) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = a[i];
}

// x = V_l b from x = 0; x and b must not alias level-l internal buffers.
// preinit: the caller already wrote the first smoother step (d and the
// level's alternate x buffer) while restricting.
template <typename T>
static int vcyc(amgh_problem *p, int l, const T *b, T *x, const int *skip, int preinit = 0)
{
    StateLevel &S = p->sl[l];
    int n = S.A.rows;
    if (sizeof(T) == sizeof(float) && l == p->fuse_c0)
        return fused_vcycle(p, (const float *)b, (float *)x, preinit, skip);
    if (l == p->Ls - 1) {
        if (sizeof(T) == sizeof(float))
            return dense_gemv32(p, n, p->Acoarse.ld32, p->Acoarse.inv32, (const float *)b, (float *)x, skip);
        return dense_gemv<T>(p, n, p->Acoarse.inv, b, x, skip);
    }
    int timed = (l == 0);
    T *tmp = (x == VBuf<T>::x(S)) ? VBuf<T>::x2(S) : VBuf<T>::x(S);
    T *d = VBuf<T>::d(S), *r = VBuf<T>::r(S);
    const T *invd = VBuf<T>::invd(S);
    T *cur = tmp, *nxt = x;
    // pre-smoothing from zero
    if (!preinit) TRY(cheb_first<T>(p, n, invd, b, d, cur, p->cr[0], skip));
    // level 0 of an FP32 cycle on the structured Kuhn cube: matrix-free operator
    const bool mf = sizeof(T) == sizeof(float) && l == 0 && p->aopts.matrix_free && p->kuhn_N > 0;
    for (int s = 1; s < p->nsteps; s++) {
        if (mf)
            TRY(kuhn_cheb_step(p, (const float *)invd, (const float *)b, (const float *)cur, (float *)d,
                               (float *)nxt, p->cd[s], p->cr[s], skip));
        else
            TRY(cheb_step<T>(p, S.A, invd, b, cur, d, nxt, p->cd[s], p->cr[s], skip, timed));
        T *t = cur;
        cur = nxt;
        nxt = t;
    }
    // coarse-grid correction
    if (mf) TRY(kuhn_residual(p, (const float *)b, (const float *)cur, (float *)r, skip));
    else TRY(residual<T>(p, S.A, b, cur, r, skip, timed));
    StateLevel &Sc = p->sl[l + 1];
    T *bc = VBuf<T>::b(Sc), *xc = VBuf<T>::x(Sc);
    if (l + 1 < p->Ls - 1) {
        TRY(restrict_first<T>(p, S.St, r, bc, VBuf<T>::invd(Sc), VBuf<T>::d(Sc), VBuf<T>::x2(Sc), p->cr[0], skip));
        TRY(vcyc<T>(p, l + 1, bc, xc, skip, 1));
    } else {
        TRY(spmv_t<T>(p, S.St, r, bc, skip, l == 0 ? KC_RESTRICT0 : KC_RESTRICT));
        TRY(vcyc<T>(p, l + 1, bc, xc, skip));
    }
    TRY(prolong_add<T>(p, S.S, xc, cur, skip));
    // post-smoothing with the same polynomial
    for (int s = 0; s < p->nsteps; s++) {
        if (mf)
            TRY(kuhn_cheb_step(p, (const float *)invd, (const float *)b, (const float *)cur, (float *)d,
                               (float *)nxt, s == 0 ? 0.0 : p->cd[s], p->cr[s], skip));
        else
            TRY(cheb_step<T>(p, S.A, invd, b, cur, d, nxt, s == 0 ? 0.0 : p->cd[s], p->cr[s], skip, timed));
        T *t = cur;
        cur = nxt;
        nxt = t;
    }
    if (cur != x) {
        timer_begin(p, KC_VEC);
        pdl_launch(k_copy<T>, dim3(ceil_div(n, 256)), dim3(256), 0, p->stream, n, cur, x, skip);
        LAUNCH_CHECK();
        timer_end(p, KC_VEC, 2.0 * sizeof(T) * n);
    }
    return AMGH_OK;
}

// algorithmic bytes of one V-cycle from level l down (value bytes vb), launch
// by launch as vcyc runs it
double vcycle_bytes(const amgh_problem *p, int l, int vb)
{
    const StateLevel &S = p->sl[l];
    const double n = S.A.rows;
    if (l == p->Ls - 1) return vb == 4 ? 4.0 * n * p->Acoarse.ld32 + 8.0 * n : 8.0 * n * n + 2.0 * vb * n;
    const double step = spmv_bytes(S.A, vb) + 4.0 * vb * n;
    double b = 4.0 * vb * n + (p->nsteps - 1) * step;                 // pre-smoothing from zero
    b += spmv_bytes(S.A, vb) + vb * n;                                 // residual
    b += spmv_bytes(S.St, vb) + 3.0 * vb * S.St.rows;                  // restriction (+ first coarse step)
    b += vcycle_bytes(p, l + 1, vb);
    b += spmv_bytes(S.S, vb) + vb * n;                                 // prolongation
    return b + p->nsteps * step;                                       // post-smoothing
}

int vcycle_run(amgh_problem *p, int l0, int prec32, const void *b, void *x, const int *skip)
{
    if (prec32) return vcyc<float>(p, l0, (const float *)b, (float *)x, skip);
    return vcyc<double>(p, l0, (const double *)b, (double *)x, skip);
}

// ------------------------------------------------------------------ graphs
// One CG iteration (SpMV + p.q, update + r.r, the whole V-cycle, r.z, p update)
// is captured once per level and precision mode on a private stream and then
// replayed with cudaGraphLaunch; all its buffers and scalars are level-owned,
// and every kernel returns at once when the loop's `done` flag is set, so the
// host can replay a whole chunk of iterations before reading the flag back.
template <typename F>
static int capture(amgh_problem *p, F body, cudaGraphExec_t *exec, int *nodes, double *bytes = nullptr)
{
    double local = 0.0;
    ByteSink sink_(&local); // the body's launches are counted per replay by the caller
    cudaStream_t orig = p->stream;
    p->stream = p->cap_stream;
    p->capturing = 1;
    amgh_set_capturing(1);
    cudaGraph_t g = nullptr;
    int st = AMGH_OK;
    if (cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) st = AMGH_ERR_CUDA;
    else {
        st = body();
        if (cudaStreamEndCapture(p->cap_stream, &g) != cudaSuccess && st == AMGH_OK) st = AMGH_ERR_CUDA;
    }
    p->stream = orig;
    p->capturing = 0;
    amgh_set_capturing(0);
    if (st != AMGH_OK) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return st;
    }
    size_t n = 0;
    cudaGraphGetNodes(g, nullptr, &n);
    cudaError_t e = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return AMGH_ERR_CUDA;
    *nodes = (int)n;
    if (bytes) *bytes = local;
    return AMGH_OK;
}

static int replay(amgh_problem *p, cudaGraphExec_t ex, int nodes)
{
    CU(cudaGraphLaunch(ex, p->stream));
    amgh_count_launch(nodes);
    return AMGH_OK;
}

static void free_graph(CgGraph &g)
{
    if (g.start) cudaGraphExecDestroy(g.start);
    if (g.iter) cudaGraphExecDestroy(g.iter);
    g = CgGraph();
}

void solver_free_graphs(amgh_problem *p)
{
    for (int l = 0; l < AMGH_MAXL; l++) {
        for (int m = 0; m < 3; m++) free_graph(p->sl[l].graph[m]);
        free_graph(p->cl[l].mgraph);
    }
}

// kernel timing needs one event pair per launch, so it runs without graphs
static bool use_graphs(amgh_problem *p) { return !p->timer.enabled; }

int graph_capture(amgh_problem *p, const std::function<int()> &body, cudaGraphExec_t *exec, int *nodes)
{
    return capture(p, body, exec, nodes, nullptr);
}

int graph_replay(amgh_problem *p, cudaGraphExec_t exec, int nodes) { return replay(p, exec, nodes); }

bool graphs_enabled(amgh_problem *p) { return use_graphs(p); }

// ------------------------------------------------------------------ AMG-CG
__global__ void k_d2f(int n, const double *__restrict__ a, float *__restrict__ b, const int *skip)
{
    if (skip && *skip) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

__global__ void k_f2d(int n, const float *__restrict__ a, double *__restrict__ b, const int *skip)
{
    if (skip && *skip) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (double)a[i];
}

// mode 0: FP64 CG + FP64 V-cycle; 1: FP32 CG + FP32 V-cycle; 2: FP64 CG + FP32
// V-cycle (the update also writes the FP32 copy of r that the V-cycle reads,
// and the SpMV gathers the FP32 z directly).
// start: z = V r;  iteration: s = A z (+ dots), p/q/x/r update, z = V r.
static int cg_body_start(amgh_problem *p, int l, int mode)
{
    StateLevel &S = p->sl[l];
    if (mode == 1) return vcyc<float>(p, l, S.gr, S.gz, &S.scal32->done);
    if (mode == 0) return vcyc<double>(p, l, S.cr, S.cz, &S.scal->done);
    // double-float CG: the V-cycle reads the hi half of r
    return vcyc<float>(p, l, (const float *)S.cr, S.gz, &S.scal->done);
}

// The V-cycle that closes a CG iteration.  Its pending timings and bytes are
// marked, so that for the iteration that converges -- whose V-cycle the
// device skips -- they can be taken back.
template <typename F>
static int closing_vcycle(amgh_problem *p, F vc)
{
    p->timer.vc_mark = p->timer.ev.size();
    const double before = g_byte_sink ? *g_byte_sink : 0.0;
    int st = vc();
    p->vc_bytes = g_byte_sink ? *g_byte_sink - before : 0.0;
    return st;
}

static int cg_body_iter(amgh_problem *p, int l, int mode)
{
    StateLevel &S = p->sl[l];
    int n = S.A.rows;
    int timed = 0; // kernel timing covers the level-0 smoother step only
    // on a smoothing level the update also takes the V-cycle's first step
    // (d and the level's other x buffer from the new residual)
    const bool pre = l < p->Ls - 1;
    if (mode == 1) {
        TRY((cg2_spmv<float, float>(p, S.red, S.A, S.gz, S.gr, S.gs, S.scal32, timed)));
        TRY((cg2_update<float, float>(p, S.red, n, S.gz, S.gs, S.gp, S.gq, S.gx, S.gr, nullptr, nullptr, S.scal32,
                                      pre ? S.fd : nullptr, pre ? S.fx : nullptr, S.invd32, p->cr[0])));
        return closing_vcycle(p, [&] { return vcyc<float>(p, l, S.gr, S.gz, &S.scal32->done, pre ? 1 : 0); });
    }
    if (mode == 0) {
        TRY((cg2_spmv<double, double>(p, S.red, S.A, S.cz, S.cr, S.cs, S.scal, timed)));
        TRY((cg2_update<double, double>(p, S.red, n, S.cz, S.cs, S.cp, S.cq, S.cx, S.cr, nullptr, nullptr, S.scal,
                                        pre ? S.vd : nullptr, pre ? S.vx : nullptr, S.invd, p->cr[0])));
        return closing_vcycle(p, [&] { return vcyc<double>(p, l, S.cr, S.cz, &S.scal->done, pre ? 1 : 0); });
    }
    TRY(dfcg_spmv(p, S.red, S.A, S.gz, S.cr, S.cs, S.scal, timed));
    // on a smoothing level the update also takes the V-cycle's first step
    // (d and the level's other x buffer from the new residual)
    if (l < p->Ls - 1) {
        TRY(dfcg_update(p, S.red, n, S.gz, S.cs, S.cp, S.cq, S.cx, S.cr, S.scal, S.invd32, S.fd, S.fx, p->cr[0]));
        return closing_vcycle(p, [&] { return vcyc<float>(p, l, (const float *)S.cr, S.gz, &S.scal->done, 1); });
    }
    TRY(dfcg_update(p, S.red, n, S.gz, S.cs, S.cp, S.cq, S.cx, S.cr, S.scal));
    return closing_vcycle(p, [&] { return vcyc<float>(p, l, (const float *)S.cr, S.gz, &S.scal->done); });
}

// PCG for A_l x = f preconditioned by V_l; the solution is left in S.cx (FP64
// modes) or S.gx (mode 1)
static int pcg_run(amgh_problem *p, int l, int mode, const void *f, double tol, int maxit, int64_t *iters)
{
    StateLevel &S = p->sl[l];
    int n = S.A.rows;
    CgScal *sc = mode == 1 ? S.scal32 : S.scal;
    if (mode == 1) TRY(cg_start<float>(p, S.red, n, (const float *)f, S.gx, S.gr, sc, tol, maxit, 1));
    else if (mode == 2) TRY(dfcg_start(p, S.red, n, (const double *)f, S.cx, S.cr, sc, tol, maxit));
    else TRY(cg_start<double>(p, S.red, n, (const double *)f, S.cx, S.cr, sc, tol, maxit, 1));
    CgGraph &g = S.graph[mode];
    bool gr = use_graphs(p);
    if (gr && !g.iter) {
        TRY(capture(p, [&] { return cg_body_start(p, l, mode); }, &g.start, &g.nodes_start, &g.bytes_start));
        TRY(capture(
            p,
            [&] {
                int st = cg_body_iter(p, l, mode);
                g.bytes_vc = p->vc_bytes;
                return st;
            },
            &g.iter, &g.nodes_iter, &g.bytes_iter));
    }
    // bytes of the start, of one iteration and of its closing V-cycle: the
    // graphs' totals, or counted on the first direct launches
    double b_start = g.bytes_start, b_iter = g.bytes_iter, b_vc = g.bytes_vc;
    if (gr) TRY(replay(p, g.start, g.nodes_start));
    else {
        b_start = 0.0;
        ByteSink bs_(&b_start);
        TRY(cg_body_start(p, l, mode));
    }
    int *hint = mode == 1 ? &p->chunk_hint32[l] : &p->chunk_hint[l];
    // first chunk: most of the previous solve's count (replays past convergence are no-ops)
    int chunk = *hint > 1 ? (*hint * 7) / 8 : 1;
    int enq = 0, prev_iters = 0;
    CgScal h;
    std::vector<size_t> it_mark, vc_mark; // direct launches: timings of each enqueued iteration
    for (;;) {
        it_mark.clear();
        vc_mark.clear();
        for (int c = 0; c < chunk; c++) {
            if (gr) TRY(replay(p, g.iter, g.nodes_iter));
            else {
                double b = 0.0;
                it_mark.push_back(p->timer.ev.size());
                {
                    ByteSink bs_(&b);
                    TRY(cg_body_iter(p, l, mode));
                }
                vc_mark.push_back(p->timer.vc_mark);
                if (enq + c == 0) {
                    b_iter = b;
                    b_vc = p->vc_bytes;
                }
            }
        }
        enq += chunk;
        TRY(read_scal(p, sc, &h));
        if (!gr) {
            // the device skipped every iteration past convergence and the
            // closing V-cycle of the converging one: their timings go
            const int ran = h.iters - prev_iters;
            size_t cut = (size_t)-1;
            if (ran >= 0 && ran < chunk) cut = it_mark[ran];
            if (h.done && ran >= 1 && ran <= chunk) cut = std::min(cut, vc_mark[ran - 1]);
            if (cut != (size_t)-1) timer_drop_from(p, cut);
        }
        prev_iters = h.iters;
        if (h.done || enq > maxit + 2) break;
        chunk = h.iters / 8 > 1 ? h.iters / 8 : 1;
    }
    if (h.iters > 0) count_bytes(b_start + (double)h.iters * b_iter - (h.done ? b_vc : 0.0));
    p->c_inner_lvl[l] += h.iters;
    if (h.iters > 0) *hint = h.iters;
    if (iters) *iters = h.iters;
    p->c_inner += h.iters;
    if (!h.done) return AMGH_ERR_NOT_CONVERGED;
    return cg_status(h);
}

// A_l y = f to relative residual tol: FP64 CG with an FP64 (precision 0) or
// FP32 (precision 2) V-cycle, or FP32 CG inside FP64 iterative refinement
// (precision 1)
int state_solve(amgh_problem *p, int l, const double *f, double *y, double tol, int64_t *iters)
{
    StateLevel &S = p->sl[l];
    int n = S.A.rows;
    int maxit = p->sopts.inner_max_iter;
    int prec = p->aopts.precision;
    if (prec != 1) {
        int st = pcg_run(p, l, prec == 2 ? 2 : 0, f, tol, maxit, iters);
        if (prec == 2) TRY(df_to_double(p, n, S.cx, S.scal, y));
        else {
            timer_begin(p, KC_VEC);
            pdl_launch(k_copy<double>, dim3(ceil_div(n, 256)), dim3(256), 0, p->stream, n, S.cx, y, nullptr);
            LAUNCH_CHECK();
            timer_end(p, KC_VEC, 16.0 * n);
        }
        return st;
    }
    // r = f - A y in FP64, FP32 PCG on A e = r / ||r||, y += ||r|| e
    TRY(ref_start(p, S.red, n, f, y, S.ry, S.rscal, tol, 50));
    CgScal h;
    TRY(read_scal(p, S.rscal, &h));
    int64_t it_total = 0;
    double inner = 1e-4;
    while (!h.done) {
        TRY(ref_to32(p, S.red, n, S.ry, S.gq, S.rscal));
        int64_t it = 0;
        int st = pcg_run(p, l, 1, S.gq, inner, maxit, &it);
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
    // precision 2: the mass CG in double-float too, Jacobi from FP32 copies
    bool df = p->aopts.precision == 2;
    if (df && p->aopts.persistent_cg && !p->parent && !p->in_batch && !p->capturing)
        return persistent_mass_single(p, l, b, x, iters);
    if (df) {
        TRY(dfcg_start(p, C.red, n, b, C.mx, C.mr, C.mscal, p->sopts.mass_tol, p->sopts.mass_max_iter));
        TRY(dfcg_jacobi(p, n, C.mr, C.mu_invdiag32, (float *)C.mz));
    } else {
        TRY(mass_start(p, C.red, n, b, C.mx, C.mr, C.mz, C.mu_invdiag, C.mscal, p->sopts.mass_tol,
                       p->sopts.mass_max_iter));
    }
    bool gr = use_graphs(p);
    CgGraph &g = C.mgraph;
    auto body = [&]() {
        if (df) {
            TRY(dfcg_spmv(p, C.red, C.Mu, (const float *)C.mz, C.mr, C.ms, C.mscal, 0));
            return dfcg_update(p, C.red, n, (const float *)C.mz, C.ms, C.mp, C.mq, C.mx, C.mr, C.mscal,
                               C.mu_invdiag32);
        }
        TRY((cg2_spmv<double, double>(p, C.red, C.Mu, C.mz, C.mr, C.ms, C.mscal, 0)));
        return cg2_update<double, double>(p, C.red, n, C.mz, C.ms, C.mp, C.mq, C.mx, C.mr, nullptr, C.mu_invdiag,
                                          C.mscal);
    };
    if (gr && !g.iter) TRY(capture(p, body, &g.iter, &g.nodes_iter, &g.bytes_iter));
    double b_iter = g.bytes_iter;
    int chunk = p->mchunk_hint[l] > 1 ? (p->mchunk_hint[l] * 7) / 8 : 1;
    int enq = 0, prev_iters = 0;
    CgScal h;
    std::vector<size_t> it_mark;
    for (;;) {
        it_mark.clear();
        for (int c = 0; c < chunk; c++) {
            if (gr) TRY(replay(p, g.iter, g.nodes_iter));
            else {
                double b = 0.0;
                it_mark.push_back(p->timer.ev.size());
                {
                    ByteSink bs_(&b);
                    TRY(body());
                }
                if (enq + c == 0) b_iter = b;
            }
        }
        enq += chunk;
        TRY(read_scal(p, C.mscal, &h));
        const int ran = h.iters - prev_iters;
        if (!gr && ran >= 0 && ran < chunk) timer_drop_from(p, it_mark[ran]); // skipped iterations
        prev_iters = h.iters;
        if (h.done || enq > p->sopts.mass_max_iter + 2) break;
        chunk = h.iters / 8 > 1 ? h.iters / 8 : 1;
    }
    count_bytes((double)h.iters * b_iter);
    p->c_mass_lvl[l] += h.iters;
    if (h.iters > 0) p->mchunk_hint[l] = h.iters;
    if (iters) *iters = h.iters;
    p->c_mass += h.iters;
    if (df) {
        TRY(df_to_double(p, n, C.mx, C.mscal, x));
    } else {
        timer_begin(p, KC_VEC);
        pdl_launch(k_copy<double>, dim3(ceil_div(n, 256)), dim3(256), 0, p->stream, n, C.mx, x, nullptr);
        LAUNCH_CHECK();
        timer_end(p, KC_VEC, 16.0 * n);
    }
    if (!h.done) return AMGH_ERR_NOT_CONVERGED;
    return cg_status(h);
}

// ------------------------------------------------------------------ Hessian
int hessian_level(amgh_problem *p, int l, const double *v, double *hv)
{
    StateLevel &S = p->sl[l];
    CtrlLevel &C = p->cl[l];
    // level 0 is the outer CG's operator; levels >= 1 occur only inside the
    // preconditioner (Algorithm MLAS) and use the preconditioner tolerance
    double tol = l == 0 ? p->sopts.inner_tol : p->sopts.precond_tol;
    TRY(spmv(p, C.Myu, v, C.t1, nullptr, KC_SPMV));
    TRY(state_solve(p, l, C.t1, C.ys, tol, nullptr));
    TRY(spmv(p, S.My, C.ys, C.t2, nullptr, KC_SPMV));
    TRY(state_solve(p, l, C.t2, C.ps, tol, nullptr));
    TRY(spmv2(p, C.Myut, C.ps, C.Mu, v, p->beta, hv, nullptr));
    if (l == 0) p->c_happ += 1;
    return AMGH_OK;
}

// ------------------------------------------------------------------ MLAS
__global__ void k_r_combine(int n, const double *__restrict__ ta, const double *__restrict__ w1,
                            const double *__restrict__ tb, double beta, double *__restrict__ out)
{
    pdl_enter();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = ta[i] + (w1[i] - tb[i]) / beta;
}

int mlas_R(amgh_problem *p, int j, const double *b, double *out)
{
    CtrlLevel &C = p->cl[j], &Cc = p->cl[j + 1];
    int n = C.Mu.rows;
    TRY(spmv(p, C.Pt, b, Cc.bc, nullptr, KC_SPMV));
    TRY(mlas_Q(p, j + 1, Cc.bc, Cc.qc));
    TRY(mass_solve(p, j, b, C.w1, nullptr));
    TRY(mass_solve(p, j + 1, Cc.bc, Cc.wc, nullptr));
    TRY(spmv(p, C.P, Cc.qc, C.ta, nullptr, KC_SPMV));
    TRY(spmv(p, C.P, Cc.wc, C.tb, nullptr, KC_SPMV));
    timer_begin(p, KC_VEC);
    pdl_launch(k_r_combine, dim3(ceil_div(n, 256)), dim3(256), 0, p->stream, n, C.ta, C.w1, C.tb, p->beta, out);
    LAUNCH_CHECK();
    timer_end(p, KC_VEC, 32.0 * n);
    return AMGH_OK;
}

static int dot_host(amgh_problem *p, RedSlot &red, int n, const double *x, const double *y, double *out);

// Q_{ell-1} b by unpreconditioned CG on H_{ell-1} from u = 0 (Sec. 5.2),
// stopping at ||r_k|| <= coarse_tol ||b|| on the recursively updated
// residual; the iterate at the iteration cap is used as it stands.
static int coarse_cg(amgh_problem *p, int j, const double *b, double *u)
{
    CtrlLevel &C = p->cl[j];
    int n = C.Mu.rows;
    double *r = C.rq, *pv = C.du, *q = C.hu;
    CU(cudaMemsetAsync(u, 0, sizeof(double) * n, p->stream));
    CU(cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, p->stream));
    CU(cudaMemcpyAsync(pv, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, p->stream));
    double ff = 0.0;
    TRY(dot_host(p, C.red, n, b, b, &ff));
    if (!(ff == ff)) return AMGH_ERR_NUMERIC;
    if (ff == 0.0) return AMGH_OK;
    double nf = sqrt(ff), rz = ff;
    double tol = p->sopts.coarse_tol;
    for (int k = 1; k <= p->sopts.coarse_max_iter; k++) {
        TRY(hessian_level(p, j, pv, q));
        p->c_coarse += 1;
        double pq = 0.0;
        TRY(dot_host(p, C.red, n, pv, q, &pq));
        if (!(pq > 0.0)) return pq == pq ? AMGH_ERR_INDEFINITE : AMGH_ERR_NUMERIC;
        double alpha = rz / pq;
        TRY(vec_axpby(p, n, 1.0, u, alpha, pv, u));
        TRY(vec_axpby(p, n, 1.0, r, -alpha, q, r));
        double rr = 0.0;
        TRY(dot_host(p, C.red, n, r, r, &rr));
        if (!(rr == rr)) return AMGH_ERR_NUMERIC;
        if (sqrt(rr) <= tol * nf) break;
        if (!(rr > 0.0)) return AMGH_ERR_INDEFINITE;
        double beta = rr / rz;
        rz = rr;
        TRY(vec_axpby(p, n, 1.0, r, beta, pv, pv));
    }
    return AMGH_OK;
}

int mlas_Q(amgh_problem *p, int j, const double *b, double *u)
{
    CtrlLevel &C = p->cl[j];
    int n = C.Mu.rows;
    if (j == p->ell - 1) {
        if (p->coarse_cg) return coarse_cg(p, j, b, u);
        return dense_gemv<double>(p, n, p->Hcoarse.inv, b, u, nullptr);
    }
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
    TRY(spmv(p, S.My, p->yd_state, C.t2, nullptr, KC_SPMV));
    TRY(state_solve(p, 0, C.t2, C.ps, p->sopts.inner_tol, nullptr));
    TRY(spmv(p, C.Myut, C.ps, b, nullptr, KC_SPMV));
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
    TRY(sync_stream(p));
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
            TRY(cg_update_outer(p, p->ored, n, u, r, pv, q, sc));
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
