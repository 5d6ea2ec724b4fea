// internal.cuh -- device data structures and kernel entry points shared by the
// translation units of the amgh library (sm_103a).
#pragma once

#include <functional>
#include <utility>

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/amgh.h"

#define AMGH_MAXL 32
#define AMGH_DENSE_MAX 4096
#define AMGH_SELL_C 32
#define AMGH_BLOCK_MAX 8 // widest column block of the block solver

// ------------------------------------------------------------------ errors
// record the CUDA error (code, file, line) for amgh_last_error
void amgh_note_error(int code, const char *file, int line);
void amgh_note_msg(const char *msg);
#define CU(call)                                                               \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) {                                               \
            amgh_note_error((int)e_, __FILE__, __LINE__);                      \
            return e_ == cudaErrorMemoryAllocation ? AMGH_ERR_OOM : AMGH_ERR_CUDA; \
        }                                                                      \
    } while (0)
#define TRY(call)                 \
    do {                          \
        int s_ = (call);          \
        if (s_ != AMGH_OK) return s_; \
    } while (0)

// count of kernels launched by this library (reported to callers)
void amgh_count_launch(int n = 1);
// blocks of `block` threads of `kernel` resident on the current device at once
int resident_grid(const void *kernel, int block);
void amgh_set_capturing(int on);
// Programmatic dependent launch.  Solve-phase kernels are launched with
// pdl_launch, which lets a kernel be scheduled while its predecessor in the
// stream (or CUDA graph) is still running; every such kernel calls
// pdl_enter() first, which waits until the predecessor has completed and its
// writes are visible, and -- for grids that fit comfortably in one wave --
// lets its own successor be scheduled right away, so launch latency overlaps
// the kernel instead of following it.  Without the launch attribute the wait
// returns at once.
#define PDL_EARLY_BLOCKS 608
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (gridDim.x * gridDim.y * gridDim.z <= PDL_EARLY_BLOCKS) asm volatile("griddepcontrol.launch_dependents;" :::);
}

template <typename... KArgs, typename... Args>
inline void pdl_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                       Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // a failed launch is reported by cudaGetLastError in LAUNCH_CHECK
    (void)cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

#define LAUNCH_CHECK()                                   \
    do {                                                 \
        amgh_count_launch();                             \
        cudaError_t e_ = cudaGetLastError();             \
        if (e_ != cudaSuccess) {                         \
            amgh_note_error((int)e_, __FILE__, __LINE__); \
            return AMGH_ERR_CUDA;                        \
        }                                                \
    } while (0)

static inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// ------------------------------------------------------------------ memory
// Device memory comes from one stream-ordered pool per device owned by the
// library (cudaMallocFromPoolAsync): allocations and frees are ordered on the
// problem's stream, never synchronise the device, and freed blocks stay in the
// pool for the next problem.  g_alloc_stream is the stream the calling thread
// is working on (set by every entry point through StreamScope).
extern thread_local cudaStream_t g_alloc_stream;
int pool_alloc(void **p, size_t bytes);
void pool_free(void *p);

struct StreamScope {
    cudaStream_t prev;
    explicit StreamScope(cudaStream_t s) : prev(g_alloc_stream) { g_alloc_stream = s; }
    ~StreamScope() { g_alloc_stream = prev; }
};

// Every device allocation of a problem goes through an Arena so destroy frees all.
struct Arena {
    std::vector<void *> ptrs;
    template <typename T>
    int alloc(T **p, int64_t count)
    {
        *p = nullptr;
        if (count <= 0) count = 1;
        void *q = nullptr;
        int st = pool_alloc(&q, (size_t)count * sizeof(T));
        if (st) return st;
        ptrs.push_back(q);
        *p = (T *)q;
        return 0;
    }
    void release(void *q);
    void free_all();
};

// Temporary device allocations released (stream-ordered) at scope exit.
struct Scratch {
    std::vector<void *> ptrs;
    template <typename T>
    int alloc(T **p, int64_t count)
    {
        *p = nullptr;
        if (count <= 0) count = 1;
        void *q = nullptr;
        int st = pool_alloc(&q, (size_t)count * sizeof(T));
        if (st) return st;
        ptrs.push_back(q);
        *p = (T *)q;
        return 0;
    }
    ~Scratch()
    {
        for (void *q : ptrs) pool_free(q);
    }
};

// ------------------------------------------------------------------ matrices
// CSR with sorted columns (int32 indices, FP64 values) plus, for operators on
// the hot path, a SELL-32 copy (slices of 32 consecutive rows, column-major
// inside a slice so a warp's loads coalesce) in FP64 and FP32.
struct DevCsr {
    int rows = 0, cols = 0, nnz = 0;
    int *rp = nullptr, *ci = nullptr;
    double *v = nullptr;
    // how the solve phase applies it: tpr = 1 -> SELL-32 below; tpr > 1 -> CSR
    // with tpr lanes per row and the FP32 copy v32
    int tpr = 1;
    float *v32 = nullptr;
    // low FP32 parts, v - (double)(float)v, in the same layout as the solve-phase
    // values (SELL or CSR): with the FP32 values they carry ~48 bits of v
    float *lo32 = nullptr;
    // most entries one lane of the applying kernels visits in a row (SELL:
    // the widest slice; CSR: ceil(longest row / tpr)); rows up to
    // ROW_UNROLL per lane are read with every load issued up front
    int wmax = 1 << 30;
    // SELL-32; ellw > 0: every slice has this width (slice s starts at
    // 32 * ellw * s, so kernels need not load the slice pointers)
    int nslices = 0, sell_nnz = 0, ellw = 0;
    int *sl_ptr = nullptr, *sl_ci = nullptr;
    double *sl_v = nullptr;
    float *sl_v32 = nullptr;
    // uniform-width SELL only: column - row as int16 when every entry fits
    // (2 instead of 4 bytes of index per stored entry)
    short *sl_ci16 = nullptr;
    // entries the solve-phase copy holds: the SELL copy leaves out entries
    // whose value is exactly zero (-1: all nnz entries are held)
    int nnz_solve = -1;
};

// ------------------------------------------------------------------ reductions
// Deterministic two-stage reductions: every block writes a partial, the last
// block to finish (atomic ticket) sums the partials in fixed order and runs a
// finaliser.  Each reduction site owns its slot so tickets never mix.
struct RedSlot {
    double *partials = nullptr; // [capacity]
    unsigned *ticket = nullptr;
    int capacity = 0;
};

// device scalars of one CG loop
struct CgScal {
    double rz, pq, alpha, beta, rr, ff, thr; // thr = tol^2 * ff
    double scale;                             // refinement: ||r||
    int done, iters, status, maxit;
    int total_iters;
    int k1; // single-reduction CG: number of alpha/beta updates so far
    float ahi, alo, bhi, blo; // alpha and beta as double-float (double-float CG)
    int pad[2];
};

enum { CG_RUNNING = 0, CG_CONVERGED = 1, CG_INDEFINITE = 2, CG_NUMERIC = 3, CG_MAXIT = 4 };

// ------------------------------------------------------------------ hierarchy
// CUDA graphs of one CG iteration (and of the CG start after the first
// residual), captured once per level and precision mode, replayed per
// iteration; `nodes` is the kernel count of one replay.
struct CgGraph {
    cudaGraphExec_t start = nullptr, iter = nullptr;
    int nodes_start = 0, nodes_iter = 0;
    // algorithmic bytes of one replay, and of the iteration's V-cycle alone
    // (skipped in the iteration that converges)
    double bytes_start = 0.0, bytes_iter = 0.0, bytes_vc = 0.0;
};

struct StateLevel {
    DevCsr A, My, S, St; // S: rows m_l, cols m_{l+1}; St = S^T
    double *invd = nullptr;   // 1 / l1 row sums
    float *invd32 = nullptr;
    int *agg = nullptr;
    int nagg = 0;
    // V-cycle work (FP64 and FP32)
    double *vb, *vx, *vx2, *vd, *vr;
    float *fb, *fx, *fx2, *fd, *fr;
    // CG work at this level (FP64): x r z p q; FP32 inner CG: same
    double *cx, *cr, *cz, *cp, *cq, *cs; // x r z p q and s = A z
    float *gx, *gr, *gz, *gp, *gq, *gs;
    double *ry; // refinement residual (FP64)
    CgScal *scal = nullptr;  // FP64 CG loop scalars
    CgScal *scal32 = nullptr; // FP32 inner CG loop scalars
    CgGraph graph[3];         // 0: FP64 CG, 1: FP32 inner CG, 2: FP64 CG + FP32 V-cycle
    CgScal *rscal = nullptr;  // refinement loop scalars
    RedSlot red;
};

struct CtrlLevel {
    DevCsr KN, Mu, P, Pt, Myu, Myut; // Myu: m_l x n_l (cross), Myut its transpose
    double *mu_invdiag = nullptr;
    float *mu_invdiag32 = nullptr;
    int *agg = nullptr;
    int nagg = 0;
    // mass CG work
    double *mx, *mr, *mz, *mp, *mq, *ms;
    CgScal *mscal = nullptr;
    CgGraph mgraph;
    // MLAS work
    double *bc, *qc, *wc, *w1, *ta, *tb, *hu, *rq, *du; // n_l each (bc, qc, wc: coarse side of R_{l-1})
    // Hessian work (state-sized at this level, and control-sized)
    double *t1, *ys, *t2, *ps;
    RedSlot red;
};

struct Dense {
    int n = 0;
    double *inv = nullptr; // explicit inverse (n x n, row-major)
    float *inv32 = nullptr; // FP32 copy for FP32 V-cycles, rows padded to ld32 (a multiple of 4)
    int ld32 = 0;
};

// Kernel classes of the solve phase: per-class launch counts, durations and
// algorithmic bytes (the *0 classes are the finest level, whose operands do
// not fit in L2; the others are the coarse levels and control-side work).
enum KClass {
    KC_CHEB0,     // Chebyshev / l1-Jacobi step, level 0
    KC_CHEB,      // the same on coarse levels (and the first step from zero)
    KC_RESID0,    // residual b - A x, level 0
    KC_RESID,
    KC_RESTRICT0, // S^T r (fused with the coarse level's first smoother step)
    KC_RESTRICT,
    KC_PROLONG0,  // x += S e
    KC_PROLONG,
    KC_CGSPMV0,   // CG operator product with its dot products, level 0
    KC_CGSPMV,
    KC_CGUPD0,    // CG vector update with its reduction, level 0
    KC_CGUPD,
    KC_COARSE,    // dense coarsest solve, fused coarse V-cycle
    KC_SPMV,      // other sparse products (M_yu, M_y, M_u, P, P^T, ...)
    KC_VEC,       // other vector kernels
    KC_N
};
static_assert(KC_N == AMGH_KCLASSES, "kernel classes of the ABI");
const char *kclass_name(int c);

struct KernelTimer {
    int enabled = 0;
    unsigned mask = 0; // classes timed (bit c = class c)
    std::vector<cudaEvent_t> ev; // pairs
    std::vector<int> cls;        // class of each pending pair
    std::vector<double> pending_bytes;
    std::vector<cudaEvent_t> pool;
    int64_t launches[KC_N] = {};
    double ms[KC_N] = {}, bytes[KC_N] = {};
    size_t vc_mark = 0; // event count before the V-cycle of the last CG iteration
};

// Algorithmic bytes of the solve phase: every launch wrapper reports its
// kernel's compulsory traffic (from sizes, not counters) to the calling
// thread's sink.  Entry points point the sink at the problem's counter; graph
// capture points it at the graph's own total, which the CG loops then add
// once per iteration actually executed.
extern thread_local double *g_byte_sink;
struct ByteSink {
    double *prev;
    explicit ByteSink(double *s) : prev(g_byte_sink) { g_byte_sink = s; }
    ~ByteSink() { g_byte_sink = prev; }
};
static inline void count_bytes(double b)
{
    if (g_byte_sink) *g_byte_sink += b;
}

struct BlockWork; // work space of the block solver (block.cu)

struct amgh_problem {
    // set on a handle made by amgh_problem_share: matrices, hierarchies and
    // dense coarse inverses belong to the parent; this handle owns only its
    // work space, desired state, streams, graphs and counters
    const amgh_problem *parent = nullptr;
    cudaEvent_t wait_ev = nullptr; // blocking-sync event for host waits (else spin)
    int in_batch = 0;              // run by the batch runtime beside other handles
    // single-column persistent mass CG (persistent_cg): scalars, block
    // partials and barrier of its cooperative launch, allocated on first use
    void *pm_bs = nullptr, *pm_p1 = nullptr, *pm_p2 = nullptr, *pm_bar = nullptr;
    int dim = 0;
    int64_t nv = 0, ne = 0;
    double beta = 0.0;
    int m = 0, n = 0;
    cudaStream_t stream = 0;
    cudaStream_t cap_stream = 0; // private stream used only to capture graphs
    int df_spmv = 1;             // FP64 CG SpMVs as double-float on the FP32 pipe
    int capturing = 0;
    Arena arena;
    // inputs on device
    double *coords = nullptr, *kappa = nullptr, *yd_state = nullptr;
    int *elems = nullptr;
    unsigned char *dir = nullptr;
    int *state_of_vertex = nullptr; // -1 for Dirichlet
    int *vertex_of_state = nullptr;
    DevCsr Kfull, Mfull;
    // options
    amgh_amg_opts aopts;
    amgh_solve_opts sopts;
    int setup_done = 0;
    int Ls = 0, Lc = 0, ell = 0;
    int coarse_cg = 0; // Q_{ell-1} by CG on H_{ell-1} (else the dense inverse)
    // fused coarse end of the FP32 V-cycle (fused.cu): first fused level or -1
    int fuse_c0 = -1, fuse_cluster = 0;
    void *fuse_table = nullptr;
    int fuse_grid = 0;       // > 0: grid scope, blocks of the cooperative launch
    void *fuse_bar = nullptr; // its barrier state
    StateLevel sl[AMGH_MAXL];
    CtrlLevel cl[AMGH_MAXL];
    Dense Acoarse;  // inverse of A[Ls-1]
    Dense Aell;     // inverse of A[ell-1] when ell-1 != Ls-1
    Dense Hcoarse;  // inverse of H[ell-1]
    int nsteps = 0;
    double cd[16], cr[16];
    // outer CG work (control-sized, level 0)
    double *ou, *or_, *oz, *op, *oq, *ob;
    CgScal *oscal = nullptr;
    RedSlot ored;
    double *dscratch = nullptr;
    Arena harena; // hierarchy (freed on re-setup)
    // host mirrors
    CgScal *h_scal = nullptr; // pinned
    // counters
    int64_t c_inner = 0, c_mass = 0, c_happ = 0, c_refine = 0, c_coarse = 0;
    double c_bytes = 0.0;  // algorithmic bytes of the solve-phase kernels run
    double vc_bytes = 0.0; // bytes of the V-cycle inside the last CG iteration body
    int64_t c_inner_lvl[AMGH_MAXL], c_mass_lvl[AMGH_MAXL];
    double t_setup = 0.0;
    KernelTimer timer;
    int chunk_hint[AMGH_MAXL];
    int chunk_hint32[AMGH_MAXL];
    int mchunk_hint[AMGH_MAXL];
    BlockWork *blk = nullptr; // allocated by the first block call
    // structured Kuhn cube (kuhn.cu): N of the N^3 grid once detected, else 0
    int kuhn_checked = 0, kuhn_N = 0;
    float *kappa32 = nullptr;
};

// class c0 for vectors / operators of the finest state or control level
// (larger than L2 on the benchmark meshes), c for every coarser one
static inline int fine_cls(const amgh_problem *p, int rows, int c0, int c)
{
    return (rows == p->m || rows == p->n) ? c0 : c;
}

// ------------------------------------------------------------------ sparse.cu
int csr_to_sell(Arena &ar, DevCsr &a, int want32, cudaStream_t s);
// pick SELL-32 or lanes-per-row CSR from the mean row length and build it
int prepare_operator(Arena &ar, DevCsr &a, cudaStream_t s, int force_tpr = 0);
// prepare_operator; for a state matrix A with aopts.autotune set, the layout
// is the one whose Chebyshev step timed fastest on this GPU
int prepare_tuned(amgh_problem *p, Arena &ar, DevCsr &a, int is_state_matrix);
// AMGH_ERR_TIMEOUT (and the flag cleared) if a staged copy timed out
int bulk_timeout_check(cudaStream_t s);
// poll limit of the staged smoother's first wait (< 0: the default; 0: give
// up at once, the copies still drain); test hook behind amgh_debug_limits
int bulk_set_first_polls(int polls);
// rounds the MIS-2 loop may take before AMGH_ERR_TIMEOUT (<= 0: n + 1)
void mis_set_round_cap(int cap);
// aggregates per prolongator row kept in registers (<= 0: the default)
void prol_set_row_cap(int cap);
// b = (float)a
int to_f32(amgh_problem *p, const double *a, int64_t n, float *b);
// build a.lo32 (after prepare_operator)
int build_lo_parts(Arena &ar, DevCsr &a, cudaStream_t s);
int csr_transpose(Arena &ar, const DevCsr &a, DevCsr &t, cudaStream_t s);
// y = A x (FP64 or FP32 SELL)
// cls: the KClass the launch is timed and counted under
int spmv(amgh_problem *p, const DevCsr &a, const double *x, double *y, const int *skip, int cls);
int spmv32(amgh_problem *p, const DevCsr &a, const float *x, float *y, const int *skip, int cls);
// y = A1 x1 + c * A2 x2 (same row count)
int spmv2(amgh_problem *p, const DevCsr &a1, const double *x1, const DevCsr &a2, const double *x2,
          double c, double *y, const int *skip);
int vec_axpby_spmv(amgh_problem *p, const DevCsr &a, const double *x, double c, double *y, const int *skip);
double spmv_bytes(const DevCsr &a, int value_bytes);

template <typename T>
struct VT;

// V-cycle / smoother kernels (templated on value type, defined in sparse.cu)
template <typename T>
int cheb_first(amgh_problem *p, int n, const T *invd, const T *b, T *d, T *x, double c, const int *skip);
template <typename T>
int cheb_step(amgh_problem *p, const DevCsr &a, const T *invd, const T *b, const T *x, T *d, T *xn,
              double cdv, double crv, const int *skip, int timed);
template <typename T>
int residual(amgh_problem *p, const DevCsr &a, const T *b, const T *x, T *r, const int *skip, int timed);
template <typename T>
int spmv_t(amgh_problem *p, const DevCsr &a, const T *x, T *y, const int *skip, int cls);
template <typename T>
int restrict_first(amgh_problem *p, const DevCsr &st, const T *r, T *bc, const T *invd_c, T *d_c, T *x_c,
                   double c0, const int *skip);
template <typename T>
int prolong_add(amgh_problem *p, const DevCsr &s, const T *e, T *x, const int *skip);
template <typename T>
int dense_gemv(amgh_problem *p, int n, const double *inv, const T *b, T *x, const int *skip);
// fused.cu: table and cluster size of the fused coarse V-cycle; one launch of it
int fused_setup(amgh_problem *p);
int fused_vcycle(amgh_problem *p, const float *b, float *x, int preinit, const int *skip);
// AMGH_ERR_TIMEOUT (flag cleared, the problem's barrier reset) if a grid
// barrier of the fused V-cycle gave up
int grid_timeout_check(amgh_problem *p);
int block_grid_timeout_check(amgh_problem *p);
int persistent_mass_single(amgh_problem *p, int l, const double *b, double *x, int64_t *iters);
int block_set_grid_polls(int polls);
int fused_set_grid_polls(int polls);
// x = inv b with the FP32 copy (rows padded to ld, 16-byte aligned)
int dense_gemv32(amgh_problem *p, int n, int ld, const float *inv32, const float *b, float *x, const int *skip);
// FP32 copy of a dense inverse with rows padded to a multiple of 4
int dense_make32(amgh_problem *p, Arena &ar, Dense &d);

// ------------------------------------------------------------------ blas.cu
int red_alloc(Arena &ar, RedSlot &slot, int capacity);
// CG building blocks (device-side scalars, skip when sc->done)
template <typename T>
int cg_start(amgh_problem *p, RedSlot &red, int n, const T *f, T *x, T *r, CgScal *sc,
             double tol, int maxit, int zero_x);
template <typename T, typename Z>
int cg2_spmv(amgh_problem *p, RedSlot &red, const DevCsr &a, const Z *z, const T *r, T *s, CgScal *sc, int timed);
template <typename T, typename Z>
int cg2_update(amgh_problem *p, RedSlot &red, int n, Z *z, const T *s, T *pv, T *q, T *x, T *r, float *r32,
               const double *invd, CgScal *sc, T *vd = nullptr, T *vx = nullptr, const T *vinvd = nullptr,
               double c0 = 0.0);
int cg_update_outer(amgh_problem *p, RedSlot &red, int n, double *x, double *r, const double *pv, const double *q,
                    CgScal *sc);
// double-float CG (vectors stored as hi / lo FP32 halves of an FP64-sized buffer)
int dfcg_start(amgh_problem *p, RedSlot &red, int n, const double *f, double *x, double *r, CgScal *sc, double tol,
               int maxit);
int dfcg_spmv(amgh_problem *p, RedSlot &red, const DevCsr &a, const float *z, const double *r, double *s,
              CgScal *sc, int timed);
// invd32 alone: Jacobi, z = D^-1 r written over z; invd32 with vd, vx: the
// V-cycle's first smoother step on the new r written to vd and vx
int dfcg_update(amgh_problem *p, RedSlot &red, int n, const float *z, const double *s, double *pv, double *q,
                double *x, double *r, CgScal *sc, const float *invd32 = nullptr, float *vd = nullptr,
                float *vx = nullptr, double c0 = 0.0);
// z = D^-1 r (FP32) from the hi half of a double-float r
int dfcg_jacobi(amgh_problem *p, int n, const double *r, const float *invd32, float *z);
int df_to_double(amgh_problem *p, int n, const double *x, const CgScal *sc, double *y);
int ref_start(amgh_problem *p, RedSlot &red, int n, const double *f, double *y, double *r,
              CgScal *rs, double tol, int maxit);
int ref_to32(amgh_problem *p, RedSlot &red, int n, const double *r, float *r32, CgScal *rs);
int ref_update(amgh_problem *p, RedSlot &red, const DevCsr &a, const double *f, double *y,
               const float *e32, double *r, CgScal *rs);
int vec_axpby(amgh_problem *p, int n, double a, const double *x, double b, const double *y,
              double *out);
int vec_fill(amgh_problem *p, int n, double v, double *x);
int vec_dot(amgh_problem *p, RedSlot &red, int n, const double *x, const double *y, double *out_dev);
int scatter_state(amgh_problem *p, int m, const int *vertex_of_state, const double *ys,
                  double *full, double scale_add_beta_u, const double *u);

// ------------------------------------------------------------------ assemble.cu
int assemble_full(amgh_problem *p);
int extract_sub(Arena &ar, const DevCsr &a, const int *rmap, int nr, const int *cmap, int nc,
                DevCsr &out, cudaStream_t s);

// ------------------------------------------------------------------ amg.cu
int amg_aggregate(amgh_problem *p, const DevCsr &a, double theta2, int *agg, int *nagg);
// aggressive first-level aggregation: the aggregates of a, aggregated once
// more on their tentative Galerkin matrix (threshold theta2 / 4), composed
int amg_aggregate_aggressive(amgh_problem *p, const DevCsr &a, double theta2, int *agg, int *nagg);
// the geometric hierarchy of a structured N x N square grid (aopts.geometric):
// fills S, St, P, Pt and the Galerkin A, M_y, K_N, M_u of every level, Ls = Lc
int geometric_hierarchy(amgh_problem *p);
int amg_prolongator(amgh_problem *p, Arena &ar, const DevCsr &a, const int *agg, int nagg,
                    int smooth, DevCsr &s);
int spgemm(amgh_problem *p, Arena &ar, const DevCsr &a, const DevCsr &b, DevCsr &c);
int symmetrize_upper(amgh_problem *p, DevCsr &c);
int galerkin(amgh_problem *p, Arena &ar, const DevCsr &rt, const DevCsr &a, const DevCsr &pm,
             int symmetric, DevCsr &c);
// the same Galerkin product for two matrices with one sparsity pattern, in one
// pass (results share row pointers and columns)
int galerkin_pair(amgh_problem *p, Arena &ar, const DevCsr &rt, const DevCsr &a1, const DevCsr &a2,
                  const DevCsr &pm, DevCsr &c1, DevCsr &c2);
int l1_invdiag(amgh_problem *p, const DevCsr &a, double *invd, float *invd32);
int diag_inv(amgh_problem *p, const DevCsr &a, double *invd);

// ------------------------------------------------------------------ dense.cu
int dense_from_csr(amgh_problem *p, const DevCsr &a, double *g);
int dense_spd_inverse(amgh_problem *p, double *g, int n, double *inv, int *info_dev);
int dense_coarse_hessian(amgh_problem *p, int c, const double *ainv, double *hinv);

// ------------------------------------------------------------------ solver.cu
int solver_alloc(amgh_problem *p);
void solver_free_graphs(amgh_problem *p);
int vcycle_run(amgh_problem *p, int l0, int prec32, const void *b, void *x, const int *skip);
int state_solve(amgh_problem *p, int l, const double *f, double *y, double tol, int64_t *iters);
int mass_solve(amgh_problem *p, int l, const double *b, double *x, int64_t *iters);
int hessian_level(amgh_problem *p, int l, const double *v, double *hv);
int mlas_Q(amgh_problem *p, int j, const double *b, double *u);
int mlas_R(amgh_problem *p, int j, const double *b, double *out);
int rhs_apply(amgh_problem *p, double *b);
int outer_solve(amgh_problem *p, const double *u0, double *u, const amgh_solve_opts *o, amgh_solve_info *info);
int sync_stream(amgh_problem *p);
// capture body() on the problem's private stream as a graph; replay it
int graph_capture(amgh_problem *p, const std::function<int()> &body, cudaGraphExec_t *exec, int *nodes);
int graph_replay(amgh_problem *p, cudaGraphExec_t exec, int nodes);
bool graphs_enabled(amgh_problem *p);

// ------------------------------------------------------------------ kuhn.cu
// matrix-free level-0 stiffness of the structured Kuhn cube
int kuhn_detect(amgh_problem *p);
int kuhn_apply(amgh_problem *p, int prec32, const void *x, void *y);
int kuhn_cheb_step(amgh_problem *p, const float *invd, const float *b, const float *x, float *d, float *xn,
                   double cdv, double crv, const int *skip);
int kuhn_residual(amgh_problem *p, const float *b, const float *x, float *r, const int *skip);

// ------------------------------------------------------------------ diag.cu
// a~_j (weighted 0) or a_j (weighted 1) by `iters` power iterations from v0
int aj_estimate(amgh_problem *p, int j, int weighted, int iters, const double *v0, double *est);

// ------------------------------------------------------------------ block.cu
// K columns (K = 2, 4, 8) advanced together; the column-major inputs hold
// ncols columns of n (or n_vertices) doubles
void block_free(amgh_problem *p);
int block_hessian_apply(amgh_problem *p, const double *u, double *hu, int ncols);
int block_precond_apply(amgh_problem *p, const double *r, double *z, int ncols);
// the first failing column's status; info accumulates outer_iters and the
// largest final_relres of the converged columns
int block_solve(amgh_problem *p, const double *yd, int ncols, double *u, const amgh_solve_opts &o,
                amgh_solve_info *info);

// per-launch timing (when enabled, outside graph capture) and byte counting of
// a solve-phase kernel of class cls; timer_end always counts the bytes
void timer_begin(amgh_problem *p, int cls);
void timer_end(amgh_problem *p, int cls, double bytes);
int timer_collect(amgh_problem *p);
// drop the pending timings recorded since `mark` (launches that the device
// skipped: the V-cycle of a CG iteration that converged)
void timer_drop_from(amgh_problem *p, size_t mark);
// bytes of one V-cycle at level l (value bytes vb) for the fused coarse launch
double vcycle_bytes(const amgh_problem *p, int l, int vb);
