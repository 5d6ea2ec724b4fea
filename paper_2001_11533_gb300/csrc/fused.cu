// fused.cu -- the coarse end of the FP32 V-cycle in one launch.
//
// Below a few hundred thousand rows a V-cycle level is a handful of kernels
// of a few microseconds each, too small to fill the GPU and each paying a
// launch.  From the first level small enough down to the dense coarsest
// solve, the whole V-cycle (pre-smoothing, residual, restriction, dense
// solve, prolongation, post-smoothing at every level, in the order of vcyc in
// solver.cu) runs in one launch, in one of two scopes:
//   cluster (fuse_coarse = 1): one thread-block cluster of 8 or 16 CTAs for
//     levels of at most FUSE_MAX_ROWS rows, phases separated by the hardware
//     cluster barrier;
//   grid (fuse_coarse = 2): a cooperative launch of one 1024-thread block per
//     SM for levels of at most GRID_FUSE_MAX_ROWS rows, phases separated by a
//     software grid barrier (an arrival counter and a generation word in
//     global memory, gridbar.cuh) whose wait is bounded: a block that gives
//     up raises the timeout flag and every block leaves at its next barrier,
//     and the host reports AMGH_ERR_TIMEOUT.
// Each barrier also orders the global memory writes of one phase before the
// reads of the next.  Every row does the same arithmetic as in the
// level-by-level kernels (the row sums and the point-wise helpers of
// spmv.cuh), so the result is the same to the bit.  Vectors written inside the
// kernel are read through L2 (ld.global.cg); the matrices, read-only, through
// the ordinary path.
#include <cooperative_groups.h>

#include "gridbar.cuh"
#include "internal.cuh"
#include "spmv.cuh"

namespace cg = cooperative_groups;

#define FUSE_TPB 1024
#define FUSE_MAX_ROWS 32768
#define GRID_FUSE_MAX_ROWS 262144
struct ClusterScope {
    __device__ bool sync()
    {
        cg::this_cluster().sync();
        return true;
    }
};
struct GridScope {
    GridBar *gb;
    unsigned nb;
    __device__ bool sync() { return grid_sync(gb, nb); }
};

struct FusedLevel {
    MatView<float> A, St, S; // St: rows of level l+1; S: rows of level l
    const float *invd;
    float *b, *x, *x2, *d, *r;
    int n;
};

struct FusedCycle {
    int c0, last, nsteps;
    float cd[16], cr[16];
    const float *cinv; // FP32 inverse of the coarsest matrix, rows padded to cld
    int cld, cn, cvec; // cvec: the coarsest level's b is 16-byte aligned
    FusedLevel lv[AMGH_MAXL];
};

// Each phase walks the rows of one level with all threads of the cluster:
// TPR consecutive threads per row, the same number of sweeps for every
// thread (rows past the end compute nothing), so warps stay converged.
template <int TPR, typename F>
__device__ __forceinline__ void sweep_rows(int n, int g, int T, F body)
{
    int slots = n * TPR;
    for (int base = 0; base < slots; base += T) body((base + g) / TPR);
}

#define TPR_DISPATCH(tpr, CALL)                                                                                   \
    switch (tpr) {                                                                                                \
    case 2: CALL(2); break;                                                                                       \
    case 4: CALL(4); break;                                                                                       \
    case 8: CALL(8); break;                                                                                       \
    case 16: CALL(16); break;                                                                                     \
    case 32: CALL(32); break;                                                                                     \
    default: CALL(1); break;                                                                                      \
    }

template <int TPR>
__device__ void ph_cheb(const FusedLevel &L, const float *b, const float *x, float *xn, float cdv, float crv, int g,
                        int T)
{
    sweep_rows<TPR>(L.n, g, T, [&](int r) {
        bool lead = r < L.n && row_leader<TPR>();
        float br = 0.f, ir = 0.f, dr = 0.f, xr = 0.f;
        if (lead) {
            br = __ldcg(b + r);
            ir = L.invd[r];
            dr = __ldcg(L.d + r);
            xr = __ldcg(x + r);
        }
        float ax = row_sum<float, TPR>(L.A, r, [&](int c) { return __ldcg(x + c); });
        if (lead) {
            float dn, xv;
            cheb_point(br, ax, ir, dr, xr, cdv, crv, dn, xv);
            L.d[r] = dn;
            xn[r] = xv;
        }
    });
}

template <int TPR>
__device__ void ph_residual(const FusedLevel &L, const float *b, const float *x, int g, int T)
{
    sweep_rows<TPR>(L.n, g, T, [&](int r) {
        bool lead = r < L.n && row_leader<TPR>();
        float br = lead ? __ldcg(b + r) : 0.f;
        float ax = row_sum<float, TPR>(L.A, r, [&](int c) { return __ldcg(x + c); });
        if (lead) L.r[r] = rsub(br, ax);
    });
}

// b_c = S^T r; with first, also the coarse level's first smoother step
// d_c = x2_c = c0 D_c^-1 b_c
template <int TPR>
__device__ void ph_restrict(const FusedLevel &L, const FusedLevel &C, int first, float c0, int g, int T)
{
    sweep_rows<TPR>(C.n, g, T, [&](int i) {
        float bv = row_sum<float, TPR>(L.St, i, [&](int c) { return __ldcg(L.r + c); });
        if (i < C.n && row_leader<TPR>()) {
            C.b[i] = bv;
            if (first) {
                float v = cheb_first_point(bv, C.invd[i], c0);
                C.d[i] = v;
                C.x2[i] = v;
            }
        }
    });
}

template <int TPR>
__device__ void ph_prolong(const FusedLevel &L, const float *e, float *x, int g, int T)
{
    sweep_rows<TPR>(L.n, g, T, [&](int i) {
        float v = row_sum<float, TPR>(L.S, i, [&](int c) { return __ldcg(e + c); });
        if (i < L.n && row_leader<TPR>()) x[i] = radd(__ldcg(x + i), v);
    });
}

template <typename Scope>
__device__ __forceinline__ void vcycle_body(const FusedCycle *__restrict__ fc, const float *b0, float *x0,
                                            int preinit, int g, int T, Scope &cl)
{
    const int c0 = fc->c0, last = fc->last, ns = fc->nsteps;
    float *cur[AMGH_MAXL], *nxt[AMGH_MAXL];
    // down-sweep: levels c0 .. last-1
    for (int l = c0; l < last; l++) {
        const FusedLevel &L = fc->lv[l];
        const float *b = l == c0 ? b0 : L.b;
        float *x = l == c0 ? x0 : L.x;
        float *c = x == L.x ? L.x2 : L.x, *nx = x;
        int pre = l == c0 ? preinit : 1;
        if (!pre) {
            for (int i = g; i < L.n; i += T) {
                float v = cheb_first_point(__ldcg(b + i), L.invd[i], fc->cr[0]);
                L.d[i] = v;
                c[i] = v;
            }
            if (!cl.sync()) return;
        }
        for (int s = 1; s < ns; s++) {
#define CALL(K) ph_cheb<K>(L, b, c, nx, fc->cd[s], fc->cr[s], g, T)
            TPR_DISPATCH(L.A.tpr, CALL)
#undef CALL
            if (!cl.sync()) return;
            float *t = c;
            c = nx;
            nx = t;
        }
#define CALL(K) ph_residual<K>(L, b, c, g, T)
        TPR_DISPATCH(L.A.tpr, CALL)
#undef CALL
        if (!cl.sync()) return;
        const FusedLevel &C = fc->lv[l + 1];
#define CALL(K) ph_restrict<K>(L, C, l + 1 < last, fc->cr[0], g, T)
        TPR_DISPATCH(L.St.tpr, CALL)
#undef CALL
        if (!cl.sync()) return;
        cur[l] = c;
        nxt[l] = nx;
    }
    // coarsest: x = A^-1 b, one warp per row
    {
        const FusedLevel &C = fc->lv[last];
        int lane = g & 31;
        for (int w = g >> 5; w < fc->cn; w += T >> 5) {
            float acc = fc->cvec ? dense_row32<true>(fc->cinv, fc->cld, w, fc->cn, C.b, lane)
                                 : dense_row32<false>(fc->cinv, fc->cld, w, fc->cn, C.b, lane);
            if (lane == 0) C.x[w] = acc;
        }
        if (!cl.sync()) return;
    }
    // up-sweep: levels last-1 .. c0
    for (int l = last - 1; l >= c0; l--) {
        const FusedLevel &L = fc->lv[l];
        const float *b = l == c0 ? b0 : L.b;
        float *x = l == c0 ? x0 : L.x;
        float *c = cur[l], *nx = nxt[l];
#define CALL(K) ph_prolong<K>(L, fc->lv[l + 1].x, c, g, T)
        TPR_DISPATCH(L.S.tpr, CALL)
#undef CALL
        if (!cl.sync()) return;
        for (int s = 0; s < ns; s++) {
#define CALL(K) ph_cheb<K>(L, b, c, nx, s == 0 ? 0.f : fc->cd[s], fc->cr[s], g, T)
            TPR_DISPATCH(L.A.tpr, CALL)
#undef CALL
            if (!cl.sync()) return;
            float *t = c;
            c = nx;
            nx = t;
        }
        if (c != x) {
            for (int i = g; i < L.n; i += T) x[i] = __ldcg(c + i);
            if (!cl.sync()) return;
        }
    }
}

__global__ void __launch_bounds__(FUSE_TPB, 1)
    k_vcycle_fused(const FusedCycle *__restrict__ fc, const float *b0, float *x0, int preinit,
                   const int *__restrict__ skip)
{
    if (skip && *skip) return; // the flag is not written while this kernel runs: uniform
    cg::cluster_group cl = cg::this_cluster();
    ClusterScope sc;
    vcycle_body(fc, b0, x0, preinit, (int)(cl.block_rank() * blockDim.x + threadIdx.x),
                (int)(cl.num_blocks() * blockDim.x), sc);
}

// the same V-cycle over the whole GPU: a cooperative launch of gridDim.x
// blocks, all resident at once, phases separated by grid_sync
__global__ void __launch_bounds__(FUSE_TPB, 1)
    k_vcycle_grid(const FusedCycle *__restrict__ fc, const float *b0, float *x0, int preinit,
                  const int *__restrict__ skip, GridBar *gb)
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (skip && *skip) return; // uniform: the flag is not written while this kernel runs
    GridScope sc{gb, gridDim.x};
    vcycle_body(fc, b0, x0, preinit, (int)(blockIdx.x * blockDim.x + threadIdx.x), (int)(gridDim.x * blockDim.x),
                sc);
}

// Fill the level table and pick the cluster size (16 CTAs where the GPU can
// co-schedule them, else 8).  p->fuse_c0 = -1 disables the fused path.
int fused_setup(amgh_problem *p)
{
    p->fuse_c0 = -1;
    p->fuse_cluster = 0;
    p->fuse_grid = 0;
    p->fuse_bar = nullptr;
    int mode = p->aopts.fuse_coarse;
    // handles sharing a hierarchy run concurrently in the batch runtime: two
    // grid-wide launches there could each hold part of the GPU, so they take
    // the level-by-level kernels
    if (mode == 2 && p->parent) mode = 0;
    if (!mode || p->Ls < 2) return AMGH_OK;
    const int maxrows = mode == 2 ? GRID_FUSE_MAX_ROWS : FUSE_MAX_ROWS;
    int c0 = -1;
    for (int l = 0; l < p->Ls - 1; l++)
        if (p->sl[l].A.rows <= maxrows) {
            c0 = l;
            break;
        }
    if (c0 < 0 || p->nsteps > 16 || !p->Acoarse.inv32) return AMGH_OK;
    FusedCycle h;
    memset(&h, 0, sizeof(h));
    h.c0 = c0;
    h.last = p->Ls - 1;
    h.nsteps = p->nsteps;
    for (int s = 0; s < p->nsteps; s++) {
        h.cd[s] = (float)p->cd[s];
        h.cr[s] = (float)p->cr[s];
    }
    h.cinv = p->Acoarse.inv32;
    h.cld = p->Acoarse.ld32;
    h.cn = p->Acoarse.n;
    h.cvec = ((uintptr_t)p->sl[h.last].fb & 15) == 0;
    for (int l = c0; l <= h.last; l++) {
        StateLevel &S = p->sl[l];
        FusedLevel &L = h.lv[l];
        L.A = view<float>(S.A);
        if (l < h.last) {
            L.St = view<float>(S.St);
            L.S = view<float>(S.S);
        }
        L.invd = S.invd32;
        L.b = S.fb;
        L.x = S.fx;
        L.x2 = S.fx2;
        L.d = S.fd;
        L.r = S.fr;
        L.n = S.A.rows;
    }
    FusedCycle *dev = nullptr;
    TRY(p->harena.alloc(&dev, 1));
    CU(cudaMemcpyAsync(dev, &h, sizeof(h), cudaMemcpyHostToDevice, p->stream));
    CU(cudaStreamSynchronize(p->stream));
    if (mode == 2) {
        // one block per SM, if one fits (cooperative launch: all resident)
        int dev_id = 0, sms = 0, per_sm = 0;
        CU(cudaGetDevice(&dev_id));
        CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev_id));
        CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_vcycle_grid, FUSE_TPB, 0));
        if (per_sm < 1 || sms < 1) return AMGH_OK;
        GridBar *bar = nullptr;
        TRY(p->harena.alloc(&bar, 1));
        CU(cudaMemsetAsync(bar, 0, sizeof(GridBar), p->stream));
        CU(cudaStreamSynchronize(p->stream));
        p->fuse_table = dev;
        p->fuse_bar = bar;
        p->fuse_grid = sms;
        p->fuse_c0 = c0;
        return AMGH_OK;
    }
    // cluster size: 16 if it can be scheduled, else 8
    int cluster = 0;
    for (int want : {16, 8}) {
        if (want > 8 &&
            cudaFuncSetAttribute(k_vcycle_fused, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = want;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(want, 1, 1);
        cfg.blockDim = dim3(FUSE_TPB, 1, 1);
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, k_vcycle_fused, &cfg) == cudaSuccess && nclusters >= 1) {
            cluster = want;
            break;
        }
        cudaGetLastError();
    }
    if (!cluster) return AMGH_OK; // no cluster launch on this device: level-by-level kernels
    p->fuse_table = dev;
    p->fuse_cluster = cluster;
    p->fuse_c0 = c0;
    return AMGH_OK;
}

int grid_timeout_check(amgh_problem *p)
{
    int h = 0;
    CU(cudaMemcpyFromSymbolAsync(&h, g_gridbar_timeout, sizeof(int), 0, cudaMemcpyDeviceToHost, p->stream));
    CU(cudaStreamSynchronize(p->stream));
    if (!h) return AMGH_OK;
    int zero = 0;
    CU(cudaMemcpyToSymbolAsync(g_gridbar_timeout, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, p->stream));
    if (p->fuse_bar) CU(cudaMemsetAsync(p->fuse_bar, 0, sizeof(GridBar), p->stream));
    CU(cudaStreamSynchronize(p->stream));
    return AMGH_ERR_TIMEOUT;
}

int fused_vcycle(amgh_problem *p, const float *b, float *x, int preinit, const int *skip)
{
    if (p->fuse_grid > 0) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.gridDim = dim3(p->fuse_grid, 1, 1);
        cfg.blockDim = dim3(FUSE_TPB, 1, 1);
        cfg.stream = p->stream;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        timer_begin(p, KC_COARSE);
        CU(cudaLaunchKernelEx(&cfg, k_vcycle_grid, (const FusedCycle *)p->fuse_table, b, x, preinit, skip,
                              (GridBar *)p->fuse_bar));
        amgh_count_launch();
        timer_end(p, KC_COARSE, vcycle_bytes(p, p->fuse_c0, 4));
        return AMGH_OK;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = p->fuse_cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(p->fuse_cluster, 1, 1);
    cfg.blockDim = dim3(FUSE_TPB, 1, 1);
    cfg.stream = p->stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    timer_begin(p, KC_COARSE);
    CU(cudaLaunchKernelEx(&cfg, k_vcycle_fused, (const FusedCycle *)p->fuse_table, b, x, preinit, skip));
    amgh_count_launch();
    timer_end(p, KC_COARSE, vcycle_bytes(p, p->fuse_c0, 4));
    return AMGH_OK;
}

// poll limit of the grid barrier waits of the fused V-cycle (-1: default)
int fused_set_grid_polls(int polls)
{
    int v = polls < 0 ? GRIDBAR_POLLS : polls;
    CU(cudaMemcpyToSymbol(g_gridbar_polls, &v, sizeof(int)));
    return AMGH_OK;
}
