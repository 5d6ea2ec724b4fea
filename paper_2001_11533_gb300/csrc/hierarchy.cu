// hierarchy.cu -- the two alternative hierarchies of the setup:
//
//   aggressive first-level coarsening (Sec. 5.1 uses it for the first level;
//   read for smoothed aggregation): the level-0 aggregates are aggregated
//   once more on their tentative Galerkin matrix S_hat^T A S_hat with the next
//   level's threshold, and every vertex takes the aggregate of its aggregate;
//
//   the geometric hierarchy of the structured N x N square grid (the
//   comparison of Sec. 5.4, Table 5): every other grid line, P1
//   interpolation on the (i,j)-(i+1,j+1) diagonal split:
//     (2I, 2J)     <- (I, J)                        weight 1
//     (2I+1, 2J)   <- (I, J), (I+1, J)              weights 1/2
//     (2I, 2J+1)   <- (I, J), (I, J+1)              weights 1/2
//     (2I+1, 2J+1) <- (I, J), (I+1, J+1)            weights 1/2
//   on all vertices for the control space (P_j) and restricted to interior
//   rows and columns for the state space (S_j).
// Both produce the same integers and values as the oracle's definitions, so
// the hierarchies stay bit-exact.
#include <math.h>

#include "internal.cuh"
#include "util.cuh"

__global__ void k_compose(int n, const int *__restrict__ agg1, const int *__restrict__ agg2, int *__restrict__ agg)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) agg[i] = agg2[agg1[i]];
}

int amg_aggregate_aggressive(amgh_problem *p, const DevCsr &a, double theta2, int *agg, int *nagg)
{
    cudaStream_t s = p->stream;
    const int n = a.rows;
    Scratch sc;
    int *agg1 = nullptr, *agg2 = nullptr;
    TRY(sc.alloc(&agg1, n));
    int n1 = 0, n2 = 0;
    TRY(amg_aggregate(p, a, theta2, agg1, &n1));
    Arena tmp;
    DevCsr sh, sht, t;
    int st = amg_prolongator(p, tmp, a, agg1, n1, 0, sh);
    if (!st) st = csr_transpose(tmp, sh, sht, s);
    if (!st) st = galerkin(p, tmp, sht, a, sh, 1, t);
    if (!st) st = sc.alloc(&agg2, n1);
    if (!st) st = amg_aggregate(p, t, theta2 * 0.25, agg2, &n2);
    if (!st) {
        k_compose<<<ceil_div(n, 256), 256, 0, s>>>(n, agg1, agg2, agg);
        cudaError_t e = cudaGetLastError();
        amgh_count_launch();
        if (e != cudaSuccess) {
            amgh_note_error((int)e, __FILE__, __LINE__);
            st = AMGH_ERR_CUDA;
        }
    }
    if (!st && cudaStreamSynchronize(s) != cudaSuccess) st = AMGH_ERR_CUDA;
    tmp.free_all();
    *nagg = n2;
    return st;
}

// ------------------------------------------------------------------ geometric
// 1 if a vertex of the N x N grid is Dirichlet exactly when it is on the boundary
__global__ void k_grid_check(int N, const int *__restrict__ state_of_vertex, int *__restrict__ bad)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N * N) return;
    int i = v % N, j = v / N;
    bool interior = i > 0 && j > 0 && i < N - 1 && j < N - 1;
    if (interior != (state_of_vertex[v] >= 0)) atomicOr(bad, 1);
}

// interior numbering of the N x N grid (row by row), -1 on the boundary
__global__ void k_grid_interior(int N, int *__restrict__ map)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N * N) return;
    int i = v % N, j = v / N;
    bool interior = i > 0 && j > 0 && i < N - 1 && j < N - 1;
    map[v] = interior ? (i - 1) + (N - 2) * (j - 1) : -1;
}

// CSR of the interpolation from the (N+1)/2 grid: one entry for a vertex on
// both even lines, two otherwise; row v starts at 2v minus the number of
// one-entry rows before it (rows with i and j even), computed in closed form
__device__ __forceinline__ int geo_row_start(int N, int v)
{
    int i = v % N, j = v / N;
    int ne = (N + 1) / 2;                                  // even i per row
    int singles = (j + 1) / 2 * ne + (j % 2 == 0 ? (i + 1) / 2 : 0); // even-even rows before v
    return 2 * v - singles;
}

__global__ void k_geo_interp(int N, int *__restrict__ rp, int *__restrict__ ci, double *__restrict__ v)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = N * N, Nc = (N + 1) / 2;
    if (r > n) return;
    rp[r] = r == n ? geo_row_start(N, n - 1) + 1 : geo_row_start(N, r);
    if (r == n) return;
    int i = r % N, j = r / N, I = i / 2, J = j / 2, k = geo_row_start(N, r);
    if (i % 2 == 0 && j % 2 == 0) {
        ci[k] = I + Nc * J;
        v[k] = 1.0;
    } else {
        ci[k] = I + Nc * J;
        v[k] = 0.5;
        ci[k + 1] = (I + (i % 2)) + Nc * (J + (j % 2));
        v[k + 1] = 0.5;
    }
}

int geometric_hierarchy(amgh_problem *p)
{
    const amgh_amg_opts &o = p->aopts;
    cudaStream_t s = p->stream;
    Arena &ar = p->harena;
    int N = (int)llround(sqrt((double)p->n));
    if (p->dim != 2 || (int64_t)N * N != p->n || N < 3) {
        amgh_note_msg("geometric hierarchy: the mesh is not an N x N square grid");
        return AMGH_ERR_INVALID_ARG;
    }
    {
        Scratch sc;
        int *bad = nullptr;
        TRY(sc.alloc(&bad, 1));
        CU(cudaMemsetAsync(bad, 0, sizeof(int), s));
        k_grid_check<<<ceil_div(p->n, 256), 256, 0, s>>>(N, p->state_of_vertex, bad);
        LAUNCH_CHECK();
        int h = 0;
        CU(cudaMemcpyAsync(&h, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        if (h) {
            amgh_note_msg("geometric hierarchy: the Dirichlet vertices are not the grid's boundary");
            return AMGH_ERR_INVALID_ARG;
        }
    }
    p->Ls = p->Lc = 1;
    for (int l = 0; l + 1 < o.max_levels && N >= 5 && N % 2 == 1 && p->cl[l].KN.rows > o.coarse_max; l++) {
        const int Nc = (N + 1) / 2;
        Scratch sc;
        int *fmap = nullptr, *cmap = nullptr;
        TRY(sc.alloc(&fmap, (int64_t)N * N));
        TRY(sc.alloc(&cmap, (int64_t)Nc * Nc));
        k_grid_interior<<<ceil_div((int64_t)N * N, 256), 256, 0, s>>>(N, fmap);
        LAUNCH_CHECK();
        k_grid_interior<<<ceil_div((int64_t)Nc * Nc, 256), 256, 0, s>>>(Nc, cmap);
        LAUNCH_CHECK();
        StateLevel &S = p->sl[l];
        CtrlLevel &C = p->cl[l];
        DevCsr &P = C.P;
        P.rows = N * N;
        P.cols = Nc * Nc;
        P.nnz = 2 * N * N - ((N + 1) / 2) * ((N + 1) / 2);
        TRY(ar.alloc(&P.rp, (int64_t)N * N + 1));
        TRY(ar.alloc(&P.ci, P.nnz));
        TRY(ar.alloc(&P.v, P.nnz));
        k_geo_interp<<<ceil_div((int64_t)N * N + 1, 256), 256, 0, s>>>(N, P.rp, P.ci, P.v);
        LAUNCH_CHECK();
        TRY(extract_sub(ar, P, fmap, (N - 2) * (N - 2), cmap, (Nc - 2) * (Nc - 2), S.S, s));
        TRY(csr_transpose(ar, S.S, S.St, s));
        TRY(galerkin_pair(p, ar, S.St, S.A, S.My, S.S, p->sl[l + 1].A, p->sl[l + 1].My));
        TRY(csr_transpose(ar, P, C.Pt, s));
        TRY(galerkin_pair(p, ar, C.Pt, C.KN, C.Mu, P, p->cl[l + 1].KN, p->cl[l + 1].Mu));
        S.nagg = (Nc - 2) * (Nc - 2);
        C.nagg = Nc * Nc;
        p->Ls = p->Lc = l + 2;
        N = Nc;
    }
    return AMGH_OK;
}
