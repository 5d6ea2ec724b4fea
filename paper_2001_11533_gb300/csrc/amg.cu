// amg.cu -- smoothed-aggregation setup on the device (Sec. 3.1; Eq.
// coarsestiffness, coarsemass): strength graph, distance-2 maximal
// independent set, aggregates, smoothed prolongator and Galerkin products.
//
// Everything that decides an integer (a strength test, a root, an aggregate
// id, a sparsity pattern) is computed so that it equals the sequential
// definition exactly:
//   strength   j ~ i iff a_ij*a_ij >= theta^2 * (a_ii*a_jj), each product
//              rounded separately (no fused multiply-add);
//   roots      the greedy distance-2 independent set in decreasing splitmix64
//              priority, obtained here by parallel rounds with fixed
//              priorities (a vertex whose priority is the largest among the
//              undecided vertices within distance 2 becomes a root; vertices
//              within distance 2 of a root leave) -- with fixed priorities
//              this returns exactly the greedy set;
//   aggregates phase 1 = root + strong neighbours (id = root rank), phase 2 =
//              strongest phase-1 neighbour (ties to the smaller id), phase 3 =
//              singletons in ascending vertex order;
//   products   C_iJ = sum over A's row i in ascending column order of
//              A_ij * B_jJ (rounded products, added in that order), so the
//              Galerkin matrices -- and the strength tests of the next level
//              -- are the same bits on every run.
#include <stdio.h>

#include "internal.cuh"
#include "util.cuh"

#define MAXROW 256

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ uint64_t splitmix_prio(uint64_t i)
{
    // splitmix64 output function (Steele, Lea & Flood 2014) of (seed ^ i)
    uint64_t z = 0x9E3779B97F4A7C15ULL ^ i;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double row_diag(int i, const int *__restrict__ rp, const int *__restrict__ ci,
                                           const double *__restrict__ v)
{
    int lo = rp[i], hi = rp[i + 1] - 1;
    while (lo <= hi) {
        int mid = (lo + hi) >> 1;
        int c = ci[mid];
        if (c == i) return v[mid];
        if (c < i) lo = mid + 1;
        else hi = mid - 1;
    }
    return 0.0;
}

__global__ void k_diag(int n, const int *__restrict__ rp, const int *__restrict__ ci, const double *__restrict__ v,
                       double *__restrict__ d)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) d[i] = row_diag(i, rp, ci, v);
}

// ------------------------------------------------------------------ strength
__global__ void k_strength(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                           const double *__restrict__ v, const double *__restrict__ d, double th2,
                           const int *__restrict__ srp, int *__restrict__ cnt, int *__restrict__ sci,
                           double *__restrict__ sv)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double di = d[i];
    int c = 0, pos = srp ? srp[i] : 0;
    for (int k = rp[i]; k < rp[i + 1]; k++) {
        int j = ci[k];
        if (j == i) continue;
        double a = v[k];
        if (__dmul_rn(a, a) >= __dmul_rn(th2, __dmul_rn(di, d[j]))) {
            if (srp) {
                sci[pos] = j;
                sv[pos] = a;
                pos++;
            }
            c++;
        }
    }
    if (!srp) cnt[i] = c;
}

// ------------------------------------------------------------------ MIS-2
// state: 0 undecided, 1 root, 2 removed
__global__ void k_mis_m1(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                         const unsigned char *__restrict__ st, int *__restrict__ m1)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    int best = -1;
    uint64_t bp = 0;
    if (st[v] == 0) {
        best = v;
        bp = splitmix_prio(v);
    }
    for (int k = rp[v]; k < rp[v + 1]; k++) {
        int u = ci[k];
        if (st[u] != 0) continue;
        uint64_t pu = splitmix_prio(u);
        if (best < 0 || pu > bp) {
            best = u;
            bp = pu;
        }
    }
    m1[v] = best;
}

__global__ void k_mis_select(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                             const int *__restrict__ m1, unsigned char *__restrict__ st)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n || st[v] != 0) return;
    int best = m1[v];
    uint64_t bp = best >= 0 ? splitmix_prio(best) : 0;
    for (int k = rp[v]; k < rp[v + 1]; k++) {
        int w = m1[ci[k]];
        if (w < 0) continue;
        uint64_t pw = splitmix_prio(w);
        if (best < 0 || pw > bp) {
            best = w;
            bp = pw;
        }
    }
    if (best == v) st[v] = 3; // new root this round (promoted below)
}

__global__ void k_mis_r1(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                         const unsigned char *__restrict__ st, unsigned char *__restrict__ r1)
{
    int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    unsigned char f = st[u] == 3;
    for (int k = rp[u]; k < rp[u + 1] && !f; k++) f = st[ci[k]] == 3;
    r1[u] = f;
}

__global__ void k_mis_r2(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                         const unsigned char *__restrict__ r1, unsigned char *__restrict__ st,
                         int *__restrict__ undecided)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    unsigned char s = st[v];
    if (s != 0) return;
    unsigned char f = r1[v];
    for (int k = rp[v]; k < rp[v + 1] && !f; k++) f = r1[ci[k]];
    if (f) st[v] = 2;
    else atomicAdd(undecided, 1);
}

__global__ void k_mis_promote(int n, unsigned char *__restrict__ st)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n && st[v] == 3) st[v] = 1;
}

// ------------------------------------------------------------------ aggregation phases
__global__ void k_root_flag(int n, const unsigned char *__restrict__ st, int *__restrict__ f)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) f[v] = st[v] == 1;
}

__global__ void k_phase1(int n, const int *__restrict__ srp, const int *__restrict__ sci,
                         const unsigned char *__restrict__ st, const int *__restrict__ rank, int *__restrict__ agg)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    if (st[v] == 1) {
        agg[v] = rank[v];
        return;
    }
    int a = -1;
    for (int k = srp[v]; k < srp[v + 1]; k++) {
        int u = sci[k];
        if (st[u] == 1) {
            a = rank[u];
            break;
        }
    }
    agg[v] = a;
}

__global__ void k_phase2(int n, const int *__restrict__ srp, const int *__restrict__ sci,
                         const double *__restrict__ sv, const int *__restrict__ agg1, int *__restrict__ agg2,
                         int *__restrict__ freeflag)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int a = agg1[i];
    if (a < 0) {
        double best = -1.0;
        int bid = -1;
        for (int k = srp[i]; k < srp[i + 1]; k++) {
            int aj = agg1[sci[k]];
            if (aj < 0) continue;
            double w = fabs(sv[k]);
            if (w > best || (w == best && aj < bid)) {
                best = w;
                bid = aj;
            }
        }
        a = bid;
    }
    agg2[i] = a;
    freeflag[i] = a < 0;
}

__global__ void k_phase3(int n, const int *__restrict__ fr, const int *__restrict__ frank, int nroots,
                         int *__restrict__ agg)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && fr[i]) agg[i] = nroots + frank[i];
}

// cap on the MIS-2 rounds (0: n + 1); lowered only by amgh_debug_limits
static int g_mis_round_cap = 0;
void mis_set_round_cap(int cap) { g_mis_round_cap = cap > 0 ? cap : 0; }
// aggregates a prolongator row may reach before k_prol hands it to
// k_prol_long (MAXROW; lowered only by amgh_debug_limits to test that path)
static int g_prol_rowcap = 0;
void prol_set_row_cap(int cap) { g_prol_rowcap = cap > 0 && cap < MAXROW ? cap : 0; }

int amg_aggregate(amgh_problem *p, const DevCsr &a, double theta2, int *agg, int *nagg_out)
{
    cudaStream_t s = p->stream;
    int n = a.rows;
    Scratch sc;
    double *d = nullptr, *sv = nullptr;
    int *cnt = nullptr, *srp = nullptr, *sci = nullptr;
    TRY(sc.alloc(&d, n));
    TRY(sc.alloc(&cnt, n + 1));
    TRY(sc.alloc(&srp, n + 1));
    int nb = ceil_div(n, 256);
    k_diag<<<nb, 256, 0, s>>>(n, a.rp, a.ci, a.v, d);
    LAUNCH_CHECK();
    k_strength<<<nb, 256, 0, s>>>(n, a.rp, a.ci, a.v, d, theta2, nullptr, cnt, nullptr, nullptr);
    LAUNCH_CHECK();
    int snnz = 0;
    TRY(exclusive_scan<int>(cnt, srp, n, s, &snnz));
    TRY(sc.alloc(&sci, snnz));
    TRY(sc.alloc(&sv, snnz));
    k_strength<<<nb, 256, 0, s>>>(n, a.rp, a.ci, a.v, d, theta2, srp, cnt, sci, sv);
    LAUNCH_CHECK();
    // MIS-2 by rounds
    unsigned char *st = nullptr, *r1 = nullptr;
    int *m1 = nullptr, *und = nullptr;
    TRY(sc.alloc(&st, n));
    TRY(sc.alloc(&r1, n));
    TRY(sc.alloc(&m1, n));
    TRY(sc.alloc(&und, 1));
    CU(cudaMemsetAsync(st, 0, n, s));
    int rounds = 0;
    for (;;) {
        CU(cudaMemsetAsync(und, 0, sizeof(int), s));
        k_mis_m1<<<nb, 256, 0, s>>>(n, srp, sci, st, m1);
        LAUNCH_CHECK();
        k_mis_select<<<nb, 256, 0, s>>>(n, srp, sci, m1, st);
        LAUNCH_CHECK();
        k_mis_r1<<<nb, 256, 0, s>>>(n, srp, sci, st, r1);
        LAUNCH_CHECK();
        k_mis_r2<<<nb, 256, 0, s>>>(n, srp, sci, r1, st, und);
        LAUNCH_CHECK();
        k_mis_promote<<<nb, 256, 0, s>>>(n, st);
        LAUNCH_CHECK();
        int h = 0;
        CU(cudaMemcpyAsync(&h, und, sizeof(int), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        rounds++;
        if (h == 0) break;
        // each round fixes at least one vertex, so n + 1 rounds always suffice
        if (rounds > (g_mis_round_cap > 0 ? g_mis_round_cap : n + 1)) return AMGH_ERR_TIMEOUT;
    }
    // phases
    int *flag = nullptr, *rank = nullptr, *agg1 = nullptr, *fr = nullptr, *frank = nullptr;
    TRY(sc.alloc(&flag, n + 1));
    TRY(sc.alloc(&rank, n + 1));
    TRY(sc.alloc(&agg1, n));
    TRY(sc.alloc(&fr, n + 1));
    TRY(sc.alloc(&frank, n + 1));
    k_root_flag<<<nb, 256, 0, s>>>(n, st, flag);
    LAUNCH_CHECK();
    int nroots = 0;
    TRY(exclusive_scan<int>(flag, rank, n, s, &nroots));
    k_phase1<<<nb, 256, 0, s>>>(n, srp, sci, st, rank, agg1);
    LAUNCH_CHECK();
    k_phase2<<<nb, 256, 0, s>>>(n, srp, sci, sv, agg1, agg, fr);
    LAUNCH_CHECK();
    int nfree = 0;
    TRY(exclusive_scan<int>(fr, frank, n, s, &nfree));
    if (nfree > 0) {
        k_phase3<<<nb, 256, 0, s>>>(n, fr, frank, nroots, agg);
        LAUNCH_CHECK();
    }
    CU(cudaStreamSynchronize(s));
    *nagg_out = nroots + nfree;
    return AMGH_OK;
}

// ------------------------------------------------------------------ prolongator
__global__ void k_rho(int n, const int *__restrict__ rp, const int *__restrict__ ci, const double *__restrict__ v,
                      unsigned long long *__restrict__ rho_bits)
{
    __shared__ unsigned long long wmax[32];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long b = 0;
    if (i < n) {
        double s = 0.0, aii = 0.0;
        for (int k = rp[i]; k < rp[i + 1]; k++) {
            s = __dadd_rn(s, fabs(v[k]));
            if (ci[k] == i) aii = v[k];
        }
        // non-negative doubles order like their bit patterns
        b = (unsigned long long)__double_as_longlong(__ddiv_rn(s, aii));
    }
    // one atomic per block: the maximum over bit patterns is the same in any order
    for (int o = 16; o; o >>= 1) {
        unsigned long long t = __shfl_xor_sync(0xffffffffu, b, o);
        b = t > b ? t : b;
    }
    int warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if ((threadIdx.x & 31) == 0) wmax[warp] = b;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < nw; w++) b = wmax[w] > b ? wmax[w] : b;
        atomicMax(rho_bits, b);
    }
}

// row i: columns {agg(j)}, values [agg(i)==J] - (omega/a_ii) * sum_{agg(j)=J} a_ij
__global__ void k_prol(int n, const int *__restrict__ rp, const int *__restrict__ ci, const double *__restrict__ v,
                       const int *__restrict__ agg, double omega, const int *__restrict__ prp,
                       int *__restrict__ cnt, int *__restrict__ pci, double *__restrict__ pv, int *__restrict__ bad,
                       int rowcap)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int cols[MAXROW];
    double acc[MAXROW];
    int c = 0;
    double aii = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; k++) {
        int J = agg[ci[k]];
        if (ci[k] == i) aii = v[k];
        int pos = c;
        bool found = false;
        for (int t = 0; t < c; t++) {
            if (cols[t] == J) {
                pos = t;
                found = true;
                break;
            }
            if (cols[t] > J) {
                pos = t;
                break;
            }
        }
        if (!found) {
            if (c >= rowcap) {
                // more aggregates than the register list holds: k_prol_long
                // takes the row (count pass: marked -1; fill pass: left to it)
                if (!prp) cnt[i] = -1;
                return;
            }
            for (int t = c; t > pos; t--) {
                cols[t] = cols[t - 1];
                acc[t] = acc[t - 1];
            }
            cols[pos] = J;
            acc[pos] = 0.0;
            c++;
        }
        acc[pos] = __dadd_rn(acc[pos], v[k]);
    }
    if (!prp) {
        cnt[i] = c;
        return;
    }
    double wi = __ddiv_rn(omega, aii);
    int ai = agg[i];
    int base = prp[i];
    for (int t = 0; t < c; t++) {
        double delta = cols[t] == ai ? 1.0 : 0.0;
        pci[base + t] = cols[t];
        pv[base + t] = __dsub_rn(delta, __dmul_rn(wi, acc[t]));
    }
}

// Rows of k_prol that reach more than MAXROW aggregates, one block per row:
// the row's (aggregate, entry) pairs are ranked in shared memory by aggregate
// and then entry position (a stable sort), after which one thread sums each
// aggregate's entries in entry order -- the order k_prol and the sequential
// definition use -- so the values are identical.  Rows longer than
// PROL_LONG_MAX entries raise `bad`.
#define PROL_LONG_MAX 8192
__global__ void __launch_bounds__(256)
    k_prol_long(const int *__restrict__ rows, int nrows, const int *__restrict__ rp, const int *__restrict__ ci,
                const double *__restrict__ v, const int *__restrict__ agg, double omega, const int *__restrict__ prp,
                int *__restrict__ cnt, int *__restrict__ pci, double *__restrict__ pv, int *__restrict__ bad)
{
    extern __shared__ __align__(16) unsigned char pl_sm[];
    if ((int)blockIdx.x >= nrows) return;
    const int i = rows[blockIdx.x];
    const int beg = rp[i], len = rp[i + 1] - beg;
    if (len > PROL_LONG_MAX) {
        if (threadIdx.x == 0) atomicOr(bad, 1);
        return;
    }
    double *sval = (double *)pl_sm;                  // values in sorted order
    int *key = (int *)(sval + PROL_LONG_MAX);         // aggregate of entry t
    int *skey = key + PROL_LONG_MAX;                  // aggregates in sorted order
    for (int t = threadIdx.x; t < len; t += blockDim.x) key[t] = agg[ci[beg + t]];
    __syncthreads();
    for (int t = threadIdx.x; t < len; t += blockDim.x) {
        const int kt = key[t];
        int r = 0;
        for (int u = 0; u < len; u++) {
            const int ku = key[u];
            r += (ku < kt) || (ku == kt && u < t);
        }
        skey[r] = kt;
        sval[r] = v[beg + t];
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    if (!prp) {
        int c = 0;
        for (int t = 0; t < len; t++) c += (t == 0 || skey[t] != skey[t - 1]);
        cnt[i] = c;
        return;
    }
    double aii = 0.0;
    for (int k = beg; k < beg + len; k++)
        if (ci[k] == i) aii = v[k];
    const double wi = __ddiv_rn(omega, aii);
    const int ai = agg[i];
    int out = prp[i];
    for (int t = 0; t < len;) {
        const int J = skey[t];
        double acc = 0.0;
        for (; t < len && skey[t] == J; t++) acc = __dadd_rn(acc, sval[t]);
        pci[out] = J;
        pv[out] = __dsub_rn(J == ai ? 1.0 : 0.0, __dmul_rn(wi, acc));
        out++;
    }
}

// rows with cnt[i] < 0 listed (any order: each row is handled alone)
__global__ void k_list_negative(int n, const int *__restrict__ cnt, int *__restrict__ list, int *__restrict__ nlist)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && cnt[i] < 0) list[atomicAdd(nlist, 1)] = i;
}

__global__ void k_tentative(int n, const int *__restrict__ agg, int *__restrict__ rp, int *__restrict__ ci,
                            double *__restrict__ v)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    rp[i] = i;
    if (i < n) {
        ci[i] = agg[i];
        v[i] = 1.0;
    }
}

int amg_prolongator(amgh_problem *p, Arena &ar, const DevCsr &a, const int *agg, int nagg, int smooth, DevCsr &S)
{
    cudaStream_t s = p->stream;
    int n = a.rows;
    S.rows = n;
    S.cols = nagg;
    int nb = ceil_div(n, 256);
    if (!smooth) {
        S.nnz = n;
        TRY(ar.alloc(&S.rp, n + 1));
        TRY(ar.alloc(&S.ci, n));
        TRY(ar.alloc(&S.v, n));
        k_tentative<<<ceil_div(n + 1, 256), 256, 0, s>>>(n, agg, S.rp, S.ci, S.v);
        LAUNCH_CHECK();
        CU(cudaStreamSynchronize(s));
        return AMGH_OK;
    }
    Scratch sc;
    unsigned long long *rho_bits = nullptr;
    int *cnt = nullptr, *bad = nullptr;
    TRY(sc.alloc(&rho_bits, 1));
    TRY(sc.alloc(&cnt, n + 1));
    TRY(sc.alloc(&bad, 1));
    CU(cudaMemsetAsync(rho_bits, 0, sizeof(unsigned long long), s));
    CU(cudaMemsetAsync(bad, 0, sizeof(int), s));
    k_rho<<<nb, 256, 0, s>>>(n, a.rp, a.ci, a.v, rho_bits);
    LAUNCH_CHECK();
    unsigned long long hb = 0;
    CU(cudaMemcpyAsync(&hb, rho_bits, sizeof(hb), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    double rho;
    memcpy(&rho, &hb, sizeof(double));
    if (!(rho > 0.0)) return AMGH_ERR_NUMERIC;
    double omega = 4.0 / (3.0 * rho);
    const int rowcap = g_prol_rowcap > 0 ? g_prol_rowcap : MAXROW;
    k_prol<<<ceil_div(n, 128), 128, 0, s>>>(n, a.rp, a.ci, a.v, agg, omega, nullptr, cnt, nullptr, nullptr, bad,
                                            rowcap);
    LAUNCH_CHECK();
    // rows over MAXROW aggregates go to the one-block-per-row kernel
    int *longrows = nullptr, *nlong_dev = nullptr;
    TRY(sc.alloc(&longrows, n));
    TRY(sc.alloc(&nlong_dev, 1));
    CU(cudaMemsetAsync(nlong_dev, 0, sizeof(int), s));
    k_list_negative<<<nb, 256, 0, s>>>(n, cnt, longrows, nlong_dev);
    LAUNCH_CHECK();
    int nlong = 0;
    CU(cudaMemcpyAsync(&nlong, nlong_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    const size_t long_smem = (size_t)PROL_LONG_MAX * (sizeof(double) + 2 * sizeof(int));
    if (nlong > 0) {
        CU(cudaFuncSetAttribute(k_prol_long, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)long_smem));
        k_prol_long<<<nlong, 256, long_smem, s>>>(longrows, nlong, a.rp, a.ci, a.v, agg, omega, nullptr, cnt, nullptr,
                                                  nullptr, bad);
        LAUNCH_CHECK();
    }
    int hbad = 0;
    CU(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (hbad) {
        amgh_note_msg("prolongator: a row of A has more than 8192 entries");
        return AMGH_ERR_INVALID_ARG;
    }
    TRY(ar.alloc(&S.rp, n + 1));
    int nnz = 0;
    TRY(exclusive_scan<int>(cnt, S.rp, n, s, &nnz));
    S.nnz = nnz;
    TRY(ar.alloc(&S.ci, nnz));
    TRY(ar.alloc(&S.v, nnz));
    k_prol<<<ceil_div(n, 128), 128, 0, s>>>(n, a.rp, a.ci, a.v, agg, omega, S.rp, cnt, S.ci, S.v, bad, rowcap);
    LAUNCH_CHECK();
    if (nlong > 0) {
        k_prol_long<<<nlong, 256, long_smem, s>>>(longrows, nlong, a.rp, a.ci, a.v, agg, omega, S.rp, cnt, S.ci,
                                                  S.v, bad);
        LAUNCH_CHECK();
    }
    CU(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (hbad) amgh_note_msg("prolongator: a row of A has more than 8192 entries");
    return hbad ? AMGH_ERR_INVALID_ARG : AMGH_OK;
}

// ------------------------------------------------------------------ SpGEMM
// C = A B for CSR matrices, every entry summed in the canonical order (A's
// row entries ascending, then B's row entries ascending; first product added
// to 0.0).  NV = 2 multiplies two pairs of matrices that share their patterns
// (A1, A2 with one pattern, B1, B2 with one pattern) in one pass, so the
// hashing is paid once for C1 = A1 B1 and C2 = A2 B2 (A and M_y, K_N and M_u
// in the Galerkin products).
//
// Candidate count of row i: u_i = sum over A's row i of the lengths of the
// B rows it selects.  Path of row i: 0 = one thread with a global hash table
// of 2^ceil(log2(2 u_i)) slots, 1 = one warp with a shared hash table
// (u_i <= WARP_TS / 2), 2 = one block with a dense shared accumulator over all
// columns (u_i > WARP_TS / 2, few columns), 3 = one block with a shared hash
// table (u_i > WARP_TS / 2, many columns, few rows).  Products with few rows
// (n <= WARP_PATH_MAX_ROWS) use the shared paths throughout.  In large
// products a thread per row with a global table wins while the tables stay
// small; rows with 64 < u_i <= WARP_TS / 2 are marked 4 and go to the warp
// path only if all such tables together would exceed GLOBAL_TABLE_MAX_BYTES
// (the 3D fine levels).
#define WARP_TS 1024
#define WARPS_PER_BLOCK 4
#define WARP_PATH_MAX_ROWS 65536
#define GLOBAL_TABLE_MAX_BYTES (8ll << 30)
#define DENSE_ROW_TPB 256
#define BH_TPB 256

template <int NV>
struct GemmVals {
    const double *a[NV];
    const double *b[NV];
};

template <int NV>
struct GemmOut {
    double *v[NV];
};

template <int NV>
struct Limits;
template <>
struct Limits<1> {
    static constexpr int dense_cols = 16384, bhash_u = 8192;
};
template <>
struct Limits<2> {
    static constexpr int dense_cols = 12288, bhash_u = 4096;
};

// set when a row reaches a SpGEMM path whose table it would overflow; the
// row is skipped and the host reports an error
__device__ int g_spgemm_bad = 0;

__device__ __forceinline__ unsigned hslot(int key, unsigned mask) { return ((unsigned)key * 2654435761u) & mask; }

// 0.0 + x for finite x (the first term of a sum that starts from +0): only -0
// changes, to +0; done on the bits, off the FP64 pipe
__device__ __forceinline__ double plus_zero(double x)
{
    return __double_as_longlong(x) == (long long)0x8000000000000000ull ? 0.0 : x;
}

__global__ void k_gemm_ub(int n, const int *__restrict__ arp, const int *__restrict__ aci,
                          const int *__restrict__ brp, long long *__restrict__ ub, int *__restrict__ path_of,
                          int small_n, int use_dense, int bhash_u, int *__restrict__ umax3,
                          unsigned long long *__restrict__ slots4)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    long long u = 0;
    for (int k = arp[i]; k < arp[i + 1]; k++) {
        int j = aci[k];
        u += brp[j + 1] - brp[j];
    }
    long long t = 2;
    while (t < 2 * u) t <<= 1;
    int path = 0;
    if (u <= WARP_TS / 2) path = small_n ? 1 : (u > 64 ? 4 : 0);
    else if (use_dense) path = 2;
    else if (small_n && u <= bhash_u) path = 3;
    path_of[i] = path;
    if (path == 3) atomicMax(umax3, (int)u);
    if (path == 4) atomicAdd(slots4, (unsigned long long)t);
    ub[i] = (u > 0 && (path == 0 || path == 4)) ? t : 0;
}

// settle the rows marked 4: warp path (no global table) or thread path
__global__ void k_gemm_settle(int n, int to_warp, int *__restrict__ path_of, long long *__restrict__ ub)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || path_of[i] != 4) return;
    path_of[i] = to_warp ? 1 : 0;
    if (to_warp) ub[i] = 0;
}

__global__ void k_is_path(int n, const int *__restrict__ path_of, int want, int *__restrict__ flag)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = path_of[i] == want;
}

__global__ void k_list(int n, const int *__restrict__ flag, const int *__restrict__ pos, int *__restrict__ list)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && flag[i]) list[pos[i]] = i;
}

// path 0: accumulate row i in canonical order in its global table; count uniques
template <int NV>
__global__ void k_gemm_hash(int n, const int *__restrict__ arp, const int *__restrict__ aci, GemmVals<NV> V,
                            const int *__restrict__ brp, const int *__restrict__ bci,
                            const long long *__restrict__ toff, const int *__restrict__ path_of,
                            int *__restrict__ tkey, GemmOut<NV> T, int *__restrict__ cnt)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || path_of[i]) return;
    long long base = toff[i];
    unsigned size = (unsigned)(toff[i + 1] - base);
    int c = 0;
    if (size > 0) {
        unsigned mask = size - 1;
        int *key = tkey + base; // all slots set to -1 by the caller
        for (int k = arp[i]; k < arp[i + 1]; k++) {
            int j = aci[k];
            double aij[NV];
#pragma unroll
            for (int q = 0; q < NV; q++) aij[q] = V.a[q][k];
            for (int e = brp[j]; e < brp[j + 1]; e++) {
                int J = bci[e];
                // the products before the probe loop, where the warp still runs
                // together: an FP64 warp instruction costs the same with one
                // active lane as with 32
                double prod[NV];
#pragma unroll
                for (int q = 0; q < NV; q++) prod[q] = __dmul_rn(aij[q], V.b[q][e]);
                unsigned h = hslot(J, mask);
                for (;;) {
                    int kk = key[h];
                    if (kk == J) {
#pragma unroll
                        for (int q = 0; q < NV; q++) T.v[q][base + h] = __dadd_rn(T.v[q][base + h], prod[q]);
                        break;
                    }
                    if (kk < 0) {
                        key[h] = J;
#pragma unroll
                        for (int q = 0; q < NV; q++) T.v[q][base + h] = plus_zero(prod[q]);
                        c++;
                        break;
                    }
                    h = (h + 1) & mask;
                }
            }
        }
    }
    cnt[i] = c;
}

// path 0 output: the table's entries in ascending column order, sorted in
// place in the output arrays (insertion sort)
template <int NV>
__device__ __forceinline__ void out_row_inplace(long long base, unsigned size, const int *__restrict__ tkey,
                                                const GemmOut<NV> &T, int b, int *__restrict__ cci,
                                                const GemmOut<NV> &C)
{
    int c = 0;
    for (unsigned u = 0; u < size; u++) {
        int key = tkey[base + u];
        if (key < 0) continue;
        int j = b + c - 1;
        while (j >= b && cci[j] > key) {
            cci[j + 1] = cci[j];
#pragma unroll
            for (int q = 0; q < NV; q++) C.v[q][j + 1] = C.v[q][j];
            j--;
        }
        cci[j + 1] = key;
#pragma unroll
        for (int q = 0; q < NV; q++) C.v[q][j + 1] = T.v[q][base + u];
        c++;
    }
}

template <int NV>
__global__ void k_gemm_out(int n, const long long *__restrict__ toff, const int *__restrict__ path_of,
                           const int *__restrict__ tkey, GemmOut<NV> T, const int *__restrict__ crp,
                           int *__restrict__ cci, GemmOut<NV> C)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || path_of[i]) return;
    long long base = toff[i];
    out_row_inplace<NV>(base, (unsigned)(toff[i + 1] - base), tkey, T, crp[i], cci, C);
}

// The same for products with short rows (on average at most OUT_AVG entries):
// each thread insertion-sorts (column, slot) pairs of its row in shared
// memory (thread t's k-th pair at [k][t], so a warp's accesses fall in
// distinct banks) and then writes every entry once; a row with more than
// OUT_CAP entries sorts in place.  Its shared memory lowers occupancy, so
// long-row products (3D) keep the kernel above.
#define OUT_TPB 128
#define OUT_CAP 48
#define OUT_AVG 24
template <int NV>
__global__ void __launch_bounds__(OUT_TPB)
    k_gemm_out_sm(int n, const long long *__restrict__ toff, const int *__restrict__ path_of,
                  const int *__restrict__ tkey, GemmOut<NV> T, const int *__restrict__ crp, int *__restrict__ cci,
                  GemmOut<NV> C)
{
    __shared__ int sk[OUT_CAP][OUT_TPB];
    __shared__ unsigned short ss[OUT_CAP][OUT_TPB];
    int t = threadIdx.x;
    int i = blockIdx.x * blockDim.x + t;
    if (i >= n || path_of[i]) return;
    long long base = toff[i];
    unsigned size = (unsigned)(toff[i + 1] - base);
    int b = crp[i], c = 0;
    if (crp[i + 1] - b > OUT_CAP || size > 65536) {
        out_row_inplace<NV>(base, size, tkey, T, b, cci, C);
        return;
    }
    for (unsigned u = 0; u < size; u++) {
        int key = tkey[base + u];
        if (key < 0) continue;
        int j = c - 1;
        while (j >= 0 && sk[j][t] > key) {
            sk[j + 1][t] = sk[j][t];
            ss[j + 1][t] = ss[j][t];
            j--;
        }
        sk[j + 1][t] = key;
        ss[j + 1][t] = (unsigned short)u;
        c++;
    }
    for (int k = 0; k < c; k++) {
        unsigned u = ss[k][t];
        cci[b + k] = sk[k][t];
#pragma unroll
        for (int q = 0; q < NV; q++) C.v[q][b + k] = T.v[q][base + u];
    }
}

// path 1: one warp per listed row.  Candidates are taken 32 at a time in
// canonical order; lanes holding the same column form a group
// (__match_any_sync) whose lowest lane finds / inserts the slot and adds the
// group's products in lane order -- so every entry receives its products in
// exactly the sequential order.  phase 0 counts, phase 1 writes the sorted row.
template <int NV>
__host__ __device__ constexpr size_t warp_smem_bytes()
{
    return (size_t)WARPS_PER_BLOCK * WARP_TS * (sizeof(int) + NV * sizeof(double)) +
           (size_t)WARPS_PER_BLOCK * 32 * NV * sizeof(double);
}

template <int NV>
__global__ void k_gemm_warp(int n, const int *__restrict__ arp, const int *__restrict__ aci, GemmVals<NV> V,
                            const int *__restrict__ brp, const int *__restrict__ bci, const int *__restrict__ list,
                            int phase, int *__restrict__ cnt, const int *__restrict__ crp, int *__restrict__ cci,
                            GemmOut<NV> C)
{
    extern __shared__ unsigned char smem_raw[];
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *keys = (int *)smem_raw + w * WARP_TS;
    double *vbase = (double *)((int *)smem_raw + WARPS_PER_BLOCK * WARP_TS);
    double *vals = vbase + (size_t)w * NV * WARP_TS; // [NV][WARP_TS]
    double *stage = vbase + (size_t)WARPS_PER_BLOCK * NV * WARP_TS + (size_t)w * NV * 32; // [NV][32]
    int li = blockIdx.x * WARPS_PER_BLOCK + w;
    if (li >= n) return; // warp-uniform; n = number of listed rows
    int i = list[li];
    // table of 2^ceil(log2(2u)) slots (u = candidate count of the row)
    int u = 0;
    for (int k = arp[i] + lane; k < arp[i + 1]; k += 32) {
        int j = aci[k];
        u += brp[j + 1] - brp[j];
    }
    for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
    unsigned ts = 2;
    while ((int)ts < 2 * u) ts <<= 1;
    if (ts > WARP_TS) { // warp-uniform
        if (lane == 0) atomicExch(&g_spgemm_bad, 1);
        return;
    }
    const unsigned mask = ts - 1;
    for (unsigned t = lane; t < ts; t += 32) keys[t] = -1;
    __syncwarp();
    for (int k = arp[i]; k < arp[i + 1]; k++) {
        int j = aci[k];
        double aij[NV];
#pragma unroll
        for (int q = 0; q < NV; q++) aij[q] = V.a[q][k];
        int qb = brp[j], qe = brp[j + 1];
        for (int q0 = qb; q0 < qe; q0 += 32) {
            int e = q0 + lane;
            bool valid = e < qe;
            int J = valid ? bci[e] : -1;
#pragma unroll
            for (int q = 0; q < NV; q++) stage[q * 32 + lane] = valid ? __dmul_rn(aij[q], V.b[q][e]) : 0.0;
            unsigned grp = __match_any_sync(0xffffffffu, J);
            __syncwarp();
            if (valid && lane == __ffs(grp) - 1) {
                unsigned h = hslot(J, mask);
                bool fresh = false;
                for (;;) {
                    int old = atomicCAS(&keys[h], -1, J);
                    if (old == -1) {
                        fresh = true;
                        break;
                    }
                    if (old == J) break;
                    h = (h + 1) & mask;
                }
#pragma unroll
                for (int q = 0; q < NV; q++) {
                    double acc = fresh ? 0.0 : vals[q * WARP_TS + h];
                    for (unsigned m = grp; m; m &= m - 1) acc = __dadd_rn(acc, stage[q * 32 + __ffs(m) - 1]);
                    vals[q * WARP_TS + h] = acc;
                }
            }
            __syncwarp();
        }
    }
    // compact the occupied slots to the front of the table
    int c = 0;
    for (unsigned t0 = 0; t0 < ts; t0 += 32) {
        unsigned t = t0 + lane;
        int key = t < ts ? keys[t] : -1;
        double val[NV];
#pragma unroll
        for (int q = 0; q < NV; q++) val[q] = t < ts ? vals[q * WARP_TS + t] : 0.0;
        unsigned occ = __ballot_sync(0xffffffffu, key >= 0);
        __syncwarp();
        if (key >= 0) {
            int pos = c + __popc(occ & ((1u << lane) - 1));
            keys[pos] = key; // pos <= t: never overwrites an unread slot
#pragma unroll
            for (int q = 0; q < NV; q++) vals[q * WARP_TS + pos] = val[q];
        }
        c += __popc(occ);
        __syncwarp();
    }
    if (phase == 0) {
        if (lane == 0) cnt[i] = c;
        return;
    }
    // rank of each key among the row's keys = its position in the sorted row
    int base = crp[i];
    for (int t = lane; t < c; t += 32) {
        int key = keys[t];
        int rank = 0;
        for (int v = 0; v < c; v++) rank += keys[v] < key;
        cci[base + rank] = key;
#pragma unroll
        for (int q = 0; q < NV; q++) C.v[q][base + rank] = vals[q * WARP_TS + t];
    }
}

// path 2: one block per listed row with a dense shared accumulator over all
// columns.  The row's products are taken one entry a_ik at a time (a barrier
// between entries) with row k of B spread over the threads; every column
// occurs once in a row of B, so each accumulator receives its products in the
// sequential order.  phase 0 counts the row's columns, phase 1 writes them in
// ascending order.
template <int NV>
__global__ void __launch_bounds__(DENSE_ROW_TPB)
    k_gemm_dense(int nlist, const int *__restrict__ list, int cols, const int *__restrict__ arp,
                 const int *__restrict__ aci, GemmVals<NV> V, const int *__restrict__ brp,
                 const int *__restrict__ bci, int phase, int *__restrict__ cnt, const int *__restrict__ crp,
                 int *__restrict__ cci, GemmOut<NV> C)
{
    extern __shared__ unsigned char smem_raw[];
    __shared__ int wsum[DENSE_ROW_TPB / 32];
    double *acc = (double *)smem_raw; // [NV][cols]
    unsigned char *seen = smem_raw + (size_t)NV * cols * sizeof(double);
    int i = list[blockIdx.x];
    int t = threadIdx.x, lane = t & 31, w = t >> 5;
    for (int J = t; J < cols; J += DENSE_ROW_TPB) {
#pragma unroll
        for (int q = 0; q < NV; q++) acc[(size_t)q * cols + J] = 0.0;
        seen[J] = 0;
    }
    __syncthreads();
    for (int k = arp[i]; k < arp[i + 1]; k++) {
        int j = aci[k];
        double aij[NV];
#pragma unroll
        for (int q = 0; q < NV; q++) aij[q] = V.a[q][k];
        for (int e = brp[j] + t; e < brp[j + 1]; e += DENSE_ROW_TPB) {
            int J = bci[e];
#pragma unroll
            for (int q = 0; q < NV; q++)
                acc[(size_t)q * cols + J] = __dadd_rn(acc[(size_t)q * cols + J], __dmul_rn(aij[q], V.b[q][e]));
            seen[J] = 1;
        }
        __syncthreads();
    }
    // each thread owns a contiguous run of columns; a block scan of the runs'
    // counts gives every column its position in the sorted row
    int per = (cols + DENSE_ROW_TPB - 1) / DENSE_ROW_TPB;
    int beg = t * per, end = min(beg + per, cols);
    int c = 0;
    for (int J = beg; J < end; J++) c += seen[J];
    int incl = c;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    int before = 0, total = 0;
    for (int q = 0; q < DENSE_ROW_TPB / 32; q++) {
        if (q < w) before += wsum[q];
        total += wsum[q];
    }
    if (phase == 0) {
        if (t == 0) cnt[i] = total;
        return;
    }
    int pos = crp[i] + before + incl - c;
    for (int J = beg; J < end; J++)
        if (seen[J]) {
            cci[pos] = J;
#pragma unroll
            for (int q = 0; q < NV; q++) C.v[q][pos] = acc[(size_t)q * cols + J];
            pos++;
        }
}

// path 3: one block per listed row with a shared hash table of ts slots; the
// products are taken as in path 2, then the occupied slots are compacted to
// the front (chunk by chunk: all reads of a chunk before its writes, which
// only land on slots already read) and sorted by column (bitonic network over
// the next power of two).  phase 0 counts, phase 1 writes the row.
template <int NV>
__global__ void __launch_bounds__(BH_TPB)
    k_gemm_bhash(int nlist, const int *__restrict__ list, int ts, const int *__restrict__ arp,
                 const int *__restrict__ aci, GemmVals<NV> V, const int *__restrict__ brp,
                 const int *__restrict__ bci, int phase, int *__restrict__ cnt, const int *__restrict__ crp,
                 int *__restrict__ cci, GemmOut<NV> C)
{
    extern __shared__ unsigned char smem_raw[];
    __shared__ int wcount[BH_TPB / 32];
    double *vals = (double *)smem_raw; // [NV][ts]
    int *keys = (int *)(vals + (size_t)NV * ts);
    const unsigned mask = (unsigned)ts - 1;
    int i = list[blockIdx.x];
    int t = threadIdx.x, lane = t & 31, w = t >> 5;
    if (t == 0) {
        long long u = 0;
        for (int k = arp[i]; k < arp[i + 1]; k++) u += brp[aci[k] + 1] - brp[aci[k]];
        wcount[0] = 2 * u <= ts;
    }
    __syncthreads();
    if (!wcount[0]) { // block-uniform
        if (t == 0) atomicExch(&g_spgemm_bad, 1);
        return;
    }
    __syncthreads();
    for (int q = t; q < ts; q += BH_TPB) keys[q] = -1;
    __syncthreads();
    for (int k = arp[i]; k < arp[i + 1]; k++) {
        int j = aci[k];
        double aij[NV];
#pragma unroll
        for (int q = 0; q < NV; q++) aij[q] = V.a[q][k];
        for (int e = brp[j] + t; e < brp[j + 1]; e += BH_TPB) {
            int J = bci[e];
            unsigned h = hslot(J, mask);
            for (;;) {
                int old = atomicCAS(&keys[h], -1, J);
                if (old == -1 || old == J) {
#pragma unroll
                    for (int q = 0; q < NV; q++) {
                        double prev = old == -1 ? 0.0 : vals[(size_t)q * ts + h];
                        vals[(size_t)q * ts + h] = __dadd_rn(prev, __dmul_rn(aij[q], V.b[q][e]));
                    }
                    break;
                }
                h = (h + 1) & mask;
            }
        }
        __syncthreads();
    }
    // compact occupied slots to the front, one chunk of BH_TPB slots at a time
    int c = 0;
    for (int base = 0; base < ts; base += BH_TPB) {
        int slot = base + t;
        int key = keys[slot];
        double val[NV];
#pragma unroll
        for (int q = 0; q < NV; q++) val[q] = vals[(size_t)q * ts + slot];
        bool occ = key >= 0;
        unsigned bal = __ballot_sync(0xffffffffu, occ);
        if (lane == 0) wcount[w] = __popc(bal);
        __syncthreads();
        int before = 0, chunk = 0;
        for (int q = 0; q < BH_TPB / 32; q++) {
            if (q < w) before += wcount[q];
            chunk += wcount[q];
        }
        int pos = c + before + __popc(bal & ((1u << lane) - 1));
        __syncthreads(); // every read of this chunk is done
        if (occ) {
            keys[pos] = key;
#pragma unroll
            for (int q = 0; q < NV; q++) vals[(size_t)q * ts + pos] = val[q];
        }
        c += chunk;
        __syncthreads();
    }
    if (phase == 0) {
        if (t == 0) cnt[i] = c;
        return;
    }
    // bitonic sort of the c entries by column (padding sorts last)
    int P = 1;
    while (P < c) P <<= 1;
    for (int q = c + t; q < P; q += BH_TPB) keys[q] = 0x7fffffff;
    __syncthreads();
    for (int kk = 2; kk <= P; kk <<= 1)
        for (int jj = kk >> 1; jj > 0; jj >>= 1) {
            for (int a = t; a < P; a += BH_TPB) {
                int b = a ^ jj;
                if (b > a) {
                    bool up = (a & kk) == 0;
                    int ka = keys[a], kb = keys[b];
                    if ((ka > kb) == up) {
                        keys[a] = kb;
                        keys[b] = ka;
#pragma unroll
                        for (int q = 0; q < NV; q++) {
                            double tv = vals[(size_t)q * ts + a];
                            vals[(size_t)q * ts + a] = vals[(size_t)q * ts + b];
                            vals[(size_t)q * ts + b] = tv;
                        }
                    }
                }
            }
            __syncthreads();
        }
    int base = crp[i];
    for (int q = t; q < c; q += BH_TPB) {
        cci[base + q] = keys[q];
#pragma unroll
        for (int r = 0; r < NV; r++) C.v[r][base + q] = vals[(size_t)r * ts + q];
    }
}

// C (pattern c, values cv[0..NV-1]) = A_q B_q for q < NV (patterns of a, b)
template <int NV>
static int spgemm_nv(amgh_problem *p, Arena &ar, const DevCsr &a, const double *const *av, const DevCsr &b,
                     const double *const *bv, DevCsr &c, double **cv)
{
    cudaStream_t s = p->stream;
    int n = a.rows;
    c.rows = n;
    c.cols = b.cols;
    GemmVals<NV> V;
    for (int q = 0; q < NV; q++) {
        V.a[q] = av[q];
        V.b[q] = bv[q];
    }
    // dynamic shared memory limits are per function and setups may run on
    // several host threads: raise them once to the most any launch can use
    // (the 48 KB default counts static memory too)
    const int dense_cols = Limits<NV>::dense_cols, bhash_u = Limits<NV>::bhash_u;
    CU(cudaFuncSetAttribute(k_gemm_warp<NV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)warp_smem_bytes<NV>()));
    CU(cudaFuncSetAttribute(k_gemm_dense<NV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)((size_t)dense_cols * (NV * sizeof(double) + 1))));
    CU(cudaFuncSetAttribute(k_gemm_bhash<NV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)((size_t)2 * bhash_u * (NV * sizeof(double) + sizeof(int)))));
    Scratch sc;
    long long *ub = nullptr, *toff = nullptr;
    int *cnt = nullptr, *tkey = nullptr, *path = nullptr, *flag = nullptr, *pos = nullptr, *umax = nullptr;
    unsigned long long *slots4 = nullptr;
    TRY(sc.alloc(&ub, n + 1));
    TRY(sc.alloc(&toff, n + 1));
    TRY(sc.alloc(&cnt, n + 1));
    TRY(sc.alloc(&path, n + 1));
    TRY(sc.alloc(&flag, n + 1));
    TRY(sc.alloc(&pos, n + 1));
    TRY(sc.alloc(&umax, 1));
    TRY(sc.alloc(&slots4, 1));
    int nb = ceil_div(n, 128);
    int use_dense = b.cols <= dense_cols;
    size_t dsmem = (size_t)b.cols * (NV * sizeof(double) + 1);
    CU(cudaMemsetAsync(umax, 0, sizeof(int), s));
    CU(cudaMemsetAsync(slots4, 0, sizeof(unsigned long long), s));
    k_gemm_ub<<<nb, 128, 0, s>>>(n, a.rp, a.ci, b.rp, ub, path, n <= WARP_PATH_MAX_ROWS, use_dense, bhash_u, umax,
                                  slots4);
    LAUNCH_CHECK();
    {
        unsigned long long sl = 0;
        CU(cudaMemcpyAsync(&sl, slots4, sizeof(sl), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        int to_warp = (long long)sl * (long long)(sizeof(int) + NV * sizeof(double)) > GLOBAL_TABLE_MAX_BYTES;
        k_gemm_settle<<<ceil_div(n, 256), 256, 0, s>>>(n, to_warp, path, ub);
        LAUNCH_CHECK();
    }
    // row lists of the warp (1), dense (2) and block-hash (3) paths
    int nlist[4] = {0, 0, 0, 0};
    int *list[4] = {nullptr, nullptr, nullptr, nullptr};
    for (int q = 1; q <= 3; q++) {
        k_is_path<<<ceil_div(n, 256), 256, 0, s>>>(n, path, q, flag);
        LAUNCH_CHECK();
        TRY(exclusive_scan<int>(flag, pos, n, s, &nlist[q]));
        if (nlist[q] > 0) {
            TRY(sc.alloc(&list[q], nlist[q]));
            k_list<<<ceil_div(n, 256), 256, 0, s>>>(n, flag, pos, list[q]);
            LAUNCH_CHECK();
        }
    }
    int ts3 = 0;
    size_t bsmem = 0;
    if (nlist[3] > 0) {
        int um = 0;
        CU(cudaMemcpyAsync(&um, umax, sizeof(int), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        ts3 = BH_TPB;
        while (ts3 < 2 * um) ts3 <<= 1;
        bsmem = (size_t)ts3 * (NV * sizeof(double) + sizeof(int));
    }
    long long tot = 0;
    TRY(exclusive_scan<long long>(ub, toff, n, s, &tot));
    GemmOut<NV> T;
    TRY(sc.alloc(&tkey, tot));
    for (int q = 0; q < NV; q++) TRY(sc.alloc(&T.v[q], tot));
    if (tot > 0) CU(cudaMemsetAsync(tkey, 0xff, sizeof(int) * (size_t)tot, s));
    k_gemm_hash<NV><<<nb, 128, 0, s>>>(n, a.rp, a.ci, V, b.rp, b.ci, toff, path, tkey, T, cnt);
    LAUNCH_CHECK();
    auto launch_lists = [&](int phase, int *cnt_, const int *crp, int *cci, GemmOut<NV> Cv) -> int {
        if (nlist[1] > 0) {
            k_gemm_warp<NV><<<ceil_div(nlist[1], WARPS_PER_BLOCK), 32 * WARPS_PER_BLOCK, warp_smem_bytes<NV>(), s>>>(
                nlist[1], a.rp, a.ci, V, b.rp, b.ci, list[1], phase, cnt_, crp, cci, Cv);
            LAUNCH_CHECK();
        }
        if (nlist[2] > 0) {
            k_gemm_dense<NV><<<nlist[2], DENSE_ROW_TPB, dsmem, s>>>(nlist[2], list[2], b.cols, a.rp, a.ci, V,
                                                                     b.rp, b.ci, phase, cnt_, crp, cci, Cv);
            LAUNCH_CHECK();
        }
        if (nlist[3] > 0) {
            k_gemm_bhash<NV><<<nlist[3], BH_TPB, bsmem, s>>>(nlist[3], list[3], ts3, a.rp, a.ci, V, b.rp, b.ci,
                                                              phase, cnt_, crp, cci, Cv);
            LAUNCH_CHECK();
        }
        return AMGH_OK;
    };
    GemmOut<NV> none;
    for (int q = 0; q < NV; q++) none.v[q] = nullptr;
    TRY(launch_lists(0, cnt, nullptr, nullptr, none));
    TRY(ar.alloc(&c.rp, n + 1));
    int nnz = 0;
    TRY(exclusive_scan<int>(cnt, c.rp, n, s, &nnz));
    c.nnz = nnz;
    TRY(ar.alloc(&c.ci, nnz));
    GemmOut<NV> Cv;
    for (int q = 0; q < NV; q++) {
        TRY(ar.alloc(&cv[q], nnz));
        Cv.v[q] = cv[q];
    }
    c.v = cv[0];
    if ((int64_t)nnz <= (int64_t)OUT_AVG * n)
        k_gemm_out_sm<NV><<<ceil_div(n, OUT_TPB), OUT_TPB, 0, s>>>(n, toff, path, tkey, T, c.rp, c.ci, Cv);
    else
        k_gemm_out<NV><<<ceil_div(n, 128), 128, 0, s>>>(n, toff, path, tkey, T, c.rp, c.ci, Cv);
    LAUNCH_CHECK();
    TRY(launch_lists(1, nullptr, c.rp, c.ci, Cv));
    int bad = 0;
    CU(cudaMemcpyFromSymbolAsync(&bad, g_spgemm_bad, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (bad) {
        int zero = 0;
        CU(cudaMemcpyToSymbolAsync(g_spgemm_bad, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s));
        CU(cudaStreamSynchronize(s));
        amgh_note_error(0, __FILE__, __LINE__);
        return AMGH_ERR_CUDA;
    }
    CU(cudaStreamSynchronize(s));
    return AMGH_OK;
}

int spgemm(amgh_problem *p, Arena &ar, const DevCsr &a, const DevCsr &b, DevCsr &c)
{
    const double *av[1] = {a.v}, *bv[1] = {b.v};
    double *cv[1] = {nullptr};
    return spgemm_nv<1>(p, ar, a, av, b, bv, c, cv);
}

// entries below the diagonal take the value of their mirror above it
__global__ void k_symm(int n, const int *__restrict__ rp, const int *__restrict__ ci, double *__restrict__ v,
                       int *__restrict__ bad)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int k = rp[i]; k < rp[i + 1]; k++) {
        int j = ci[k];
        if (j >= i) break;
        int lo = rp[j], hi = rp[j + 1] - 1, pos = -1;
        while (lo <= hi) {
            int mid = (lo + hi) >> 1;
            int cm = ci[mid];
            if (cm == i) {
                pos = mid;
                break;
            }
            if (cm < i) lo = mid + 1;
            else hi = mid - 1;
        }
        if (pos < 0) {
            atomicOr(bad, 1);
            return;
        }
        v[k] = v[pos];
    }
}

int symmetrize_upper(amgh_problem *p, DevCsr &c)
{
    cudaStream_t s = p->stream;
    Scratch sc;
    int *bad = nullptr;
    TRY(sc.alloc(&bad, 1));
    CU(cudaMemsetAsync(bad, 0, sizeof(int), s));
    k_symm<<<ceil_div(c.rows, 256), 256, 0, s>>>(c.rows, c.rp, c.ci, c.v, bad);
    LAUNCH_CHECK();
    int h = 0;
    CU(cudaMemcpyAsync(&h, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (h) amgh_note_msg("Galerkin product: sparsity pattern not symmetric");
    return h ? AMGH_ERR_INVALID_ARG : AMGH_OK;
}

int galerkin(amgh_problem *p, Arena &ar, const DevCsr &rt, const DevCsr &a, const DevCsr &pm, int symmetric,
             DevCsr &c)
{
    Arena tmp;
    DevCsr ap;
    int st = spgemm(p, tmp, a, pm, ap);
    if (st == AMGH_OK) st = spgemm(p, ar, rt, ap, c);
    tmp.free_all();
    if (st) return st;
    if (symmetric) TRY(symmetrize_upper(p, c));
    return AMGH_OK;
}

// c1 = rt a1 pm and c2 = rt a2 pm for a1, a2 with one sparsity pattern (A and
// M_y, or K_N and M_u): both products share their hashing and the result's
// pattern (c2 uses c1's row pointers and columns); both made exactly symmetric
int galerkin_pair(amgh_problem *p, Arena &ar, const DevCsr &rt, const DevCsr &a1, const DevCsr &a2,
                  const DevCsr &pm, DevCsr &c1, DevCsr &c2)
{
    if (a1.rows != a2.rows || a1.nnz != a2.nnz) return AMGH_ERR_INVALID_ARG;
    Arena tmp;
    DevCsr ap;
    double *apv[2] = {nullptr, nullptr};
    const double *av[2] = {a1.v, a2.v}, *pv[2] = {pm.v, pm.v};
    int st = spgemm_nv<2>(p, tmp, a1, av, pm, pv, ap, apv);
    if (st == AMGH_OK) {
        const double *rv[2] = {rt.v, rt.v}, *bv[2] = {apv[0], apv[1]};
        double *cv[2] = {nullptr, nullptr};
        st = spgemm_nv<2>(p, ar, rt, rv, ap, bv, c1, cv);
        if (st == AMGH_OK) {
            c2 = DevCsr();
            c2.rows = c1.rows;
            c2.cols = c1.cols;
            c2.nnz = c1.nnz;
            c2.rp = c1.rp;
            c2.ci = c1.ci;
            c1.v = cv[0];
            c2.v = cv[1];
        }
    }
    tmp.free_all();
    if (st) return st;
    TRY(symmetrize_upper(p, c1));
    TRY(symmetrize_upper(p, c2));
    return AMGH_OK;
}

// ------------------------------------------------------------------ diagonals
__global__ void k_l1(int n, const int *__restrict__ rp, const double *__restrict__ v, double *__restrict__ invd,
                     float *__restrict__ invd32)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; k++) s += fabs(v[k]);
    double r = 1.0 / s;
    invd[i] = r;
    if (invd32) invd32[i] = (float)r;
}

int l1_invdiag(amgh_problem *p, const DevCsr &a, double *invd, float *invd32)
{
    k_l1<<<ceil_div(a.rows, 256), 256, 0, p->stream>>>(a.rows, a.rp, a.v, invd, invd32);
    LAUNCH_CHECK();
    return AMGH_OK;
}

__global__ void k_dinv(int n, const int *__restrict__ rp, const int *__restrict__ ci, const double *__restrict__ v,
                       double *__restrict__ invd)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) invd[i] = 1.0 / row_diag(i, rp, ci, v);
}

int diag_inv(amgh_problem *p, const DevCsr &a, double *invd)
{
    k_dinv<<<ceil_div(a.rows, 256), 256, 0, p->stream>>>(a.rows, a.rp, a.ci, a.v, invd);
    LAUNCH_CHECK();
    return AMGH_OK;
}
