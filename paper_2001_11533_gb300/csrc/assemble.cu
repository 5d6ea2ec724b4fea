// assemble.cu -- P1 stiffness and mass assembly on the device (Sec. 2:
// [A]_ij = a(phi_j, phi_i) = int kappa grad phi_j . grad phi_i, [M]_ij =
// (phi_j, phi_i)).
//
// One thread owns one matrix row (one vertex).  It walks the elements that
// contain its vertex in ascending element id and adds that element's row to
// its entries, so every entry receives its element contributions in the same
// order on every run.  All element arithmetic uses explicit round-to-nearest
// intrinsics (no fused multiply-add), so the assembled values are
// reproducible bit for bit and equal to the sequential definition:
//   e_k = p_k - p_0, D = det[e_1 .. e_d], grad(lambda_k) = c_k / D with
//   2D: c_1 = (e2y, -e2x), c_2 = (-e1y, e1x);  3D: c_1 = e2 x e3, c_2 = e3 x e1,
//   c_3 = e1 x e2;  c_0 = -(c_1 + ... + c_d);
//   K_ab = (kappa / (d! |D|)) (c_a . c_b);  M_ab = |D| (1 + delta_ab) / (d! (d+1)(d+2)).
#include "internal.cuh"
#include "util.cuh"

#define MAXROW 256

__global__ void k_check_elems(int64_t ne, int d1, const int *__restrict__ el, int64_t nv, int *__restrict__ bad)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    for (int a = 0; a < d1; a++) {
        int v = el[e * d1 + a];
        if (v < 0 || v >= nv) atomicOr(bad, 1);
        for (int b = 0; b < a; b++)
            if (el[e * d1 + b] == v) atomicOr(bad, 2);
    }
}

__global__ void k_vcount(int64_t ne, int d1, const int *__restrict__ el, int *__restrict__ cnt)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    for (int a = 0; a < d1; a++) atomicAdd(&cnt[el[e * d1 + a]], 1);
}

__global__ void k_vfill(int64_t ne, int d1, const int *__restrict__ el, const int *__restrict__ vptr,
                        int *__restrict__ cursor, int *__restrict__ vel)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    for (int a = 0; a < d1; a++) {
        int v = el[e * d1 + a];
        vel[vptr[v] + atomicAdd(&cursor[v], 1)] = (int)e;
    }
}

__global__ void k_sort_int_rows(int rows, const int *__restrict__ rp, int *__restrict__ a)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    int b = rp[r], e = rp[r + 1];
    for (int k = b + 1; k < e; k++) {
        int x = a[k], j = k - 1;
        while (j >= b && a[j] > x) {
            a[j + 1] = a[j];
            j--;
        }
        a[j + 1] = x;
    }
}

// neighbours of vertex v (sorted, unique) into buf; returns count or -1
__device__ int row_pattern(int v, int d1, const int *__restrict__ el, const int *__restrict__ vptr,
                           const int *__restrict__ vel, int *buf)
{
    int cnt = 0;
    for (int q = vptr[v]; q < vptr[v + 1]; q++) {
        int64_t e = vel[q];
        for (int a = 0; a < d1; a++) {
            int w = el[e * d1 + a];
            // insert w into sorted buf if absent
            int pos = cnt;
            bool dup = false;
            for (int t = 0; t < cnt; t++) {
                if (buf[t] == w) {
                    dup = true;
                    break;
                }
                if (buf[t] > w) {
                    pos = t;
                    break;
                }
            }
            if (dup) continue;
            if (cnt >= MAXROW) return -1;
            for (int t = cnt; t > pos; t--) buf[t] = buf[t - 1];
            buf[pos] = w;
            cnt++;
        }
    }
    return cnt;
}

__global__ void k_row_count(int nv, int d1, const int *__restrict__ el, const int *__restrict__ vptr,
                            const int *__restrict__ vel, int *__restrict__ cnt, int *__restrict__ bad)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    int buf[MAXROW];
    int c = row_pattern(v, d1, el, vptr, vel, buf);
    if (c < 0) {
        atomicOr(bad, 4);
        c = 0;
    }
    cnt[v] = c;
}

__global__ void k_row_fill(int nv, int d1, const int *__restrict__ el, const int *__restrict__ vptr,
                           const int *__restrict__ vel, const int *__restrict__ rp, int *__restrict__ ci)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    int buf[MAXROW];
    int c = row_pattern(v, d1, el, vptr, vel, buf);
    for (int t = 0; t < c; t++) ci[rp[v] + t] = buf[t];
}

// cofactor gradients c[a][k] (scaled by D) and |D| of one element
__device__ void element_geometry(int dim, const double *__restrict__ X, const int *ev, double c[4][3],
                                 double *absdet)
{
    if (dim == 2) {
        const double *p0 = X + 2 * (int64_t)ev[0], *p1 = X + 2 * (int64_t)ev[1], *p2 = X + 2 * (int64_t)ev[2];
        double e1x = __dsub_rn(p1[0], p0[0]), e1y = __dsub_rn(p1[1], p0[1]);
        double e2x = __dsub_rn(p2[0], p0[0]), e2y = __dsub_rn(p2[1], p0[1]);
        double det = __dsub_rn(__dmul_rn(e1x, e2y), __dmul_rn(e1y, e2x));
        c[1][0] = e2y;
        c[1][1] = -e2x;
        c[2][0] = -e1y;
        c[2][1] = e1x;
        c[0][0] = -__dadd_rn(c[1][0], c[2][0]);
        c[0][1] = -__dadd_rn(c[1][1], c[2][1]);
        *absdet = fabs(det);
    } else {
        const double *p0 = X + 3 * (int64_t)ev[0], *p1 = X + 3 * (int64_t)ev[1], *p2 = X + 3 * (int64_t)ev[2],
                     *p3 = X + 3 * (int64_t)ev[3];
        double e1[3], e2[3], e3[3];
        for (int k = 0; k < 3; k++) {
            e1[k] = __dsub_rn(p1[k], p0[k]);
            e2[k] = __dsub_rn(p2[k], p0[k]);
            e3[k] = __dsub_rn(p3[k], p0[k]);
        }
        c[1][0] = __dsub_rn(__dmul_rn(e2[1], e3[2]), __dmul_rn(e2[2], e3[1]));
        c[1][1] = __dsub_rn(__dmul_rn(e2[2], e3[0]), __dmul_rn(e2[0], e3[2]));
        c[1][2] = __dsub_rn(__dmul_rn(e2[0], e3[1]), __dmul_rn(e2[1], e3[0]));
        c[2][0] = __dsub_rn(__dmul_rn(e3[1], e1[2]), __dmul_rn(e3[2], e1[1]));
        c[2][1] = __dsub_rn(__dmul_rn(e3[2], e1[0]), __dmul_rn(e3[0], e1[2]));
        c[2][2] = __dsub_rn(__dmul_rn(e3[0], e1[1]), __dmul_rn(e3[1], e1[0]));
        c[3][0] = __dsub_rn(__dmul_rn(e1[1], e2[2]), __dmul_rn(e1[2], e2[1]));
        c[3][1] = __dsub_rn(__dmul_rn(e1[2], e2[0]), __dmul_rn(e1[0], e2[2]));
        c[3][2] = __dsub_rn(__dmul_rn(e1[0], e2[1]), __dmul_rn(e1[1], e2[0]));
        for (int k = 0; k < 3; k++) c[0][k] = -__dadd_rn(__dadd_rn(c[1][k], c[2][k]), c[3][k]);
        double det = __dadd_rn(__dadd_rn(__dmul_rn(e1[0], c[1][0]), __dmul_rn(e1[1], c[1][1])),
                               __dmul_rn(e1[2], c[1][2]));
        *absdet = fabs(det);
    }
}

__global__ void k_degenerate(int64_t ne, int dim, const double *__restrict__ X, const int *__restrict__ el,
                             int *__restrict__ bad)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    int ev[4];
    for (int a = 0; a <= dim; a++) ev[a] = el[e * (dim + 1) + a];
    double c[4][3], ad;
    element_geometry(dim, X, ev, c, &ad);
    if (!(ad > 0.0) || isinf(ad)) atomicOr(bad, 8);
}

__global__ void k_row_values(int nv, int dim, const double *__restrict__ X, const int *__restrict__ el,
                             const double *__restrict__ kappa, const int *__restrict__ vptr,
                             const int *__restrict__ vel, const int *__restrict__ rp, const int *__restrict__ ci,
                             double *__restrict__ Kv, double *__restrict__ Mv)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    int d1 = dim + 1;
    int beg = rp[v], len = rp[v + 1] - beg;
    for (int t = 0; t < len; t++) {
        Kv[beg + t] = 0.0;
        Mv[beg + t] = 0.0;
    }
    for (int q = vptr[v]; q < vptr[v + 1]; q++) {
        int64_t e = vel[q];
        int ev[4];
        int a = 0;
        for (int k = 0; k < d1; k++) {
            ev[k] = el[e * d1 + k];
            if (ev[k] == v) a = k;
        }
        double c[4][3], absdet;
        element_geometry(dim, X, ev, c, &absdet);
        double coef, mdiag, moff;
        if (dim == 2) {
            coef = __ddiv_rn(kappa[e], 2.0 * absdet);
            mdiag = __ddiv_rn(absdet, 12.0);
            moff = __ddiv_rn(absdet, 24.0);
        } else {
            coef = __ddiv_rn(kappa[e], __dmul_rn(6.0, absdet));
            mdiag = __ddiv_rn(absdet, 60.0);
            moff = __ddiv_rn(absdet, 120.0);
        }
        for (int b = 0; b < d1; b++) {
            double dd;
            if (dim == 2)
                dd = __dadd_rn(__dmul_rn(c[a][0], c[b][0]), __dmul_rn(c[a][1], c[b][1]));
            else
                dd = __dadd_rn(__dadd_rn(__dmul_rn(c[a][0], c[b][0]), __dmul_rn(c[a][1], c[b][1])),
                               __dmul_rn(c[a][2], c[b][2]));
            double kab = __dmul_rn(coef, dd);
            double mab = (a == b) ? mdiag : moff;
            // column position of ev[b] in row v (sorted): binary search
            int lo = 0, hi = len - 1, w = ev[b], pos = -1;
            while (lo <= hi) {
                int mid = (lo + hi) >> 1;
                int cm = ci[beg + mid];
                if (cm == w) {
                    pos = mid;
                    break;
                }
                if (cm < w) lo = mid + 1;
                else hi = mid - 1;
            }
            Kv[beg + pos] = __dadd_rn(Kv[beg + pos], kab);
            Mv[beg + pos] = __dadd_rn(Mv[beg + pos], mab);
        }
    }
}

// state numbering: state id = rank of the vertex among non-Dirichlet vertices
__global__ void k_not_dir(int64_t nv, const unsigned char *__restrict__ dir, int *__restrict__ flag)
{
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < nv) flag[v] = dir[v] ? 0 : 1;
}

__global__ void k_state_maps(int64_t nv, const unsigned char *__restrict__ dir, const int *__restrict__ rank,
                             int *__restrict__ sov, int *__restrict__ vos)
{
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    if (dir[v]) sov[v] = -1;
    else {
        sov[v] = rank[v];
        vos[rank[v]] = (int)v;
    }
}

int assemble_full(amgh_problem *p)
{
    cudaStream_t s = p->stream;
    int nv = (int)p->nv;
    int d1 = p->dim + 1;
    int64_t ne = p->ne;
    Scratch sc;
    int *bad = nullptr, *cnt = nullptr, *vptr = nullptr, *cur = nullptr, *vel = nullptr, *rcnt = nullptr;
    TRY(sc.alloc(&bad, 1));
    CU(cudaMemsetAsync(bad, 0, sizeof(int), s));
    int eb = (int)((ne + 255) / 256);
    k_check_elems<<<eb, 256, 0, s>>>(ne, d1, p->elems, p->nv, bad);
    LAUNCH_CHECK();
    int hbad = 0;
    CU(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (hbad) return AMGH_ERR_INVALID_ARG;
    k_degenerate<<<eb, 256, 0, s>>>(ne, p->dim, p->coords, p->elems, bad);
    LAUNCH_CHECK();
    // vertex -> element incidence, ascending element id
    TRY(sc.alloc(&cnt, nv + 1));
    TRY(sc.alloc(&vptr, nv + 1));
    TRY(sc.alloc(&cur, nv + 1));
    CU(cudaMemsetAsync(cnt, 0, sizeof(int) * (nv + 1), s));
    CU(cudaMemsetAsync(cur, 0, sizeof(int) * (nv + 1), s));
    k_vcount<<<eb, 256, 0, s>>>(ne, d1, p->elems, cnt);
    LAUNCH_CHECK();
    int ninc = 0;
    TRY(exclusive_scan<int>(cnt, vptr, nv, s, &ninc));
    TRY(sc.alloc(&vel, ninc));
    k_vfill<<<eb, 256, 0, s>>>(ne, d1, p->elems, vptr, cur, vel);
    LAUNCH_CHECK();
    k_sort_int_rows<<<ceil_div(nv, 128), 128, 0, s>>>(nv, vptr, vel);
    LAUNCH_CHECK();
    // row patterns
    TRY(sc.alloc(&rcnt, nv + 1));
    k_row_count<<<ceil_div(nv, 128), 128, 0, s>>>(nv, d1, p->elems, vptr, vel, rcnt, bad);
    LAUNCH_CHECK();
    CU(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (hbad) return AMGH_ERR_INVALID_ARG;
    DevCsr &K = p->Kfull, &M = p->Mfull;
    K.rows = K.cols = M.rows = M.cols = nv;
    TRY(p->arena.alloc(&K.rp, nv + 1));
    int nnz = 0;
    TRY(exclusive_scan<int>(rcnt, K.rp, nv, s, &nnz));
    K.nnz = M.nnz = nnz;
    TRY(p->arena.alloc(&K.ci, nnz));
    TRY(p->arena.alloc(&K.v, nnz));
    TRY(p->arena.alloc(&M.v, nnz));
    M.rp = K.rp;
    M.ci = K.ci;
    k_row_fill<<<ceil_div(nv, 128), 128, 0, s>>>(nv, d1, p->elems, vptr, vel, K.rp, K.ci);
    LAUNCH_CHECK();
    k_row_values<<<ceil_div(nv, 128), 128, 0, s>>>(nv, p->dim, p->coords, p->elems, p->kappa, vptr, vel, K.rp,
                                                   K.ci, K.v, M.v);
    LAUNCH_CHECK();
    // state numbering
    int *flag = nullptr, *rank = nullptr;
    TRY(sc.alloc(&flag, nv + 1));
    TRY(sc.alloc(&rank, nv + 1));
    k_not_dir<<<ceil_div(nv, 256), 256, 0, s>>>(nv, p->dir, flag);
    LAUNCH_CHECK();
    int m = 0;
    TRY(exclusive_scan<int>(flag, rank, nv, s, &m));
    // every vertex on the Dirichlet boundary: the state space is empty and the
    // problem of Sec. 2 degenerates (y = 0 for every control)
    if (m == 0) return AMGH_ERR_INVALID_ARG;
    p->m = m;
    p->n = nv;
    TRY(p->arena.alloc(&p->state_of_vertex, nv));
    TRY(p->arena.alloc(&p->vertex_of_state, m));
    k_state_maps<<<ceil_div(nv, 256), 256, 0, s>>>(nv, p->dir, rank, p->state_of_vertex, p->vertex_of_state);
    LAUNCH_CHECK();
    CU(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (hbad) return AMGH_ERR_INVALID_ARG;
    return AMGH_OK;
}

// ------------------------------------------------------------------ extraction
__global__ void k_sub_count(int rows, const int *__restrict__ rp, const int *__restrict__ ci,
                            const int *__restrict__ rmap, const int *__restrict__ cmap, int *__restrict__ cnt)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows) return;
    int ri = rmap ? rmap[i] : i;
    if (ri < 0) return;
    int c = 0;
    for (int k = rp[i]; k < rp[i + 1]; k++) c += (cmap ? cmap[ci[k]] : ci[k]) >= 0;
    cnt[ri] = c;
}

__global__ void k_sub_fill(int rows, const int *__restrict__ rp, const int *__restrict__ ci,
                           const double *__restrict__ v, const int *__restrict__ rmap, const int *__restrict__ cmap,
                           const int *__restrict__ orp, int *__restrict__ oci, double *__restrict__ ov)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows) return;
    int ri = rmap ? rmap[i] : i;
    if (ri < 0) return;
    int pos = orp[ri];
    for (int k = rp[i]; k < rp[i + 1]; k++) {
        int c = cmap ? cmap[ci[k]] : ci[k];
        if (c < 0) continue;
        oci[pos] = c;
        ov[pos] = v[k];
        pos++;
    }
}

// rows with rmap >= 0 and columns with cmap >= 0 (NULL map = identity), renumbered;
// cmap must be increasing on kept columns so rows stay sorted
int extract_sub(Arena &ar, const DevCsr &a, const int *rmap, int nr, const int *cmap, int nc, DevCsr &out,
                cudaStream_t s)
{
    out.rows = nr;
    out.cols = nc;
    Scratch sc;
    int *cnt = nullptr;
    TRY(sc.alloc(&cnt, nr + 1));
    CU(cudaMemsetAsync(cnt, 0, sizeof(int) * (nr + 1), s));
    k_sub_count<<<ceil_div(a.rows, 256), 256, 0, s>>>(a.rows, a.rp, a.ci, rmap, cmap, cnt);
    LAUNCH_CHECK();
    TRY(ar.alloc(&out.rp, nr + 1));
    int nnz = 0;
    TRY(exclusive_scan<int>(cnt, out.rp, nr, s, &nnz));
    out.nnz = nnz;
    TRY(ar.alloc(&out.ci, nnz));
    TRY(ar.alloc(&out.v, nnz));
    k_sub_fill<<<ceil_div(a.rows, 256), 256, 0, s>>>(a.rows, a.rp, a.ci, a.v, rmap, cmap, out.rp, out.ci, out.v);
    LAUNCH_CHECK();
    CU(cudaStreamSynchronize(s));
    return AMGH_OK;
}
