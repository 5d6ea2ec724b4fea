// kuhn.cu -- matrix-free stiffness operator of the structured Kuhn cube.
//
// On the N^3 vertex grid of the unit cube split into 6 Kuhn tetrahedra per
// cell (the meshes of the 3D workloads: cell-major, the 6 tetrahedra of a
// cell in lexicographic order of the axis permutation (a, b, c), each the
// path o, o + e_a, o + e_a + e_b, o + (1,1,1)), every tetrahedron is the same
// simplex up to a permutation of the axes.  Its barycentric gradients are
// -e_a/h, (e_a - e_b)/h, (e_b - e_c)/h, e_c/h and its volume h^3/6, so the P1
// element stiffness (Sec. 2) is kappa_T h/6 times the tridiagonal matrix
//   [ 1 -1  0  0 ]
//   [-1  2 -1  0 ]
//   [ 0 -1  2 -1 ]
//   [ 0  0 -1  1 ]
// in path order.  The state stiffness A (Dirichlet vertices eliminated) is
// applied without storing it:
//   (A x)_v = h/6 ( x_v sum_T kappa_T d_L(T) - sum_T kappa_T (x_prev(T) + x_next(T)) )
// over the 24 tetrahedra T containing v, L(T) the position of v on T's path,
// d_L = 1 at the path ends and 2 inside, prev/next its path neighbours (zero
// on Dirichlet vertices).  The only per-element data is kappa, so the matrix
// stream of 8-12 bytes per stored entry (15 per row) becomes ~6 x (value
// bytes) per vertex.  Results equal the assembled product up to rounding.
#include <math.h>

#include "internal.cuh"
#include "spmv.cuh"

// axis permutations in lexicographic order (the element order of the mesh)
__constant__ int c_perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

// 0 if element e is not the Kuhn tetrahedron the structured grid puts there
__global__ void k_kuhn_check(int N, int64_t ne, const int *__restrict__ elems, const double *__restrict__ coords,
                             double h, int *__restrict__ bad)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < ne) {
        const int64_t cell = e / 6;
        const int t = (int)(e % 6), M = N - 1;
        const int ci = (int)(cell % M), cj = (int)((cell / M) % M), ck = (int)(cell / ((int64_t)M * M));
        const int64_t step[3] = {1, N, (int64_t)N * N};
        const int64_t base = ci + (int64_t)N * cj + (int64_t)N * N * ck;
        const int a = c_perm[t][0], b = c_perm[t][1];
        const int64_t want[4] = {base, base + step[a], base + step[a] + step[b], base + 1 + N + (int64_t)N * N};
        for (int q = 0; q < 4; q++)
            if (elems[4 * e + q] != want[q]) atomicOr(bad, 1);
    }
    const int64_t nv = (int64_t)N * N * N;
    if (e < nv) {
        const int i = (int)(e % N), j = (int)((e / N) % N), k = (int)(e / ((int64_t)N * N));
        const double tol = 1e-12;
        if (fabs(coords[3 * e] - i * h) > tol || fabs(coords[3 * e + 1] - j * h) > tol ||
            fabs(coords[3 * e + 2] - k * h) > tol)
            atomicOr(bad, 2);
    }
}

__global__ void k_to_f32_kappa(int64_t n, const double *__restrict__ a, float *__restrict__ b)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

// Consecutive path points of a Kuhn tetrahedron differ by one unit vector and
// the element matrix couples only consecutive points, so the operator is a
// 7-point stencil: the off-diagonal coefficient of the edge v -- v+e is minus
// h/6 times the sum of kappa over the tetrahedra whose path runs along that
// edge.  (The assembled matrix has the 15-point pattern of the mesh; its 8
// other entries per row are exact zeros.)  Index 0..5 of the axis neighbours
// +x, -x, +y, -y, +z, -z, -1 for any other offset.
__host__ __device__ constexpr int kuhn_nbr(int di, int dj, int dk)
{
    return (di == 1 && dj == 0 && dk == 0)    ? 0
           : (di == -1 && dj == 0 && dk == 0) ? 1
           : (di == 0 && dj == 1 && dk == 0)  ? 2
           : (di == 0 && dj == -1 && dk == 0) ? 3
           : (di == 0 && dj == 0 && dk == 1)  ? 4
           : (di == 0 && dj == 0 && dk == -1) ? 5
                                              : -1;
}

// (A x)_r for state row r.  The row's 6 off-diagonal coefficients and its
// diagonal are first summed from the kappa of the 24 tetrahedra around the
// vertex (cells dk, dj, di = 0, 1 in that order, tetrahedra t = 0..5; every
// index below is a compile-time constant once the loops are unrolled), then
// the 6 neighbour values are loaded together and combined in a fixed order.
template <typename T, typename K>
__device__ __forceinline__ T kuhn_row(int N, T h6, const K *__restrict__ kappa, const int *__restrict__ sov,
                                      const int *__restrict__ vos, const T *__restrict__ x, int r)
{
    const int64_t v = vos[r];
    const int i = (int)(v % N), j = (int)((v / N) % N), k = (int)(v / ((int64_t)N * N));
    const int M = N - 1;
    constexpr int PERM[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    T coef[6];
#pragma unroll
    for (int q = 0; q < 6; q++) coef[q] = (T)0;
    T diag = (T)0;
#pragma unroll
    for (int dk = 0; dk < 2; dk++)
#pragma unroll
        for (int dj = 0; dj < 2; dj++)
#pragma unroll
            for (int di = 0; di < 2; di++) {
                const int oi = i - di, oj = j - dj, ok = k - dk;
                if (oi < 0 || oj < 0 || ok < 0 || oi >= M || oj >= M || ok >= M) continue;
                const int dmask = di | (dj << 1) | (dk << 2);
                const int s = di + dj + dk;
                const int64_t cell = oi + (int64_t)M * (oj + (int64_t)M * ok);
#pragma unroll
                for (int t = 0; t < 6; t++) {
                    const int a = PERM[t][0], b = PERM[t][1], c = PERM[t][2];
                    int L = -1;
                    if (s == 0) L = 0;
                    else if (s == 3) L = 3;
                    else if (s == 1 && ((dmask >> a) & 1)) L = 1;
                    else if (s == 2 && !((dmask >> c) & 1)) L = 2;
                    if (L < 0) continue;
                    // path points p_0..p_3 of the tetrahedron relative to its cell
                    const int px[4] = {0, a == 0, (a == 0) + (b == 0), 1};
                    const int py[4] = {0, a == 1, (a == 1) + (b == 1), 1};
                    const int pz[4] = {0, a == 2, (a == 2) + (b == 2), 1};
                    const T kt = (T)kappa[6 * cell + t];
                    diag += kt * (T)((L == 0 || L == 3) ? 1 : 2);
                    if (L > 0) coef[kuhn_nbr(px[L - 1] - di, py[L - 1] - dj, pz[L - 1] - dk)] += kt;
                    if (L < 3) coef[kuhn_nbr(px[L + 1] - di, py[L + 1] - dj, pz[L + 1] - dk)] += kt;
                }
            }
    constexpr int OFF[6][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
    T xn[6];
#pragma unroll
    for (int q = 0; q < 6; q++) {
        const int ni = i + OFF[q][0], nj = j + OFF[q][1], nk = k + OFF[q][2];
        int st = -1;
        if (ni >= 0 && nj >= 0 && nk >= 0 && ni < N && nj < N && nk < N)
            st = sov[ni + (int64_t)N * nj + (int64_t)N * N * nk];
        xn[q] = st >= 0 ? x[st] : (T)0;
    }
    T off = (T)0;
#pragma unroll
    for (int q = 0; q < 6; q++) off += coef[q] * xn[q];
    return h6 * (diag * x[r] - off);
}

template <typename T, typename K>
__global__ void k_kuhn_apply(int m, int N, T h6, const K *__restrict__ kappa, const int *__restrict__ sov,
                             const int *__restrict__ vos, const T *__restrict__ x, T *__restrict__ y)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < m) y[r] = kuhn_row<T, K>(N, h6, kappa, sov, vos, x, r);
}

// Chebyshev step of the level-0 smoother with the matrix-free operator:
// d' = c_d d + c_r D^-1 (b - A x), x' = x + d'
__global__ void k_kuhn_cheb(int m, int N, float h6, const float *__restrict__ kappa, const int *__restrict__ sov,
                            const int *__restrict__ vos, const float *__restrict__ invd, const float *__restrict__ b,
                            const float *__restrict__ x, float *__restrict__ d, float *__restrict__ xn, float cdv,
                            float crv, const int *__restrict__ skip)
{
    pdl_enter();
    if (skip && *skip) return;
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= m) return;
    float br = b[r], ir = invd[r], dr = d[r], xr = x[r];
    float ax = kuhn_row<float, float>(N, h6, kappa, sov, vos, x, r);
    float dn, xv;
    cheb_point(br, ax, ir, dr, xr, cdv, crv, dn, xv);
    d[r] = dn;
    xn[r] = xv;
}

__global__ void k_kuhn_residual(int m, int N, float h6, const float *__restrict__ kappa, const int *__restrict__ sov,
                                const int *__restrict__ vos, const float *__restrict__ b, const float *__restrict__ x,
                                float *__restrict__ res, const int *__restrict__ skip)
{
    pdl_enter();
    if (skip && *skip) return;
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < m) res[r] = rsub(b[r], kuhn_row<float, float>(N, h6, kappa, sov, vos, x, r));
}

// sets p->kuhn_N to N if the mesh is the structured Kuhn cube (and fills
// kappa32), else to 0; returns a status
int kuhn_detect(amgh_problem *p)
{
    if (p->kuhn_checked) return AMGH_OK;
    p->kuhn_checked = 1;
    p->kuhn_N = 0;
    if (p->dim != 3) return AMGH_OK;
    const int N = (int)llround(cbrt((double)p->nv));
    if (N < 2 || (int64_t)N * N * N != p->nv || p->ne != 6LL * (N - 1) * (N - 1) * (N - 1)) return AMGH_OK;
    cudaStream_t s = p->stream;
    Scratch sc;
    int *bad = nullptr;
    TRY(sc.alloc(&bad, 1));
    CU(cudaMemsetAsync(bad, 0, sizeof(int), s));
    const int64_t work = p->ne > p->nv ? p->ne : p->nv;
    k_kuhn_check<<<ceil_div(work, 256), 256, 0, s>>>(N, p->ne, p->elems, p->coords, 1.0 / (N - 1), bad);
    LAUNCH_CHECK();
    int h = 0;
    CU(cudaMemcpyAsync(&h, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (h) return AMGH_OK;
    TRY(p->arena.alloc(&p->kappa32, p->ne));
    k_to_f32_kappa<<<ceil_div(p->ne, 256), 256, 0, s>>>(p->ne, p->kappa, p->kappa32);
    LAUNCH_CHECK();
    CU(cudaStreamSynchronize(s));
    p->kuhn_N = N;
    return AMGH_OK;
}

// compulsory bytes per state row: kappa of one cell (6 per vertex, read once
// with cache reuse between neighbouring rows), the vertex map entry of the
// row and of the vertex, x and y
static double kuhn_bytes(const amgh_problem *p, int vb, int kb)
{
    return (double)p->m * (2.0 * vb + 8.0) + (double)p->ne * kb;
}

int kuhn_apply(amgh_problem *p, int prec32, const void *x, void *y)
{
    const int N = p->kuhn_N, m = p->m;
    const double h6 = 1.0 / (6.0 * (N - 1));
    timer_begin(p, KC_SPMV);
    if (prec32)
        k_kuhn_apply<float, float><<<ceil_div(m, 256), 256, 0, p->stream>>>(m, N, (float)h6, p->kappa32,
                                                                            p->state_of_vertex, p->vertex_of_state,
                                                                            (const float *)x, (float *)y);
    else
        k_kuhn_apply<double, double><<<ceil_div(m, 256), 256, 0, p->stream>>>(m, N, h6, p->kappa,
                                                                              p->state_of_vertex, p->vertex_of_state,
                                                                              (const double *)x, (double *)y);
    LAUNCH_CHECK();
    timer_end(p, KC_SPMV, prec32 ? kuhn_bytes(p, 4, 4) : kuhn_bytes(p, 8, 8));
    return AMGH_OK;
}

int kuhn_cheb_step(amgh_problem *p, const float *invd, const float *b, const float *x, float *d, float *xn,
                   double cdv, double crv, const int *skip)
{
    const int N = p->kuhn_N, m = p->m;
    timer_begin(p, KC_CHEB0);
    pdl_launch(k_kuhn_cheb, dim3(ceil_div(m, 256)), dim3(256), 0, p->stream, m, N, (float)(1.0 / (6.0 * (N - 1))),
               (const float *)p->kappa32, (const int *)p->state_of_vertex, (const int *)p->vertex_of_state, invd, b, x,
               d, xn, (float)cdv, (float)crv, skip);
    LAUNCH_CHECK();
    timer_end(p, KC_CHEB0, kuhn_bytes(p, 4, 4) + 4.0 * 4 * m);
    return AMGH_OK;
}

int kuhn_residual(amgh_problem *p, const float *b, const float *x, float *r, const int *skip)
{
    const int N = p->kuhn_N, m = p->m;
    timer_begin(p, KC_RESID0);
    pdl_launch(k_kuhn_residual, dim3(ceil_div(m, 256)), dim3(256), 0, p->stream, m, N,
               (float)(1.0 / (6.0 * (N - 1))), (const float *)p->kappa32, (const int *)p->state_of_vertex,
               (const int *)p->vertex_of_state, b, x, r, skip);
    LAUNCH_CHECK();
    timer_end(p, KC_RESID0, kuhn_bytes(p, 4, 4) + 4.0 * m);
    return AMGH_OK;
}
