// noalloc.cu -- aggregation of a caller's matrix without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs while another
// framework's caching allocator owns the device memory budget, processes
// under a hard memory cap, or latency-critical paths where an allocation (and
// the device synchronisation cudaFree implies) is not acceptable.  For them
// amgh_aggregate_noalloc runs the same aggregation kernels as amgh_amg_setup
// on a matrix the caller already holds on the device, taking every scratch
// array from one fixed buffer that is part of the library image
// (g_noalloc_scratch below) instead of allocating.
//
// Limits: at most NOALLOC_MAX_ROWS rows and NOALLOC_MAX_NNZ stored entries.
// The buffer exists once per device that loads the library and stays until
// the process exits.  Every call shares it, so calls that overlap on the GPU
// (on different streams, or from different threads) race and must be
// serialised by the caller.  A call clears what must start at zero itself;
// nothing depends on a previous call's contents.
#include <mutex>

#include "internal.cuh"

#define NOALLOC_MAX_ROWS 32768
#define NOALLOC_MAX_NNZ 262144
#define NOALLOC_BYTES (5u << 20)

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

// aggregation kernels of amg.cu (launched unchanged)
__global__ void k_diag(int n, const int *__restrict__ rp, const int *__restrict__ ci, const double *__restrict__ v,
                       double *__restrict__ d);
__global__ void k_strength(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                           const double *__restrict__ v, const double *__restrict__ d, double th2,
                           const int *__restrict__ srp, int *__restrict__ cnt, int *__restrict__ sci,
                           double *__restrict__ sv);
__global__ void k_mis_m1(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                         const unsigned char *__restrict__ st, int *__restrict__ m1);
__global__ void k_mis_select(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                             const int *__restrict__ m1, unsigned char *__restrict__ st);
__global__ void k_mis_r1(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                         const unsigned char *__restrict__ st, unsigned char *__restrict__ r1);
__global__ void k_mis_r2(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                         const unsigned char *__restrict__ r1, unsigned char *__restrict__ st,
                         int *__restrict__ undecided);
__global__ void k_mis_promote(int n, unsigned char *__restrict__ st);
__global__ void k_root_flag(int n, const unsigned char *__restrict__ st, int *__restrict__ f);
__global__ void k_phase1(int n, const int *__restrict__ srp, const int *__restrict__ sci,
                         const unsigned char *__restrict__ st, const int *__restrict__ rank, int *__restrict__ agg);
__global__ void k_phase2(int n, const int *__restrict__ srp, const int *__restrict__ sci,
                         const double *__restrict__ sv, const int *__restrict__ agg1, int *__restrict__ agg2,
                         int *__restrict__ freeflag);
__global__ void k_phase3(int n, const int *__restrict__ fr, const int *__restrict__ frank, int nroots,
                         int *__restrict__ agg);

// exclusive prefix sum of n <= NOALLOC_MAX_ROWS ints by one block; total -> *total
__global__ void k_noalloc_scan(const int *__restrict__ in, int n, int *__restrict__ out, int *__restrict__ total)
{
    __shared__ int sh[1024];
    int chunk = (n + 1023) / 1024;
    int beg = threadIdx.x * chunk, end = min(beg + chunk, n);
    int s = 0;
    for (int i = beg; i < end; i++) s += in[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        int t = (int)threadIdx.x >= off ? sh[threadIdx.x - off] : 0;
        __syncthreads();
        sh[threadIdx.x] += t;
        __syncthreads();
    }
    int run = threadIdx.x ? sh[threadIdx.x - 1] : 0;
    for (int i = beg; i < end; i++) {
        int v = in[i];
        out[i] = run;
        run += v;
    }
    if (threadIdx.x == 1023) {
        out[n] = sh[1023];
        *total = sh[1023];
    }
}

// Address of g_noalloc_scratch on the current device.  The host-side name of a
// __device__ array is only a stand-in, so the device address is looked up
// once per device (with that device current) and cached.
static int scratch_address(unsigned char **out)
{
    static std::mutex mu;
    static unsigned char *addr[64] = {nullptr};
    int dev = 0;
    CU(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return AMGH_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return AMGH_ERR_CUDA;
        addr[dev] = (unsigned char *)p;
    }
    *out = addr[dev];
    return AMGH_OK;
}

// carve `count` elements of T from the scratch cursor (256-byte aligned)
template <typename T>
static T *carve(unsigned char *base, size_t &off, size_t count)
{
    off = (off + 255) & ~(size_t)255;
    T *p = (T *)(base + off);
    off += count * sizeof(T);
    return p;
}

static int scan_host_total(const int *in, int n, int *out, int *tot_dev, cudaStream_t s, int *total)
{
    k_noalloc_scan<<<1, 1024, 0, s>>>(in, n, out, tot_dev);
    amgh_count_launch();
    CU(cudaGetLastError());
    CU(cudaMemcpyAsync(total, tot_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    return AMGH_OK;
}

extern "C" int amgh_aggregate_noalloc(int n, const int32_t *rp, const int32_t *ci, const double *v, double theta,
                                      void *stream, int32_t *agg, int32_t *nagg)
{
    if (n <= 0 || !rp || !ci || !v || !agg || !nagg || !(theta >= 0.0)) return AMGH_ERR_INVALID_ARG;
    if (n > NOALLOC_MAX_ROWS) return AMGH_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int first = -1, nnz = 0;
    CU(cudaMemcpyAsync(&first, rp, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(&nnz, rp + n, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    // a CSR must start at entry 0; the entry count bounds every scratch array
    if (first != 0 || nnz < 0 || nnz > NOALLOC_MAX_NNZ) return AMGH_ERR_INVALID_ARG;
    unsigned char *base = nullptr;
    TRY(scratch_address(&base));
    size_t off = 0;
    double *d = carve<double>(base, off, n);
    double *sv = carve<double>(base, off, nnz);
    int *cnt = carve<int>(base, off, n + 1);
    int *srp = carve<int>(base, off, n + 1);
    int *sci = carve<int>(base, off, nnz);
    int *m1 = carve<int>(base, off, n);
    int *flag = carve<int>(base, off, n + 1);
    int *rank = carve<int>(base, off, n + 1);
    int *agg1 = carve<int>(base, off, n);
    int *fr = carve<int>(base, off, n + 1);
    int *frank = carve<int>(base, off, n + 1);
    int *und = carve<int>(base, off, 4);
    int *tot = carve<int>(base, off, 4);
    unsigned char *st = carve<unsigned char>(base, off, n);
    unsigned char *r1 = carve<unsigned char>(base, off, n);
    if (off > NOALLOC_BYTES) return AMGH_ERR_INVALID_ARG;
    int nb = ceil_div(n, 256);
    double th2 = theta * theta;
    k_diag<<<nb, 256, 0, s>>>(n, rp, ci, v, d);
    LAUNCH_CHECK();
    k_strength<<<nb, 256, 0, s>>>(n, rp, ci, v, d, th2, nullptr, cnt, nullptr, nullptr);
    LAUNCH_CHECK();
    int snnz = 0;
    TRY(scan_host_total(cnt, n, srp, tot, s, &snnz));
    k_strength<<<nb, 256, 0, s>>>(n, rp, ci, v, d, th2, srp, cnt, sci, sv);
    LAUNCH_CHECK();
    // distance-2 independent set by rounds (state must start at zero)
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
        if (rounds > n + 1) return AMGH_ERR_TIMEOUT;
    }
    // phases 1-3
    k_root_flag<<<nb, 256, 0, s>>>(n, st, flag);
    LAUNCH_CHECK();
    int nroots = 0;
    TRY(scan_host_total(flag, n, rank, tot, s, &nroots));
    k_phase1<<<nb, 256, 0, s>>>(n, srp, sci, st, rank, agg1);
    LAUNCH_CHECK();
    k_phase2<<<nb, 256, 0, s>>>(n, srp, sci, sv, agg1, agg, fr);
    LAUNCH_CHECK();
    int nfree = 0;
    TRY(scan_host_total(fr, n, frank, tot, s, &nfree));
    if (nfree > 0) {
        k_phase3<<<nb, 256, 0, s>>>(n, fr, frank, nroots, agg);
        LAUNCH_CHECK();
    }
    CU(cudaStreamSynchronize(s));
    *nagg = nroots + nfree;
    return AMGH_OK;
}
