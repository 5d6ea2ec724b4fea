// util.cu -- arena, launch counting, scans and kernel timing shared by the
// amgh translation units.
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <mutex>

#include "internal.cuh"
#include "util.cuh"

static std::atomic<long long> g_launches{0};
static thread_local int g_capturing = 0;
// launches recorded while a graph is being captured are counted per replay instead
void amgh_count_launch(int n)
{
    if (!g_capturing) g_launches += n;
}
void amgh_set_capturing(int on) { g_capturing = on; }

static std::mutex g_err_mu;
static char g_last_error[256] = "";
static thread_local char g_err_copy[256];

void amgh_note_error(int code, const char *file, int line)
{
    const char *base = strrchr(file, '/');
    std::lock_guard<std::mutex> lock(g_err_mu);
    snprintf(g_last_error, sizeof(g_last_error), "%s (%d) at %s:%d", cudaGetErrorName((cudaError_t)code), code,
             base ? base + 1 : file, line);
}

void amgh_note_msg(const char *msg)
{
    std::lock_guard<std::mutex> lock(g_err_mu);
    snprintf(g_last_error, sizeof(g_last_error), "%s", msg);
}

extern "C" const char *amgh_last_error(void)
{
    std::lock_guard<std::mutex> lock(g_err_mu);
    memcpy(g_err_copy, g_last_error, sizeof(g_err_copy));
    return g_err_copy;
}

// blocks of `block` threads of `kernel` that fit on the current device at once
// (occupancy x SM count), cached per kernel and device
int resident_grid(const void *kernel, int block)
{
    static std::mutex mu;
    static std::vector<std::pair<std::pair<const void *, int>, int>> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1 << 30;
    {
        std::lock_guard<std::mutex> lock(mu);
        for (auto &e : cache)
            if (e.first.first == kernel && e.first.second == dev) return e.second;
    }
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, 0) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        return 1 << 30;
    }
    int g = per_sm * sms;
    std::lock_guard<std::mutex> lock(mu);
    cache.push_back({{kernel, dev}, g});
    return g;
}
extern "C" int64_t amgh_launch_count(void) { return (int64_t)g_launches.load(); }

// ------------------------------------------------------------------ memory pool
thread_local cudaStream_t g_alloc_stream = 0;

static cudaMemPool_t device_pool()
{
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) return nullptr;
        // keep freed memory in the pool (no release at synchronisation points)
        uint64_t keep = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        pools[dev] = pool;
    }
    return pools[dev];
}

int pool_alloc(void **p, size_t bytes)
{
    cudaMemPool_t pool = device_pool();
    if (!pool) return AMGH_ERR_CUDA;
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, g_alloc_stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return e == cudaErrorMemoryAllocation ? AMGH_ERR_OOM : AMGH_ERR_CUDA;
    }
    return AMGH_OK;
}

void pool_free(void *p)
{
    if (p) cudaFreeAsync(p, g_alloc_stream);
}

void Arena::release(void *q)
{
    for (auto &x : ptrs)
        if (x == q) {
            pool_free(q);
            x = nullptr;
        }
}

void Arena::free_all()
{
    for (void *q : ptrs)
        if (q) pool_free(q);
    ptrs.clear();
}

// ------------------------------------------------------------------ scans
// Exclusive prefix sum of `n` values into out[0..n] (out[n] = total), in three
// passes: per-block sums, a single-block scan of the block sums, per-block
// scans with the block offset.  Integer addition, so the result is exact.
template <typename T>
__global__ void k_scan_blocksum(const T *__restrict__ in, int64_t n, T *__restrict__ bsum)
{
    __shared__ T sh[1024];
    int64_t i = (int64_t)blockIdx.x * 1024 + threadIdx.x;
    sh[threadIdx.x] = i < n ? in[i] : (T)0;
    __syncthreads();
    for (int s = 512; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) bsum[blockIdx.x] = sh[0];
}

template <typename T>
__global__ void k_scan_single(T *__restrict__ a, int64_t n, T *__restrict__ total)
{
    // one block of 1024 threads; each thread scans a contiguous chunk
    __shared__ T sh[1024];
    int64_t chunk = (n + 1023) / 1024;
    int64_t beg = threadIdx.x * chunk, end = beg + chunk < n ? beg + chunk : n;
    T s = 0;
    for (int64_t i = beg; i < end; i++) s += a[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    // Hillis-Steele inclusive scan of the 1024 chunk sums
    for (int off = 1; off < 1024; off <<= 1) {
        T v = (int)threadIdx.x >= off ? sh[threadIdx.x - off] : (T)0;
        __syncthreads();
        sh[threadIdx.x] += v;
        __syncthreads();
    }
    T run = threadIdx.x ? sh[threadIdx.x - 1] : (T)0;
    for (int64_t i = beg; i < end; i++) {
        T v = a[i];
        a[i] = run;
        run += v;
    }
    if (threadIdx.x == 1023 && total) *total = sh[1023];
}

template <typename T>
__global__ void k_scan_apply(const T *__restrict__ in, int64_t n, const T *__restrict__ boff,
                             T *__restrict__ out)
{
    __shared__ T sh[1024];
    int64_t i = (int64_t)blockIdx.x * 1024 + threadIdx.x;
    T v = i < n ? in[i] : (T)0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        T t = (int)threadIdx.x >= off ? sh[threadIdx.x - off] : (T)0;
        __syncthreads();
        sh[threadIdx.x] += t;
        __syncthreads();
    }
    if (i < n) out[i] = boff[blockIdx.x] + sh[threadIdx.x] - v;
}

template <typename T>
__global__ void k_set_total(T *out, int64_t n, const T *total) { out[n] = *total; }

template <typename T>
int exclusive_scan(const T *in, T *out, int64_t n, cudaStream_t s, T *total_host)
{
    // out has n+1 entries; in may alias out only if in == out is not required
    int nb = ceil_div(n > 0 ? n : 1, 1024);
    Scratch sc;
    T *bsum = nullptr, *tot = nullptr;
    TRY(sc.alloc(&bsum, nb));
    TRY(sc.alloc(&tot, 1));
    k_scan_blocksum<T><<<nb, 1024, 0, s>>>(in, n, bsum);
    LAUNCH_CHECK();
    k_scan_single<T><<<1, 1024, 0, s>>>(bsum, nb, tot);
    LAUNCH_CHECK();
    k_scan_apply<T><<<nb, 1024, 0, s>>>(in, n, bsum, out);
    LAUNCH_CHECK();
    k_set_total<T><<<1, 1, 0, s>>>(out, n, tot);
    LAUNCH_CHECK();
    if (total_host) {
        CU(cudaMemcpyAsync(total_host, tot, sizeof(T), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
    }
    return AMGH_OK; // bsum / tot are freed in stream order
}

template int exclusive_scan<int>(const int *, int *, int64_t, cudaStream_t, int *);
template int exclusive_scan<long long>(const long long *, long long *, int64_t, cudaStream_t,
                                       long long *);

// ------------------------------------------------------------------ timing
// Events come from a per-problem pool so that timing a launch costs two
// cudaEventRecord calls and no allocation.
static cudaEvent_t pool_get(KernelTimer &t)
{
    if (!t.pool.empty()) {
        cudaEvent_t e = t.pool.back();
        t.pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

thread_local double *g_byte_sink = nullptr;

const char *kclass_name(int c)
{
    static const char *names[KC_N] = {"cheb_step_l0", "cheb_step_coarse", "residual_l0", "residual_coarse",
                                      "restrict_l0", "restrict_coarse", "prolong_l0", "prolong_coarse",
                                      "cg_spmv_l0", "cg_spmv_coarse", "cg_update_l0", "cg_update_coarse",
                                      "coarsest", "spmv_other", "vector_other"};
    return c >= 0 && c < KC_N ? names[c] : "?";
}

void timer_begin(amgh_problem *p, int cls)
{
    if (cls < 0 || !p->timer.enabled || p->capturing || !(p->timer.mask >> cls & 1u)) return;
    cudaEvent_t a = pool_get(p->timer);
    cudaEventRecord(a, p->stream);
    p->timer.ev.push_back(a);
}

void timer_end(amgh_problem *p, int cls, double bytes)
{
    count_bytes(bytes);
    if (cls < 0 || !p->timer.enabled || p->capturing || !(p->timer.mask >> cls & 1u)) return;
    cudaEvent_t b = pool_get(p->timer);
    cudaEventRecord(b, p->stream);
    p->timer.ev.push_back(b);
    p->timer.cls.push_back(cls);
    p->timer.pending_bytes.push_back(bytes);
}

void timer_drop_from(amgh_problem *p, size_t mark)
{
    KernelTimer &t = p->timer;
    if (mark >= t.ev.size()) return;
    for (size_t k = mark; k < t.ev.size(); k++) t.pool.push_back(t.ev[k]);
    t.ev.resize(mark);
    t.cls.resize(mark / 2);
    t.pending_bytes.resize(mark / 2);
}

int timer_collect(amgh_problem *p)
{
    KernelTimer &t = p->timer;
    if (t.ev.empty()) return AMGH_OK;
    CU(cudaStreamSynchronize(p->stream));
    for (size_t k = 0; k + 1 < t.ev.size(); k += 2) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, t.ev[k], t.ev[k + 1]);
        int c = t.cls[k / 2];
        t.ms[c] += ms;
        t.launches[c] += 1;
        t.bytes[c] += t.pending_bytes[k / 2];
    }
    for (auto e : t.ev) t.pool.push_back(e);
    t.ev.clear();
    t.cls.clear();
    t.pending_bytes.clear();
    return AMGH_OK;
}
