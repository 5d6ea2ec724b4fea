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
// Exclusive prefix sum of `n` values into out[0..n] (out[n] = total).  Up to
// SCAN_ONE values: one block, each thread a contiguous chunk.  Beyond: three
// passes (per-block sums, a single-block scan of the block sums, per-block
// scans with the block offset; the last block also writes the total).  Integer
// addition, so the result is exact in any order.  in == out is allowed: every
// element is read and then written by the same thread.
#define SCAN_ONE 16384

// inclusive scan of one value per thread over a block of 1024 threads
template <typename T>
__device__ __forceinline__ T block_incl_scan(T v, T *wsum)
{
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        T t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) wsum[warp] = v;
    __syncthreads();
    if (warp == 0) {
        T w = wsum[lane];
        for (int o = 1; o < 32; o <<= 1) {
            T t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    return warp ? v + wsum[warp - 1] : v;
}

template <typename T>
__global__ void __launch_bounds__(1024) k_scan_one(const T *in, int64_t n, T *out)
{
    __shared__ T wsum[32];
    int chunk = (int)((n + 1023) / 1024);
    int64_t beg = (int64_t)threadIdx.x * chunk, end = beg + chunk < n ? beg + chunk : n;
    T s = 0;
    for (int64_t i = beg; i < end; i++) s += in[i];
    T incl = block_incl_scan<T>(s, wsum);
    T run = incl - s;
    for (int64_t i = beg; i < end; i++) {
        T v = in[i];
        out[i] = run;
        run += v;
    }
    if (threadIdx.x == 1023) out[n] = incl;
}

template <typename T>
__global__ void __launch_bounds__(1024) k_scan_blocksum(const T *__restrict__ in, int64_t n, T *__restrict__ bsum)
{
    __shared__ T wsum[32];
    int64_t i = (int64_t)blockIdx.x * 1024 + threadIdx.x;
    T incl = block_incl_scan<T>(i < n ? in[i] : (T)0, wsum);
    if (threadIdx.x == 1023) bsum[blockIdx.x] = incl;
}

template <typename T>
__global__ void __launch_bounds__(1024) k_scan_apply(const T *in, int64_t n, const T *__restrict__ boff, T *out)
{
    __shared__ T wsum[32];
    int64_t i = (int64_t)blockIdx.x * 1024 + threadIdx.x;
    T v = i < n ? in[i] : (T)0;
    T incl = block_incl_scan<T>(v, wsum);
    if (i < n) out[i] = boff[blockIdx.x] + incl - v;
    if (i == n - 1) out[n] = boff[blockIdx.x] + incl;
}

template <typename T>
int exclusive_scan(const T *in, T *out, int64_t n, cudaStream_t s, T *total_host)
{
    if (n <= SCAN_ONE) {
        k_scan_one<T><<<1, 1024, 0, s>>>(in, n, out);
        LAUNCH_CHECK();
    } else {
        int nb = (int)ceil_div(n, 1024);
        Scratch sc;
        T *bsum = nullptr;
        TRY(sc.alloc(&bsum, nb + 1));
        k_scan_blocksum<T><<<nb, 1024, 0, s>>>(in, n, bsum);
        LAUNCH_CHECK();
        k_scan_one<T><<<1, 1024, 0, s>>>(bsum, nb, bsum); // block offsets, in place
        LAUNCH_CHECK();
        k_scan_apply<T><<<nb, 1024, 0, s>>>(in, n, bsum, out);
        LAUNCH_CHECK();
    } // bsum is freed in stream order
    if (total_host) {
        CU(cudaMemcpyAsync(total_host, out + n, sizeof(T), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
    }
    return AMGH_OK;
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
