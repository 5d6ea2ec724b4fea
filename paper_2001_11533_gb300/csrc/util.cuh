// util.cuh -- device helpers: fixed-order warp/block reductions, scans.
#pragma once

#include "internal.cuh"

template <typename T>
int exclusive_scan(const T *in, T *out, int64_t n, cudaStream_t s, T *total_host);

// Butterfly sum inside a warp: the same lanes combine in the same order on
// every run, so the result is deterministic.
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int warp_max_int(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Sum over a block of blockDim.x (multiple of 32, <= 1024) threads; result
// valid in thread 0.  Fixed order: warp butterflies, then warp 0 sums the
// per-warp values.
__device__ __forceinline__ double block_sum(double v, double *sh32)
{
    v = warp_sum(v);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh32[w] = v;
    __syncthreads();
    int nw = blockDim.x >> 5;
    double t = 0.0;
    if (w == 0) {
        t = l < nw ? sh32[l] : 0.0;
        t = warp_sum(t);
    }
    __syncthreads();
    return t;
}

// Last-block finalisation of a two-stage reduction with NV values per block.
// Returns true in thread 0 of the block that finished last; `tot` then holds
// the fixed-order sums of all partials.  partials layout: [NV][gridDim.x].
template <int NV>
__device__ bool reduce_last_block(const double (&val)[NV], double *partials, unsigned *ticket,
                                  double (&tot)[NV])
{
    __shared__ double sh32[NV][32];
    __shared__ bool is_last;
    int nb = gridDim.x;
#pragma unroll
    for (int q = 0; q < NV; q++) {
        double v = warp_sum(val[q]);
        int w = threadIdx.x >> 5, l = threadIdx.x & 31;
        if (l == 0) sh32[q][w] = v;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        int nw = blockDim.x >> 5;
#pragma unroll
        for (int q = 0; q < NV; q++) {
            double t = (int)threadIdx.x < nw ? sh32[q][threadIdx.x] : 0.0;
            t = warp_sum(t);
            if (threadIdx.x == 0) partials[q * nb + blockIdx.x] = t;
        }
    }
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned t = atomicAdd(ticket, 1u);
        is_last = (t == (unsigned)nb - 1);
    }
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
    // fixed-order sum of the nb partials: thread t sums t, t+B, ...; then tree
#pragma unroll
    for (int q = 0; q < NV; q++) {
        double s = 0.0;
        for (int b = threadIdx.x; b < nb; b += blockDim.x) s += ((volatile double *)partials)[q * nb + b];
        s = warp_sum(s);
        int w = threadIdx.x >> 5, l = threadIdx.x & 31;
        if (l == 0) sh32[q][w] = s;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        int nw = blockDim.x >> 5;
#pragma unroll
        for (int q = 0; q < NV; q++) {
            double t = (int)threadIdx.x < nw ? sh32[q][threadIdx.x] : 0.0;
            tot[q] = warp_sum(t);
        }
    }
    if (threadIdx.x == 0) *ticket = 0u;
    return threadIdx.x == 0;
}
