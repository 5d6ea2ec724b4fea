// df.cuh -- double-float arithmetic: a value is carried as an unevaluated sum
// hi + lo of two FP32 numbers (about 48 significant bits).  Sums use Knuth's
// error-free two-sum, products the exact FMA residual (Dekker / Knuth; see
// also Hida, Li & Bailey, "Library for double-double and quad-double
// arithmetic", 2000, for the float-pair algorithms).  On GB300 the FP32 pipe
// is ~64x wider than the FP64 pipe, so FP64-accurate vector and SpMV work is
// done this way instead of in FP64.
#pragma once

struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF df_make(float hi, float lo) { return DF{hi, lo}; }

// exact sum a + b = s + e
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// exact when |a| >= |b|
__device__ __forceinline__ void quick_two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    e = b - (s - a);
}

// acc += b (b a plain float), lo not renormalised (accumulator form)
__device__ __forceinline__ void df_add(DF &a, float b)
{
    float s, e;
    two_sum(a.hi, b, s, e);
    a.hi = s;
    a.lo += e;
}

__device__ __forceinline__ void df_merge(DF &a, const DF &b)
{
    df_add(a, b.hi);
    a.lo += b.lo;
}

// normalised x + y, accurate under cancellation (both halves summed with
// two-sum, then renormalised twice)
__device__ __forceinline__ DF df_add2(DF x, DF y)
{
    float s1, e1, s2, e2;
    two_sum(x.hi, y.hi, s1, e1);
    two_sum(x.lo, y.lo, s2, e2);
    e1 += s2;
    quick_two_sum(s1, e1, s1, e1);
    e1 += e2;
    DF r;
    quick_two_sum(s1, e1, r.hi, r.lo);
    return r;
}

// normalised x + y with the low halves added without error compensation
// (relative error ~2^-44 of |x| + |y|): the cheap form for reduction trees
__device__ __forceinline__ DF df_add_fast(DF x, DF y)
{
    float s, e;
    two_sum(x.hi, y.hi, s, e);
    e += x.lo + y.lo;
    DF r;
    quick_two_sum(s, e, r.hi, r.lo);
    return r;
}

// normalised x * y
__device__ __forceinline__ DF df_mul2(DF x, DF y)
{
    float p = x.hi * y.hi;
    float e = fmaf(x.hi, y.hi, -p);
    e += x.hi * y.lo + x.lo * y.hi;
    DF r;
    quick_two_sum(p, e, r.hi, r.lo);
    return r;
}

// normalised x * f (f a plain float)
__device__ __forceinline__ DF df_mulf(DF x, float f)
{
    float p = x.hi * f;
    float e = fmaf(x.hi, f, -p);
    e += x.lo * f;
    DF r;
    quick_two_sum(p, e, r.hi, r.lo);
    return r;
}

// a_hi*z exactly as p + e, plus the small terms; all added into acc
__device__ __forceinline__ void df_fma(DF &acc, float ahi, float alo, float z)
{
    float p = ahi * z;
    float e = fmaf(ahi, z, -p);
    df_add(acc, p);
    acc.lo += e + alo * z;
}

__device__ __forceinline__ void df_fma2(DF &acc, float ahi, float alo, float zhi, float zlo)
{
    float p = ahi * zhi;
    float e = fmaf(ahi, zhi, -p);
    df_add(acc, p);
    acc.lo += e + (ahi * zlo + alo * zhi);
}

__device__ __forceinline__ double df_to_double(DF x) { return (double)x.hi + (double)x.lo; }

__device__ __forceinline__ DF df_from_double(double d)
{
    float hi = (float)d;
    return DF{hi, (float)(d - (double)hi)};
}

// butterfly sum of a DF value over a warp (fixed order)
__device__ __forceinline__ DF df_warp_sum(DF v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        DF w = {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
        v = df_add_fast(v, w);
    }
    return v;
}

// Sum over the grid of NV double-float values per thread: warp butterflies,
// then warp 0 of each block, then the last block to finish sums the blocks'
// partials (double-float, two FP32 halves in each 8-byte slot of partials,
// [NV][gridDim.x]) in fixed order.  Returns true in thread 0 of that block,
// with the sums (as FP64) in tot.  Every FP64 instruction costs ~64 FP32
// issue slots on GB300, so the tree stays on the FP32 pipe.
template <int NV>
__device__ bool reduce_df_last_block(const DF (&val)[NV], double *partials, unsigned *ticket, double (&tot)[NV])
{
    // the partial sums stay double-float (two FP32 halves in each 8-byte
    // slot): on GB300 every FP64 instruction costs ~64 FP32 issue slots
    __shared__ DF shw[NV][32];
    __shared__ bool is_last;
    float2 *part = reinterpret_cast<float2 *>(partials);
    int nb = gridDim.x, w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; q++) {
        DF s = df_warp_sum(val[q]);
        if (l == 0) shw[q][w] = s;
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int q = 0; q < NV; q++) {
            DF t = l < nw ? shw[q][l] : DF{0.f, 0.f};
            t = df_warp_sum(t);
            if (l == 0) part[q * nb + blockIdx.x] = make_float2(t.hi, t.lo);
        }
        if (l == 0) {
            __threadfence();
            unsigned tk = atomicAdd(ticket, 1u);
            is_last = (tk == (unsigned)nb - 1);
        }
    }
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
#pragma unroll
    for (int q = 0; q < NV; q++) {
        DF s = {0.f, 0.f};
        for (int b = threadIdx.x; b < nb; b += blockDim.x) {
            float2 v = __ldcg(&part[q * nb + b]); // L2: written by other blocks
            s = df_add_fast(s, DF{v.x, v.y});
        }
        s = df_warp_sum(s);
        if (l == 0) shw[q][w] = s;
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int q = 0; q < NV; q++) {
            DF t = l < nw ? shw[q][l] : DF{0.f, 0.f};
            t = df_warp_sum(t);
            tot[q] = df_to_double(t);
        }
        if (l == 0) *ticket = 0u;
    }
    return threadIdx.x == 0;
}
