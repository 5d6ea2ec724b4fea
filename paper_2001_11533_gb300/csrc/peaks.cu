// peaks.cu -- the FP64 rates that bound the dense coarsest-level kernels.
//
// The dense factorisation, triangular inverse and products behind the exact
// coarsest solves run in FP64, and the GPU's FP64 rate is far below its FP32
// and low-precision tensor rates.  This measures it both ways the hardware
// offers: fused multiply-adds on the FP64 pipe (eight independent chains per
// thread, every SM busy) and the FP64 tensor instruction mma.m8n8k4.f64
// (four independent accumulators per warp).  The measured figures are the
// denominators of the dense kernels' roofline.
#include "internal.cuh"

__global__ void k_peak_dfma(double *out, int iters, double s)
{
    double a[8];
#pragma unroll
    for (int k = 0; k < 8; k++) a[k] = threadIdx.x * 1e-3 + k;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < 8; k++) a[k] = fma(a[k], s, 1e-9);
    }
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < 8; k++) t += a[k];
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = t;
}

// D = A B + C on an 8 x 8 x 4 tile per warp: A (8 x 4, row) and B (4 x 8,
// col) one double per lane, C and D two doubles per lane
__global__ void k_peak_dmma(double *out, int iters)
{
    int lane = threadIdx.x & 31;
    double a = 1e-3 * lane, b = 1e-3 * (31 - lane);
    double c[4][2];
#pragma unroll
    for (int k = 0; k < 4; k++) c[k][0] = c[k][1] = 0.0;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < 4; k++)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                         : "+d"(c[k][0]), "+d"(c[k][1])
                         : "d"(a), "d"(b));
    }
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < 4; k++) t += c[k][0] + c[k][1];
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = t;
}

extern "C" int amgh_fp64_peak(int kind, void *stream, double *tflops)
{
    if (!tflops || kind < 0 || kind > 1) return AMGH_ERR_INVALID_ARG;
    *tflops = 0.0;
    cudaStream_t s = (cudaStream_t)stream;
    StreamScope ss(s);
    int dev = 0, sms = 0;
    CU(cudaGetDevice(&dev));
    CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int threads = 256, blocks = sms * 8;
    const int iters = kind == 0 ? 2048 : 512; // about 10 ms each
    Scratch sc;
    double *out = nullptr;
    TRY(sc.alloc(&out, (int64_t)blocks * threads));
    auto launch = [&]() {
        if (kind == 0) k_peak_dfma<<<blocks, threads, 0, s>>>(out, iters, 0.9999999);
        else k_peak_dmma<<<blocks, threads, 0, s>>>(out, iters);
        return cudaGetLastError();
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = 0.f;
    cudaError_t err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    if (err == cudaSuccess) err = launch(); // warm-up
    if (err == cudaSuccess) err = cudaEventRecord(e0, s);
    if (err == cudaSuccess) err = launch();
    if (err == cudaSuccess) err = cudaEventRecord(e1, s);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (err != cudaSuccess) {
        amgh_note_error((int)err, __FILE__, __LINE__);
        return AMGH_ERR_CUDA;
    }
    double flops = kind == 0 ? 2.0 * 8 * iters * (double)blocks * threads
                             : 512.0 * 4 * iters * (double)blocks * (threads / 32);
    *tflops = ms > 0.f ? flops / (ms * 1e-3) * 1e-12 : 0.0;
    return AMGH_OK;
}
