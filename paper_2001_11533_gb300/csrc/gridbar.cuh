// gridbar.cuh -- a bounded software barrier over every block of a cooperative
// launch (all blocks resident at once): an arrival counter and a generation
// word in global memory.  The last block to arrive resets the counter and
// advances the generation; the others poll the generation at most
// g_gridbar_polls times, leaving early once any block has given up.  A block
// that gives up raises g_gridbar_timeout; every block then leaves at its next
// barrier, and the host turns the flag into AMGH_ERR_TIMEOUT.  The barrier
// also orders each block's global writes before the next phase's reads.
//
// The flag and the poll limit have internal linkage: every translation unit
// that includes this file has its own, read and reset by its own host code.
#pragma once

#define GRIDBAR_POLLS (1 << 20)

// arrival counter and generation (zero at rest)
struct GridBar {
    unsigned count, gen;
};

static __device__ int g_gridbar_timeout = 0;
// poll limit of every wait; lowered only by amgh_debug_grid_polls (tests of
// the timeout path)
static __device__ int g_gridbar_polls = GRIDBAR_POLLS;

// Returns false if this block gave up or another one has.
__device__ __forceinline__ bool grid_sync(GridBar *gb, unsigned nblocks)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = &gb->gen;
        volatile int *vto = &g_gridbar_timeout;
        const int limit = *(volatile int *)&g_gridbar_polls;
        const unsigned g0 = *vgen;
        int good = 1;
        __threadfence(); // this block's writes of the phase before its arrival
        if (atomicAdd(&gb->count, 1u) == nblocks - 1) {
            atomicExch(&gb->count, 0u);
            __threadfence();
            atomicAdd(&gb->gen, 1u);
        } else {
            for (int polls = 0; *vgen == g0; polls++) {
                if (polls >= limit || *vto) {
                    atomicExch(&g_gridbar_timeout, 1);
                    good = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}
