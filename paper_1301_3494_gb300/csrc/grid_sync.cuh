// Bounded grid-wide barrier for cooperative launches.
#pragma once
#include <cstdint>

#include "internal.h"

namespace pd {

// Grid-wide barrier with a time bound (the launch is cooperative, so all blocks are resident).
// bar[0] = arrival count, bar[1] = generation, bar[2] = abort flag.  On expiry the block sets
// ERRBIT_TIMEOUT and the abort flag, and every later barrier returns false at once.
// Ordering: each block's thread 0 fences at GPU scope before it arrives and after it sees the new
// generation, and the closing __syncthreads orders the block's other threads after thread 0, so
// every load after the barrier (L1-cached or asynchronous) sees what any block wrote before it.
static __device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned nblocks, unsigned* err) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* vbar = bar;
        int ok = vbar[2] == 0u;
        if (ok) {
            const unsigned gen = vbar[1];
            __threadfence();
            if (atomicAdd(&bar[0], 1u) == nblocks - 1u) {
                atomicExch(&bar[0], 0u);
                __threadfence();
                atomicAdd(&bar[1], 1u);
            } else {
                uint64_t t0;
                asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
                while (vbar[1] == gen) {
                    if (vbar[2]) { ok = 0; break; }
                    uint64_t t;
                    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
                    if (t - t0 > 2000000000ull) {
                        atomicOr(err, ERRBIT_TIMEOUT);
                        atomicExch(&bar[2], 1u);
                        ok = 0;
                        break;
                    }
                }
            }
            __threadfence();
        }
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

}  // namespace pd
