// dwt_grid.cuh -- the bounded grid-wide wait of the cooperative coset-table
// sweeps (dwt_tree.cu, dwt_treep.cu).
//
// flags[3] counts arrivals; flags[2] is set by the first CTA that gives up.
// Every CTA of a cooperative launch (all resident) calls grid_wait the same
// number of times with its own running target.
#pragma once

#include <cuda_runtime.h>

namespace dwt {

constexpr unsigned long long kGridWaitNs = 2000000000ull;   // about two seconds

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// All CTAs arrive at flags[3]; returns false, with flags[2] set, when the wait
// gives up after kGridWaitNs or another CTA gave up first.  ok: one int of the
// CTA's shared memory.
__device__ __forceinline__ bool grid_wait(unsigned* flags, unsigned& target, int* ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        target += gridDim.x;
        __threadfence();
        asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(flags + 3), "r"(1u) : "memory");
        int good = 1;
        const unsigned long long t0 = global_ns();
        while ((int)(ld_acquire_gpu(flags + 3) - target) < 0) {
            if (*(volatile unsigned*)(flags + 2)) {
                good = 0;
                break;
            }
            if (global_ns() - t0 > kGridWaitNs) {
                atomicExch(flags + 2, 1u);
                good = 0;
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
        *ok = good;
    }
    __syncthreads();
    return *ok != 0;
}

}  // namespace dwt
