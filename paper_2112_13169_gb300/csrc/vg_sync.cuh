// vg_sync.cuh -- the grid-wide barrier of the persistent, cooperative
// launches (k_batch.cu, k_frame.cu).
//
// The CTAs arrive on a counter in global memory; the last of the
// gridDim.x + bar_extra arrivals resets the counter and opens the next
// generation.  Every wait has a deadline: a CTA that has waited bar_ns
// nanoseconds of the GPU's global timer (or that sees the error flag) sets
// the error flag and gives up, so that a launch whose CTAs are not all
// resident, or a fault injected through bar_extra, ends with an error the
// host can read instead of a hung GPU.  The launches are cooperative, so
// all their CTAs are resident together and a barrier only waits for the
// slowest CTA.
#pragma once

#include "vg_internal.cuh"

namespace vg {

__device__ __forceinline__ int64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return (int64_t)t;
}

// C: a control block with bar_count, bar_gen, error, bar_extra (unsigned)
// and bar_ns (int64_t).  Returns false (for every thread of the CTA) when
// the launch has failed.
template <class C>
__device__ bool grid_sync(C *ctl, unsigned nblocks) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned *gen = &ctl->bar_gen;
        volatile unsigned *err = &ctl->error;
        const unsigned g = *gen;
        const unsigned expect = nblocks + ctl->bar_extra;
        const int64_t limit = ctl->bar_ns;
        __threadfence();
        const unsigned arrived = atomicAdd(&ctl->bar_count, 1u) + 1u;
        if (arrived == expect) {
            atomicExch(&ctl->bar_count, 0u);
            __threadfence();
            atomicAdd(&ctl->bar_gen, 1u);
        } else {
            const int64_t t0 = global_ns();
            while (*gen == g) {
                if (*err || global_ns() - t0 > limit) {
                    atomicExch(&ctl->error, 1u);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        if (*err) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

}  // namespace vg
