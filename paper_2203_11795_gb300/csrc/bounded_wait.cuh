// Bounded device-side waits: every spin on a counter another CTA advances gives up after a time
// budget read from %globaltimer, records FFTU_ERR_TIMEOUT in a status word the host reads, and
// lets the kernel return.  Nothing traps: the context stays usable after an expired wait.
#pragma once

#include <cuda_runtime.h>

#include "fftu.h"

namespace fftu {

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Spin until *ctr >= target (gpu-scope acquire) or limit_ns has passed.  On expiry the first error
// wins in *status and the result is false.
__device__ __forceinline__ bool wait_counter_geq(const unsigned *ctr, unsigned target, long long limit_ns,
                                                 int *status) {
    const unsigned long long t0 = globaltimer_ns();
    for (;;) {
        unsigned v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
        if (v >= target) return true;
        if ((long long)(globaltimer_ns() - t0) > limit_ns) {
            atomicCAS(status, 0, (int)FFTU_ERR_TIMEOUT);
            return false;
        }
        __nanosleep(64);
    }
}

}  // namespace fftu
