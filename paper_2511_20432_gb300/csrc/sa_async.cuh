// Device helpers shared by the kernels: mbarrier and bulk asynchronous copy
// (TMA engine) primitives in inline PTX, the global timer, bounded waits.
#pragma once
#include <cuda_runtime.h>

namespace sa_dev {

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes,
                                          unsigned long long* bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for a chunk: false after ~1 s (the caller flags the error).
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (long long it = 0; it < (1ll << 26); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63) == 63 && global_ns() - t0 > 1000000000ull) return false;
    }
    return false;
}

// Orders this thread's earlier generic-proxy accesses (and those it has
// acquired) before its later async-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async;" ::: "memory");
}

// Grid barrier of a cooperative launch.  *count is zero at launch and only
// grows: barrier k (nb counts them, every thread of every block alike)
// completes when it reaches k x gridDim.x.  Thread 0 posts its block's arrival
// with a release reduction (no reply to wait for) and polls with acquire
// loads; a wait over 2 s or 2^30 polls, or a timeout flagged elsewhere, sets
// timeout_flag in *err and returns false.
__device__ __forceinline__ bool count_barrier(unsigned* count, unsigned& nb, int* err,
                                              int timeout_flag) {
    __shared__ int ok;
    __syncthreads();
    ++nb;
    if (threadIdx.x == 0) {
        ok = 1;
        const unsigned target = nb * gridDim.x;
        asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(count), "r"(1u) : "memory");
        const unsigned long long t0 = global_ns();
        long long spins = 0;
        for (;;) {
            unsigned v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
            if ((int)(v - target) >= 0) break;
            if ((++spins & 255) == 0) {
                if (global_ns() - t0 > 2000000000ull || spins > (1ll << 30)) {
                    atomicOr(err, timeout_flag);
                    ok = 0;
                    break;
                }
                if (*((volatile int*)err) & timeout_flag) {
                    ok = 0;
                    break;
                }
            }
        }
    }
    __syncthreads();
    return ok != 0;
}

}  // namespace sa_dev
