// Device helpers shared by the kernels: mbarrier, bulk asynchronous copy
// (TMA engine) and per-thread asynchronous copy primitives in inline PTX, the
// global timer, bounded waits.
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

// Per-thread asynchronous copies global -> shared (cp.async, no registers
// held while in flight): 16-byte chunks bypassing L1 (.cg: data other blocks
// may have written in the same launch), or 4/8/16-byte elements through L1
// (.ca: data constant during the launch).  The issuing thread waits for all
// of its copies with cp_async_wait_all; other threads see them after a block
// barrier that follows that wait.
__device__ __forceinline__ void cp_async_cg16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
template <int kBytes>
__device__ __forceinline__ void cp_async_ca(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_u32(dst)), "l"(src), "n"(kBytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

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
