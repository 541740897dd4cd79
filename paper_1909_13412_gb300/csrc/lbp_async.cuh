// lbp_async.cuh -- inline-PTX helpers for the asynchronous data movement of
// liblbp's kernels on sm_103a: mbarrier phases (init, arrive, transaction
// counts, bounded waits) and bulk copies into shared memory.  Every wait is
// bounded: a kernel that gives up records it and leaves cleanly.
#pragma once

#include <cuda_runtime.h>

namespace lbp {
namespace async {

// bound of the drain waits at exit, in SM clock cycles (~0.5 s at 2 GHz); each
// try_wait poll may itself suspend the thread for a short, hardware-chosen time
constexpr long long DRAIN_CYCLES = 1ll << 30;

__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned bar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait: true when the phase completed; false when `bound` cycles
// passed or the CTA's abort flag (if given) is set
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, long long bound,
                                          const volatile int *abort_flag) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (abort_flag && *abort_flag) return false;
        if (clock64() - t0 > bound) return false;
    }
    return true;
}

__device__ __forceinline__ void bulk_g2s(unsigned dst, const void *src, unsigned bytes, unsigned bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}


}  // namespace async
}  // namespace lbp

namespace lbp {
namespace async {

// 3-D tiled bulk tensor copy global -> shared through a tensor map (TMA),
// completing on an mbarrier with a transaction byte count.  Coordinates in
// elements, innermost first; out-of-range (including negative) coordinates
// read zeros.
__device__ __forceinline__ void tma_load_3d(unsigned dst, const void *tmap, int x, int y, int z, unsigned bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

}  // namespace async
}  // namespace lbp
