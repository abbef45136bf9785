// Shared-memory staging primitives of the tiled finest-level kernels
// (k_sweep.cu, k_resid.cu): 16-byte cp.async copies with commit groups, and
// TMA tensor copies (cp.async.bulk.tensor) completed on mbarriers whose waits
// are bounded.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

namespace cdi {
namespace stage {

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
// the issuing thread's arrival; the phase completes once `bytes` have landed
__device__ __forceinline__ void mbar_arrive_tx(unsigned bar, unsigned bytes) {
    if (bytes)
        asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(bar),
                     "r"(bytes)
                     : "memory");
    else
        asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// wait for the phase of the given parity; gives up (false) only after 2^20
// polls and one second
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity) {
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    for (long polls = 0;; ++polls) {
        if (mbar_try(bar, parity)) return true;
        if (polls > (1L << 20) && globaltimer() - t0 > 1000000000ull) return false;
    }
}
// one z plane (box 72 x rows x 1) of a 3D FP32 tensor into shared memory, completed on mbarrier bar
__device__ __forceinline__ void tma_plane(unsigned dst, const CUtensorMap* map, int x, int y, int z, unsigned bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(dst),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}
// order this thread's generic shared-memory writes before later TMA writes to the same bytes
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

}  // namespace stage
}  // namespace cdi
