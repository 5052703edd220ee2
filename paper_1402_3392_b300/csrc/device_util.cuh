// device_util.cuh -- small sm_103a building blocks shared by the coder kernels:
// lane masks, mbarrier and bulk-copy (TMA) wrappers in inline PTX, bounded
// waits and the device status word.
#pragma once

#include <cstdint>

#include "rans.h"

namespace rans {

constexpr uint32_t kLog2M = RANS_LOG2_M;
constexpr uint32_t kM = RANS_M;
constexpr uint32_t kL = RANS_L;
constexpr uint32_t kFull = 0xFFFFFFFFu;

// Longest time a kernel waits for one mbarrier phase before it reports
// RANS_ERR_TIMEOUT instead of waiting forever (nanoseconds of %globaltimer).
constexpr uint64_t kWaitNs = 200ull * 1000 * 1000;

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}
__device__ __forceinline__ uint32_t lanemask_ge() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_ge;" : "=r"(m));
    return m;
}
__device__ __forceinline__ uint32_t lane_id() {
    uint32_t l;
    asm("mov.u32 %0, %%laneid;" : "=r"(l));
    return l;
}

__device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }

// v, a value every lane of the (full) warp holds, passed through a warp
// reduction (REDUX) and so known to the compiler as warp-uniform.  The
// batched decoder passes its read positions and ring addresses through it:
// measured faster on B300, with the same instructions executed per opcode
// (ncu), i.e. through the compiler's scheduling of the step alone.
__device__ __forceinline__ uint32_t warp_uniform(uint32_t v) {
    return __reduce_or_sync(kFull, v);
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// First error wins; later errors do not overwrite it.
__device__ __forceinline__ void report(uint32_t *status, uint32_t code) {
    atomicCAS(status, 0u, code);
}

// ---- checked builds ---------------------------------------------------------
// Compiled with -DRANS_CHECKED (a test build), RANS_CHECK(cond) counts a failed
// invariant in this translation unit's counter and yields cond, so that an
// access it guards is skipped; in normal builds it is `true` and cond is not
// evaluated.  take_check_failures() (host) reads and clears the counter.
#ifdef RANS_CHECKED
static __device__ unsigned long long g_check_failures;
__device__ __forceinline__ bool check_ok(bool ok) {
    if (!ok) atomicAdd(&g_check_failures, 1ull);
    return ok;
}
#define RANS_CHECK(cond) (::rans::check_ok(cond))
static inline uint64_t take_check_failures() {
    unsigned long long v = 0, zero = 0;
    if (cudaMemcpyFromSymbol(&v, g_check_failures, sizeof v) != cudaSuccess ||
        cudaMemcpyToSymbol(g_check_failures, &zero, sizeof zero) != cudaSuccess)
        return ~0ull;
    return v;
}
#else
__device__ __forceinline__ constexpr bool check_off() { return true; }
#define RANS_CHECK(cond) (::rans::check_off())
#endif

// ---- mbarrier ---------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}
__device__ __forceinline__ bool mbar_test_wait(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for phase `parity` of barrier `bar` for at most kWaitNs; false if it
// gave up.  The slow path polls without blocking so the bound is wall time.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (;;) {
        if (mbar_test_wait(bar, parity)) return true;
        if (globaltimer_ns() - t0 > kWaitNs) return false;
        __nanosleep(256);
    }
}

// ---- bulk copies (TMA, non-tensor) -------------------------------------------
// global -> shared, completion counted on an mbarrier.  dst, src 16-byte
// aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes,
                                         uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}
// As bulk_g2s, preceded by arming `bar` for `bytes`, both only where `pred`
// holds (predicated instructions: the calling warp does not branch).
__device__ __forceinline__ void bulk_g2s_armed_if(bool pred, uint32_t dst, const void *src,
                                                  uint32_t bytes, uint32_t bar) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.u32 p, %4, 0;\n\t"
        "@p mbarrier.arrive.expect_tx.shared::cta.b64 _, [%3], %2;\n\t"
        "@p cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n\t"
        "}" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar), "r"(uint32_t(pred))
        : "memory");
}
// shared -> global, tracked by bulk async-groups of the issuing thread.
__device__ __forceinline__ void bulk_s2g(void *dst, uint32_t src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(src),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() {
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
template <int N>
__device__ __forceinline__ void bulk_wait() {
    asm volatile("cp.async.bulk.wait_group %0;" ::"n"(N) : "memory");
}
// Make generic-proxy shared-memory writes visible to the async proxy (TMA).
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ uint32_t ld_u16_global(const uint8_t *p) {
    return *reinterpret_cast<const uint16_t *>(p);
}

}  // namespace rans
