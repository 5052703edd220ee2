// rans_check.cu -- diagnostic of the coder kernels' failure path: a bounded
// device-side wait that runs out ends the kernel with a status, not a hang.
#include <cuda_runtime.h>

#include "device_util.cuh"
#include "encode_core.cuh"
#include "host_util.h"

namespace rans {
namespace {

// Look-back words of a two-chunk message (per chunk, per group, group
// accumulator), for lookback_wait_kernel.
__device__ uint64_t g_look_words[6];

// One warp waits on an mbarrier that no thread or copy ever completes, with
// the coder kernels' bounded wait; the status records that it gave up.
__global__ void __launch_bounds__(32) bounded_wait_kernel(uint32_t *status) {
    __shared__ __align__(8) uint64_t bar;
    const uint32_t b = smem_addr(&bar);
    if (threadIdx.x == 0) {
        mbar_init(b, 1);
        fence_mbar_init();
    }
    __syncwarp();
    const bool ok = mbar_wait_bounded(b, 0);
    const uint32_t st = __any_sync(kFull, !ok) ? RANS_ERR_TIMEOUT : RANS_OK;
    if (threadIdx.x == 0) *status = st;
}

// One warp looks back from chunk 1 of a two-chunk message whose chunk 0
// never publishes its size, with the encoder's own look-back and a 200 ms
// bound: it gives up, marks chunk 1 failed, and the kernel writes
// RANS_ERR_TIMEOUT (RANS_OK if the look-back did anything else).
__global__ void __launch_bounds__(32) lookback_wait_kernel(uint32_t *status) {
    const uint32_t lane = threadIdx.x;
    if (lane < 6) g_look_words[lane] = 0;
    __syncwarp();
    const enc::LookBack lb{g_look_words, g_look_words + 2, g_look_words + 4, 2, kWaitNs};
    uint64_t excl = 0;
    const bool done = enc::chunk_offset(lb, 1, 0, lane, excl);
    __syncwarp();
    if (lane == 0) {
        const bool failed = (g_look_words[1] & ~enc::kLookValue) == enc::kLookFailed;
        *status = !done && failed ? RANS_ERR_TIMEOUT : RANS_OK;
    }
}

// Exhaustive check of the encoders' divisions.  CTA (i, part) takes
// frequency f = 1 + i and the part-th slice of kDivSlice states of the range
// an encoder divides by f: after renormalization x lies in the precursor set
// [f L / M, f b L / M) = [f * 2^(16 - lm), f * 2^(32 - lm)) (M = 2^lm, L = b =
// 2^16).  Each x is divided by the product's own code (METHOD 0: the
// multiply-high with the table's reciprocal; METHOD 1: the adaptive coder's
// float estimate and correction) and the quotient q checked against the
// definition of floor(x / f): q * f <= x < (q + 1) * f, in 64 bits.  Counts
// go to out[0] (checked) and out[1] (wrong); out[2] keeps the smallest
// f << 32 | x that was wrong.
constexpr uint32_t kDivThreads = 256;
constexpr uint64_t kDivSlice = 1ull << 22;

template <int METHOD>
__global__ void __launch_bounds__(kDivThreads)
    division_check_kernel(uint32_t lm, unsigned long long *out) {
    const uint32_t f = 1u + blockIdx.x;
    const uint64_t lo = uint64_t(f) << (16 - lm), hi = uint64_t(f) << (32 - lm);
    const uint64_t a = lo + uint64_t(blockIdx.y) * kDivSlice;
    if (a >= hi) return;
    const uint32_t a32 = uint32_t(a);                                // hi <= 2^32
    const uint32_t n = uint32_t(umin64(hi, a + kDivSlice) - a);      // <= kDivSlice
    uint32_t m_lo = 0, k = 0;
    if (METHOD == 0) enc::reciprocal(f, m_lo, k);
    unsigned long long wrong = 0, first = ~0ull;
    for (uint32_t i = threadIdx.x; i < n; i += kDivThreads) {
        const uint32_t x = a32 + i;
        uint32_t q, r = 0;
        if (METHOD == 0) {
            q = enc::div_reciprocal(x, m_lo, k);
        } else {
            q = enc::div_float(x, f, r);
        }
        const uint64_t qf = uint64_t(q) * f;
        bool ok = qf <= x && uint64_t(x) - qf < f;
        if (METHOD == 1) ok = ok && r == uint32_t(uint64_t(x) - qf);
        if (!ok) {
            ++wrong;
            first = umin64(first, (uint64_t(f) << 32) | x);
        }
    }
    __shared__ unsigned long long s_wrong, s_first;
    if (threadIdx.x == 0) {
        s_wrong = 0;
        s_first = ~0ull;
    }
    __syncthreads();
    if (wrong) {
        atomicAdd(&s_wrong, wrong);
        atomicMin(&s_first, first);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(out, (unsigned long long)n);
        if (s_wrong) {
            atomicAdd(out + 1, s_wrong);
            atomicMin(out + 2, s_first);
        }
    }
}

__global__ void division_check_init(unsigned long long *out) {
    out[0] = out[1] = out[3] = 0;
    out[2] = ~0ull;
}

#ifdef RANS_CHECKED
// Checked builds: one invariant that fails on purpose, so a test can see the
// counters work.
__global__ void check_selftest_kernel() {
    if (threadIdx.x == 0) RANS_CHECK(false);
}
#endif

}  // namespace
}  // namespace rans

using namespace rans;

#ifdef RANS_CHECKED
uint64_t rans_check_failures_check() { return take_check_failures(); }
#endif

extern "C" int rans_debug_check_selftest(rans_stream_t stream) {
#ifdef RANS_CHECKED
    check_selftest_kernel<<<1, 32, 0, reinterpret_cast<cudaStream_t>(stream)>>>();
    return check_launch();
#else
    (void)stream;
    return RANS_ERR_INVALID_ARG;
#endif
}

extern "C" int rans_check_bounded_wait(uint32_t *d_status, rans_stream_t stream) {
    if (!d_status) return RANS_ERR_INVALID_ARG;
    bounded_wait_kernel<<<1, 32, 0, reinterpret_cast<cudaStream_t>(stream)>>>(d_status);
    return check_launch();
}

extern "C" int rans_check_lookback_wait(uint32_t *d_status, rans_stream_t stream) {
    if (!d_status) return RANS_ERR_INVALID_ARG;
    lookback_wait_kernel<<<1, 32, 0, reinterpret_cast<cudaStream_t>(stream)>>>(d_status);
    return check_launch();
}

extern "C" int rans_check_division(uint32_t method, uint32_t log2m, uint64_t *d_result,
                                   rans_stream_t stream) {
    if (!d_result || (reinterpret_cast<uintptr_t>(d_result) & 7u) || method > 1 ||
        log2m < 12 || log2m > 14 || (method == 1 && log2m != 12))
        return RANS_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    unsigned long long *out = reinterpret_cast<unsigned long long *>(d_result);
    division_check_init<<<1, 1, 0, st>>>(out);
    int rc = check_launch();
    if (rc != RANS_OK) return rc;
    // frequencies 1 .. M - 1; the largest range, (M - 1) * 2^(32 - lm) - (M - 1)
    // * 2^(16 - lm) states, sets the slices per frequency
    const uint32_t nf = (1u << log2m) - 1;
    const uint64_t span = (uint64_t(nf) << (32 - log2m)) - (uint64_t(nf) << (16 - log2m));
    const dim3 grid(nf, unsigned((span + kDivSlice - 1) / kDivSlice));
    if (method == 0) division_check_kernel<0><<<grid, kDivThreads, 0, st>>>(log2m, out);
    else division_check_kernel<1><<<grid, kDivThreads, 0, st>>>(log2m, out);
    return check_launch();
}
