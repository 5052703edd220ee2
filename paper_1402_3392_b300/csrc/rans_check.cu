// rans_check.cu -- diagnostic of the coder kernels' failure path: a bounded
// device-side wait that runs out ends the kernel with a status, not a hang.
#include <cuda_runtime.h>

#include "decode_core.cuh"
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

// The table decoder's data-pipe work without its arithmetic: the ceiling of
// the SM's L1/shared-memory pipe for the decode step's access mix.  Same
// shape as the plain decoder of large messages (12-warp CTAs, 3 per SM, a
// 16 KiB table per CTA and a 4 KiB ring per warp).  Per step lane j loads the
// table entry of a slot taken from its state (32 random words of the
// 4096-word table, as the decode step's slot lookup), the word at rp + 2j of
// the warp's ring (a contiguous 64-byte window, as the renormalization
// read), and stores one byte to 32 consecutive bytes of the warp's 4 KiB of
// out (as the decoded symbols).  The next state is a multiply-add of both
// loads, so every warp's steps form a chain as the decoder's do; rp moves 24
// bytes a step, about a step's words.  36 warps of such chains ask the pipe
// for several wavefronts a cycle, so the rate this kernel reaches is the
// pipe's.
constexpr int kCeilWarps = dec::kWarpsOne;
constexpr uint32_t kCeilSmem = dec::kTableBytes + dec::kWarpRing + kCeilWarps * dec::kWarpRing;
constexpr uint32_t kCeilOutPerWarp = 4096;

__device__ __forceinline__ uint32_t ceil_mix(uint32_t v) {  // a fixed scramble of v
    v ^= v >> 16;
    v *= 0x7FEB352Du;
    v ^= v >> 15;
    v *= 0x846CA68Bu;
    return v ^ (v >> 16);
}

__global__ void __launch_bounds__(kCeilWarps * 32, 3)
    gather_ceiling_kernel(uint32_t steps, uint8_t *out, uint32_t *sink) {
    extern __shared__ __align__(128) uint8_t smem[];
    uint32_t *tab = reinterpret_cast<uint32_t *>(smem);
    const uint32_t raw = smem_addr(smem + dec::kTableBytes);
    const uint32_t rings_s = (raw + dec::kWarpRing - 1) & ~(dec::kWarpRing - 1);
    uint32_t *rings = reinterpret_cast<uint32_t *>(smem + dec::kTableBytes + (rings_s - raw));
    for (uint32_t i = threadIdx.x; i < kM; i += blockDim.x) tab[i] = ceil_mix(i);
    for (uint32_t i = threadIdx.x; i < kCeilWarps * dec::kWarpRing / 4; i += blockDim.x)
        rings[i] = ceil_mix(i ^ 0x9E3779B9u);
    __syncthreads();
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    const uint32_t tab_s = smem_addr(tab), ring_s = rings_s + warp * dec::kWarpRing;
    uint8_t *o = out + (uint64_t(blockIdx.x) * kCeilWarps + warp) * kCeilOutPerWarp + lane;
    uint32_t x = ceil_mix(blockIdx.x * blockDim.x + threadIdx.x + 1u), rp = 0;
    for (uint32_t t = 0; t < steps; t += 16) {
#pragma unroll
        for (uint32_t u = 0; u < 16; ++u) {
            const uint32_t e = dec::ld_table(dec::imad(x & (kM - 1), 4u, tab_s));
            const uint32_t w = dec::ld_ring_u16(dec::word_at<dec::kWarpRing>(rp, lane, ring_s));
            x = dec::imad(x, 0x9E3779B1u, e ^ w);
            o[((t + u) * 32u) & (kCeilOutPerWarp - 1)] = uint8_t(e);
            rp += 24u;
        }
    }
    if (x == 0u) atomicAdd(sink, 1u);  // keeps the chain live
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

extern "C" uint32_t rans_check_cta_warps(uint64_t n_units, uint32_t sms, const int32_t *per_sm,
                                         uint32_t max_warps) {
    if (!per_sm || max_warps == 0 || max_warps > 32) return 0;
    return rans::balanced_cta_warps(n_units, sms, per_sm, max_warps);
}

extern "C" uint64_t rans_check_gather_ceiling_warps(void) {
    static_assert(3 * (kCeilSmem + 1024) <= 233472, "three CTAs per SM");
    if (cudaFuncSetAttribute(gather_ceiling_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(kCeilSmem)) != cudaSuccess)
        return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gather_ceiling_kernel,
                                                      kCeilWarps * 32, kCeilSmem) != cudaSuccess ||
        per_sm <= 0)
        return 0;
    return uint64_t(per_sm) * uint64_t(sm_count()) * kCeilWarps;
}

extern "C" int rans_check_gather_ceiling(uint32_t steps, uint8_t *d_out, uint64_t out_size,
                                         uint32_t *d_sink, rans_stream_t stream) {
    const uint64_t warps = rans_check_gather_ceiling_warps();
    if (!warps) return RANS_ERR_CUDA;
    if (!d_out || !d_sink || steps == 0 || (steps & 15u)) return RANS_ERR_INVALID_ARG;
    if (out_size < warps * kCeilOutPerWarp) return RANS_ERR_BUFFER_TOO_SMALL;
    gather_ceiling_kernel<<<unsigned(warps / kCeilWarps), kCeilWarps * 32, kCeilSmem,
                            reinterpret_cast<cudaStream_t>(stream)>>>(steps, d_out, d_sink);
    return check_launch();
}
