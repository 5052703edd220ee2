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
