// host_util.h -- host-side helpers shared by the entry points of the library:
// argument checks, message geometry and per-device launch facts.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "rans.h"

namespace rans {

constexpr uint64_t round16(uint64_t v) { return (v + 15u) & ~uint64_t(15); }
constexpr uint64_t ceil_div(uint64_t a, uint64_t b) { return (a + b - 1) / b; }

// Geometry of a message of n symbols: chunk count and the byte offset of the
// data region (header + offset table, padded to 16 bytes).
struct MessageGeometry {
    uint64_t n_chunks;
    uint64_t data0;
};

inline bool params_ok(const rans_params *p) {
    return p && p->n_lanes >= 1 && p->n_lanes <= RANS_MAX_LANES && p->chunk_symbols >= 1;
}

inline MessageGeometry geometry(uint64_t n, const rans_params *p) {
    MessageGeometry g;
    g.n_chunks = ceil_div(n, p->chunk_symbols);
    g.data0 = round16(32 + 4 * (g.n_chunks + 1));
    return g;
}

// The model must be a valid static table: 1..256 symbols, frequencies that
// sum to M.  Sets *const_sym to the symbol with f = M, or 0xFFFFFFFF.
inline bool table_ok(const uint16_t *freq, uint32_t n_alpha, uint32_t *const_sym) {
    if (!freq || n_alpha == 0 || n_alpha > RANS_MAX_ALPHABET) return false;
    uint32_t sum = 0, cs = 0xFFFFFFFFu;
    for (uint32_t s = 0; s < n_alpha; ++s) {
        sum += freq[s];
        if (freq[s] == RANS_M) cs = s;
    }
    if (const_sym) *const_sym = cs;
    return sum == RANS_M;
}

// A plain message's model may also have M = 2^13 or 2^14 (b = 2^16 >= M
// keeps one renormalization per symbol): true if the frequencies sum to 2^12,
// 2^13 or 2^14, with *log2m set to that exponent.
inline bool table_log2m(const uint16_t *freq, uint32_t n_alpha, uint32_t *log2m) {
    if (!freq || n_alpha == 0 || n_alpha > RANS_MAX_ALPHABET) return false;
    uint32_t sum = 0;
    for (uint32_t s = 0; s < n_alpha; ++s) sum += freq[s];
    for (uint32_t lm = RANS_LOG2_M; lm <= RANS_LOG2_M_MAX; ++lm)
        if (sum == (1u << lm)) {
            *log2m = lm;
            return true;
        }
    return false;
}

inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Number of SMs of the current device (cached per device).
int sm_count();

// Two non-blocking streams per device, one for host-to-device and one for
// device-to-host copies, created on a device's first use and kept.
struct CopyStreams {
    cudaStream_t in = nullptr, out = nullptr;
};
int copy_streams(CopyStreams *cs);

// Stream `waiter` waits for the work enqueued on `signaler` so far.
bool join(cudaStream_t waiter, cudaStream_t signaler);

// CTA size, 1 .. max_warps warps, for a launch whose n units (chunks, one
// per warp at a time) all start at once: the one that gives the busiest SM
// the fewest warps, the larger of equal ones.  per_sm[w] (w = 1 .. max_warps)
// is the number of w-warp CTAs an SM holds (0: none fits).  A launch of more
// than one wave of max_warps-warp CTAs (or one that fits no CTA) keeps
// max_warps.
inline uint32_t balanced_cta_warps(uint64_t n, uint64_t sms, const int *per_sm,
                                   uint32_t max_warps) {
    if (sms == 0 || max_warps == 0 || per_sm[max_warps] <= 0 ||
        n > uint64_t(per_sm[max_warps]) * sms * max_warps)
        return max_warps;
    auto cdiv = [](uint64_t a, uint64_t b) { return (a + b - 1) / b; };
    uint32_t warps = max_warps;
    uint64_t best = cdiv(cdiv(n, max_warps), sms) * max_warps;
    for (uint32_t w = max_warps - 1; w >= 1; --w) {
        const uint64_t ctas = cdiv(n, w);
        if (per_sm[w] <= 0 || ctas > uint64_t(per_sm[w]) * sms) continue;
        const uint64_t busiest = cdiv(ctas, sms) * w;
        if (busiest < best) {
            best = busiest;
            warps = w;
        }
    }
    return warps;
}

inline int check_launch() {
    return cudaGetLastError() == cudaSuccess ? RANS_OK : RANS_ERR_CUDA;
}

}  // namespace rans
