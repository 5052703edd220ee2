// rans_host.cpp -- host-only entry points of the C ABI: model quantization,
// size queries, status strings, and the per-device SM count cache.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

#include "host_util.h"

namespace rans {

int sm_count() {
    static std::mutex mu;
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
    std::lock_guard<std::mutex> lock(mu);
    if (cached[dev] == 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
            n = 148;
        cached[dev] = n;
    }
    return cached[dev];
}

}  // namespace rans

using namespace rans;

extern "C" uint32_t rans_version(void) { return RANS_VERSION; }

extern "C" const char *rans_status_string(int status) {
    switch (status) {
        case RANS_OK: return "ok";
        case RANS_ERR_INVALID_ARG: return "invalid argument";
        case RANS_ERR_ZERO_FREQ: return "symbol with zero frequency";
        case RANS_ERR_BUFFER_TOO_SMALL: return "buffer too small";
        case RANS_ERR_CORRUPT: return "corrupt message";
        case RANS_ERR_TIMEOUT: return "device wait timed out";
        case RANS_ERR_CUDA: return "CUDA error";
        case RANS_ERR_OOM: return "out of memory budget";
        default: return "unknown status";
    }
}

// Static model quantization (the rule is stated in rans.h).  Remainders are
// compared exactly in 128-bit integers.
extern "C" int rans_quantize_table(const uint64_t *weights, uint32_t n, uint32_t log2_M,
                                   uint16_t *freq_out) {
    using u128 = unsigned __int128;
    if (!weights || !freq_out || n == 0 || n > 4096 || log2_M == 0 || log2_M > 15)
        return RANS_ERR_INVALID_ARG;
    const uint64_t M = uint64_t(1) << log2_M;
    u128 W = 0;
    uint64_t nonzero = 0;
    for (uint32_t s = 0; s < n; ++s) {
        W += weights[s];
        nonzero += weights[s] != 0;
    }
    if (W == 0 || (W >> 64) != 0 || nonzero > M) return RANS_ERR_INVALID_ARG;

    std::vector<uint64_t> f(n);
    std::vector<u128> rem(n);
    uint64_t total = 0;
    for (uint32_t s = 0; s < n; ++s) {
        const u128 scaled = u128(weights[s]) << log2_M;
        f[s] = uint64_t(scaled / W);
        rem[s] = scaled % W;
        if (weights[s] != 0 && f[s] == 0) f[s] = 1;
        total += f[s];
    }
    if (total < M) {
        std::vector<uint32_t> order;
        order.reserve(nonzero);
        for (uint32_t s = 0; s < n; ++s)
            if (weights[s] != 0) order.push_back(s);
        std::stable_sort(order.begin(), order.end(),
                         [&](uint32_t a, uint32_t b) { return rem[a] > rem[b]; });
        for (size_t k = 0; total < M; ++k, ++total) f[order[k % order.size()]] += 1;
    }
    while (total > M) {
        const auto it = std::max_element(f.begin(), f.end());  // first maximum
        *it -= 1;
        --total;
    }
    for (uint32_t s = 0; s < n; ++s) freq_out[s] = uint16_t(f[s]);
    return RANS_OK;
}

extern "C" uint64_t rans_max_encoded_size(uint64_t n_symbols, const rans_params *params) {
    if (!params_ok(params)) return 0;
    const MessageGeometry g = geometry(n_symbols, params);
    return g.data0 + round16(4ull * params->n_lanes * g.n_chunks + 2ull * n_symbols);
}

// A byte-wise chunk holds at most two bytes per symbol and up to 3 bytes of
// padding.
extern "C" uint64_t rans_max_encoded_size_bytes(uint64_t n_symbols, const rans_params *params) {
    if (!params_ok(params)) return 0;
    const MessageGeometry g = geometry(n_symbols, params);
    return g.data0 + round16((4ull * params->n_lanes + 3) * g.n_chunks + 2ull * n_symbols);
}

// A bypass message can hold a raw word after every symbol as well.
extern "C" uint64_t rans_max_encoded_size_bypass(uint64_t n_symbols, const rans_params *params) {
    if (!params_ok(params)) return 0;
    const MessageGeometry g = geometry(n_symbols, params);
    return g.data0 + round16(4ull * params->n_lanes * g.n_chunks + 4ull * n_symbols);
}
