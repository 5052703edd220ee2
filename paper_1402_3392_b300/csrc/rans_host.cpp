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

// Two non-blocking streams per device (host-to-device copies and
// device-to-host copies), created on first use and kept for the process.
int copy_streams(CopyStreams *cs) {
    static std::mutex mu;
    static CopyStreams per_dev[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return RANS_ERR_CUDA;
    std::lock_guard<std::mutex> lock(mu);
    CopyStreams &c = per_dev[dev];
    if (!c.in) {
        if (cudaStreamCreateWithFlags(&c.in, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&c.out, cudaStreamNonBlocking) != cudaSuccess) {
            c.in = c.out = nullptr;
            return RANS_ERR_CUDA;
        }
    }
    *cs = c;
    return RANS_OK;
}

// stream `waiter` waits for the work enqueued on `signaler` so far.
bool join(cudaStream_t waiter, cudaStream_t signaler) {
    cudaEvent_t ev;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return false;
    const bool ok = cudaEventRecord(ev, signaler) == cudaSuccess &&
                    cudaStreamWaitEvent(waiter, ev, 0) == cudaSuccess;
    cudaEventDestroy(ev);  // released once the event has completed
    return ok;
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

// ---------------------------------------------------------------------------
// Prefix codes for the instrumented-decoder messages (Section 4).
// ---------------------------------------------------------------------------

// Optimal code lengths <= max_len by package-merge (Larmore and Hirschberg,
// 1990), coin-collector form: list_max holds the used symbols by (weight,
// index); list_d merges the used symbols with the packages of list_{d+1}
// (consecutive pairs, weight the sum, an odd last item dropped) by weight,
// a symbol before a package of equal weight.  The first 2(n - 1) items of
// list_1 are chosen; a chosen package stands for the first two unchosen-yet
// items of the next list, so the choice is carried down level by level as a
// count: every chosen symbol item adds 1 to that symbol's length, and the
// chosen packages of list_d choose the first 2 * (their number) items of
// list_{d+1}.
extern "C" int rans_prefix_lengths(const uint64_t *weights, uint32_t n_alpha, uint32_t max_len,
                                   uint8_t *lengths_out) {
    using u128 = unsigned __int128;
    if (!weights || !lengths_out || n_alpha == 0 || n_alpha > RANS_MAX_ALPHABET || max_len == 0 ||
        max_len > RANS_PREFIX_MAX_LEN)
        return RANS_ERR_INVALID_ARG;
    std::vector<uint32_t> order;
    for (uint32_t s = 0; s < n_alpha; ++s)
        if (weights[s]) order.push_back(s);
    const uint32_t n = uint32_t(order.size());
    if (n == 0 || n > (1u << max_len)) return RANS_ERR_INVALID_ARG;
    std::stable_sort(order.begin(), order.end(),
                     [&](uint32_t a, uint32_t b) { return weights[a] < weights[b]; });
    std::fill(lengths_out, lengths_out + n_alpha, uint8_t(0));
    if (n == 1) {
        lengths_out[order[0]] = 1;
        return RANS_OK;
    }
    struct Item {
        u128 w;
        int32_t sym;  // symbol, or -1 for a package
    };
    std::vector<std::vector<Item>> lists(max_len + 1);
    for (uint32_t s : order) lists[max_len].push_back({weights[s], int32_t(s)});
    for (uint32_t d = max_len - 1; d >= 1; --d) {
        const std::vector<Item> &finer = lists[d + 1];
        std::vector<Item> &cur = lists[d];
        size_t li = 0, pi = 0;
        const size_t n_pk = finer.size() / 2;
        while (li < n || pi < n_pk) {
            const bool take_leaf =
                li < n && (pi >= n_pk || u128(weights[order[li]]) <= finer[2 * pi].w + finer[2 * pi + 1].w);
            if (take_leaf) {
                cur.push_back({weights[order[li]], int32_t(order[li])});
                ++li;
            } else {
                cur.push_back({finer[2 * pi].w + finer[2 * pi + 1].w, -1});
                ++pi;
            }
        }
    }
    size_t chosen = 2 * size_t(n - 1);
    for (uint32_t d = 1; d <= max_len && chosen; ++d) {
        size_t packages = 0;
        for (size_t i = 0; i < chosen && i < lists[d].size(); ++i) {
            if (lists[d][i].sym >= 0) ++lengths_out[lists[d][i].sym];
            else ++packages;
        }
        chosen = 2 * packages;
    }
    return RANS_OK;
}

// Canonical codes: symbols in order of (length, symbol) get consecutive
// codes; moving to a longer length appends zero bits.  Checks lengths <=
// RANS_PREFIX_MAX_LEN, at least one code, and Kraft's inequality.
extern "C" int rans_prefix_codes(const uint8_t *lengths, uint32_t n_alpha, uint16_t *codes_out) {
    if (!lengths || !codes_out || n_alpha == 0 || n_alpha > RANS_MAX_ALPHABET)
        return RANS_ERR_INVALID_ARG;
    std::vector<uint32_t> order;
    uint32_t kraft = 0;  // in units of 2^-RANS_PREFIX_MAX_LEN
    for (uint32_t s = 0; s < n_alpha; ++s) {
        if (lengths[s] > RANS_PREFIX_MAX_LEN) return RANS_ERR_INVALID_ARG;
        if (lengths[s]) {
            order.push_back(s);
            kraft += 1u << (RANS_PREFIX_MAX_LEN - lengths[s]);
        }
    }
    if (order.empty() || kraft > (1u << RANS_PREFIX_MAX_LEN)) return RANS_ERR_INVALID_ARG;
    std::stable_sort(order.begin(), order.end(),
                     [&](uint32_t a, uint32_t b) { return lengths[a] < lengths[b]; });
    std::fill(codes_out, codes_out + n_alpha, uint16_t(0));
    uint32_t code = 0, len = lengths[order[0]];
    for (uint32_t s : order) {
        code <<= lengths[s] - len;
        len = lengths[s];
        codes_out[s] = uint16_t(code++);
    }
    return RANS_OK;
}

// A chunk of a prefix message holds at most ceil(12 n_c / 32) + 2N words: a
// coder's decoder reads at most one word more than its codes fill.
extern "C" uint64_t rans_max_encoded_size_prefix(uint64_t n_symbols, const rans_params *params) {
    if (!params_ok(params)) return 0;
    const MessageGeometry g = geometry(n_symbols, params);
    return g.data0 + round16(4ull * ((n_symbols * RANS_PREFIX_MAX_LEN + 31) / 32 +
                                     g.n_chunks * (2ull * params->n_lanes + 1)));
}

// Checked builds (-DRANS_CHECKED): the failed invariants of all kernels since
// the last call, summed over the files that define kernels.
#ifdef RANS_CHECKED
uint64_t rans_check_failures_decode();
uint64_t rans_check_failures_encode();
uint64_t rans_check_failures_batch();
uint64_t rans_check_failures_prefix();
uint64_t rans_check_failures_check();
#endif

extern "C" int rans_debug_checks(uint64_t *failures) {
#ifdef RANS_CHECKED
    if (!failures) return RANS_ERR_INVALID_ARG;
    if (cudaDeviceSynchronize() != cudaSuccess) return RANS_ERR_CUDA;
    const uint64_t parts[] = {rans_check_failures_decode(), rans_check_failures_encode(),
                              rans_check_failures_batch(), rans_check_failures_prefix(),
                              rans_check_failures_check()};
    uint64_t sum = 0;
    for (uint64_t v : parts) {
        if (v == ~0ull) return RANS_ERR_CUDA;
        sum += v;
    }
    *failures = sum;
    return RANS_OK;
#else
    (void)failures;
    return RANS_ERR_INVALID_ARG;
#endif
}
