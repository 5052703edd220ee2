// rans_encode.cu -- single-message GPU encoder: one warp per chunk
// (encode_core.cuh).  A whole message is coded and placed in one launch (each
// warp finds its chunk's offset by look-back over the sizes before it and
// copies the chunk into the message); pieces of a message (host-memory
// encoding) use a scan of the chunk sizes and a separate copy.
#include <algorithm>
#include <deque>
#include <mutex>

#include <cuda_runtime.h>

#include "encode_core.cuh"
#include "host_util.h"

namespace rans {
namespace {

using enc::kSmemBytes;
using enc::kWarps;
using enc::ScratchLayout;
using enc::scratch_layout;
using enc::adaptive_ctx_stride;

struct EncodeParams {
    const uint8_t *sym;
    uint8_t *words;      // scratch: n_chunks slots of slot_bytes
    uint32_t *states;    // scratch: n_chunks * N final states
    uint32_t *wstart;    // scratch: first word byte of each slot
    uint32_t *sizes;     // scratch: chunk bytes 4N + 2W
    uint32_t *status;
    uint64_t n_sym;
    uint32_t N;
    uint32_t CS;
    uint32_t n_chunks;
    uint32_t slot_bytes;
    uint32_t c_begin, c_end;  // chunks [c_begin, c_end) are coded by this launch
    uint32_t log2m;           // plain messages: log2 M (12, 13 or 14)
    const uint16_t *raw;  // bypass messages: raw word of each symbol
    uint32_t *ctx;        // adaptive messages: scratch, pass 1's words per chunk
    uint64_t ctx_stride;  // u32 words per chunk in ctx
    uint32_t n_alpha;     // adaptive-n messages: the alphabet size n
    // Whole messages placed by the coder itself: the message and where its
    // pieces are, and the chunk ticket (zeroed before the launch).
    enc::Placement pl;
    uint32_t *ticket;
    uint16_t freq[RANS_MAX_ALPHABET];
    uint8_t raw_words[RANS_MAX_ALPHABET];  // bypass: raw words symbol s carries (0 or 1)
};

// Message kinds: plain (version 1), bypass (version 2: a raw word after every
// symbol that carries one), byte-wise (version 3: b = 2^8) and adaptive
// (version 4: binary symbols, one adaptive context per coder).
constexpr int kPlain = 0, kBypass = 1, kBytes = 2, kAdaptive = 3;
// Plain messages with M = 2^13 or 2^14 (16-byte table entries).
constexpr int kWide = 4;
// Adaptive models over n symbols (version 6), per coder, with room for 3, 7
// or 15 boundaries (n <= 4, 8, 16): pass 1 stores each symbol's (B, f).
constexpr int kAdaptN4 = 5, kAdaptN8 = 6, kAdaptN16 = 7;
template <int KIND>
struct AdaptN {
    static constexpr bool kOn = KIND == kAdaptN4 || KIND == kAdaptN8 || KIND == kAdaptN16;
    static constexpr int kNB = KIND == kAdaptN4 ? 3 : KIND == kAdaptN8 ? 7 : 15;
};

// PLACE: the next chunk number from the ticket counter (the order the warps
// start their chunks), else chunks strided over the grid's warps.
template <bool PLACE>
__device__ __forceinline__ uint32_t next_chunk(const EncodeParams &p, uint32_t c, uint32_t lane) {
    if (!PLACE) return c + gridDim.x * kWarps;
    uint32_t t = 0;
    if (lane == 0) t = atomicAdd(p.ticket, 1u);
    return p.c_begin + __shfl_sync(kFull, t, 0);
}

// LAT: encode_chunk's latency form (plain chunks of 32 coders, messages of
// few chunks).
template <int NT, int KIND, bool PLACE = false, bool LAT = false>
__device__ __forceinline__ void encode_body(const EncodeParams &p) {
    constexpr bool RAW = KIND == kBypass;
    constexpr bool BYTES = KIND == kBytes;
    constexpr bool ADAPT = KIND == kAdaptive;
    constexpr bool WIDE = KIND == kWide;
    constexpr bool ADAPTN = AdaptN<KIND>::kOn;
    extern __shared__ __align__(128) uint8_t smem[];
    const enc::Smem sm = enc::smem_layout(smem);
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    if (WIDE)
        enc::build_wide_encode_table(p.freq, p.log2m, reinterpret_cast<uint4 *>(sm.tab),
                                     reinterpret_cast<uint32_t *>(sm.rings));
    else if (!ADAPT && !ADAPTN)  // adaptive models need no table
        enc::build_encode_table(p.freq, sm.tab, reinterpret_cast<uint32_t *>(sm.rings),
                                RAW ? p.raw_words : nullptr);
    const uint32_t ring_s = sm.rings_s + warp * enc::kRing;
    const uint32_t ge = lanemask_ge();
    uint32_t acc = 0;
    // PLACE: a chunk is placed after the warp's next chunk is coded (its
    // last chunk at the end), when the chunks before it have long been
    // published: the look-back rarely waits.  Trying at once, without
    // waiting, measured slower (1 GiB: 1.515 against 1.430 ms).
    constexpr uint32_t kNone = 0xFFFFFFFFu;
    constexpr int kCopyU = ADAPT || ADAPTN ? 2 : 4;
    uint32_t pending = kNone;
    for (uint32_t c = PLACE ? next_chunk<true>(p, 0, lane) : p.c_begin + blockIdx.x * kWarps + warp;
         c < p.c_end; c = next_chunk<PLACE>(p, c, lane)) {
        const uint64_t first = uint64_t(c) * p.CS;
        const uint32_t n_c = uint32_t(umin64(p.CS, p.n_sym - first));
        uint32_t *ctx = ADAPT || ADAPTN ? p.ctx + uint64_t(c) * p.ctx_stride : nullptr;
        if (ADAPT) enc::adaptive_forward<NT>(p.sym + first, n_c, p.N, ctx, lane, acc);
        if (ADAPTN)
            enc::adaptive_n_forward<NT, AdaptN<KIND>::kNB>(p.sym + first, n_c, p.N, p.n_alpha, ctx,
                                                          lane, acc);
        enc::encode_chunk<NT, !RAW && !ADAPT && !ADAPTN, RAW, BYTES, ADAPT, WIDE, ADAPTN, false, LAT>(
            p.sym + first, n_c, p.N, p.words + uint64_t(c) * p.slot_bytes, p.slot_bytes,
            p.wstart + c, p.sizes + c, p.states + uint64_t(c) * p.N, sm.tab_s, ring_s, ge, lane,
            acc, RAW ? p.raw + first : nullptr, ctx);
        if (PLACE) {
            enc::chunk_coded(p.pl, c, lane, acc);
            if (pending != kNone) enc::place_chunk<BYTES, kCopyU>(p.pl, pending, lane);
            pending = c;
        }
    }
    // The last chunk's copy, with the coding registers free: twice the
    // blocks in flight (1 GiB: 1250 -> 1238 us).  Plain chunks of 32 coders
    // and wide ones only: the other kernels then spilled.
    constexpr int kLastU = (KIND == kPlain && NT == 32) || WIDE ? 8 : kCopyU;
    if (PLACE && pending != kNone) enc::place_chunk<BYTES, kLastU>(p.pl, pending, lane);
    // Symbols with f_s = 0 leave the table's flag bit in acc.
    if (__any_sync(kFull, acc & enc::kZeroFlag) && lane == 0) report(p.status, RANS_ERR_ZERO_FREQ);
    if (lane == 0) bulk_wait<0>();
}

// Four CTAs per SM (64 registers) for every kind but the 13/14-bit models,
// whose 16-byte table entries need more registers than that (two or three
// CTAs per SM), and the plain 32-coder kernel: left unbounded it takes 80
// registers (three CTAs per SM) for its two register sets of prefetched
// symbols, and ran faster so than held to 64 with spills (measured on B300,
// 1 GiB: 1246 against 1257 us).  The others need the bound.
template <int NT, int KIND, bool PLACE, bool LAT = false>
__global__ void __launch_bounds__(enc::kThreads, KIND == kPlain && NT == 32 ? 0 : 4)
    encode_kernel(const __grid_constant__ EncodeParams p) {
    encode_body<NT, KIND, PLACE, LAT>(p);
}

template <int NT, bool PLACE>
__global__ void __launch_bounds__(enc::kThreads)
    encode_kernel_wide(const __grid_constant__ EncodeParams p) {
    encode_body<NT, kWide, PLACE>(p);
}

// After a placing launch: a rejected message has size 0 (the last chunk may
// have written the header before another chunk reported).
__global__ void settle_kernel(const uint32_t *status, uint64_t *out_size) {
    if (*status != RANS_OK) *out_size = 0;
}

struct FinalizeParams {
    uint8_t *out;
    uint64_t *out_size;
    const uint32_t *sizes;
    const uint32_t *status;
    uint64_t n_sym;
    uint32_t N, CS, n_chunks, data0, version, log2m;
};

constexpr int kScanThreads = 1024;
__global__ void __launch_bounds__(kScanThreads)
    finalize_kernel(const __grid_constant__ FinalizeParams p) {
    __shared__ uint32_t warp_sums[32];
    __shared__ uint64_t carry_s;
    if (*p.status != RANS_OK) {
        if (threadIdx.x == 0) *p.out_size = 0;
        return;
    }
    enc::finalize_message(p.out, p.out_size, p.sizes, p.n_sym, p.N, p.CS, p.n_chunks, p.data0,
                          warp_sums, &carry_s, p.version, p.log2m);
}

struct PackParams {
    uint8_t *out;
    const uint8_t *words;
    const uint32_t *states;
    const uint32_t *wstart;
    const uint32_t *status;
    const uint32_t *offs;     // chunk offsets, or nullptr: out's own offset table
    uint32_t N, n_chunks, data0, slot_bytes;
    uint32_t c_begin, c_end;  // chunks packed by this launch
};

constexpr int kPackThreads = 256;
template <bool BYTES>
__global__ void __launch_bounds__(kPackThreads) pack_kernel(const __grid_constant__ PackParams p) {
    if (*p.status != RANS_OK) return;
    for (uint32_t c = p.c_begin + blockIdx.x; c < p.c_end; c += gridDim.x)
        enc::pack_chunk<BYTES>(p.out, p.data0, p.words, p.states, p.wstart, p.N, p.slot_bytes, c,
                               p.offs);
}

// Plain messages of 32 coders and up to this many chunks take the encoder's
// latency form (encode_chunk's LAT): up to a wave and a third of the placing
// coder's warps (3 CTAs of 8 warps per SM on 148 SMs), where the SM has too
// few warps to hide a step's latencies.  Measured on B300 (chunks of 64 Ki
// symbols, latency form against the other): 1184 chunks 202.0 -> 165.3 us,
// 2368 chunks 251.9 -> 232.7 us; with each step's ballot and store deferred
// into the next step, 2960 chunks 312.6 -> 304.8 us, 4144 chunks 419.2 ->
// 404.0 us, 4736 chunks 430.7 -> 416.2 us, but 5328 chunks 470.7 -> 477.8 us
// and 7104 chunks 579.2 -> 605.2 us.
constexpr uint32_t kLatMaxChunks = 4736;

// Dynamic shared memory of a CTA of w warps: the table, the rings' alignment
// slack, w rings and the CTA-state words.  The single-message kernels touch
// only the table and their warps' rings.
constexpr uint32_t smem_for_warps(uint64_t w) {
    return uint32_t(enc::kTabBytes + enc::kRing + w * enc::kRing + 64);
}

// Resident CTAs per SM of `kernel` with CTAs of w = 1 .. kWarps warps
// (per_sm[w]; 0 where none fits), computed once per device and kernel.
const int *occupancy_by_warps(void (*kernel)(EncodeParams)) {
    struct Entry {
        int dev;
        void (*k)(EncodeParams);
        int per_sm[kWarps + 1];
    };
    static std::mutex mu;
    static std::deque<Entry> cache;  // push_back leaves earlier entries in place
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    for (const Entry &e : cache)
        if (e.dev == dev && e.k == kernel) return e.per_sm;
    Entry e{dev, kernel, {0}};
    for (uint64_t w = 1; w <= uint64_t(kWarps); ++w)
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&e.per_sm[w], kernel, int(w * 32),
                                                          smem_for_warps(w)) != cudaSuccess)
            return nullptr;
    cache.push_back(e);
    return cache.back().per_sm;
}

template <int NT, int KIND, bool PLACE = false>
int launch_encode(const EncodeParams &p, cudaStream_t stream) {
    void (*kernel)(EncodeParams);
    if constexpr (KIND == kWide) kernel = encode_kernel_wide<NT, PLACE>;
    else if constexpr (KIND == kPlain && NT == 32)
        kernel = p.c_end - p.c_begin <= kLatMaxChunks ? encode_kernel<NT, KIND, PLACE, true>
                                                      : encode_kernel<NT, KIND, PLACE, false>;
    else kernel = encode_kernel<NT, KIND, PLACE>;
    const int *per_sm = occupancy_by_warps(kernel);
    if (!per_sm || per_sm[kWarps] <= 0) return RANS_ERR_CUDA;
    const uint64_t n = p.c_end - p.c_begin, sms = sm_count();
    // Warps per CTA: kWarps, but a placing launch whose chunks all start at
    // once (at most one wave) takes the CTA size that gives the busiest SM the
    // fewest warps, the larger of equal ones: the message is done when that
    // SM's chunks are, and the others wait for it.  Its chunks come from the
    // ticket counter, so any CTA size covers them all.  Measured on B300
    // (chunks of 64 Ki symbols, 8-warp CTAs against the chosen size): plain
    // 148 chunks 129.0 -> 105.6 us (1 warp), 592 chunks 149.9 -> 130.4 us (4
    // warps), 2960 chunks 306.3 -> 271.7 us; adaptive-n models over 16
    // symbols, 4096 chunks, 2407 -> 2263 us; over 8, 1405 -> 1301 us.
    uint64_t warps = kWarps;
    if constexpr (PLACE && KIND != kWide) warps = balanced_cta_warps(n, sms, per_sm, kWarps);
    const uint64_t want = ceil_div(n, warps);
    const uint64_t cap = uint64_t(per_sm[warps]) * sms;
    const unsigned grid = unsigned(std::max<uint64_t>(1, std::min(want, cap)));
    kernel<<<grid, unsigned(warps * 32), smem_for_warps(warps), stream>>>(p);
    return check_launch();
}

// Code and place a whole message of n_chunks > 0 chunks (ep complete but for
// the placement fields): zero the look-back words and the ticket, launch the
// placing coder, then settle the size.
int encode_placed(EncodeParams &ep, const ScratchLayout &sl, uint8_t *scr, uint8_t *d_out,
                  uint64_t *d_out_size, uint32_t data0, uint32_t version, int kind,
                  cudaStream_t st) {
    enc::Placement &m = ep.pl;
    m.out = d_out;
    m.out_size = d_out_size;
    m.status = ep.status;
    m.words = ep.words;
    m.states = ep.states;
    m.wstart = ep.wstart;
    m.sizes = ep.sizes;
    m.lb = enc::scratch_lookback(scr, sl, ep.n_chunks, ep.CS, ep.N);
    m.n_sym = ep.n_sym;
    m.N = ep.N;
    m.CS = ep.CS;
    m.data0 = data0;
    m.slot_bytes = ep.slot_bytes;
    m.version = version;
    m.log2m = ep.log2m;
    ep.ticket = reinterpret_cast<uint32_t *>(scr + sl.ticket);
    ep.c_begin = 0;  // the placed coder always covers the whole message
    if (cudaMemsetAsync(scr + sl.look, 0, sl.total - sl.look, st) != cudaSuccess)
        return RANS_ERR_CUDA;
    const bool n32 = ep.N == 32;
    int rc;
    switch (kind) {
        case kWide: rc = n32 ? launch_encode<32, kWide, true>(ep, st) : launch_encode<0, kWide, true>(ep, st); break;
        case kAdaptive: rc = n32 ? launch_encode<32, kAdaptive, true>(ep, st) : launch_encode<0, kAdaptive, true>(ep, st); break;
        case kAdaptN4: rc = n32 ? launch_encode<32, kAdaptN4, true>(ep, st) : launch_encode<0, kAdaptN4, true>(ep, st); break;
        case kAdaptN8: rc = n32 ? launch_encode<32, kAdaptN8, true>(ep, st) : launch_encode<0, kAdaptN8, true>(ep, st); break;
        case kAdaptN16: rc = n32 ? launch_encode<32, kAdaptN16, true>(ep, st) : launch_encode<0, kAdaptN16, true>(ep, st); break;
        case kBypass: rc = n32 ? launch_encode<32, kBypass, true>(ep, st) : launch_encode<0, kBypass, true>(ep, st); break;
        case kBytes: rc = n32 ? launch_encode<32, kBytes, true>(ep, st) : launch_encode<0, kBytes, true>(ep, st); break;
        default: rc = n32 ? launch_encode<32, kPlain, true>(ep, st) : launch_encode<0, kPlain, true>(ep, st); break;
    }
    if (rc != RANS_OK) return rc;
    settle_kernel<<<1, 1, 0, st>>>(ep.status, d_out_size);
    return check_launch();
}

// The header of a message without chunks.
int encode_empty(uint8_t *d_out, uint64_t *d_out_size, uint32_t *d_status, uint64_t n_sym,
                 const rans_params *params, uint32_t data0, uint32_t version, uint32_t log2m,
                 cudaStream_t st) {
    FinalizeParams fp{};
    fp.out = d_out;
    fp.out_size = d_out_size;
    fp.status = d_status;
    fp.n_sym = n_sym;
    fp.N = params->n_lanes;
    fp.CS = params->chunk_symbols;
    fp.n_chunks = 0;
    fp.data0 = data0;
    fp.version = version;
    fp.log2m = log2m;
    finalize_kernel<<<1, kScanThreads, 0, st>>>(fp);
    return check_launch();
}

}  // namespace
}  // namespace rans

using namespace rans;

extern "C" uint64_t rans_encode_scratch_size(uint64_t n_symbols, const rans_params *params) {
    if (!params_ok(params)) return 0;
    const MessageGeometry g = geometry(n_symbols, params);
    return scratch_layout(g.n_chunks, params->n_lanes, params->chunk_symbols).total;
}

extern "C" uint64_t rans_encode_scratch_size_bypass(uint64_t n_symbols, const rans_params *params) {
    if (!params_ok(params)) return 0;
    const MessageGeometry g = geometry(n_symbols, params);
    return scratch_layout(g.n_chunks, params->n_lanes, params->chunk_symbols, 2).total;
}

// rans_encode and rans_encode_bypass: raw_words == nullptr for a plain
// message, else a bypass message with d_raw[i] after symbol i where
// raw_words[symbol] = 1.
static int encode_message(const uint8_t *d_symbols, const uint16_t *d_raw, uint64_t n_symbols,
                          const uint16_t *h_freq, const uint8_t *raw_words, uint32_t n_alpha,
                          const rans_params *params, uint8_t *d_out, uint64_t out_cap,
                          uint64_t *d_out_size, uint32_t *d_status, void *d_scratch,
                          uint64_t scratch_cap, rans_stream_t stream, bool bytes = false,
                          bool adaptive = false, uint32_t adaptive_n = 0) {
    // Plain messages may use M = 2^13 or 2^14 (the table's sum); the other
    // kinds keep M = 2^12.  adaptive_n > 0: adaptive models over that many
    // symbols (the model argument is not used).
    const bool plain = raw_words == nullptr && !bytes && !adaptive && !adaptive_n;
    uint32_t lm = RANS_LOG2_M;
    if (!params_ok(params) ||
        !(plain ? table_log2m(h_freq, n_alpha, &lm) : table_ok(h_freq, n_alpha, nullptr)) ||
        !d_out || !d_out_size || !d_status || !d_scratch || !aligned16(d_out) ||
        !aligned16(d_scratch))
        return RANS_ERR_INVALID_ARG;
    if (n_symbols && !d_symbols) return RANS_ERR_INVALID_ARG;
    const bool bypass = raw_words != nullptr;
    if (bypass && n_symbols && (!d_raw || (reinterpret_cast<uintptr_t>(d_raw) & 1u)))
        return RANS_ERR_INVALID_ARG;
    const uint32_t wps = bypass ? 2u : 1u;
    const MessageGeometry g = geometry(n_symbols, params);
    // Offsets are u32: the worst-case data region must fit.
    if (g.n_chunks > 0xFFFFFFFEull ||
        (4ull * params->n_lanes + (bytes ? 3u : 0u)) * g.n_chunks + 2ull * wps * n_symbols >
            0xFFFFFFF0ull)
        return RANS_ERR_INVALID_ARG;
    const ScratchLayout sl =
        scratch_layout(g.n_chunks, params->n_lanes, params->chunk_symbols, wps);
    const uint64_t max_out = bypass  ? rans_max_encoded_size_bypass(n_symbols, params)
                             : bytes ? rans_max_encoded_size_bytes(n_symbols, params)
                                     : rans_max_encoded_size(n_symbols, params);
    const uint64_t ctx_stride = adaptive_n ? uint64_t(params->chunk_symbols)
                                           : adaptive_ctx_stride(params->chunk_symbols,
                                                                 params->n_lanes);
    const uint64_t need_scratch =
        adaptive || adaptive_n ? sl.ctx + round16(4 * g.n_chunks * ctx_stride) : sl.total;
    if (out_cap < max_out || scratch_cap < need_scratch) return RANS_ERR_BUFFER_TOO_SMALL;

    EncodeParams ep{};
    if (bypass) {
        for (uint32_t s = 0; s < n_alpha; ++s) {
            if (raw_words[s] > 1) return RANS_ERR_INVALID_ARG;
            ep.raw_words[s] = raw_words[s];
        }
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(d_status, 0, sizeof(uint32_t), st) != cudaSuccess) return RANS_ERR_CUDA;
    uint8_t *scr = static_cast<uint8_t *>(d_scratch);

    ep.sym = d_symbols;
    ep.raw = d_raw;
    ep.words = scr + sl.words;
    ep.states = reinterpret_cast<uint32_t *>(scr + sl.states);
    ep.wstart = reinterpret_cast<uint32_t *>(scr + sl.wstart);
    ep.sizes = reinterpret_cast<uint32_t *>(scr + sl.sizes);
    ep.ctx = reinterpret_cast<uint32_t *>(scr + sl.ctx);
    ep.ctx_stride = ctx_stride;
    ep.status = d_status;
    ep.n_sym = n_symbols;
    ep.N = params->n_lanes;
    ep.CS = params->chunk_symbols;
    ep.n_chunks = uint32_t(g.n_chunks);
    ep.slot_bytes = sl.slot_bytes;
    ep.c_begin = 0;
    ep.c_end = ep.n_chunks;
    ep.log2m = lm;
    ep.n_alpha = adaptive_n;
    for (uint32_t s = 0; s < n_alpha; ++s) ep.freq[s] = h_freq[s];

    const uint32_t version = bypass       ? RANS_VERSION_BYPASS
                             : bytes      ? RANS_VERSION_BYTES
                             : adaptive   ? RANS_VERSION_ADAPTIVE
                             : adaptive_n ? RANS_VERSION_ADAPTIVE_N
                                          : RANS_VERSION;
    // adaptive-n headers record n beside log2 M
    const uint32_t hdr_lm = adaptive_n ? lm | (adaptive_n << 16) : lm;
    ep.log2m = hdr_lm;
    if (g.n_chunks == 0)
        return encode_empty(d_out, d_out_size, d_status, n_symbols, params, uint32_t(g.data0),
                            version, hdr_lm, st);
    const int kind = adaptive_n      ? (adaptive_n <= 4 ? kAdaptN4 : adaptive_n <= 8 ? kAdaptN8
                                                                                  : kAdaptN16)
                     : lm != RANS_LOG2_M ? kWide
                     : adaptive        ? kAdaptive
                     : bypass          ? kBypass
                     : bytes           ? kBytes
                                       : kPlain;
    return encode_placed(ep, sl, scr, d_out, d_out_size, uint32_t(g.data0), version, kind, st);
}

extern "C" uint64_t rans_encode_scratch_size_adaptive(uint64_t n_symbols, const rans_params *params) {
    if (!params_ok(params)) return 0;
    const MessageGeometry g = geometry(n_symbols, params);
    return scratch_layout(g.n_chunks, params->n_lanes, params->chunk_symbols).ctx +
           round16(4 * g.n_chunks *
                   adaptive_ctx_stride(params->chunk_symbols, params->n_lanes));
}

extern "C" int rans_encode_adaptive(const uint8_t *d_symbols, uint64_t n_symbols,
                                    const rans_params *params, uint8_t *d_out, uint64_t out_cap,
                                    uint64_t *d_out_size, uint32_t *d_status, void *d_scratch,
                                    uint64_t scratch_cap, rans_stream_t stream) {
    const uint16_t any_model[2] = {RANS_M / 2, RANS_M / 2};  // the contexts need no table
    return encode_message(d_symbols, nullptr, n_symbols, any_model, nullptr, 2, params, d_out,
                          out_cap, d_out_size, d_status, d_scratch, scratch_cap, stream, false,
                          true);
}

extern "C" uint64_t rans_encode_scratch_size_adaptive_n(uint64_t n_symbols,
                                                        const rans_params *params) {
    if (!params_ok(params)) return 0;
    const MessageGeometry g = geometry(n_symbols, params);
    return scratch_layout(g.n_chunks, params->n_lanes, params->chunk_symbols).ctx +
           round16(4 * g.n_chunks * uint64_t(params->chunk_symbols));
}

extern "C" int rans_encode_adaptive_n(const uint8_t *d_symbols, uint64_t n_symbols,
                                      uint32_t n_alpha, const rans_params *params, uint8_t *d_out,
                                      uint64_t out_cap, uint64_t *d_out_size, uint32_t *d_status,
                                      void *d_scratch, uint64_t scratch_cap,
                                      rans_stream_t stream) {
    if (n_alpha < 2 || n_alpha > RANS_ADAPTIVE_N_MAX) return RANS_ERR_INVALID_ARG;
    const uint16_t any_model[2] = {RANS_M / 2, RANS_M / 2};  // the models need no table
    return encode_message(d_symbols, nullptr, n_symbols, any_model, nullptr, 2, params, d_out,
                          out_cap, d_out_size, d_status, d_scratch, scratch_cap, stream, false,
                          false, n_alpha);
}

extern "C" int rans_encode_bytes(const uint8_t *d_symbols, uint64_t n_symbols,
                                 const uint16_t *h_freq, uint32_t n_alpha,
                                 const rans_params *params, uint8_t *d_out, uint64_t out_cap,
                                 uint64_t *d_out_size, uint32_t *d_status, void *d_scratch,
                                 uint64_t scratch_cap, rans_stream_t stream) {
    return encode_message(d_symbols, nullptr, n_symbols, h_freq, nullptr, n_alpha, params, d_out,
                          out_cap, d_out_size, d_status, d_scratch, scratch_cap, stream, true);
}

extern "C" int rans_encode(const uint8_t *d_symbols, uint64_t n_symbols, const uint16_t *h_freq,
                           uint32_t n_alpha, const rans_params *params, uint8_t *d_out,
                           uint64_t out_cap, uint64_t *d_out_size, uint32_t *d_status,
                           void *d_scratch, uint64_t scratch_cap, rans_stream_t stream) {
    return encode_message(d_symbols, nullptr, n_symbols, h_freq, nullptr, n_alpha, params, d_out,
                          out_cap, d_out_size, d_status, d_scratch, scratch_cap, stream);
}

extern "C" int rans_encode_bypass(const uint8_t *d_symbols, const uint16_t *d_raw,
                                  uint64_t n_symbols, const uint16_t *h_freq,
                                  const uint8_t *h_raw_words, uint32_t n_alpha,
                                  const rans_params *params, uint8_t *d_out, uint64_t out_cap,
                                  uint64_t *d_out_size, uint32_t *d_status, void *d_scratch,
                                  uint64_t scratch_cap, rans_stream_t stream) {
    if (!h_raw_words) return RANS_ERR_INVALID_ARG;
    return encode_message(d_symbols, d_raw, n_symbols, h_freq, h_raw_words, n_alpha, params,
                          d_out, out_cap, d_out_size, d_status, d_scratch, scratch_cap, stream);
}

// ---------------------------------------------------------------------------
// rans_encode_static_scratch: the same encoder with its scratch in a
// file-scope device array, for callers that must not allocate device memory.
// ---------------------------------------------------------------------------
namespace rans {
namespace {

// Held by every GPU that loads this library, for the life of the process.
static __device__ __align__(256) uint8_t g_static_scratch[RANS_STATIC_SCRATCH_BYTES];

// Device address of g_static_scratch per device, looked up on the first call
// made with that device current.  The host-side name of the array is only a
// stand-in for the symbol, never a device address, so it is never passed to a
// kernel.  The address is kept for the life of the process: a reset of the
// device's context (cudaDeviceReset) would leave it stale, which rans.h
// states as a limit of this entry point.
std::mutex g_static_mu;
uint8_t *g_static_ptr[64] = {nullptr};

int static_scratch_address(uint8_t **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return RANS_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (g_static_ptr[dev] == nullptr) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || p == nullptr)
            return RANS_ERR_CUDA;
        g_static_ptr[dev] = static_cast<uint8_t *>(p);
    }
    *out = g_static_ptr[dev];
    return RANS_OK;
}

}  // namespace
}  // namespace rans

extern "C" int rans_encode_static_scratch(const uint8_t *d_symbols, uint64_t n_symbols,
                                          const uint16_t *h_freq, uint32_t n_alpha,
                                          const rans_params *params, uint8_t *d_out,
                                          uint64_t out_cap, uint64_t *d_out_size,
                                          uint32_t *d_status, rans_stream_t stream) {
    // The model may sum to 2^12, 2^13 or 2^14, as for rans_encode.
    uint32_t lm = RANS_LOG2_M;
    if (!params_ok(params) || !table_log2m(h_freq, n_alpha, &lm) || !d_out || !d_out_size ||
        !d_status || !aligned16(d_out))
        return RANS_ERR_INVALID_ARG;
    if (n_symbols && !d_symbols) return RANS_ERR_INVALID_ARG;
    const MessageGeometry g = geometry(n_symbols, params);
    if (g.n_chunks > 0xFFFFFFFEull ||
        4ull * params->n_lanes * g.n_chunks + 2ull * n_symbols > 0xFFFFFFF0ull)
        return RANS_ERR_INVALID_ARG;
    const ScratchLayout sl = scratch_layout(g.n_chunks, params->n_lanes, params->chunk_symbols);
    if (sl.total > RANS_STATIC_SCRATCH_BYTES) return RANS_ERR_BUFFER_TOO_SMALL;
    if (out_cap < rans_max_encoded_size(n_symbols, params)) return RANS_ERR_BUFFER_TOO_SMALL;
    uint8_t *scr = nullptr;
    if (static_scratch_address(&scr) != RANS_OK) return RANS_ERR_CUDA;

    // Only the look-back words and the ticket start at zero (encode_placed
    // clears them): the coder writes every word, state, size and offset
    // before they are read.
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(d_status, 0, sizeof(uint32_t), st) != cudaSuccess) return RANS_ERR_CUDA;

    EncodeParams ep{};
    ep.sym = d_symbols;
    ep.words = scr + sl.words;
    ep.states = reinterpret_cast<uint32_t *>(scr + sl.states);
    ep.wstart = reinterpret_cast<uint32_t *>(scr + sl.wstart);
    ep.sizes = reinterpret_cast<uint32_t *>(scr + sl.sizes);
    ep.status = d_status;
    ep.n_sym = n_symbols;
    ep.N = params->n_lanes;
    ep.CS = params->chunk_symbols;
    ep.n_chunks = uint32_t(g.n_chunks);
    ep.slot_bytes = sl.slot_bytes;
    ep.c_begin = 0;
    ep.c_end = ep.n_chunks;
    ep.log2m = lm;
    for (uint32_t s = 0; s < n_alpha; ++s) ep.freq[s] = h_freq[s];
    if (g.n_chunks == 0)
        return encode_empty(d_out, d_out_size, d_status, n_symbols, params, uint32_t(g.data0),
                            RANS_VERSION, lm, st);
    return encode_placed(ep, sl, scr, d_out, d_out_size, uint32_t(g.data0), RANS_VERSION,
                         lm != RANS_LOG2_M ? kWide : kPlain, st);
}

// ---------------------------------------------------------------------------
// rans_encode_host: encoding from and to host memory, copies overlapped with
// coding.
// ---------------------------------------------------------------------------
namespace rans {
namespace {

constexpr uint64_t kHostPieceSymbols = 32ull << 20;  // about this many symbols per piece
constexpr uint32_t kHostMaxPieces = 256;

struct RangeOffsetsParams {
    const uint32_t *sizes;
    uint32_t *d_offs;      // device copy of the offset table
    uint32_t *msg_offs;    // the message's offset table (device or page-locked host memory)
    uint64_t *running;     // data bytes of the chunks before c_begin; advanced past c_end
    uint32_t c_begin, c_end;
};

// One CTA: the offsets of chunks [c_begin, c_end), after those before them.
__global__ void __launch_bounds__(kScanThreads)
    range_offsets_kernel(const __grid_constant__ RangeOffsetsParams p) {
    __shared__ uint32_t warp_sums[32];
    __shared__ uint64_t carry_s;
    const uint64_t total = enc::scan_sizes(p.sizes, p.c_begin, p.c_end, *p.running, p.d_offs,
                                           p.msg_offs, warp_sums, &carry_s);
    if (threadIdx.x == 0) *p.running = total;
}

struct HeaderParams {
    uint8_t *out;
    uint64_t *d_size;
    const uint64_t *running;
    const uint32_t *status;
    uint64_t n_sym;
    uint32_t N, CS, n_chunks, data0, log2m;
};

__global__ void host_header_kernel(const __grid_constant__ HeaderParams p) {
    if (*p.status != RANS_OK) {
        *p.d_size = 0;
        return;
    }
    enc::write_header(p.out, p.d_size, p.n_sym, p.N, p.CS, p.n_chunks, p.data0,
                      uint32_t(*p.running), RANS_VERSION, p.log2m);
}

// Work space: [symbols][encode scratch][device offsets][running, status,
// size][message, for a pageable output buffer].
struct HostWork {
    uint64_t sym, scratch, offs, misc, msg, total;
};

HostWork host_work(uint64_t n_symbols, const rans_params *params) {
    const MessageGeometry g = geometry(n_symbols, params);
    HostWork w;
    w.sym = 0;
    w.scratch = round16(n_symbols);
    w.offs = w.scratch + scratch_layout(g.n_chunks, params->n_lanes, params->chunk_symbols).total;
    w.misc = w.offs + round16(4 * (g.n_chunks + 1));
    w.msg = w.misc + 64;
    w.total = w.msg + round16(rans_max_encoded_size(n_symbols, params));
    return w;
}

}  // namespace
}  // namespace rans

extern "C" uint64_t rans_encode_host_work_size(uint64_t n_symbols, const rans_params *params) {
    if (!params_ok(params)) return 0;
    return host_work(n_symbols, params).total;
}

extern "C" int rans_encode_host(const uint8_t *h_symbols, uint64_t n_symbols,
                                const uint16_t *h_freq, uint32_t n_alpha,
                                const rans_params *params, uint8_t *h_out, uint64_t out_cap,
                                uint64_t *h_out_size, uint32_t *h_status, void *d_work,
                                uint64_t work_cap, rans_stream_t stream) {
    uint32_t lm = RANS_LOG2_M;
    if (!params_ok(params) || !table_log2m(h_freq, n_alpha, &lm) || !h_out || !h_out_size ||
        !h_status || !d_work || !aligned16(d_work) || (n_symbols && !h_symbols))
        return RANS_ERR_INVALID_ARG;
    const MessageGeometry g = geometry(n_symbols, params);
    if (g.n_chunks > 0xFFFFFFFEull ||
        4ull * params->n_lanes * g.n_chunks + 2ull * n_symbols > 0xFFFFFFF0ull)
        return RANS_ERR_INVALID_ARG;
    const uint64_t max_out = rans_max_encoded_size(n_symbols, params);
    const HostWork hw = host_work(n_symbols, params);
    if (out_cap < max_out || work_cap < hw.total) return RANS_ERR_BUFFER_TOO_SMALL;

    // A page-locked, 16-byte aligned output buffer is written by the kernels
    // through its device address, piece by piece (the pack writes 16-byte
    // blocks); any other gets the message from device memory once the coding
    // is done.
    uint8_t *out_dev = nullptr;
    cudaPointerAttributes attr{};
    if (cudaPointerGetAttributes(&attr, h_out) == cudaSuccess && attr.type == cudaMemoryTypeHost &&
        attr.devicePointer != nullptr && aligned16(attr.devicePointer))
        out_dev = static_cast<uint8_t *>(attr.devicePointer);
    else
        cudaGetLastError();  // a pageable pointer may leave an error behind
    uint8_t *w = static_cast<uint8_t *>(d_work);
    const bool staged = out_dev == nullptr;
    if (staged) out_dev = w + hw.msg;

    const ScratchLayout sl = scratch_layout(g.n_chunks, params->n_lanes, params->chunk_symbols);
    uint8_t *scr = w + hw.scratch;
    uint64_t *running = reinterpret_cast<uint64_t *>(w + hw.misc);
    uint32_t *d_status = reinterpret_cast<uint32_t *>(w + hw.misc + 8);
    uint64_t *d_size = reinterpret_cast<uint64_t *>(w + hw.misc + 16);
    uint32_t *d_offs = reinterpret_cast<uint32_t *>(w + hw.offs);

    EncodeParams ep{};
    ep.sym = w + hw.sym;
    ep.words = scr + sl.words;
    ep.states = reinterpret_cast<uint32_t *>(scr + sl.states);
    ep.wstart = reinterpret_cast<uint32_t *>(scr + sl.wstart);
    ep.sizes = reinterpret_cast<uint32_t *>(scr + sl.sizes);
    ep.status = d_status;
    ep.n_sym = n_symbols;
    ep.N = params->n_lanes;
    ep.CS = params->chunk_symbols;
    ep.n_chunks = uint32_t(g.n_chunks);
    ep.slot_bytes = sl.slot_bytes;
    ep.log2m = lm;
    for (uint32_t s = 0; s < n_alpha; ++s) ep.freq[s] = h_freq[s];

    CopyStreams cs;
    int rc = copy_streams(&cs);
    if (rc != RANS_OK) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(w + hw.misc, 0, 64, st) != cudaSuccess || !join(cs.in, st) ||
        !join(cs.out, st))
        return RANS_ERR_CUDA;

    // Pieces of whole chunks: the symbols of piece k are copied in on one
    // stream, coded and given their offsets on the caller's stream, and
    // packed into the output on a third, so the copy-in of piece k+1 and the
    // output of piece k-1 overlap the coding of piece k.
    const uint32_t nc = ep.n_chunks;
    const uint32_t per_piece = uint32_t(std::max<uint64_t>(
        std::max<uint64_t>(1, ceil_div(kHostPieceSymbols, ep.CS)), ceil_div(nc, kHostMaxPieces)));
    for (uint64_t c0 = 0; c0 < nc; c0 += per_piece) {
        const uint64_t c1 = std::min<uint64_t>(nc, c0 + per_piece);
        const uint64_t s0 = c0 * ep.CS, s1 = std::min<uint64_t>(n_symbols, c1 * ep.CS);
        if (cudaMemcpyAsync(w + hw.sym + s0, h_symbols + s0, s1 - s0, cudaMemcpyHostToDevice,
                            cs.in) != cudaSuccess ||
            !join(st, cs.in))
            return RANS_ERR_CUDA;
        ep.c_begin = uint32_t(c0);
        ep.c_end = uint32_t(c1);
        if (lm != RANS_LOG2_M)
            rc = ep.N == 32 ? launch_encode<32, kWide>(ep, st) : launch_encode<0, kWide>(ep, st);
        else
            rc = ep.N == 32 ? launch_encode<32, kPlain>(ep, st) : launch_encode<0, kPlain>(ep, st);
        if (rc != RANS_OK) return rc;
        RangeOffsetsParams rp{};
        rp.sizes = ep.sizes;
        rp.d_offs = d_offs;
        rp.msg_offs = reinterpret_cast<uint32_t *>(out_dev + 32);
        rp.running = running;
        rp.c_begin = uint32_t(c0);
        rp.c_end = uint32_t(c1);
        range_offsets_kernel<<<1, kScanThreads, 0, st>>>(rp);
        if (check_launch() != RANS_OK || !join(cs.out, st)) return RANS_ERR_CUDA;
        PackParams pp{};
        pp.out = out_dev;
        pp.words = ep.words;
        pp.states = ep.states;
        pp.wstart = ep.wstart;
        pp.status = d_status;
        pp.offs = d_offs;
        pp.N = ep.N;
        pp.n_chunks = nc;
        pp.data0 = uint32_t(g.data0);
        pp.slot_bytes = ep.slot_bytes;
        pp.c_begin = uint32_t(c0);
        pp.c_end = uint32_t(c1);
        const unsigned grid = unsigned(std::min<uint64_t>(c1 - c0, 65535ull * 8));
        pack_kernel<false><<<grid, kPackThreads, 0, cs.out>>>(pp);
        if (check_launch() != RANS_OK) return RANS_ERR_CUDA;
    }
    if (!join(cs.out, st)) return RANS_ERR_CUDA;
    HeaderParams hp{};
    hp.out = out_dev;
    hp.d_size = d_size;
    hp.running = running;
    hp.status = d_status;
    hp.n_sym = n_symbols;
    hp.N = ep.N;
    hp.CS = ep.CS;
    hp.n_chunks = nc;
    hp.data0 = uint32_t(g.data0);
    hp.log2m = lm;
    host_header_kernel<<<1, 1, 0, cs.out>>>(hp);
    if (check_launch() != RANS_OK ||
        cudaMemcpyAsync(h_status, d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, cs.out) !=
            cudaSuccess ||
        cudaMemcpyAsync(h_out_size, d_size, sizeof(uint64_t), cudaMemcpyDeviceToHost, cs.out) !=
            cudaSuccess ||
        !join(st, cs.out))
        return RANS_ERR_CUDA;
    if (staged) {
        // Pageable output: the size is known once the work is done.
        if (cudaStreamSynchronize(st) != cudaSuccess) return RANS_ERR_CUDA;
        if (*h_out_size &&
            cudaMemcpy(h_out, out_dev, *h_out_size, cudaMemcpyDeviceToHost) != cudaSuccess)
            return RANS_ERR_CUDA;
    }
    return RANS_OK;
}

#ifdef RANS_CHECKED
// Checked builds: failed invariants of this file's kernels since the last call.
uint64_t rans_check_failures_encode() { return rans::take_check_failures(); }
#endif
