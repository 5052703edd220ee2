// rans_decode.cu -- single-message GPU decoder: one warp per chunk, the
// chunk's N interleaved coders on the warp's lanes (decode_core.cuh), one
// slot table per CTA built from the message's model, in CTAs of 8 or 12
// warps (chosen per launch from the kind and the chunk count).
#include <algorithm>
#include <atomic>
#include <mutex>

#include <cuda_runtime.h>

#include "decode_core.cuh"
#include "host_util.h"

namespace rans {
namespace {


struct DecodeParams {
    const uint8_t *msg;
    uint8_t *out;
    uint32_t *status;
    uint64_t msg_size;
    uint64_t n_sym;
    uint32_t N;
    uint32_t CS;
    uint32_t n_chunks;
    uint32_t data0;
    uint32_t c_begin;   // chunks [c_begin, c_end) are decoded by this launch
    uint32_t c_end;
    uint32_t kind;      // kPlain, kBypass (raw words after their symbols) or kBytes
    uint32_t warp_major;  // 1: chunks dealt warp-major across the grid (set by the launcher)
    uint16_t *raw_out;  // bypass messages: raw word (or 0) per symbol
    uint16_t freq[RANS_MAX_ALPHABET];
    uint8_t raw_words[RANS_MAX_ALPHABET];  // bypass: raw words symbol s carries (0 or 1)
    uint32_t log2m;                        // plain messages: log2 M (12, 13 or 14)
    uint32_t n_alpha;                      // adaptive-n messages: the alphabet size n
    uint8_t plen[RANS_MAX_ALPHABET];       // prefix messages: code lengths (0: no code)
    uint16_t pcode[RANS_MAX_ALPHABET];     // prefix messages: canonical codes
};

// Message kinds: plain (version 1), bypass (version 2: raw words after their
// symbols), byte-wise (version 3: b = 2^8, digits breadth-first per step) and
// adaptive (version 4: binary symbols, one adaptive context per coder) and
// prefix (version 5: canonical prefix codes in their decoder's read order).
constexpr int kPlain = dec::kKindPlain, kBypass = dec::kKindRaw, kBytes = dec::kKindBytes,
              kAdaptive = dec::kKindAdaptive, kPrefix = dec::kKindPrefix,
              kWide13 = dec::kKindWide13, kWide14 = dec::kKindWide14,
              kBinary = dec::kKindBinary, kAdaptN4 = dec::kKindAdaptN4,
              kAdaptN8 = dec::kKindAdaptN8, kAdaptN16 = dec::kKindAdaptN16,
              kPlainEarly = dec::kKindPlainEarly, kPlainSpec = dec::kKindPlainSpec,
              kBytesLat = dec::kKindBytesLat;

// Dynamic shared memory of the W-warp kernel for KIND: the shape's layout,
// and for the entry-ahead step one entry ring per warp after it (aligned to
// its size, with that much slack).
template <int KIND, int W>
constexpr uint32_t smem_bytes() {
    return dec::Shape<W>::kSmemBytes + (KIND == kPlainSpec ? (W + 1) * dec::kERing : 0u);
}

// NT = 32: every chunk uses all 32 lanes; NT = 0: runtime N.  W: warps per
// CTA (dec::Shape).  A warp decodes one chunk at a time.
template <int NT, int KIND, int W>
__device__ __forceinline__ void decode_body(const DecodeParams &p) {
    constexpr bool RAW = KIND == kBypass;
    constexpr bool BYTES = KIND == kBytes || KIND == kBytesLat;
    constexpr bool ADAPTIVE = KIND == kAdaptive;
    constexpr bool PREFIX = KIND == kPrefix;
    constexpr bool WIDE = KIND == kWide13 || KIND == kWide14;
    constexpr bool BINARY = KIND == kBinary;  // a plain message with a binary model
    constexpr bool ADAPTN = dec::AdaptN<KIND>::kOn;
    extern __shared__ __align__(128) uint8_t smem[];
    const dec::Smem sm = dec::smem_layout<W>(smem);
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    uint32_t &hdr_ok = sm.misc[0];
    uint32_t &const_sym = sm.misc[1];

    if (threadIdx.x == 0) {
        hdr_ok = dec::header_ok(p.msg, p.msg_size, p.data0, p.n_sym, p.N, p.CS, p.n_chunks,
                                RAW ? RANS_VERSION_BYPASS : BYTES ? RANS_VERSION_BYTES
                                : ADAPTIVE                        ? RANS_VERSION_ADAPTIVE
                                : PREFIX                          ? RANS_VERSION_PREFIX
                                : ADAPTN                          ? RANS_VERSION_ADAPTIVE_N
                                                                  : RANS_VERSION,
                                WIDE     ? dec::WideBits<KIND>::kLog2
                                : ADAPTN ? uint32_t(kLog2M) | (p.n_alpha << 16)
                                         : uint32_t(kLog2M));
        const_sym = dec::kNoConst;
    }
    if (RAW && threadIdx.x < RANS_MAX_ALPHABET) sm.flags[threadIdx.x] = p.raw_words[threadIdx.x];
    if (ADAPTIVE || BINARY || ADAPTN) __syncthreads();  // no table: contexts, or f_0 and f_1
    else if (PREFIX) dec::build_prefix_table<W>(p.plen, p.pcode, sm.tab);
    else if (WIDE)
        dec::build_wide_table<W>(p.freq, dec::WideBits<KIND>::kLog2, reinterpret_cast<uint8_t *>(sm.tab),
                              sm.fb, sm.rings, &const_sym);  // rings unused yet
    else dec::build_slot_table<W>(p.freq, sm.tab, sm.rings, &const_sym);  // rings unused yet
    if (!hdr_ok) {
        if (threadIdx.x == 0) report(p.status, RANS_ERR_CORRUPT);
        return;
    }
    dec::WarpRings wr = dec::rings_init(sm, warp, lane);
    const uint32_t cs = const_sym;
    const uint32_t *offs = reinterpret_cast<const uint32_t *>(p.msg + 32);
    const uint32_t data_end = offs[p.n_chunks];
    const uint32_t lt = lanemask_lt();
    const uint32_t n_units = p.c_end - p.c_begin;
    // The entry-ahead step: each warp's entry ring after the shape's layout.
    // It and the byte-wise latency form deal chunks warp-major, so that a
    // message of few chunks spreads over the SMs one warp each rather than
    // filling a few CTAs.
    constexpr bool SPEC = KIND == kPlainSpec;
    constexpr bool WARP_MAJOR = SPEC || KIND == kBytesLat;
    const uint32_t ering_s =
        SPEC ? ((smem_addr(smem + dec::Shape<W>::kSmemBytes) + dec::kERing - 1) &
                ~(dec::kERing - 1)) + warp * dec::kERing
             : 0u;
    const uint32_t q0 = (WARP_MAJOR || p.warp_major) ? warp * gridDim.x + blockIdx.x
                                                     : blockIdx.x * W + warp;

    // 32-step groups for plain chunks in the 12-warp shape, the early-word
    // step and 13/14-bit chunks (measured on B300: early-word 297 chunks 166.0
    // -> 161.3 us, 2368 chunks 191.7 -> 187.1 us; 14-bit model 1 GiB 1104 ->
    // 1084 us, 4000 chunks 295 -> 288 us; slower with them: adaptive models
    // over 16 symbols 1991 -> 2322 us, binary contexts 295 -> 309 us, the
    // byte-wise latency form 193 -> 195 us at 296 chunks, binary models in
    // 8-warp CTAs 232 -> 240 us at 4000 chunks)
    constexpr bool LONG =
        (W == dec::kWarpsOne && KIND == kPlain) || KIND == kPlainEarly || WIDE;
    for (uint32_t q = q0; q < n_units; q += gridDim.x * W) {
        const uint32_t c = p.c_begin + q;
        uint32_t st;
        if (RAW)
            st = dec::decode_chunks<NT, false, kBypass>(wr, sm.tab_s, p.msg, p.data0, offs,
                                                        data_end, c, 1, p.n_sym, p.CS, p.N, p.out,
                                                        cs, lane, lt, p.raw_out, sm.flags_s,
                                                        cs != dec::kNoConst &&
                                                            sm.flags[cs & 0xFFu]);
        else if (BYTES || ADAPTIVE || PREFIX)
            st = dec::decode_chunks<NT, false, KIND>(wr, sm.tab_s, p.msg, p.data0, offs, data_end,
                                                     c, 1, p.n_sym, p.CS, p.N, p.out, cs, lane,
                                                     lt);
        else if (WIDE)  // the f/B table goes where bypass messages keep their flags
            st = dec::decode_chunks<NT, false, KIND, false, LONG>(
                wr, sm.tab_s, p.msg, p.data0, offs, data_end, c, 1, p.n_sym, p.CS, p.N, p.out, cs,
                lane, lt, nullptr, sm.fb_s);
        else if (ADAPTN)  // n rides in the flag argument
            st = dec::decode_chunks<NT, false, KIND>(wr, 0, p.msg, p.data0, offs, data_end, c, 1,
                                                     p.n_sym, p.CS, p.N, p.out, cs, lane, lt,
                                                     nullptr, p.n_alpha);
        else if (BINARY)  // f_0 and f_1 ride in the table and flag arguments
            st = dec::decode_chunks<NT, false, KIND, false, LONG>(
                wr, p.freq[0], p.msg, p.data0, offs, data_end, c, 1, p.n_sym, p.CS, p.N, p.out,
                cs, lane, lt, nullptr, p.freq[1]);
        else  // plain (KIND kPlain, kPlainEarly or kPlainSpec; the entry ring rides in flags_s)
            st = dec::decode_chunks<NT, false, KIND, false, LONG>(
                wr, sm.tab_s, p.msg, p.data0, offs, data_end, c, 1, p.n_sym, p.CS, p.N, p.out, cs,
                lane, lt, nullptr, ering_s);
        if (st != RANS_OK && lane == 0) report(p.status, st);
        if (wr.timeouts) break;
    }
}

// The two CTA shapes as kernels.  8 warps: bound by the CTA's threads alone,
// the form these kernels were measured fastest with (a bound of 4 CTAs per SM
// let bypass and 13/14-bit decoding take more registers, 5-10% slower).
// 12 warps: 3 CTAs per SM, which caps a thread at 56 registers.
template <int NT, int KIND>
__global__ void __launch_bounds__(dec::kThreads)
    decode_kernel(const __grid_constant__ DecodeParams p) {
    decode_body<NT, KIND, dec::kWarps>(p);
}
template <int NT, int KIND>
__global__ void __launch_bounds__(dec::Shape<dec::kWarpsOne>::kThreads,
                                  dec::Shape<dec::kWarpsOne>::kCtasPerSm)
    decode_kernel12(const __grid_constant__ DecodeParams p) {
    decode_body<NT, KIND, dec::kWarpsOne>(p);
}

template <int NT, int KIND, int W>
constexpr void (*kernel_for())(DecodeParams) {
    if constexpr (W == dec::kWarps) return decode_kernel<NT, KIND>;
    else return decode_kernel12<NT, KIND>;
}

// Resident CTAs of the W-warp kernel for <NT, KIND> on the whole GPU (0 on error);
// sets its shared-memory limit once per device.
template <int NT, int KIND, int W>
uint64_t resident_ctas() {
    using S = dec::Shape<W>;
    // Set once per device; concurrent first calls may both set it (harmless).
    static std::atomic<bool> configured[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !configured[dev].load()) {
        if (cudaFuncSetAttribute(kernel_for<NT, KIND, W>(),
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(smem_bytes<KIND, W>())) != cudaSuccess)
            return 0;
        configured[dev].store(true);
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel_for<NT, KIND, W>(),
                                                      S::kThreads, smem_bytes<KIND, W>()) !=
            cudaSuccess ||
        per_sm <= 0)
        return 0;
    return uint64_t(per_sm) * sm_count();
}

template <int NT, int KIND, int W>
int launch_shape(DecodeParams &p, uint64_t cap, cudaStream_t stream) {
    using S = dec::Shape<W>;
    // The entry-ahead step and the byte-wise latency form deal chunks
    // warp-major: a CTA per chunk up to the resident limit.  So does every
    // launch of at most one wave of chunks: all its CTAs are resident at once,
    // so each SM gets its share of chunks to within one per CTA, where whole
    // CTAs of W chunks left some SMs a CTA more than others.  Measured on
    // B300 (chunks of 64 Ki symbols, block-major against warp-major): plain
    // 2400 chunks 219.6 -> 205.4 us, 4000 chunks 266.7 -> 244.2 us; byte-wise
    // 4000 chunks 422.0 -> 391.0 us; adaptive-n over 8 symbols, 4096 chunks,
    // 910 -> 822 us.  Launches of more than a wave stay block-major (1 GiB:
    // 839 -> 978 us warp-major).
    const uint64_t n_range = p.c_end - p.c_begin;
    p.warp_major = n_range <= cap * W ? 1u : 0u;
    const uint64_t want = (KIND == kPlainSpec || KIND == kBytesLat || p.warp_major)
                              ? n_range
                              : ceil_div(n_range, uint64_t(W));
    const unsigned grid = unsigned(std::max<uint64_t>(1, std::min(want, cap)));
    kernel_for<NT, KIND, W>()<<<grid, S::kThreads, smem_bytes<KIND, W>(), stream>>>(p);
    return check_launch();
}

// A warp decodes one chunk.  Plain messages under one wave of chunks: 8-warp
// CTAs, where more resident warps gain nothing and the 64-register form has
// the shorter step (one 1 MiB chunk: 2.41 against 2.44 ms); up to two chunks
// per SM with the entry-ahead step (kSpecMaxChunks), up to half a
// wave with the early-word step (dec::kKindPlainEarly), whose step is
// shorter on an SM with few warps and costs a data-pipe wavefront on a full
// one (measured, µs, committed step against it: 1 chunk 164.7 / 158.8, 1184
// chunks 171.6 / 167.6, 2368 chunks 192.5 / 189.1, 3552 chunks 220.4 /
// 221.4, 4700 chunks 267.4 / 270.1; one 1 MiB chunk 73.2 / 70.5 ns a
// step).  Plain messages
// of a wave or more, and byte-wise messages: 12-warp CTAs.  The other kinds:
// 8-warp CTAs (dec::Shape).  Two chunks side by side in a warp of an 8-warp
// CTA were faster than one per warp in 8-warp CTAs from five waves up; one
// per warp in 12-warp CTAs beats both (32256 chunks of 64 Ki symbols, 6.8
// waves: 1636 against 1814 us), so single messages no longer pair chunks.
// Plain messages of up to this many chunks, two per SM, take the entry-ahead
// step (dec::kKindPlainSpec), one chunk per CTA.  Measured on B300 (chunks of
// 64 Ki symbols, against the early-word step): 1 chunk of 1 MiB 2312 -> 2149
// us, 148 chunks 166.8 -> 150.7 us, 296 chunks 166.3 -> 152.4 us; at 444 to
// 1184 chunks the two are within 1 %.
constexpr uint64_t kSpecMaxChunks = 296;
// Byte-wise messages of up to this many chunks (24 per SM) take the latency
// form (dec::kKindBytesLat), chunks dealt warp-major.  Measured on B300
// (chunks of 64 Ki symbols, against the block-major two-pass form): 888
// chunks 276 -> 207 us, 1776 chunks 277 -> 225 us, 2369 chunks 327 -> 285
// us, 3552 chunks 327 -> 323 us, 4736 chunks 424 -> 453 us.
constexpr uint64_t kBytesLatMaxChunks = 3552;

template <int NT, int KIND>
int launch_decode(DecodeParams &p, cudaStream_t stream) {
    const uint64_t n_range = p.c_end - p.c_begin;
    if constexpr (KIND == kPlain || KIND == kBinary) {
        const uint64_t cap8 = resident_ctas<NT, KIND, dec::kWarps>();
        if (!cap8) return RANS_ERR_CUDA;
        if constexpr (KIND == kPlain) {
            if (n_range <= kSpecMaxChunks) {
                const uint64_t cap_s = resident_ctas<NT, kPlainSpec, dec::kWarps>();
                if (!cap_s) return RANS_ERR_CUDA;
                return launch_shape<NT, kPlainSpec, dec::kWarps>(p, cap_s, stream);
            }
            if (2 * n_range <= cap8 * dec::kWarps) {
                const uint64_t cap_e = resident_ctas<NT, kPlainEarly, dec::kWarps>();
                if (!cap_e) return RANS_ERR_CUDA;
                return launch_shape<NT, kPlainEarly, dec::kWarps>(p, cap_e, stream);
            }
        }
        if (n_range < cap8 * dec::kWarps)
            return launch_shape<NT, KIND, dec::kWarps>(p, cap8, stream);
    }
    if constexpr (KIND == kBytes) {
        if (n_range <= kBytesLatMaxChunks) {
            const uint64_t cap_l = resident_ctas<NT, kBytesLat, dec::kWarpsOne>();
            if (!cap_l) return RANS_ERR_CUDA;
            return launch_shape<NT, kBytesLat, dec::kWarpsOne>(p, cap_l, stream);
        }
    }
    if constexpr (KIND == kPlain || KIND == kBytes || KIND == kBinary) {
        const uint64_t cap = resident_ctas<NT, KIND, dec::kWarpsOne>();
        if (!cap) return RANS_ERR_CUDA;
        return launch_shape<NT, KIND, dec::kWarpsOne>(p, cap, stream);
    } else {
        const uint64_t cap = resident_ctas<NT, KIND, dec::kWarps>();
        if (!cap) return RANS_ERR_CUDA;
        return launch_shape<NT, KIND, dec::kWarps>(p, cap, stream);
    }
}

}  // namespace
}  // namespace rans

using namespace rans;

// Checks the arguments shared by the decode entry points and fills p (all
// chunks); msg may be a host or a device address.
// wide_ok: a plain message, whose model may also sum to 2^13 or 2^14 (the
// kind is then kWide13 or kWide14).
static int prepare_decode(const uint8_t *msg, uint64_t msg_size, const uint16_t *h_freq,
                          uint32_t n_alpha, const rans_params *params, uint64_t n_symbols,
                          DecodeParams &p, bool wide_ok = false) {
    uint32_t lm = RANS_LOG2_M;
    if (!msg || !params_ok(params) ||
        !(wide_ok ? table_log2m(h_freq, n_alpha, &lm) : table_ok(h_freq, n_alpha, nullptr)))
        return RANS_ERR_INVALID_ARG;
    const MessageGeometry g = geometry(n_symbols, params);
    if (g.n_chunks > 0xFFFFFFFEull) return RANS_ERR_INVALID_ARG;
    if (msg_size < g.data0 || (msg_size & 15u) || msg_size < 48 ||
        msg_size - g.data0 > 0xFFFFFFFFull + 15)
        return RANS_ERR_INVALID_ARG;
    p = DecodeParams{};
    p.msg_size = msg_size;
    p.n_sym = n_symbols;
    p.N = params->n_lanes;
    p.CS = params->chunk_symbols;
    p.n_chunks = uint32_t(g.n_chunks);
    p.data0 = uint32_t(g.data0);
    p.c_begin = 0;
    p.c_end = p.n_chunks;
    p.log2m = lm;
    p.kind = lm == 13 ? kWide13 : lm == 14 ? kWide14 : kPlain;
    for (uint32_t s = 0; s < n_alpha; ++s) p.freq[s] = h_freq[s];
    // symbols 0 and 1 only, both possible: the table-free binary decoder
    bool binary = lm == RANS_LOG2_M && n_alpha >= 2 && p.freq[0] > 0 && p.freq[1] > 0 &&
                  p.freq[0] + p.freq[1] == RANS_M;
    for (uint32_t s = 2; binary && s < n_alpha; ++s) binary = p.freq[s] == 0;
    if (binary) p.kind = kBinary;
    return RANS_OK;
}

static int launch_range(DecodeParams p, uint32_t c_begin, uint32_t c_end, cudaStream_t st) {
    p.c_begin = c_begin;
    p.c_end = c_end;
    if (p.kind == kBypass)
        return p.N == 32 ? launch_decode<32, kBypass>(p, st) : launch_decode<0, kBypass>(p, st);
    if (p.kind == kBytes)
        return p.N == 32 ? launch_decode<32, kBytes>(p, st) : launch_decode<0, kBytes>(p, st);
    if (p.kind == kAdaptive)
        return p.N == 32 ? launch_decode<32, kAdaptive>(p, st) : launch_decode<0, kAdaptive>(p, st);
    if (p.kind == kPrefix)
        return p.N == 32 ? launch_decode<32, kPrefix>(p, st) : launch_decode<0, kPrefix>(p, st);
    if (p.kind == kWide13)
        return p.N == 32 ? launch_decode<32, kWide13>(p, st) : launch_decode<0, kWide13>(p, st);
    if (p.kind == kWide14)
        return p.N == 32 ? launch_decode<32, kWide14>(p, st) : launch_decode<0, kWide14>(p, st);
    if (p.kind == kBinary)
        return p.N == 32 ? launch_decode<32, kBinary>(p, st) : launch_decode<0, kBinary>(p, st);
    if (p.kind == kAdaptN4)
        return p.N == 32 ? launch_decode<32, kAdaptN4>(p, st) : launch_decode<0, kAdaptN4>(p, st);
    if (p.kind == kAdaptN8)
        return p.N == 32 ? launch_decode<32, kAdaptN8>(p, st) : launch_decode<0, kAdaptN8>(p, st);
    if (p.kind == kAdaptN16)
        return p.N == 32 ? launch_decode<32, kAdaptN16>(p, st) : launch_decode<0, kAdaptN16>(p, st);
    return p.N == 32 ? launch_decode<32, kPlain>(p, st) : launch_decode<0, kPlain>(p, st);
}

extern "C" int rans_decode(const uint8_t *d_msg, uint64_t msg_size, const uint16_t *h_freq,
                           uint32_t n_alpha, const rans_params *params, uint8_t *d_symbols,
                           uint64_t n_symbols, uint32_t *d_status, rans_stream_t stream) {
    DecodeParams p;
    const int rc = prepare_decode(d_msg, msg_size, h_freq, n_alpha, params, n_symbols, p, true);
    if (rc != RANS_OK) return rc;
    if (!d_status || !aligned16(d_msg) || (n_symbols && !d_symbols)) return RANS_ERR_INVALID_ARG;
    p.msg = d_msg;
    p.out = d_symbols;
    p.status = d_status;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(d_status, 0, sizeof(uint32_t), st) != cudaSuccess) return RANS_ERR_CUDA;
    return launch_range(p, 0, p.n_chunks, st);
}

extern "C" int rans_decode_bypass(const uint8_t *d_msg, uint64_t msg_size, const uint16_t *h_freq,
                                  const uint8_t *h_raw_words, uint32_t n_alpha,
                                  const rans_params *params, uint8_t *d_symbols, uint16_t *d_raw,
                                  uint64_t n_symbols, uint32_t *d_status, rans_stream_t stream) {
    DecodeParams p;
    const int rc = prepare_decode(d_msg, msg_size, h_freq, n_alpha, params, n_symbols, p);
    if (rc != RANS_OK) return rc;
    if (!d_status || !aligned16(d_msg) || !h_raw_words || (n_symbols && (!d_symbols || !d_raw)) ||
        (reinterpret_cast<uintptr_t>(d_raw) & 1u))
        return RANS_ERR_INVALID_ARG;
    for (uint32_t s = 0; s < n_alpha; ++s) {
        if (h_raw_words[s] > 1) return RANS_ERR_INVALID_ARG;
        p.raw_words[s] = h_raw_words[s];
    }
    p.msg = d_msg;
    p.out = d_symbols;
    p.raw_out = d_raw;
    p.kind = kBypass;
    p.status = d_status;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(d_status, 0, sizeof(uint32_t), st) != cudaSuccess) return RANS_ERR_CUDA;
    return launch_range(p, 0, p.n_chunks, st);
}

extern "C" int rans_decode_bytes(const uint8_t *d_msg, uint64_t msg_size, const uint16_t *h_freq,
                                 uint32_t n_alpha, const rans_params *params, uint8_t *d_symbols,
                                 uint64_t n_symbols, uint32_t *d_status, rans_stream_t stream) {
    DecodeParams p;
    const int rc = prepare_decode(d_msg, msg_size, h_freq, n_alpha, params, n_symbols, p);
    if (rc != RANS_OK) return rc;
    if (!d_status || !aligned16(d_msg) || (n_symbols && !d_symbols)) return RANS_ERR_INVALID_ARG;
    p.msg = d_msg;
    p.out = d_symbols;
    p.status = d_status;
    p.kind = kBytes;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(d_status, 0, sizeof(uint32_t), st) != cudaSuccess) return RANS_ERR_CUDA;
    return launch_range(p, 0, p.n_chunks, st);
}

extern "C" int rans_decode_adaptive(const uint8_t *d_msg, uint64_t msg_size,
                                    const rans_params *params, uint8_t *d_symbols,
                                    uint64_t n_symbols, uint32_t *d_status, rans_stream_t stream) {
    uint16_t any_model[2] = {RANS_M / 2, RANS_M / 2};  // the contexts need no table
    DecodeParams p;
    const int rc = prepare_decode(d_msg, msg_size, any_model, 2, params, n_symbols, p);
    if (rc != RANS_OK) return rc;
    if (!d_status || !aligned16(d_msg) || (n_symbols && !d_symbols)) return RANS_ERR_INVALID_ARG;
    p.msg = d_msg;
    p.out = d_symbols;
    p.status = d_status;
    p.kind = kAdaptive;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(d_status, 0, sizeof(uint32_t), st) != cudaSuccess) return RANS_ERR_CUDA;
    return launch_range(p, 0, p.n_chunks, st);
}

extern "C" int rans_decode_adaptive_n(const uint8_t *d_msg, uint64_t msg_size, uint32_t n_alpha,
                                      const rans_params *params, uint8_t *d_symbols,
                                      uint64_t n_symbols, uint32_t *d_status,
                                      rans_stream_t stream) {
    if (n_alpha < 2 || n_alpha > RANS_ADAPTIVE_N_MAX) return RANS_ERR_INVALID_ARG;
    uint16_t any_model[2] = {RANS_M / 2, RANS_M / 2};  // the models need no table
    DecodeParams p;
    const int rc = prepare_decode(d_msg, msg_size, any_model, 2, params, n_symbols, p);
    if (rc != RANS_OK) return rc;
    if (!d_status || !aligned16(d_msg) || (n_symbols && !d_symbols)) return RANS_ERR_INVALID_ARG;
    p.msg = d_msg;
    p.out = d_symbols;
    p.status = d_status;
    p.n_alpha = n_alpha;
    p.kind = n_alpha <= 4 ? kAdaptN4 : n_alpha <= 8 ? kAdaptN8 : kAdaptN16;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(d_status, 0, sizeof(uint32_t), st) != cudaSuccess) return RANS_ERR_CUDA;
    return launch_range(p, 0, p.n_chunks, st);
}

extern "C" int rans_decode_prefix(const uint8_t *d_msg, uint64_t msg_size, const uint8_t *h_lengths,
                                  uint32_t n_alpha, const rans_params *params, uint8_t *d_symbols,
                                  uint64_t n_symbols, uint32_t *d_status, rans_stream_t stream) {
    uint16_t any_model[2] = {RANS_M / 2, RANS_M / 2};  // the code table replaces the model
    uint16_t codes[RANS_MAX_ALPHABET];
    DecodeParams p;
    int rc = prepare_decode(d_msg, msg_size, any_model, 2, params, n_symbols, p);
    if (rc != RANS_OK) return rc;
    if (!d_status || !aligned16(d_msg) || (n_symbols && !d_symbols)) return RANS_ERR_INVALID_ARG;
    if ((rc = rans_prefix_codes(h_lengths, n_alpha, codes)) != RANS_OK) return rc;
    for (uint32_t s = 0; s < n_alpha; ++s) {
        p.plen[s] = h_lengths[s];
        p.pcode[s] = codes[s];
    }
    p.msg = d_msg;
    p.out = d_symbols;
    p.status = d_status;
    p.kind = kPrefix;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(d_status, 0, sizeof(uint32_t), st) != cudaSuccess) return RANS_ERR_CUDA;
    return launch_range(p, 0, p.n_chunks, st);
}

// ---------------------------------------------------------------------------
// Decoding from and to host memory, copies overlapped with decoding.
// ---------------------------------------------------------------------------

namespace {

constexpr uint64_t kPieceSymbols = 32ull << 20;  // about this many symbols per piece
constexpr uint32_t kMaxPieces = 256;

}  // namespace

extern "C" uint64_t rans_decode_host_work_size(uint64_t msg_size, uint64_t n_symbols) {
    return round16(msg_size) + round16(n_symbols) + 16;
}

extern "C" int rans_decode_host(const uint8_t *h_msg, uint64_t msg_size, const uint16_t *h_freq,
                                uint32_t n_alpha, const rans_params *params, uint8_t *h_symbols,
                                uint64_t n_symbols, uint32_t *h_status, void *d_work,
                                uint64_t work_cap, rans_stream_t stream) {
    DecodeParams p;
    int rc = prepare_decode(h_msg, msg_size, h_freq, n_alpha, params, n_symbols, p, true);
    if (rc != RANS_OK) return rc;
    if (!h_status || !d_work || !aligned16(d_work) || (n_symbols && !h_symbols))
        return RANS_ERR_INVALID_ARG;
    if (work_cap < rans_decode_host_work_size(msg_size, n_symbols)) return RANS_ERR_BUFFER_TOO_SMALL;
    uint8_t *d_msg = static_cast<uint8_t *>(d_work);
    uint8_t *d_out = d_msg + round16(msg_size);
    uint32_t *d_status = reinterpret_cast<uint32_t *>(d_out + round16(n_symbols));
    p.msg = d_msg;
    p.out = d_out;
    p.status = d_status;

    // Pieces of whole chunks; piece k's message bytes are copied in on one
    // stream, decoded on the caller's stream, and its symbols copied out on a
    // third, so copies in both directions overlap each other and decoding.
    // The split reads the offset table in host memory; if it is not
    // increasing and in range the whole message is one piece (the kernel
    // then reports the damage).
    const uint32_t nc = p.n_chunks;
    const uint32_t per_piece = uint32_t(std::max<uint64_t>(
        std::max<uint64_t>(1, ceil_div(kPieceSymbols, p.CS)), ceil_div(nc, kMaxPieces)));
    const uint32_t *offs = reinterpret_cast<const uint32_t *>(h_msg + 32);
    bool split = nc > per_piece;
    for (uint32_t c = 0; split && c < nc; ++c)
        split = offs[c] <= offs[c + 1] && uint64_t(p.data0) + offs[c + 1] <= msg_size;

    CopyStreams cs;
    if ((rc = copy_streams(&cs)) != RANS_OK) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(d_status, 0, sizeof(uint32_t), st) != cudaSuccess || !join(cs.in, st) ||
        !join(cs.out, st))
        return RANS_ERR_CUDA;
    uint64_t copied = 0;  // message bytes [0, copied) are on their way in
    for (uint64_t c0 = 0; c0 < nc || c0 == 0; c0 += per_piece) {
        const uint64_t c1 = split ? std::min<uint64_t>(nc, c0 + per_piece) : nc;
        const uint64_t hi = c1 == nc ? msg_size
                                     : std::min<uint64_t>(msg_size, round16(p.data0 + offs[c1]));
        if (hi > copied &&
            cudaMemcpyAsync(d_msg + copied, h_msg + copied, hi - copied, cudaMemcpyHostToDevice,
                            cs.in) != cudaSuccess)
            return RANS_ERR_CUDA;
        copied = std::max(copied, hi);
        if (!join(st, cs.in)) return RANS_ERR_CUDA;
        if ((rc = launch_range(p, uint32_t(c0), uint32_t(c1), st)) != RANS_OK) return rc;
        if (!join(cs.out, st)) return RANS_ERR_CUDA;
        const uint64_t s0 = c0 * p.CS, s1 = std::min<uint64_t>(n_symbols, c1 * p.CS);
        if (s1 > s0 && cudaMemcpyAsync(h_symbols + s0, d_out + s0, s1 - s0, cudaMemcpyDeviceToHost,
                                       cs.out) != cudaSuccess)
            return RANS_ERR_CUDA;
        if (c1 >= nc) break;
    }
    if (cudaMemcpyAsync(h_status, d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, cs.out) !=
            cudaSuccess ||
        !join(st, cs.out))
        return RANS_ERR_CUDA;
    return RANS_OK;
}

#ifdef RANS_CHECKED
// Checked builds: failed invariants of this file's kernels since the last call.
uint64_t rans_check_failures_decode() { return rans::take_check_failures(); }
#endif
