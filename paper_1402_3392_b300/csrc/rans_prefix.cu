// rans_prefix.cu -- Section 4 of the paper on the GPU: N prefix coders (a
// canonical code, lengths <= 12) interleaved into one stream in the order
// their decoders read it, with no metadata.
//
// The receiver's decoder (decode_core.cuh, decode_step_prefix) holds up to
// 43 bits per coder and, before each symbol, reads one 32-bit word if it
// holds fewer than 12; the reads of one step are taken in lane order.  The
// encoder below runs that read schedule beside its own coding, in one
// forward pass per chunk -- Section 4's instrumented decoder run as a
// coroutine with the encoders.  At every step it gives each read its
// position in the chunk (ballot + popc over the lanes, as the decoder
// does), and every word a coder completes goes to the oldest position that
// coder has been given.  A coder's decoder is never more than 43 bits ahead
// of its encoder, so at most two positions wait for words at any time and
// the coroutine needs no buffer beyond two registers per lane.
#include <algorithm>

#include <cuda_runtime.h>

#include "encode_core.cuh"
#include "host_util.h"

namespace rans {
namespace {

constexpr int kPfxWarps = 8;
constexpr uint32_t kPfxGroup = 16;           // steps whose symbols are loaded together
constexpr uint32_t kPfxMaxLen = RANS_PREFIX_MAX_LEN;
constexpr uint32_t kNoPos = 0xFFFFFFFFu;

struct PrefixEncodeParams {
    const uint8_t *sym;
    uint8_t *slots;       // chunk c's words at slots + c * slot_bytes
    uint32_t *sizes;      // bytes of each chunk
    uint32_t *status;
    uint64_t n_sym;
    uint32_t N, CS, n_chunks, slot_bytes;
    // The message's placement: where it goes, the look-back words (the
    // scratch's enc::LookBack) and the chunk ticket, zeroed before the launch.
    uint8_t *out;
    uint64_t *out_size;
    uint32_t data0;
    enc::LookBack lb;
    uint32_t *ticket;
    uint32_t code[RANS_MAX_ALPHABET];  // len << 16 | code; len 0: symbol not in the code
};

// The coder state of one lane: the bits not yet in a completed word (acc,
// na of them), the bits its decoder holds (held = read - consumed), and the
// positions of reads still waiting for a word (q0 oldest; kNoPos = none).
struct PfxLane {
    uint64_t acc;
    uint32_t na, held, q0, q1;
};

// One step: the decoder's read (if it holds fewer than 12 bits), then the
// symbol's code appended; a completed word goes to the oldest waiting read.
// (slot_words: the slot's capacity, for the checks of checked builds.)
template <bool FULL>
__device__ __forceinline__ void prefix_enc_step(PfxLane &c, bool active, uint32_t s,
                                                const uint32_t *tab, uint32_t *slot, uint32_t &wpos,
                                                uint32_t &err, uint32_t lt, uint32_t slot_words) {
    const bool on = FULL || active;
    const bool need = on && c.held < kPfxMaxLen;
    const uint32_t m = __ballot_sync(kFull, need);
    if (need) {
        const uint32_t pos = wpos + __popc(m & lt);
        if (c.q0 == kNoPos) c.q0 = pos;
        else c.q1 = pos;
        c.held += 32;
    }
    wpos += __popc(m);
    if (on) {
        const uint32_t e = tab[s];
        const uint32_t len = e >> 16;
        err |= uint32_t(len == 0);
        c.acc = (c.acc << len) | (e & 0xFFFFu);
        c.na += len;
        c.held -= len;
        if (c.na >= 32) {
            c.na -= 32;
            if (RANS_CHECK(c.q0 < slot_words)) slot[c.q0] = uint32_t(c.acc >> c.na);
            c.q0 = c.q1;
            c.q1 = kNoPos;
        }
    }
}

// One chunk of n_c symbols, N coders on the warp's lanes: words to slot,
// the chunk's byte size to *size.
template <int NT>
__device__ __forceinline__ void prefix_encode_chunk(const uint8_t *sym, uint32_t n_c, uint32_t N_rt,
                                                    uint32_t *slot, uint32_t slot_words,
                                                    uint32_t *size, const uint32_t *tab,
                                                    uint32_t lane, uint32_t lt, uint32_t &err) {
    const uint32_t N = NT ? NT : N_rt;
    const bool lane_on = lane < N;
    const uint32_t T = n_c / N, rem = n_c % N, G = T / kPfxGroup;
    const uint8_t *sp = sym + lane;
    PfxLane c{0, 0, 0, kNoPos, kNoPos};
    uint32_t wpos = 0;
    uint32_t cur[kPfxGroup];
    if (G) {
#pragma unroll
        for (uint32_t u = 0; u < kPfxGroup; ++u) cur[u] = lane_on ? sp[uint64_t(u) * N] : 0u;
    }
    for (uint32_t g = 0; g < G; ++g) {
        uint32_t nxt[kPfxGroup];
        const bool more = lane_on && g + 1 < G;
        const uint64_t base = uint64_t(g + 1) * kPfxGroup;
#pragma unroll
        for (uint32_t u = 0; u < kPfxGroup; ++u) nxt[u] = more ? sp[(base + u) * N] : 0u;
#pragma unroll
        for (uint32_t u = 0; u < kPfxGroup; ++u)
            prefix_enc_step<NT == 32>(c, lane_on, cur[u], tab, slot, wpos, err, lt, slot_words);
#pragma unroll
        for (uint32_t u = 0; u < kPfxGroup; ++u) cur[u] = nxt[u];
    }
    for (uint32_t t = G * kPfxGroup; t < T; ++t) {
        const uint32_t s = lane_on ? sp[uint64_t(t) * N] : 0u;
        prefix_enc_step<NT == 32>(c, lane_on, s, tab, slot, wpos, err, lt, slot_words);
    }
    if (rem) {
        const bool act = lane < rem;
        const uint32_t s = act ? sp[uint64_t(T) * N] : 0u;
        prefix_enc_step<false>(c, act, s, tab, slot, wpos, err, lt, slot_words);
    }
    // Flush: the last bits padded with zeros, then zero words for the reads
    // the decoder makes beyond them (at most one).
    if (c.na) {
        if (RANS_CHECK(c.q0 < slot_words)) slot[c.q0] = uint32_t(c.acc << (32 - c.na));
        c.q0 = c.q1;
        c.q1 = kNoPos;
    }
    if (c.q0 != kNoPos && RANS_CHECK(c.q0 < slot_words)) slot[c.q0] = 0u;
    if (c.q1 != kNoPos && RANS_CHECK(c.q1 < slot_words)) slot[c.q1] = 0u;
    RANS_CHECK(wpos <= slot_words);
    if (lane == 0) *size = 4u * wpos;
}

// Place coded chunk c: its offset by look-back (enc::chunk_offset), the
// offset table entry, its words copied to their place, and -- for the last
// chunk -- the header.
__device__ __forceinline__ void prefix_place(const PrefixEncodeParams &p, uint32_t c,
                                             uint32_t lane) {
    const uint32_t size = p.sizes[c];
    uint64_t excl;
    if (!enc::chunk_offset(p.lb, c, size, lane, excl)) {
        if (lane == 0) report(p.status, RANS_ERR_TIMEOUT);
        return;
    }
    if (lane == 0) reinterpret_cast<uint32_t *>(p.out + 32)[c] = uint32_t(excl);
    enc::copy_bytes<false, 4, true>(p.out, uint64_t(p.data0) + excl, p.slots,
                                    uint64_t(c) * p.slot_bytes, size, lane, 32);
    if (c + 1 == p.n_chunks && lane == 0)
        enc::write_header(p.out, p.out_size, p.n_sym, p.N, p.CS, p.n_chunks, p.data0,
                          uint32_t(excl + size), RANS_VERSION_PREFIX);
}

// Warps take chunks in order from a counter, code each into its slot,
// publish its size, and place it after the warp's next chunk (the last one
// at the end; see enc::chunk_offset).
template <int NT>
__global__ void __launch_bounds__(kPfxWarps * 32)
    prefix_encode_kernel(const __grid_constant__ PrefixEncodeParams p) {
    __shared__ uint32_t tab[RANS_MAX_ALPHABET];
    for (uint32_t i = threadIdx.x; i < RANS_MAX_ALPHABET; i += blockDim.x) tab[i] = p.code[i];
    __syncthreads();
    const uint32_t lane = lane_id(), lt = lanemask_lt();
    uint32_t err = 0;
    constexpr uint32_t kNone = 0xFFFFFFFFu;
    uint32_t pending = kNone;
    auto next = [&]() {
        uint32_t t = 0;
        if (lane == 0) t = atomicAdd(p.ticket, 1u);
        return __shfl_sync(kFull, t, 0);
    };
    for (uint32_t c = next(); c < p.n_chunks; c = next()) {
        const uint64_t first = uint64_t(c) * p.CS;
        const uint32_t n_c = uint32_t(umin64(p.CS, p.n_sym - first));
        prefix_encode_chunk<NT>(p.sym + first, n_c, p.N,
                                reinterpret_cast<uint32_t *>(p.slots + uint64_t(c) * p.slot_bytes),
                                p.slot_bytes / 4, p.sizes + c, tab, lane, lt, err);
        __syncwarp();  // the chunk's words and size are written
        // A symbol without a code is reported before the size is published.
        if (__any_sync(kFull, err) && lane == 0) report(p.status, RANS_ERR_ZERO_FREQ);
        enc::publish_size(p.lb, c, p.sizes[c], lane);
        if (pending != kNone) prefix_place(p, pending, lane);
        pending = c;
    }
    if (pending != kNone) prefix_place(p, pending, lane);
}

// After the placing launch: a rejected message has size 0.
__global__ void prefix_settle_kernel(const uint32_t *status, uint64_t *out_size) {
    if (*status != RANS_OK) *out_size = 0;
}

struct PrefixFinalizeParams {
    uint8_t *out;
    uint64_t *out_size;
    const uint32_t *sizes;
    const uint32_t *status;
    uint64_t n_sym;
    uint32_t N, CS, n_chunks, data0;
};

constexpr int kFinThreads = 1024;
__global__ void __launch_bounds__(kFinThreads)
    prefix_finalize_kernel(const __grid_constant__ PrefixFinalizeParams p) {
    __shared__ uint32_t warp_sums[32];
    __shared__ uint64_t carry_s;
    if (*p.status != RANS_OK) {
        if (threadIdx.x == 0) *p.out_size = 0;
        return;
    }
    enc::finalize_message(p.out, p.out_size, p.sizes, p.n_sym, p.N, p.CS, p.n_chunks, p.data0,
                          warp_sums, &carry_s, RANS_VERSION_PREFIX);
}

// Worst-case words of a chunk of CS symbols: ceil(12 CS / 32) + 2N, plus one.
uint32_t prefix_slot_bytes(uint32_t CS, uint32_t N) {
    return uint32_t(round16(4ull * ((uint64_t(CS) * kPfxMaxLen + 31) / 32 + 2ull * N + 1)));
}

// Scratch of a prefix message: the chunk slots, then the chunk sizes, then
// the look-back words and the ticket (as in enc::ScratchLayout).
struct PrefixScratch {
    uint64_t sizes, look, glook, gacc, ticket, total;
};
PrefixScratch prefix_scratch(uint64_t n_chunks, uint32_t slot_bytes) {
    PrefixScratch s{};
    const uint64_t n_groups = (n_chunks + 31) / 32;
    s.sizes = n_chunks * slot_bytes;
    s.look = s.sizes + round16(4 * n_chunks) + 16;  // 16 readable bytes past the last slot
    s.glook = s.look + round16(8 * n_chunks);
    s.gacc = s.glook + round16(8 * n_groups);
    s.ticket = s.gacc + round16(8 * n_groups);
    s.total = s.ticket + 16;
    return s;
}

}  // namespace
}  // namespace rans

using namespace rans;

extern "C" uint64_t rans_encode_scratch_size_prefix(uint64_t n_symbols, const rans_params *params) {
    if (!params_ok(params)) return 0;
    const MessageGeometry g = geometry(n_symbols, params);
    return prefix_scratch(g.n_chunks, prefix_slot_bytes(params->chunk_symbols, params->n_lanes))
        .total;
}

extern "C" int rans_encode_prefix(const uint8_t *d_symbols, uint64_t n_symbols,
                                  const uint8_t *h_lengths, uint32_t n_alpha,
                                  const rans_params *params, uint8_t *d_out, uint64_t out_cap,
                                  uint64_t *d_out_size, uint32_t *d_status, void *d_scratch,
                                  uint64_t scratch_cap, rans_stream_t stream) {
    uint16_t codes[RANS_MAX_ALPHABET];
    if (!params_ok(params) || !d_out || !d_out_size || !d_status || !d_scratch ||
        !aligned16(d_out) || !aligned16(d_scratch) || (n_symbols && !d_symbols))
        return RANS_ERR_INVALID_ARG;
    int rc = rans_prefix_codes(h_lengths, n_alpha, codes);
    if (rc != RANS_OK) return rc;
    const MessageGeometry g = geometry(n_symbols, params);
    const uint64_t data_max = rans_max_encoded_size_prefix(n_symbols, params) - g.data0;
    if (g.n_chunks > 0xFFFFFFFEull || data_max > 0xFFFFFFF0ull) return RANS_ERR_INVALID_ARG;
    const uint32_t slot_bytes = prefix_slot_bytes(params->chunk_symbols, params->n_lanes);
    if (out_cap < rans_max_encoded_size_prefix(n_symbols, params) ||
        scratch_cap < rans_encode_scratch_size_prefix(n_symbols, params))
        return RANS_ERR_BUFFER_TOO_SMALL;

    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(d_status, 0, sizeof(uint32_t), st) != cudaSuccess) return RANS_ERR_CUDA;
    uint8_t *scr = static_cast<uint8_t *>(d_scratch);
    const PrefixScratch ps = prefix_scratch(g.n_chunks, slot_bytes);
    if (g.n_chunks == 0) {
        PrefixFinalizeParams fp{};
        fp.out = d_out;
        fp.out_size = d_out_size;
        fp.status = d_status;
        fp.n_sym = n_symbols;
        fp.N = params->n_lanes;
        fp.CS = params->chunk_symbols;
        fp.data0 = uint32_t(g.data0);
        prefix_finalize_kernel<<<1, kFinThreads, 0, st>>>(fp);
        return check_launch();
    }
    PrefixEncodeParams ep{};
    ep.sym = d_symbols;
    ep.slots = scr;
    ep.sizes = reinterpret_cast<uint32_t *>(scr + ps.sizes);
    ep.status = d_status;
    ep.n_sym = n_symbols;
    ep.N = params->n_lanes;
    ep.CS = params->chunk_symbols;
    ep.n_chunks = uint32_t(g.n_chunks);
    ep.slot_bytes = slot_bytes;
    ep.out = d_out;
    ep.out_size = d_out_size;
    ep.data0 = uint32_t(g.data0);
    ep.lb.look = reinterpret_cast<uint64_t *>(scr + ps.look);
    ep.lb.glook = reinterpret_cast<uint64_t *>(scr + ps.glook);
    ep.lb.gacc = reinterpret_cast<uint64_t *>(scr + ps.gacc);
    ep.lb.n_chunks = ep.n_chunks;
    // As for rans_encode: a second plus a microsecond per step of a chunk.
    ep.lb.wait_ns = 1000000000ull + 1000ull * (ep.CS / ep.N + 1);
    ep.ticket = reinterpret_cast<uint32_t *>(scr + ps.ticket);
    for (uint32_t s = 0; s < n_alpha; ++s)
        ep.code[s] = h_lengths[s] ? (uint32_t(h_lengths[s]) << 16) | codes[s] : 0u;
    if (cudaMemsetAsync(scr + ps.look, 0, ps.total - ps.look, st) != cudaSuccess)
        return RANS_ERR_CUDA;
    auto kernel = ep.N == 32 ? prefix_encode_kernel<32> : prefix_encode_kernel<0>;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kPfxWarps * 32, 0) !=
            cudaSuccess ||
        per_sm <= 0)
        return RANS_ERR_CUDA;
    const uint64_t want = ceil_div(g.n_chunks, kPfxWarps);
    const unsigned grid =
        unsigned(std::max<uint64_t>(1, std::min<uint64_t>(want, uint64_t(per_sm) * sm_count())));
    kernel<<<grid, kPfxWarps * 32, 0, st>>>(ep);
    if (check_launch() != RANS_OK) return RANS_ERR_CUDA;
    prefix_settle_kernel<<<1, 1, 0, st>>>(d_status, d_out_size);
    return check_launch();
}

#ifdef RANS_CHECKED
// Checked builds: failed invariants of this file's kernels since the last call.
uint64_t rans_check_failures_prefix() { return rans::take_check_failures(); }
#endif
