// encode_core.cuh -- the encoder's building blocks, shared by the
// single-message entry points (rans_encode.cu) and the batched persistent
// kernel (rans_batch.cu).
//
// One warp encodes one chunk; lane j is coder j of the chunk's N interleaved
// rANS coders.  The encoder runs over the chunk backwards, step T-1 down to 0
// (Section 2: the encoder processes the message from last to first and writes
// backwards).  Per step every lane with a symbol renormalizes at most once
// (b = 2^16 >= M, Section 5) and then applies C (Algorithm 1 Encode):
//     if x >= f_s * 2^20:  emit x mod 2^16;  x = floor(x / 2^16)
//     x = floor(x / f_s) * M + B_s + (x mod f_s)
// In the serial interleaved order of Section 3 the emissions of one step come
// from coder N-1 down to coder 0, and the buffer is written backwards, so the
// lanes place their words with a reverse-lane prefix count:
//     lane j stores at write_pos - 2 * popc(emit_mask & lanes_at_or_above_j)
// (the packed store of Sections 5 and 6).  floor(x / f_s) is an exact
// multiply-high by ceil(2^(32+k) / f_s), k = ceil(log2 f_s).
//
// Words are staged in a per-warp shared-memory ring and leave as 512-byte bulk
// stores (TMA) into a worst-case scratch slot per chunk.  A whole message is
// then placed in the same launch: each warp publishes its chunk's size, finds
// the sizes of the chunks before it (decoupled look-back), writes its offset
// and copies the chunk to its place.  Pieces of a message (host-memory
// encoding) and batches of streams use a scan of the sizes and a separate
// copy instead.
#pragma once

#include <cstdint>

#include "adapt_model.cuh"
#include "device_util.cuh"
#include "host_util.h"

namespace rans {
namespace enc {

constexpr int kWarps = 8;
constexpr uint32_t kThreads = kWarps * 32;
constexpr uint32_t kSeg = 512;
constexpr uint32_t kNSeg = 8;
constexpr uint32_t kRing = kSeg * kNSeg;  // 4 KiB per warp, aligned to 4 KiB in shared space
constexpr uint32_t kGroup = 16;
// A step writes at most 32 words = 64 bytes, so a group writes at most 1 KiB
// and touches at most three segments.
static_assert(kGroup * 64 <= 2 * kSeg, "a group must fit in two segments");
// Shared memory: [encode table: 256 entries of 8 bytes, or of 16 for wide
// models][alignment slack][one ring per warp][a few words of CTA state].
constexpr uint32_t kTabBytes = 256 * 16;
constexpr uint32_t kMiscOffset = kTabBytes + kRing + kWarps * kRing;
constexpr uint32_t kSmemBytes = kMiscOffset + 64;
constexpr uint32_t kZeroFlag = 1u << 19;  // encode-table bit marking f_s = 0
constexpr uint32_t kRawFlag = 1u << 18;   // encode-table bit: the symbol carries a raw word
constexpr uint32_t kL8 = 1u << 23;         // byte-wise messages: L = 2^23, b = 2^8
// Adaptive messages: binary symbols, each coder's context p (probability of
// a 0 scaled to M) starts at M/2 and moves by (target - p) >> kAdaptRate.
constexpr uint32_t kAdaptRate = 5;
constexpr uint32_t kAdaptP0 = kM / 2;

// Scratch of one message, all sections 16-byte aligned: one worst-case slot
// of words per chunk (written backwards from its end), then the chunks'
// final states, first-word offsets and byte sizes, then the look-back words
// (one per chunk, two per group of 32 chunks) and the chunk ticket counter,
// zeroed before each launch that places the chunks itself.
struct ScratchLayout {
    uint64_t words, states, wstart, sizes, look, glook, gacc, ticket, ctx, total;
    uint32_t slot_bytes;
};

// words_per_symbol: 1, or 2 for bypass messages (a raw word after a symbol).
__host__ __device__ inline ScratchLayout scratch_layout(uint64_t n_chunks, uint32_t N, uint32_t CS,
                                                        uint32_t words_per_symbol = 1) {
    ScratchLayout s{};
    s.slot_bytes = uint32_t((2ull * words_per_symbol * CS + kSeg - 1) / kSeg * kSeg);
    s.words = 0;
    s.states = (n_chunks * s.slot_bytes + 16 + 15) & ~uint64_t(15);
    s.wstart = s.states + ((n_chunks * N * 4 + 15) & ~uint64_t(15));
    s.sizes = s.wstart + ((n_chunks * 4 + 15) & ~uint64_t(15));
    const uint64_t n_groups = (n_chunks + 31) / 32;
    s.look = s.sizes + ((n_chunks * 4 + 15) & ~uint64_t(15));
    s.glook = s.look + ((n_chunks * 8 + 15) & ~uint64_t(15));
    s.gacc = s.glook + ((n_groups * 8 + 15) & ~uint64_t(15));
    s.ticket = s.gacc + ((n_groups * 8 + 15) & ~uint64_t(15));
    s.total = s.ticket + 16;
    s.ctx = s.total;  // adaptive messages: the contexts' words (adaptive_ctx_stride) follow
    return s;
}

struct Smem {
    uint2 *tab;
    uint32_t tab_s;
    uint32_t rings_s;  // 4 KiB aligned
    uint8_t *rings;
    uint32_t *misc;
};

__device__ __forceinline__ Smem smem_layout(uint8_t *smem) {
    Smem s;
    s.tab = reinterpret_cast<uint2 *>(smem);
    s.tab_s = smem_addr(smem);
    const uint32_t raw = smem_addr(smem + kTabBytes);
    s.rings_s = (raw + kRing - 1) & ~(kRing - 1);
    s.rings = smem + kTabBytes + (s.rings_s - raw);
    s.misc = reinterpret_cast<uint32_t *>(smem + kMiscOffset);
    return s;
}

// floor(x / f) by a multiplication (Granlund and Montgomery, "Division by
// invariant integers using multiplication", 1994): with k = ceil(log2 f) and
// m = ceil(2^(32+k) / f) = 2^32 + m_lo, the quotient is floor(x * m /
// 2^(32+k)).  m is 2^(32+k)/f + e with 0 <= e < 1, so the error x*e/2^(32+k)
// < 2^-k <= 1/f never carries x/f past the next integer.
// The encoders divide only states x of the precursor set I_s = [f L / M,
// f b L / M), x < f * 2^(32 - lm) for M = 2^lm (Section 2; b = L = 2^16, and
// below that for byte-wise coding).  With m < 2^(32+k)/f + 1 that gives
// x * m < 2^(64+k-lm) + f * 2^(32-lm) - 2^(32+k)/f, below 2^64 (k = lm: f <=
// 2^k makes f * 2^(32-lm) <= 2^32 <= 2^(32+k)/f; k < lm: both terms are
// below 2^63).  So the product fits in 64 bits and one 64-bit multiply-add,
// x * m_lo + x * 2^32, gives it exactly (for x up to 2^32 it would not fit;
// the division check runs this code over every x of every I_s).
// Measured on B300 against the 33-bit-sum form (x + umulhi(x, m_lo)) >> k:
// 1 GiB encode 1425 -> 1284 us.  reciprocal() gives (m_lo, k);
// div_reciprocal() takes k from the low 5 bits of kbits (the funnel shift's
// wrap mode), so a table word holding k in bits 12..16 can be passed whole.
__host__ __device__ inline void reciprocal(uint32_t f, uint32_t &m_lo, uint32_t &k) {
    k = 0;
    while ((1u << k) < f) ++k;
    const uint64_t m = ((1ull << (32 + k)) + f - 1) / f;
    m_lo = uint32_t(m - (1ull << 32));
}
__device__ __forceinline__ uint32_t div_reciprocal(uint32_t x, uint32_t m_lo, uint32_t kbits) {
    const uint64_t xm = uint64_t(x) * m_lo + (uint64_t(x) << 32);
    return __funnelshift_r(uint32_t(xm >> 32), 0u, kbits);
}

// floor(x / f) and x mod f for 1 <= f < M and x < f * 2^20, as the adaptive
// coder computes them: a float estimate rounded towards zero at every step
// (reciprocal, conversion, product), so never above x/f and, since x/f <
// 2^20 and each rounding loses less than 2^-23 relative, below it by less
// than 1; then one exact correction by the remainder.
__device__ __forceinline__ uint32_t div_float(uint32_t x, uint32_t f, uint32_t &r) {
    const float rf = __frcp_rz(float(f));
    uint32_t q = __float2uint_rz(__fmul_rz(__uint2float_rz(x), rf));
    r = x - q * f;
    if (r >= f) {
        ++q;
        r -= f;
    }
    return q;
}

// Encode-table entry for symbol s with frequency f (1 <= f <= M):
//   .x = m_lo = ceil(2^(32+k) / f) - 2^32,  k = ceil(log2 f)   (0 <= m_lo < 2^32)
//   .y = (M - f) << 20 | k << 12 | B_s
// floor(x/f) = div_reciprocal(x, m_lo, k) for every x < 2^32.
// Emit test: x >= f * 2^20  <=>  x > f * 2^20 - 1 = ~((M - f) << 20)  (u32).
// Built by the whole CTA; cum: 257 words of free shared memory.  Returns the
// sum of the frequencies to every thread.
// raw_words (bypass messages, may be null): symbol s carries raw_words[s]
// (0 or 1) raw words; marked by kRawFlag in .y.
__device__ __forceinline__ uint2 encode_entry(uint32_t f, uint32_t B) {
    uint2 t;
    uint32_t k;
    reciprocal(f, t.x, k);
    t.y = ((kM - (f & (2 * kM - 1))) << 20) | (k << 12) | (B & (kM - 1));
    return t;
}
__device__ __noinline__ static uint32_t build_encode_table(const uint16_t *freq, uint2 *tab,
                                                           uint32_t *cum,
                                                           const uint8_t *raw_words = nullptr) {
    const uint32_t tid = threadIdx.x;
    if (tid < 32) {
        uint32_t v[8], run = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            v[k] = run;
            run += freq[tid * 8 + k];
        }
        uint32_t incl = run;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, incl, d);
            if (tid >= uint32_t(d)) incl += y;
        }
        const uint32_t excl = incl - run;
#pragma unroll
        for (int k = 0; k < 8; ++k) cum[tid * 8 + k] = excl + v[k];
        if (tid == 31) cum[256] = incl;
    }
    __syncthreads();
    for (uint32_t s = tid; s < 256; s += blockDim.x) {
        const uint32_t f = freq[s];
        uint2 t;
        if (f == 0) {
            t = make_uint2(0u, kZeroFlag);  // never emits, leaves x unchanged
        } else {
            t = encode_entry(f, cum[s]);
            if (raw_words && raw_words[s]) t.y |= kRawFlag;  // the shift uses k's 5 bits only
        }
        tab[s] = t;
    }
    const uint32_t total = cum[256];
    __syncthreads();
    return total;
}

// Wide models (M = 2^lm, lm 13 or 14; b = 2^16 >= M, one renormalization
// per symbol): entry s of 16 bytes, built by the whole CTA (cum: 257 words of
// free shared memory; returns the frequencies' sum):
//   .x = m_lo as above (exact division for every x < 2^32, f up to 2^14)
//   .y = f * 2^(32 - lm) - 1: the emit test is x > .y   (f = M: never)
//   .z = M - f             .w = B_s | k << 24
// A symbol with f = 0: .y = ~0 (never emits), .x = .z = 0, .w = kZeroFlag
// (k = 0, so q = x and x is left unchanged).
__device__ __noinline__ static uint32_t build_wide_encode_table(const uint16_t *freq, uint32_t lm,
                                                                uint4 *tab, uint32_t *cum) {
    const uint32_t tid = threadIdx.x, M = 1u << lm;
    if (tid < 32) {
        uint32_t v[8], run = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            v[k] = run;
            run += freq[tid * 8 + k];
        }
        uint32_t incl = run;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, incl, d);
            if (tid >= uint32_t(d)) incl += y;
        }
        const uint32_t excl = incl - run;
#pragma unroll
        for (int k = 0; k < 8; ++k) cum[tid * 8 + k] = excl + v[k];
        if (tid == 31) cum[256] = incl;
    }
    __syncthreads();
    for (uint32_t s = tid; s < 256; s += blockDim.x) {
        const uint32_t f = freq[s];
        uint4 t;
        if (f == 0) {
            t = make_uint4(0u, 0xFFFFFFFFu, 0u, kZeroFlag);
        } else {
            uint32_t k;
            reciprocal(f, t.x, k);
            t.y = uint32_t((uint64_t(f) << (32 - lm)) - 1);
            t.z = M - f;
            t.w = (cum[s] & 0xFFFFu) | (k << 24);
        }
        tab[s] = t;
    }
    const uint32_t total = cum[256];
    __syncthreads();
    return total;
}

__device__ __forceinline__ uint4 ld_enc_table4(uint32_t a) {
    uint4 v;
    asm("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "r"(a));
    return v;
}

__device__ __forceinline__ uint2 ld_enc_table(uint32_t a) {
    uint2 v;
    asm("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a));
    return v;
}
__device__ __forceinline__ void st_ring_u8(uint32_t a, uint32_t v) {
    asm volatile("st.shared.u8 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void st_ring_u16(uint32_t a, uint32_t v) {
    asm volatile("st.shared.u16 [%0], %1;" ::"r"(a), "h"(uint16_t(v)) : "memory");
}
// The store above made by the lanes with p set, as one predicated store (the
// emitting lanes of a step; measured on B300: 3000-stream batched encode
// 6.98 -> 6.76 ms against a branch around st_ring_u16).
__device__ __forceinline__ void st_ring_u16_if(bool p, uint32_t a, uint32_t v) {
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q st.shared.u16 [%0], %1;\n\t}" ::"r"(a),
        "h"(uint16_t(v)), "r"(uint32_t(p))
        : "memory");
}

// a * b + c (mod 2^32) as one multiply-add.
__device__ __forceinline__ uint32_t imad_u32(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t r;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
    return r;
}

// Shared address of the 16-bit word that the k-th emitting lane from the top
// stores below write position wp.  RING > 0: wp is the byte position in the
// chunk's slot, which lives in the warp's ring (aligned to RING) at
// wp mod RING.  RING = 0: wp is the shared address of the write position
// itself, for groups whose stores cannot pass below the ring's start (one
// multiply-add, no wrap).
template <uint32_t RING>
__device__ __forceinline__ uint32_t store_at(uint32_t wp, uint32_t k, uint32_t ring_s) {
    return RING ? ((wp - 2u * k) & (RING - 1)) | ring_s : imad_u32(k, 0u - 2u, wp);
}

// Encode one step with the symbol's table entry t (lanes with on set):
// renormalize (emit the low 16 bits if x >= f_s * 2^20), then x = C(s, x).
// wp is the warp-uniform write position (bytes, counting down); ring_s is
// the warp's 4 KiB-aligned ring.
template <bool FULL, uint32_t RING>
__device__ __forceinline__ void encode_with(uint32_t &x, uint32_t &wp, bool on, uint2 t,
                                            uint32_t ring_s, uint32_t ge) {
    const bool emit = on && (x > ~(t.y & 0xFFF00000u));
    const uint32_t m = __ballot_sync(kFull, emit);
    st_ring_u16_if(emit, store_at<RING>(wp, __popc(m & ge), ring_s), x);
    x = emit ? x >> 16 : x;
    if (RING) wp -= 2u * __popc(m);
    else wp = imad_u32(__popc(m), 0u - 2u, wp);
    if (on) {
        const uint32_t q = div_reciprocal(x, t.x, t.y >> 12);  // floor(x / f_s)
        x = x + q * (t.y >> 20) + (t.y & 0xFFFu);
    }
}
// The step with the entry from the shared-memory table (acc collects the
// entries' flags).
template <bool FULL, uint32_t RING = kRing>
__device__ __forceinline__ void encode_step(uint32_t &x, uint32_t &wp, uint32_t &acc, bool active,
                                            uint32_t s, uint32_t tab_s, uint32_t ring_s,
                                            uint32_t ge) {
    const uint2 t = ld_enc_table(tab_s + (s << 3));
    const bool on = FULL || active;
    if (on) acc |= t.y;
    encode_with<FULL, RING>(x, wp, on, t, ring_s, ge);
}
// The step with a binary model (f_0 + f_1 = M, both > 0; rABS, Section 2):
// the entries of symbols 0 and 1 (encode_entry) are held in registers and
// selected by the symbol, no table.  acc collects the symbols: above 1, one
// the model does not have.
template <bool FULL, uint32_t RING = kRing>
__device__ __forceinline__ void encode_step_binary(uint32_t &x, uint32_t &wp, uint32_t &acc,
                                                   bool active, uint32_t s, uint2 e0, uint2 e1,
                                                   uint32_t ring_s, uint32_t ge) {
    const bool on = FULL || active;
    if (on) acc |= s;
    const uint2 t = s ? e1 : e0;
    encode_with<FULL, RING>(x, wp, on, t, ring_s, ge);
}

// One step with a wide model: as encode_step with the 16-byte entry.
template <bool FULL, uint32_t RING = kRing>
__device__ __forceinline__ void encode_step_wide(uint32_t &x, uint32_t &wp, uint32_t &acc,
                                                 bool active, uint32_t s, uint32_t tab_s,
                                                 uint32_t ring_s, uint32_t ge) {
    const uint4 t = ld_enc_table4(tab_s + (s << 4));
    const bool on = FULL || active;
    if (on) acc |= t.w;
    const bool emit = on && x > t.y;
    const uint32_t m = __ballot_sync(kFull, emit);
    if (emit) {
        st_ring_u16(store_at<RING>(wp, __popc(m & ge), ring_s), x);
        x >>= 16;
    }
    if (RING) wp -= 2u * __popc(m);
    else wp = imad_u32(__popc(m), 0u - 2u, wp);
    if (on) {
        const uint32_t q = div_reciprocal(x, t.x, t.w >> 24);
        x = x + q * t.z + (t.w & 0xFFFFu);
    }
}

// One step of a byte-wise chunk (b = 2^8 < M, Section 5): a lane emits
// k = [x >= f*2^19] + [x >= f*2^27] bytes (x must end below f*2^19 = the top
// of I_s) before coding.  The decoder reads a step's bytes breadth-first --
// first pass: one byte for every lane that needs one, lanes in order; second
// pass: the second byte of the lanes that need two -- so in the backwards-
// filled buffer the step's second-pass bytes sit above its first-pass bytes.
// A lane's first-pass byte is the one its decoder reads first: the higher of
// two.
template <bool FULL>
__device__ __forceinline__ void encode_step_bytes(uint32_t &x, uint32_t &wp, uint32_t &acc,
                                                  bool active, uint32_t s, uint32_t tab_s,
                                                  uint32_t ring_s, uint32_t ge) {
    const uint2 t = ld_enc_table(tab_s + (s << 3));
    const bool on = FULL || active;
    if (on) acc |= t.y;
    const uint32_t thr = (kM - (t.y >> 20)) << 19;  // f * 2^19; 2^31 for f = M or f = 0
    const bool e1 = on && x >= thr;
    const bool e2 = e1 && (x >> 8) >= thr;
    const uint32_t m1 = __ballot_sync(kFull, e1);
    const uint32_t m2 = __ballot_sync(kFull, e2);
    const uint32_t lt = ~ge;
    const uint32_t n1 = __popc(m1), n2 = __popc(m2);
    if (e2) st_ring_u8(((wp - n2 + __popc(m2 & lt)) & (kRing - 1)) | ring_s, x);
    if (e1) st_ring_u8(((wp - n2 - n1 + __popc(m1 & lt)) & (kRing - 1)) | ring_s, e2 ? x >> 8 : x);
    if (e1) x >>= e2 ? 16 : 8;
    wp -= n1 + n2;
    if (on) {
        const uint32_t q = div_reciprocal(x, t.x, t.y >> 12);
        x = x + q * (t.y >> 20) + (t.y & 0xFFFu);
    }
}

// After a 0, p += (M - p) >> rate; after a 1, p -= p >> rate -- both as
// p + floor((T - p) / 2^rate), T = M or 2^rate - 1 (s is 0 or 1 here, any
// nonzero symbol counting as a 1).
__device__ __forceinline__ uint32_t adapt_ctx(uint32_t p, uint32_t s) {
    const uint32_t one = s != 0u;
    return p + uint32_t(int32_t((kM - p) - one * (kM - ((1u << kAdaptRate) - 1))) >> kAdaptRate);
}

// Adaptive scratch of one chunk, in u32 words: for each full group g of
// kGroup steps and each coder, word [g*N + lane] = the context at the
// group's first step | the group's symbols as bits << 16 (bit v: step
// g*kGroup + v); above the last full group, word [(t - top0)*N + lane] = the
// context of step t (top0 = G*kGroup - G, G = full groups).
__host__ __device__ constexpr uint64_t adaptive_ctx_stride(uint32_t CS, uint32_t N) {
    return (uint64_t(CS) + kGroup - 1) / kGroup + uint64_t(kGroup) * N;
}
static_assert(kGroup <= 16, "a group's symbol bits share a word with the context");

// Adaptive chunks, pass 1: run every coder's context forwards over its own
// symbols (a group's symbols loaded while the previous group updates) and
// store the words above.  A symbol other than 0 or 1 sets kZeroFlag.
template <int NT>
__device__ __forceinline__ void adaptive_forward(const uint8_t *sym, uint32_t n_c, uint32_t N_rt,
                                                 uint32_t *ctx, uint32_t lane, uint32_t &acc) {
    const uint32_t N = NT ? NT : N_rt;
    if (lane >= N) return;
    const uint32_t T_full = n_c / N, G = T_full / kGroup, top0 = G * kGroup - G;
    const uint8_t *sp = sym + lane;
    uint32_t *cp = ctx + lane;
    uint32_t p = kAdaptP0, bad = 0, nxt[kGroup];
    if (G) {
#pragma unroll
        for (uint32_t u = 0; u < kGroup; ++u) nxt[u] = sp[uint64_t(u) * N];
    }
    for (uint32_t g = 0; g < G; ++g) {
        uint32_t bits = 0;  // bit u: step g*kGroup + u
#pragma unroll
        for (uint32_t u = 0; u < kGroup; ++u) {
            bad |= nxt[u];
            bits |= uint32_t(nxt[u] != 0u) << u;
        }
        const bool more = g + 1 < G;
        const uint64_t base = uint64_t(g + 1) * kGroup;
#pragma unroll
        for (uint32_t u = 0; u < kGroup; ++u) nxt[u] = more ? sp[(base + u) * N] : 0u;
        cp[uint64_t(g) * N] = p | bits << 16;
#pragma unroll
        for (uint32_t u = 0; u < kGroup; ++u) p = adapt_ctx(p, (bits >> u) & 1u);
    }
    const uint32_t T_end = T_full + (lane < n_c % N ? 1u : 0u);
    for (uint32_t t = G * kGroup; t < T_end; ++t) {
        const uint32_t s = sp[uint64_t(t) * N];
        cp[uint64_t(t - top0) * N] = p;
        bad |= s;
        p = adapt_ctx(p, s);
    }
    if (bad > 1u) acc |= kZeroFlag;
}

// Pass 1 of an adaptive-n chunk (adapt_model.cuh): run every coder's model
// forwards over its own symbols and store, for each symbol, the word
// B_s | f_s << 16 it is coded with at words[t * N + lane] (step t).  A symbol
// >= n sets kZeroFlag.
template <int NT, int NB>
__device__ __forceinline__ void adaptive_n_forward(const uint8_t *sym, uint32_t n_c, uint32_t N_rt,
                                                   uint32_t n, uint32_t *words, uint32_t lane,
                                                   uint32_t &acc) {
    const uint32_t N = NT ? NT : N_rt;
    if (lane >= N) return;
    const uint32_t T_end = n_c / N + (lane < n_c % N ? 1u : 0u), nm = kM - n;
    uint32_t cm[NB];
    adapt::init<NB>(cm, n);
    bool bad = false;
    for (uint32_t t = 0; t < T_end; ++t) {
        const uint32_t s = sym[uint64_t(t) * N + lane];
        bad |= s >= n;
        uint32_t B = 0, F = kM;
        bool le[NB];
        if constexpr (NB < 15) {
            // B = C_s and F = C_{s+1} from the boundaries' sides (le is true
            // below s + 1), as the decoder finds them.  Measured on B300 (256
            // Mi symbols): n = 8 1553 -> 1407 us, n = 4 1122 -> 1091 us, but n
            // = 16 2412 -> 2499 us, which keeps the two compares.
#pragma unroll
            for (int i = 0; i < NB; ++i) {
                le[i] = uint32_t(i + 1) <= s;
                B = le[i] ? cm[i] : B;
            }
#pragma unroll
            for (int i = NB - 1; i >= 0; --i) F = le[i] ? F : cm[i];
        } else {
#pragma unroll
            for (int i = 0; i < NB; ++i) {
                const uint32_t b = uint32_t(i + 1);
                B = b == s ? cm[i] : B;
                F = b == s + 1 ? cm[i] : F;
                le[i] = b <= s;
            }
        }
        words[uint64_t(t) * N + lane] = B | ((F - B) << 16);
        adapt::update<NB>(cm, le, nm);
    }
    if (bad) acc |= kZeroFlag;
}

// Pass 2 of an adaptive-n chunk, one step: the symbol's stored word gives
// B = w & 0xFFFF and f = w >> 16; renormalize (emit if x >= f * 2^20), then
// C with the exact float-estimate division.
template <bool FULL>
__device__ __forceinline__ void encode_step_bf(uint32_t &x, uint32_t &wp, bool active, uint32_t w,
                                               uint32_t ring_s, uint32_t ge) {
    const bool on = FULL || active;
    const uint32_t f = w >> 16;
    const bool emit = on && x >= (f << 20);
    const uint32_t m = __ballot_sync(kFull, emit);
    if (emit) {
        st_ring_u16(((wp - 2u * __popc(m & ge)) & (kRing - 1)) | ring_s, x);
        x >>= 16;
    }
    wp -= 2u * __popc(m);
    if (on) {
        uint32_t r;
        const uint32_t q = div_float(x, f, r);
        x = (q << kLog2M) + (w & 0xFFFFu) + r;
    }
}

// Adaptive chunks, pass 2, one step: symbol s (0 or 1) coded with the stored
// context p: f = p or M - p, B = 0 or p.  floor(x/f) comes from a float
// estimate rounded towards zero throughout -- never above x/f, and below it
// by less than 1 since x < f * 2^20 here -- and one exact correction.
template <bool FULL>
__device__ __forceinline__ void encode_step_adaptive(uint32_t &x, uint32_t &wp, bool active,
                                                     uint32_t s, uint32_t p, uint32_t ring_s,
                                                     uint32_t ge) {
    const bool on = FULL || active;
    const bool one = s != 0u;
    const uint32_t f = one ? kM - p : p;
    const bool emit = on && x >= (f << 20);
    const uint32_t m = __ballot_sync(kFull, emit);
    if (emit) {
        st_ring_u16(((wp - 2u * __popc(m & ge)) & (kRing - 1)) | ring_s, x);
        x >>= 16;
    }
    wp -= 2u * __popc(m);
    if (on) {
        uint32_t r;
        const uint32_t q = div_float(x, f, r);
        x = (q << kLog2M) + (one ? p : 0u) + r;
    }
}

// The step of a chunk of the byte-wise, wide, binary or plain kind.
// RING = 0 (plain, binary and wide chunks only): wp is an absolute shared
// address (store_at).  e0, e1: a binary model's entries.
template <bool FULL, bool BYTES, bool WIDE, uint32_t RING = kRing, bool BINARY = false>
__device__ __forceinline__ void coded_step(uint32_t &x, uint32_t &wp, uint32_t &acc, bool active,
                                           uint32_t s, uint32_t tab_s, uint32_t ring_s,
                                           uint32_t ge, uint2 e0 = {}, uint2 e1 = {}) {
    static_assert(RING || !BYTES, "byte-wise steps address the ring by offset");
    if (BINARY) encode_step_binary<FULL, RING>(x, wp, acc, active, s, e0, e1, ring_s, ge);
    else if (BYTES) encode_step_bytes<FULL>(x, wp, acc, active, s, tab_s, ring_s, ge);
    else if (WIDE) encode_step_wide<FULL, RING>(x, wp, acc, active, s, tab_s, ring_s, ge);
    else encode_step<FULL, RING>(x, wp, acc, active, s, tab_s, ring_s, ge);
}

// A step stores at most 32 words (64 bytes), so a group of kGroup steps
// stores within [wp - kGroup * 64, wp).  When the write position's ring
// offset is at least that, none of the group's stores wraps below the
// ring's start (3 groups in 4 with a 4 KiB ring).  Used by the batched
// encoder's groups (measured on B300: 10,000 streams 23.57 -> 23.37 ms); in
// the single-message encoder, whose groups also load the next group's
// symbols, the second copy of the unrolled group made it slower (1 GiB:
// 1408 -> 1474 us), so that one always wraps.
constexpr uint32_t kGroupBytes = kGroup * 64u;
__device__ __forceinline__ bool group_is_linear(uint32_t wp) {
    return (wp & (kRing - 1)) >= kGroupBytes;
}

// One step of a bypass chunk (Section 3): a lane whose symbol carries a raw
// word rw sends it before encoding the symbol, so in the stream (decoder
// order) it follows that lane's renormalization word.  One reverse-lane
// prefix over both kinds of word places them: the words of lanes >= j fill
// [wp - 2A, wp), lane j's own at the bottom (renormalization word first).
template <bool FULL>
__device__ __forceinline__ void encode_step_raw(uint32_t &x, uint32_t &wp, uint32_t &acc,
                                                bool active, uint32_t s, uint32_t rw,
                                                uint32_t tab_s, uint32_t ring_s, uint32_t ge) {
    const uint2 t = ld_enc_table(tab_s + (s << 3));
    const bool on = FULL || active;
    if (on) acc |= t.y;
    const bool emit = on && (x > ~(t.y & 0xFFF00000u));
    const bool has = on && (t.y & kRawFlag) != 0u;
    const uint32_t m = __ballot_sync(kFull, emit);
    const uint32_t mr = __ballot_sync(kFull, has);
    const uint32_t pos = wp - 2u * (__popc(m & ge) + __popc(mr & ge));
    if (has) st_ring_u16(((pos + 2u * uint32_t(emit)) & (kRing - 1)) | ring_s, rw);
    if (emit) {
        st_ring_u16((pos & (kRing - 1)) | ring_s, x);
        x >>= 16;
    }
    wp -= 2u * (__popc(m) + __popc(mr));
    if (on) {
        const uint32_t q = div_reciprocal(x, t.x, t.y >> 12);
        x = x + q * (t.y >> 20) + (t.y & 0xFFFu);
    }
}

// Encode n_c symbols starting at sym with N coders into the worst-case slot
// slot_base[0, slot_bytes).  Writes the chunk's first-word offset *wstart,
// byte size *size and final states states[0..N).  acc collects the table
// words of every symbol coded (kZeroFlag marks a symbol without probability).
// PREFETCH: load the next group's symbols while coding this one.  RAW: a
// bypass chunk, raw[i] is the raw word of symbol i (used where the symbol
// carries one); groups are halved so that a group still writes at most 1 KiB.
// BYTES: a byte-wise chunk (at most 2 bytes per symbol, size padded to 4).
// ADAPT: an adaptive chunk; ctx holds the chunk's words from adaptive_forward.
// WIDE: a wide model's 16-byte table entries (encode_step_wide).
// BINARY: a binary model whose symbols' entries are e0 and e1 (no table; acc
// then collects the symbols themselves).
// LAT (plain chunks of 32 coders with PREFETCH): the form for warps whose
// chain of dependent steps sets the pace, on an SM with few of them: each
// step's table entry is loaded during the step before, and the new state is
// computed ahead of the ballot and the word's store, which are deferred to
// the next step.  Measured on B300, against the form below (before the
// deferral; with it one 1 MiB chunk takes 1211 us): one 1 MiB chunk 1991 -> 1347 us,
// 592 chunks of 64 Ki symbols 190.6 -> 156.5 us, but one wave (3552 chunks)
// 319.0 -> 327.2 us and 1 GiB 1236 -> 1283 us; with the deferral it is the
// faster form up to 4736 chunks (the launcher's choice: rans_encode.cu
// kLatMaxChunks).  Either form alone gains nothing (1 MiB
// chunk: 1985 -> 1948 us with the early table loads, 1988 -> 2000 us with
// the state first).
template <int NT, bool PREFETCH, bool RAW = false, bool BYTES = false, bool ADAPT = false,
          bool WIDE = false, bool ADAPTN = false, bool BINARY = false, bool LAT = false>
__device__ __forceinline__ void encode_chunk(const uint8_t *sym, uint32_t n_c, uint32_t N_rt,
                                             uint8_t *slot_base, uint32_t slot_bytes,
                                             uint32_t *wstart, uint32_t *size, uint32_t *states,
                                             uint32_t tab_s, uint32_t ring_s, uint32_t ge,
                                             uint32_t lane, uint32_t &acc,
                                             const uint16_t *raw = nullptr,
                                             const uint32_t *ctx = nullptr, uint2 e0 = {},
                                             uint2 e1 = {}) {
    static_assert(!((RAW || ADAPT || ADAPTN) && PREFETCH), "these chunks load each group up front");
    static_assert(!(BINARY && (RAW || BYTES || ADAPT || WIDE || ADAPTN || PREFETCH)),
                  "binary chunks are plain and load each group up front");
    static_assert(!LAT || (PREFETCH && NT == 32 && !RAW && !BYTES && !ADAPT && !WIDE && !ADAPTN),
                  "the latency form is for plain chunks of 32 coders");
    constexpr uint32_t kG = RAW ? kGroup / 2 : kGroup;
    const uint32_t N = NT ? NT : N_rt;
    const uint8_t *symp = sym + lane;
    const uint16_t *rawp = RAW ? raw + lane : nullptr;
    const uint32_t *ctxp = (ADAPT || ADAPTN) ? ctx + lane : nullptr;
    uint32_t x = BYTES ? kL8 : kL;
    uint32_t wp = slot_bytes;               // words occupy [wp, slot_bytes)
    uint32_t flushed = slot_bytes / kSeg;   // segments >= flushed are stored

    // Store every segment that lies entirely at or above wp.  The next group
    // writes into the segments holding wp-1 .. wp-1024, whose ring slots last
    // held segments at least five newer stores back.  wp and flushed are
    // warp-uniform; only lane 0 issues and waits.
    auto service = [&]() {
        // Checked builds: the words so far fit the slot (wp has not wrapped).
        RANS_CHECK(wp <= slot_bytes);
        const uint32_t done = (wp + kSeg - 1) / kSeg;
        if (flushed > done) {
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
                for (uint32_t sg = flushed; sg > done;) {
                    --sg;
                    if (RANS_CHECK(uint64_t(sg + 1) * kSeg <= slot_bytes))
                        bulk_s2g(slot_base + uint64_t(sg) * kSeg, ring_s + (sg % kNSeg) * kSeg,
                                 kSeg);
                    bulk_commit();
                }
                bulk_wait_read<5>();
            }
            __syncwarp();
            flushed = done;
        }
    };

    const uint32_t T_full = n_c / N, rem = n_c % N;
    const uint32_t top0 = ADAPT ? T_full / kGroup * (kGroup - 1) : 0u;  // see adaptive_ctx_stride
    const bool lane_on = lane < N;
    if (rem) {
        const bool act = lane < rem;
        const uint32_t s = act && !ADAPTN ? symp[uint64_t(T_full) * N] : 0u;
        if (ADAPTN) {
            const uint32_t w = act ? ctxp[uint64_t(T_full) * N] : 0u;
            encode_step_bf<false>(x, wp, act, w, ring_s, ge);
        } else if (ADAPT) {
            const uint32_t pw = act ? ctxp[uint64_t(T_full - top0) * N] : kAdaptP0;
            encode_step_adaptive<false>(x, wp, act, s, pw, ring_s, ge);
        } else if (RAW) {
            const uint32_t rw = act ? rawp[uint64_t(T_full) * N] : 0u;
            encode_step_raw<false>(x, wp, acc, act, s, rw, tab_s, ring_s, ge);
        } else {
            coded_step<false, BYTES, WIDE, kRing, BINARY>(x, wp, acc, act, s, tab_s, ring_s, ge, e0,
                                                             e1);
        }
    }
    int64_t t = int64_t(T_full) - 1;
    for (uint32_t r = T_full % kG; r > 0; --r, --t) {
        service();
        const uint32_t s = lane_on && !ADAPTN ? symp[uint64_t(t) * N] : 0u;
        if (ADAPTN) {
            const uint32_t w = lane_on ? ctxp[uint64_t(t) * N] : 0u;
            encode_step_bf<NT == 32>(x, wp, lane_on, w, ring_s, ge);
        } else if (ADAPT) {
            const uint32_t pw = lane_on ? ctxp[uint64_t(t - top0) * N] : kAdaptP0;
            encode_step_adaptive<NT == 32>(x, wp, lane_on, s, pw, ring_s, ge);
        } else if (RAW) {
            const uint32_t rw = lane_on ? rawp[uint64_t(t) * N] : 0u;
            encode_step_raw<NT == 32>(x, wp, acc, lane_on, s, rw, tab_s, ring_s, ge);
        } else {
            coded_step<NT == 32, BYTES, WIDE, kRing, BINARY>(x, wp, acc, lane_on, s, tab_s, ring_s,
                                                                  ge, e0, e1);
        }
    }
    if (ADAPTN) {
        // Groups of kGroup steps, each step's stored (B, f) word loaded up front.
        for (; t >= 0; t -= kGroup) {
            uint32_t cw[kGroup];
#pragma unroll
            for (uint32_t u = 0; u < kGroup; ++u) cw[u] = lane_on ? ctxp[uint64_t(t - u) * N] : 0u;
            service();
#pragma unroll
            for (uint32_t u = 0; u < kGroup; ++u)
                encode_step_bf<NT == 32>(x, wp, lane_on, cw[u], ring_s, ge);
        }
    } else if (ADAPT) {
        // Groups of kGroup steps coded from pass 1's words alone (the next
        // group's word loaded ahead): the contexts are re-run forwards from
        // the group's first step into registers, two per word, then the group
        // is coded backwards.
        uint32_t wn = 0;
        if (t >= 0 && lane_on) wn = ctxp[uint64_t((t + 1) / kGroup - 1) * N];
        for (; t >= 0; t -= kGroup) {
            const uint32_t w = wn;
            const int64_t tn = t - int64_t(kGroup);
            if (tn >= 0 && lane_on) wn = ctxp[uint64_t((tn + 1) / kGroup - 1) * N];
            service();
            const uint32_t bits = w >> 16;  // bit v: step t - (kGroup - 1) + v
            uint32_t pv[kGroup / 2];
            uint32_t pc = w & 0xFFFFu;
#pragma unroll
            for (uint32_t v = 0; v < kGroup; ++v) {
                if (v & 1u) pv[v >> 1] |= pc << 16;
                else pv[v >> 1] = pc;
                pc = adapt_ctx(pc, (bits >> v) & 1u);
            }
#pragma unroll
            for (uint32_t u = 0; u < kGroup; ++u) {  // step t - u
                const uint32_t v = kGroup - 1 - u;
                encode_step_adaptive<NT == 32>(x, wp, lane_on, (bits >> v) & 1u,
                                               (v & 1u) ? pv[v >> 1] >> 16 : pv[v >> 1] & 0xFFFFu,
                                               ring_s, ge);
            }
        }
    } else if (PREFETCH && (BYTES || WIDE || NT != 32)) {
        // Groups of kGroup steps, symbols of the next group loaded ahead and
        // copied over at the group's end (the two-set form below took more
        // registers here: byte-wise chunks and plain ones of fewer than 32
        // coders spilled at their 64, 13/14-bit ones went from 94 to 108 and
        // three CTAs per SM to two).
        // 13/14-bit models also ask L2 for the group after the next one, as
        // the two-set form below does (1 GiB 1565 -> 1536 us, 8192 chunks 881
        // -> 842 us); byte-wise chunks ran slower with it (2109 -> 2135 us).
        uint32_t cur[kGroup], nxt[kGroup];
        const int64_t pf_step = -int64_t(lane & (kGroup - 1));
        if (t >= 0) {
#pragma unroll
            for (uint32_t u = 0; u < kGroup; ++u) cur[u] = lane_on ? symp[uint64_t(t - u) * N] : 0u;
        }
        for (; t >= 0; t -= kGroup) {
            const int64_t tn = t - int64_t(kGroup);
            if constexpr (WIDE) {
                const int64_t tp = tn - int64_t(kGroup);
                if (tp >= int64_t(kGroup) - 1 && lane_on)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(
                        __cvta_generic_to_global(symp + uint64_t(tp + pf_step) * N)));
            }
#pragma unroll
            for (uint32_t u = 0; u < kGroup; ++u)
                nxt[u] = (tn >= 0 && lane_on) ? symp[uint64_t(tn - u) * N] : 0u;
            service();
#pragma unroll
            for (uint32_t u = 0; u < kGroup; ++u)
                coded_step<NT == 32, BYTES, WIDE>(x, wp, acc, lane_on, cur[u], tab_s, ring_s, ge);
#pragma unroll
            for (uint32_t u = 0; u < kGroup; ++u) cur[u] = nxt[u];
        }
    } else if (PREFETCH) {
        // Groups of kGroup steps, symbols of the next group loaded ahead
        // into the other of two register sets (no copy between groups; the
        // loads of a group guarded once; measured on B300, 1 GiB: 1284 ->
        // 1246 us).  Outside the latency form, the group after the one
        // loaded is asked into L2 as well, lane j the line of its step
        // j mod 16 (the group's 512 bytes are four 128-byte lines): 1 GiB
        // 1234 -> 1200 us, 8192 chunks 679 -> 647 us; the latency form runs
        // no faster with it.
        uint32_t sa[kGroup], sb[kGroup];
        const int64_t pf_step = -int64_t(lane & (kGroup - 1));
        auto load = [&](uint32_t(&d)[kGroup], int64_t tg) {
            if (tg < 0) return;  // no group left to load
            if constexpr (!LAT) {
                const int64_t tn = tg - int64_t(kGroup);
                if (tn >= int64_t(kGroup) - 1)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(
                        __cvta_generic_to_global(symp + uint64_t(tn + pf_step) * N)));
            }
#pragma unroll
            for (uint32_t u = 0; u < kGroup; ++u)
                d[u] = (NT == 32 || lane_on) ? symp[uint64_t(tg - u) * N] : 0u;
        };
        auto code = [&](const uint32_t(&c)[kGroup]) {
            service();
            if constexpr (LAT) {
                // Each step's ballot and word store are deferred to the next
                // step and written between its own state-update operations,
                // so that the two dependent chains overlap in the warp's
                // in-order issue (the same stores in the same order; one
                // 1 MiB chunk 1353 -> 1211 us).
                uint2 tn = ld_enc_table(tab_s + (c[0] << 3));
                bool pe = false;     // the previous step emits a word
                uint32_t pw = 0u;    // its state, whose low 16 bits are the word
#pragma unroll
                for (uint32_t u = 0; u < kGroup; ++u) {
                    const uint2 t = tn;
                    if (u + 1 < kGroup) tn = ld_enc_table(tab_s + (c[u + 1] << 3));
                    acc |= t.y;
                    const bool emit = x > ~(t.y & 0xFFF00000u);
                    const uint32_t mp = __ballot_sync(kFull, pe);
                    const uint32_t xs = emit ? x >> 16 : x;
                    const uint32_t kp = __popc(mp & ge);
                    const uint32_t q = div_reciprocal(xs, t.x, t.y >> 12);  // floor(x / f_s)
                    st_ring_u16_if(pe, store_at<kRing>(wp, kp, ring_s), pw);
                    const uint32_t xn = xs + q * (t.y >> 20) + (t.y & 0xFFFu);
                    wp -= 2u * __popc(mp);
                    pe = emit;
                    pw = x;
                    x = xn;
                }
                const uint32_t mp = __ballot_sync(kFull, pe);
                st_ring_u16_if(pe, store_at<kRing>(wp, __popc(mp & ge), ring_s), pw);
                wp -= 2u * __popc(mp);
            } else {
#pragma unroll
                for (uint32_t u = 0; u < kGroup; ++u)
                    coded_step<NT == 32, BYTES, WIDE>(x, wp, acc, lane_on, c[u], tab_s, ring_s, ge);
            }
        };
        load(sa, t);
        while (t >= 0) {
            load(sb, t - int64_t(kGroup));
            code(sa);
            t -= kGroup;
            if (t < 0) break;
            load(sa, t - int64_t(kGroup));
            code(sb);
            t -= kGroup;
        }
    } else {
        // Groups of kG steps; a group's symbols are loaded together up front,
        // after lanes 0.. have asked L2 for the symbols of the group two
        // ahead (at most 32 * kG bytes: four 128-byte lines), which no
        // register holds meanwhile (measured on B300: 3000-stream batched
        // encode 6.74 -> 6.52 ms, the binary workload 383 -> 377 us).
        for (; t >= 0; t -= kG) {
            uint32_t cur[kG], curw[kG];
            {
                const int64_t tn = t - int64_t(2 * kG);  // last step of the group two ahead
                if (tn >= int64_t(kG) - 1 && lane < (kG * N + 127) / 128) {
                    const uint8_t *a = sym + uint64_t(tn - (kG - 1)) * N + 128u * lane;
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(__cvta_generic_to_global(a)));
                }
            }
#pragma unroll
            for (uint32_t u = 0; u < kG; ++u) {
                cur[u] = lane_on ? symp[uint64_t(t - u) * N] : 0u;
                if (RAW) curw[u] = lane_on ? rawp[uint64_t(t - u) * N] : 0u;
            }
            service();
            if (!RAW && !BYTES && group_is_linear(wp)) {
                const uint32_t a0 = ring_s + (wp & (kRing - 1));
                uint32_t wa = a0;
#pragma unroll
                for (uint32_t u = 0; u < kG; ++u)
                    coded_step<NT == 32, BYTES, WIDE, (RAW || BYTES ? kRing : 0u), BINARY>(
                        x, wa, acc, lane_on, cur[u], tab_s, ring_s, ge, e0, e1);
                wp -= a0 - wa;
            } else {
#pragma unroll
                for (uint32_t u = 0; u < kG; ++u) {
                    if (RAW)
                        encode_step_raw<NT == 32>(x, wp, acc, lane_on, cur[u], curw[u], tab_s,
                                                  ring_s, ge);
                    else
                        coded_step<NT == 32, BYTES, WIDE, kRing, BINARY>(
                            x, wp, acc, lane_on, cur[u], tab_s, ring_s, ge, e0, e1);
                }
            }
        }
    }

    // Store what is left: complete segments, then the partial one rounded
    // down to 16 bytes (bytes below wp are scratch garbage nobody reads).
    fence_proxy_async_smem();
    __syncwarp();
    if (lane == 0) {
        const uint32_t done = (wp + kSeg - 1) / kSeg;
        for (uint32_t sg = flushed; sg > done;) {
            --sg;
            if (RANS_CHECK(uint64_t(sg + 1) * kSeg <= slot_bytes))
                bulk_s2g(slot_base + uint64_t(sg) * kSeg, ring_s + (sg % kNSeg) * kSeg, kSeg);
        }
        const uint32_t lo = wp & ~15u, hi = done * kSeg;
        if (lo < hi && RANS_CHECK(wp <= slot_bytes && hi <= slot_bytes))
            bulk_s2g(slot_base + lo, ring_s + (lo & (kRing - 1)), hi - lo);
        bulk_commit();
        bulk_wait_read<0>();
        *wstart = wp;
        *size = BYTES ? (4 * N + (slot_bytes - wp) + 3) & ~3u : 4 * N + (slot_bytes - wp);
    }
    __syncwarp();
    if (lane < N) states[lane] = x;
}

// With a whole CTA (blockDim.x a multiple of 32): offsets of chunks
// [c_begin, c_end) = carry + the exclusive prefix of their sizes, written to
// offs_a[c] and, if not null, offs_b[c].  Returns (to every thread) carry +
// the sizes' total.  warp_sums: 32 words of shared memory, carry_s: one.
__device__ __forceinline__ uint64_t scan_sizes(const uint32_t *sizes, uint32_t c_begin,
                                               uint32_t c_end, uint64_t carry, uint32_t *offs_a,
                                               uint32_t *offs_b, uint32_t *warp_sums,
                                               uint64_t *carry_s) {
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nt = blockDim.x;
    if (tid == 0) *carry_s = carry;
    __syncthreads();
    for (uint64_t base = c_begin; base < c_end; base += nt) {
        const uint64_t i = base + tid;
        const uint32_t v = i < c_end ? sizes[i] : 0u;
        uint32_t incl = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, incl, d);
            if (lane >= uint32_t(d)) incl += y;
        }
        if (lane == 31) warp_sums[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const uint32_t w = lane < nt / 32 ? warp_sums[lane] : 0u;
            uint32_t wi = w;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(kFull, wi, d);
                if (lane >= uint32_t(d)) wi += y;
            }
            if (lane < nt / 32) warp_sums[lane] = wi - w;  // exclusive prefix of warp totals
        }
        __syncthreads();
        const uint64_t c0 = *carry_s;
        if (i < c_end) {
            const uint32_t o = uint32_t(c0 + warp_sums[warp] + incl - v);
            offs_a[i] = o;
            if (offs_b) offs_b[i] = o;
        }
        __syncthreads();
        if (tid == nt - 1) *carry_s = c0 + warp_sums[warp] + incl;
        __syncthreads();
    }
    return *carry_s;
}

// One thread: the header, the offset table's last entry (total data bytes),
// the zero padding before and after the data region, and the message size.
__device__ __forceinline__ void write_header(uint8_t *out, uint64_t *out_size, uint64_t n_sym,
                                             uint32_t N, uint32_t CS, uint32_t n_chunks,
                                             uint32_t data0, uint32_t total, uint32_t version,
                                             uint32_t log2m = kLog2M) {
    uint32_t *h = reinterpret_cast<uint32_t *>(out);
    h[0] = RANS_MAGIC;
    h[1] = version;
    h[2] = N;
    h[3] = log2m;
    h[4] = uint32_t(n_sym);
    h[5] = uint32_t(n_sym >> 32);
    h[6] = CS;
    h[7] = n_chunks;
    reinterpret_cast<uint32_t *>(out + 32)[n_chunks] = total;
    for (uint32_t b = 32 + 4 * (n_chunks + 1); b < data0; ++b) out[b] = 0;
    const uint64_t end = uint64_t(data0) + total;
    for (uint64_t b = end; b < round16(end); ++b) out[b] = 0;
    *out_size = round16(end);
}

// With a whole CTA: exclusive scan of the chunk sizes into the offset table,
// the header, zero padding, and the message size.  blockDim.x is a multiple
// of 32; warp_sums: 32 words of shared memory, carry: one.
__device__ __forceinline__ void finalize_message(uint8_t *out, uint64_t *out_size,
                                                 const uint32_t *sizes, uint64_t n_sym, uint32_t N,
                                                 uint32_t CS, uint32_t n_chunks, uint32_t data0,
                                                 uint32_t *warp_sums, uint64_t *carry_s,
                                                 uint32_t version = RANS_VERSION,
                                                 uint32_t log2m = kLog2M) {
    uint32_t *offs = reinterpret_cast<uint32_t *>(out + 32);
    const uint64_t total = scan_sizes(sizes, 0, n_chunks, 0, offs, nullptr, warp_sums, carry_s);
    if (threadIdx.x == 0)
        write_header(out, out_size, n_sym, N, CS, n_chunks, data0, uint32_t(total), version,
                     log2m);
}

// Copy chunk c (states, then words) to its place in the message.  The
// destination is only 2-byte aligned, so whole 16-byte destination blocks are
// assembled from two aligned 16-byte source loads and a funnel shift (the
// source-to-destination shift is the same for every block of a chunk); the
// partial blocks at both ends are written in 16-bit units.  U blocks per
// thread are in flight.  L2: source loads go through L2 only (ld.global.cg),
// for words that arrived there by bulk copies in the same launch.
template <bool L2>
__device__ __forceinline__ uint4 ld_src16(const uint8_t *p) {
    return L2 ? __ldcg(reinterpret_cast<const uint4 *>(p)) : *reinterpret_cast<const uint4 *>(p);
}
template <bool L2>
__device__ __forceinline__ uint16_t ld_src2(const uint8_t *p) {
    return L2 ? __ldcg(reinterpret_cast<const unsigned short *>(p))
              : *reinterpret_cast<const uint16_t *>(p);
}
template <bool L2>
__device__ __forceinline__ uint8_t ld_src1(const uint8_t *p) {
    return L2 ? uint8_t(__ldcg(reinterpret_cast<const unsigned char *>(p))) : *p;
}

template <int K, int U, bool L2>  // K = (source shift in bytes) / 4; rs = 8 * (shift mod 4)
__device__ __forceinline__ void pack_blocks(uint8_t *out, const uint8_t *src, uint64_t B0,
                                            uint64_t B1, uint64_t s_minus_d, uint32_t rs,
                                            uint32_t t, uint32_t nt) {
    const bool need_hi = K > 0 || rs != 0;
    const uint64_t stride = 16ull * nt;
    for (uint64_t B = B0 + 16ull * t; B < B1; B += U * stride) {
        uint4 v[U][2];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t Bu = B + u * stride;
            const uint64_t sa = (Bu + s_minus_d) & ~uint64_t(15);
            v[u][0] = v[u][1] = make_uint4(0u, 0u, 0u, 0u);
            if (Bu < B1) {
                v[u][0] = ld_src16<L2>(src + sa);
                if (need_hi) v[u][1] = ld_src16<L2>(src + sa + 16);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t Bu = B + u * stride;
            if (Bu >= B1) break;
            const uint32_t w[8] = {v[u][0].x, v[u][0].y, v[u][0].z, v[u][0].w,
                                   v[u][1].x, v[u][1].y, v[u][1].z, v[u][1].w};
            uint4 r;
            r.x = __funnelshift_r(w[K + 0], w[K + 1], rs);
            r.y = __funnelshift_r(w[K + 1], w[K + 2], rs);
            r.z = __funnelshift_r(w[K + 2], w[K + 3], rs);
            r.w = __funnelshift_r(w[K + 3], w[K + 4], rs);
            *reinterpret_cast<uint4 *>(out + Bu) = r;
        }
    }
}

// Threads t of nt: bytes s0 .. s0+len of words (16-byte aligned base) to
// out + d0.  d0 and s0 are even and len is even, except with BYTES (any
// byte).  U: 16-byte blocks in flight per thread; L2: loads through L2 only
// (ld_src16).  words must have 16 readable bytes past s0 + len.
template <bool BYTES, int U, bool L2>
__device__ __forceinline__ void copy_bytes(uint8_t *out, uint64_t d0, const uint8_t *words,
                                           uint64_t s0, uint64_t len, uint32_t t, uint32_t nt) {
    const uint64_t d1 = d0 + len;
    const uint64_t B0 = round16(d0), B1 = d1 & ~uint64_t(15);
    const uint64_t head_end = B0 < d1 ? B0 : d1;
    if (BYTES) {
        for (uint64_t b = d0 + t; b < head_end; b += nt) out[b] = ld_src1<L2>(words + s0 + (b - d0));
    } else {
        for (uint64_t b = d0 + 2ull * t; b < head_end; b += 2ull * nt)
            *reinterpret_cast<uint16_t *>(out + b) = ld_src2<L2>(words + s0 + (b - d0));
    }
    if (B0 < B1) {
        const uint64_t s_minus_d = s0 - d0;  // modulo 2^64
        const uint32_t sh = uint32_t(s_minus_d & 15u);
        const uint32_t rs = 8u * (sh & 3u);
        switch (sh >> 2) {
            case 0: pack_blocks<0, U, L2>(out, words, B0, B1, s_minus_d, rs, t, nt); break;
            case 1: pack_blocks<1, U, L2>(out, words, B0, B1, s_minus_d, rs, t, nt); break;
            case 2: pack_blocks<2, U, L2>(out, words, B0, B1, s_minus_d, rs, t, nt); break;
            default: pack_blocks<3, U, L2>(out, words, B0, B1, s_minus_d, rs, t, nt); break;
        }
    }
    const uint64_t tail_start = B1 > head_end ? B1 : head_end;
    if (BYTES) {
        for (uint64_t b = tail_start + t; b < d1; b += nt) out[b] = ld_src1<L2>(words + s0 + (b - d0));
    } else {
        for (uint64_t b = tail_start + 2ull * t; b < d1; b += 2ull * nt)
            *reinterpret_cast<uint16_t *>(out + b) = ld_src2<L2>(words + s0 + (b - d0));
    }
}

// Threads t of nt: chunk c of a message from scratch (words base, states,
// wstart) into out at message byte D.  The words buffer must have 16
// readable bytes past its last slot.
// BYTES: the chunk's byte count may be odd and its start in the slot too;
// the chunk is padded with zeros to a multiple of 4 bytes.
template <bool BYTES, int U, bool L2>
__device__ __forceinline__ void pack_chunk_at(uint8_t *out, uint64_t D, const uint8_t *words,
                                              const uint32_t *states, const uint32_t *wstart,
                                              uint32_t N, uint32_t slot_bytes, uint32_t c,
                                              uint32_t t, uint32_t nt) {
    uint16_t *dst16 = reinterpret_cast<uint16_t *>(out + D);
    const uint32_t *st = states + uint64_t(c) * N;
    for (uint32_t i = t; i < 2 * N; i += nt) dst16[i] = uint16_t(st[i >> 1] >> ((i & 1) * 16));
    const uint32_t ws = wstart[c];
    const uint64_t d1 = D + 4ull * N + (slot_bytes - ws);
    copy_bytes<BYTES, U, L2>(out, D + 4ull * N, words, uint64_t(c) * slot_bytes + ws,
                             slot_bytes - ws, t, nt);
    if (BYTES) {
        const uint64_t end = D + ((d1 - D + 3) & ~uint64_t(3));
        for (uint64_t b = d1 + t; b < end; b += nt) out[b] = 0;
    }
}

// With a whole CTA: chunk c of a message (offset table already written in
// out, or offs_in) from scratch into out.
template <bool BYTES = false>
__device__ __forceinline__ void pack_chunk(uint8_t *out, uint32_t data0, const uint8_t *words,
                                           const uint32_t *states, const uint32_t *wstart,
                                           uint32_t N, uint32_t slot_bytes, uint32_t c,
                                           const uint32_t *offs_in = nullptr) {
    const uint32_t *offs = offs_in ? offs_in : reinterpret_cast<const uint32_t *>(out + 32);
    pack_chunk_at<BYTES, 1, false>(out, uint64_t(data0) + offs[c], words, states, wstart, N,
                                   slot_bytes, c, threadIdx.x, blockDim.x);
}

// ---- single-pass placement: decoupled look-back over the chunk sizes -------
// Order completed async-proxy (bulk copy) writes to global memory before the
// issuing thread's later generic-proxy accesses.
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}
// Publication between CTAs: release / acquire at GPU scope.
__device__ __forceinline__ void st_release_u64(uint64_t *p, uint64_t v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_acquire_u64(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// look[c] holds a flag in its top two bits and a byte count below them:
// kLookSize = chunk c's own size, kLookPrefix = the bytes of chunks 0..c
// (inclusive prefix), kLookFailed = a wait before it gave up; zero: nothing
// published yet.  glook[g] says the same of group g = chunks 32g .. 32g+31
// (kLookSize = the group's total once all its chunks are published,
// kLookPrefix = the bytes of chunks 0 .. 32g+31), and gacc[g] counts the
// group's published chunks (<< 40) and sums their sizes.  A look-back reads
// the chunks before c in its group, then whole groups: 32 groups (1024
// chunks) per round.
constexpr uint64_t kLookSize = 1ull << 62;
constexpr uint64_t kLookPrefix = 2ull << 62;
constexpr uint64_t kLookFailed = 3ull << 62;
constexpr uint64_t kLookValue = (1ull << 62) - 1;

struct LookBack {
    uint64_t *look, *glook, *gacc;
    uint32_t n_chunks;
    uint64_t wait_ns;  // bound of the waits of one call
};

// One warp, once chunk c is in its slot: publishes its size, and its
// group's total if it is the group's last chunk to be published (group 0's
// total is its prefix too).  A group's total never replaces its prefix.
__device__ __forceinline__ void publish_size(const LookBack &lb, uint32_t c, uint32_t size,
                                             uint32_t lane) {
    if (lane != 0) return;
    st_release_u64(lb.look + c, (c == 0 ? kLookPrefix : kLookSize) | size);
    const uint32_t g = c / 32, members = min(32u, lb.n_chunks - 32 * g);
    const unsigned long long old =
        atomicAdd(reinterpret_cast<unsigned long long *>(lb.gacc + g), (1ull << 40) | size);
    if ((old >> 40) + 1 == members) {
        const uint64_t total = (old & ((1ull << 40) - 1)) + size;
        atomicCAS(reinterpret_cast<unsigned long long *>(lb.glook + g), 0ull,
                  (g == 0 ? kLookPrefix : kLookSize) | total);
    }
}

// One warp: chunk c will never be coded (its stream was rejected); chunks
// after it give up at once instead of waiting for it.
__device__ __forceinline__ void publish_failed(const LookBack &lb, uint32_t c, uint32_t lane) {
    if (lane == 0) st_release_u64(lb.look + c, kLookFailed);
}

// One round of a look-back: lane i reads entry q - i (own = the lane has an
// entry, else it contributes `none`), waiting for it until t0 + wait_ns.
// Adds the entries up to the nearest prefix to sum and sets `found` if there
// was one; false if an entry stayed unpublished or says failed.
__device__ __forceinline__ bool look_round(const uint64_t *q, bool own, uint64_t none, uint64_t t0,
                                           uint64_t wait_ns, uint32_t lane, uint64_t &sum,
                                           bool &found) {
    uint64_t v = none;
    if (own) {
        v = ld_acquire_u64(q - lane);
        for (uint32_t ns = 64; (v >> 62) == 0 && globaltimer_ns() - t0 <= wait_ns;) {
            __nanosleep(ns);
            ns = ns < 4096 ? 2 * ns : ns;
            v = ld_acquire_u64(q - lane);
        }
    }
    const uint64_t flag = v & ~kLookValue;
    if (__any_sync(kFull, flag == 0 || flag == kLookFailed)) return false;
    const uint32_t pref = __ballot_sync(kFull, flag == kLookPrefix);
    const uint32_t stop = pref ? __ffs(pref) - 1 : 31;  // the nearest prefix
    unsigned long long add = lane <= stop ? (v & kLookValue) : 0ull;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) add += __shfl_xor_sync(kFull, add, d);
    sum += add;
    found = pref != 0;
    return true;
}

// One warp: the bytes before chunk c (of `size` bytes, published), from the
// nearest published prefix, in `excl`; publishes c's prefix (and its
// group's, if c is the group's last chunk).  Waits for entries not yet
// published.  Chunks take their numbers from a counter in the order the
// warps start them, so every chunk (or group) waited for is being coded by
// running warps, which publish sizes before they wait for anything: each
// wait ends.  The waits of a call share the deadline now + wait_ns; false if
// it passed or a chunk before gave up (look[c] then says failed).
__device__ __forceinline__ bool chunk_offset(const LookBack &lb, uint32_t c, uint32_t size,
                                             uint32_t lane, uint64_t &excl) {
    excl = 0;
    if (c == 0) return true;
    const uint64_t t0 = globaltimer_ns();
    const uint32_t g = c / 32, i = c % 32;
    uint64_t sum = 0;
    bool found = false;
    // The chunks before c in its group (lanes at or past i add nothing).
    bool ok = look_round(lb.look + (c - 1), lane < i, kLookSize, t0, lb.wait_ns, lane, sum, found);
    // Then whole groups, nearest first (before group 0: the message start).
    for (uint32_t j = g; ok && !found; j -= 32)
        ok = look_round(lb.glook + (int64_t(j) - 1), j >= 1 + lane, kLookPrefix, t0, lb.wait_ns,
                        lane, sum, found);
    if (!ok) {
        if (lane == 0) st_release_u64(lb.look + c, kLookFailed);
        return false;
    }
    excl = sum;
    if (lane == 0) {
        st_release_u64(lb.look + c, kLookPrefix | (sum + size));
        if (i == 31 || c + 1 == lb.n_chunks) st_release_u64(lb.glook + g, kLookPrefix | (sum + size));
    }
    return true;
}

// A message whose coder warps place its chunks themselves.
struct Placement {
    uint8_t *out;
    uint64_t *out_size;
    uint32_t *status;
    const uint8_t *words;      // the chunk slots
    const uint32_t *states;    // N final states per chunk
    const uint32_t *wstart;    // first word byte of each slot
    const uint32_t *sizes;     // chunk bytes
    LookBack lb;               // look-back words, n_chunks, wait bound
    uint64_t n_sym;
    uint32_t N, CS, data0, slot_bytes, version, log2m;
};

// Chunk c is coded (its slot, state, start and size written by this warp):
// wait until the slot's bulk stores have completed, report a symbol without
// probability (acc), publish the chunk's size.
__device__ __forceinline__ void chunk_coded(const Placement &m, uint32_t c, uint32_t lane,
                                            uint32_t acc) {
    if (lane == 0) {
        bulk_wait<0>();
        fence_proxy_async_global();
    }
    __syncwarp();
    if (__any_sync(kFull, acc & kZeroFlag) && lane == 0) report(m.status, RANS_ERR_ZERO_FREQ);
    publish_size(m.lb, c, m.sizes[c], lane);
}

// Place coded chunk c: its offset by look-back, the offset table entry, the
// chunk copied to its place, and -- for the message's last chunk -- the
// header, the last offset, the padding and the message size.  U: 16-byte
// blocks each lane copies at a time.
template <bool BYTES, int U>
__device__ __forceinline__ void place_chunk(const Placement &m, uint32_t c, uint32_t lane) {
    const uint32_t size = m.sizes[c];
    uint64_t excl;
    if (!chunk_offset(m.lb, c, size, lane, excl)) {
        if (lane == 0) report(m.status, RANS_ERR_TIMEOUT);
        return;
    }
    if (lane == 0) reinterpret_cast<uint32_t *>(m.out + 32)[c] = uint32_t(excl);
    pack_chunk_at<BYTES, U, true>(m.out, uint64_t(m.data0) + excl, m.words, m.states, m.wstart,
                                  m.N, m.slot_bytes, c, lane, 32);
    if (c + 1 == m.lb.n_chunks && lane == 0)
        write_header(m.out, m.out_size, m.n_sym, m.N, m.CS, m.lb.n_chunks, m.data0,
                     uint32_t(excl + size), m.version, m.log2m);
}

// The look-back words of a message's scratch (zeroed before its launch).
__host__ __device__ inline LookBack scratch_lookback(uint8_t *scr, const ScratchLayout &sl,
                                                     uint32_t n_chunks, uint32_t CS, uint32_t N) {
    LookBack lb;
    lb.look = reinterpret_cast<uint64_t *>(scr + sl.look);
    lb.glook = reinterpret_cast<uint64_t *>(scr + sl.glook);
    lb.gacc = reinterpret_cast<uint64_t *>(scr + sl.gacc);
    lb.n_chunks = n_chunks;
    // Every wait ends once the chunks started before it are coded: allow a
    // second plus a microsecond per step of a chunk (several times the
    // coding time of one chunk on a loaded GPU).
    lb.wait_ns = 1000000000ull + 1000ull * (CS / N + 1);
    return lb;
}

}  // namespace enc
}  // namespace rans
