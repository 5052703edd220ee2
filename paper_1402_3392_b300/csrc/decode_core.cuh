// decode_core.cuh -- the decoder's building blocks, shared by the single-message
// kernel (rans_decode.cu) and the batched persistent kernel (rans_batch.cu).
//
// A warp decodes one chunk, or two chunks side by side; lane j is coder j of
// each chunk's N interleaved rANS coders.  Per step every lane decodes one
// symbol of each chunk (Algorithm 1 Decode, Section 2):
//     slot = x mod M;  (s, f_s, slot - B_s) from a slot table in shared memory
//     x    = f_s * floor(x / M) + slot - B_s
// and then renormalizes at most once (b = 2^16 >= M, Section 5): the lanes
// with x < L form renorm_mask = ballot(x < L); a lane reads the word at
// read_pos + popc(renorm_mask & lanes_below_me) and read_pos advances by
// popc(renorm_mask) -- the packed load of Section 6.  Two chunks' state
// chains are independent, so their steps overlap in one instruction stream.
//
// Each chunk's compressed words stream into a shared-memory ring through
// bulk copies (TMA, cp.async.bulk) completed on mbarriers; decoded bytes go
// out as one coalesced 32-byte store per chunk and step.
#pragma once

#include <cstdint>
#include <type_traits>

#include "adapt_model.cuh"
#include "device_util.cuh"
#include "host_util.h"

namespace rans {
namespace dec {

constexpr int kWarps = 8;                 // warps per CTA (the default shape)
constexpr uint32_t kThreads = kWarps * 32;
constexpr uint32_t kBuildThreads = 256;   // threads that build a table: one per symbol
static_assert(kThreads >= kBuildThreads, "a table build needs 256 threads");
constexpr uint32_t kChains = 2;           // chunks a warp decodes side by side
constexpr uint32_t kChunksPerCta = kWarps * kChains;
constexpr uint32_t kWarpRing = 4096;      // ring bytes per warp (4 KiB aligned)
constexpr uint32_t kNSeg = 4;             // ring segments (and mbarriers) per chunk

// Ring geometry of one chunk in flight: a ring of NSEG segments of SEG bytes,
// checked every GROUP steps.  A step reads at most STEP bytes (32 words = 64
// bytes; 128 with raw words, two words per lane), so a group reads at most
// GROUP * STEP bytes.  Ring event k (due once the read position rp reaches
// (k - NSEG + 1) * SEG) issues the copy of segment k into the slot that
// segment k - NSEG has left, and waits for segment k - LAG.  After the events
// due at rp, the segments up to floor(rp / SEG) + NSEG - 1 - LAG are in:
// enough for the next group when LAG <= NSEG - 1 - ceil(GROUP * STEP / SEG).
// A copy is waited for LAG segments (LAG * SEG bytes of words) after it is
// issued.
template <uint32_t SEG, uint32_t NSEG, uint32_t GROUP, uint32_t STEP = 64>
struct Geometry {
    static constexpr uint32_t kSeg = SEG;
    static constexpr uint32_t kNSeg = NSEG;
    static constexpr uint32_t kRing = SEG * NSEG;
    static constexpr uint32_t kGroup = GROUP;
    static constexpr uint32_t kStep = STEP;
    static constexpr uint32_t kLag = NSEG - 1 - (GROUP * STEP + SEG - 1) / SEG;
    static_assert((kRing & (kRing - 1)) == 0, "the ring is indexed by masking");
    static_assert(NSEG - 1 >= (GROUP * STEP + SEG - 1) / SEG + 1, "a copy must be issued ahead of use");
    static_assert(NSEG <= 32, "one phase bit per segment");
};
// One chunk per warp: the warp's whole 4 KiB as one ring, 1 KiB copies,
// waited 2 KiB after issue.  Two chunks per warp: 2 KiB each, 512-byte
// copies, waited 512 bytes after issue.  Copies are large because each one
// costs the warp an issue, a wait and bookkeeping.  With raw words (bypass
// messages, one chunk per warp): 1 KiB copies waited 1 KiB after issue.
using GeoOne = Geometry<1024, kNSeg, 16>;
// 32-step groups (half the ring-event checks and branches a step) for the
// 12-warp kernel's plain chunks, where the SM is full, for the early-word
// step and for 13/14-bit chunks.  Measured on B300: 1
// GiB 851 -> 840 us, 10656 chunks 546 -> 538 us; the byte-wise and binary
// steps spill with them (byte-wise 1 GiB 1288 -> 1298 us), and 8-warp CTAs
// under a wave gain nothing (4000 chunks 243 -> 248 us).
using GeoOneLong = Geometry<1024, kNSeg, 32>;
using GeoPair = Geometry<512, kNSeg, 16>;
using GeoRaw = Geometry<1024, kNSeg, 16, 128>;
// Prefix messages read up to one 32-bit word per lane and step: as GeoRaw.
using GeoPrefix = Geometry<1024, kNSeg, 16, 128>;
// The entry-ahead step (kKindPlainSpec) reads 64 bytes a step but converts
// the words up to 2 KiB past rp before every group: with 128 counted per
// step a copy is waited one segment after its issue, which keeps
// [rp, rp + 2 KiB) in after the events due at rp.
using GeoSpec = Geometry<1024, kNSeg, 16, 128>;
static_assert(GeoSpec::kLag == 1 && GeoSpec::kSeg * (GeoSpec::kNSeg - 1 - GeoSpec::kLag) >= 2048,
              "the entry-ahead step converts 2 KiB of resident words ahead");
static_assert(GeoOne::kRing == kWarpRing && GeoOneLong::kRing == kWarpRing &&
                  GeoPair::kRing * kChains == kWarpRing &&
                  GeoRaw::kRing == kWarpRing,
              "ring sizes");

constexpr uint32_t kTableBytes = kM * 4;
// Shared memory of a CTA of W warps: [slot table 16 KiB][alignment slack 4
// KiB][4 KiB ring per warp][kNSeg mbarriers per chunk slot][a few words of
// CTA state][256 raw-word flags][256 (B, f) words].
//
// Two CTA shapes.  W = 8 with 4 CTAs per SM (32 warps, 64 registers a
// thread) is the default.  W = 12 with 3 CTAs per SM (36 warps, at most 56
// registers) lets each 16 KiB slot table serve 12 rings; it is used where a
// warp decodes one chunk of a plain or byte-wise message.  Measured on B300
// with the same message decoded by both shapes: 1 GiB plain 889 -> 866 us,
// byte-wise 788 -> 832 GB/s; chunk pairs, bypass, adaptive and prefix
// chunks are slower with 12 (batched decode 1325 -> 1254 GB/s).
template <int W>
struct Shape {
    static constexpr int kWarps = W;
    static constexpr uint32_t kThreads = W * 32;
    static constexpr int kCtasPerSm = W == 12 ? 3 : 4;
    static constexpr uint32_t kChunksPerCta = W * kChains;
    static constexpr uint32_t kBarOffset = kTableBytes + kWarpRing + W * kWarpRing;
    static constexpr uint32_t kMiscOffset = kBarOffset + kChunksPerCta * kNSeg * 8;
    static constexpr uint32_t kFlagsOffset = kMiscOffset + 64;  // 256 raw-word flags (bypass)
    static constexpr uint32_t kFbOffset = kFlagsOffset + 256;   // 256 words B << 16 | f (wide)
    static constexpr uint32_t kSmemBytes = kFbOffset + 1024;
    static_assert(W == 8 || W == 12, "the two measured shapes");
    static_assert(kThreads >= kBuildThreads, "a table build needs 256 threads");
    static_assert(kCtasPerSm * (kSmemBytes + 1024) <= 233472, "CTAs per SM fit in shared memory");
};
constexpr int kWarpsOne = 12;  // the shape for one plain or byte-wise chunk per warp
constexpr uint32_t kBarOffset = Shape<kWarps>::kBarOffset;
constexpr uint32_t kMiscOffset = Shape<kWarps>::kMiscOffset;
constexpr uint32_t kFlagsOffset = Shape<kWarps>::kFlagsOffset;
constexpr uint32_t kFbOffset = Shape<kWarps>::kFbOffset;
constexpr uint32_t kSmemBytes = Shape<kWarps>::kSmemBytes;
constexpr uint32_t kNoConst = 0xFFFFFFFFu;
// Byte-wise messages (version 3): L = 2^23, b = 2^8, I = [2^23, 2^31).
constexpr uint32_t kL8 = 1u << 23;
// Message kinds: plain (version 1), bypass (2: raw words after symbols),
// byte-wise (3: b = 2^8, digits breadth-first), adaptive (4: binary symbols,
// one adaptive context per coder), prefix (5: canonical prefix codes muxed in
// their decoder's read order, Section 4).
constexpr int kKindPlain = 0, kKindRaw = 1, kKindBytes = 2, kKindAdaptive = 3, kKindPrefix = 4;
// Plain messages at 13 or 14 bits of probability resolution (M = 2^13 or
// 2^14, b = 2^16 >= M: still one renormalization per symbol, Section 5).
// Their model takes a slot -> symbol byte table (M bytes, in the table area)
// and a symbol -> (B_s << 16 | f_s) table of 256 words.
constexpr int kKindWide13 = 5, kKindWide14 = 6;
// Plain messages whose model has two symbols, 0 and 1, both with f > 0 (a
// binary model, rABS in the paper's terms, Section 2): D needs no table.
// The same bitstream as kKindPlain; only the decoder's step differs.
constexpr int kKindBinary = 7;
// Adaptive models over n symbols, one per coder (version 6, adapt_model.cuh),
// with register room for 3, 7 or 15 boundaries (n <= 4, 8, 16).
constexpr int kKindAdaptN4 = 8, kKindAdaptN8 = 9, kKindAdaptN16 = 10;
// Plain messages decoded with the step's word taken early (decode_step's
// EARLY form): the plain bitstream, for messages under one wave of chunks,
// where a warp's chain of dependent steps, not the SM's pipes, sets the pace.
constexpr int kKindPlainEarly = 11;
// Plain messages decoded with the next step's table entry taken early
// (decode_step_spec): the plain bitstream, for messages of at most two chunks
// per SM, where a single warp's chain of dependent steps is all that sets
// the pace.  Beside its word ring each warp keeps an entry ring: for every
// word of the stream ahead, the slot-table entry of the state that word
// would complete (its slot is the word's low 12 bits), kERing bytes (1024
// entries, so 2 KiB of stream positions) per warp.
constexpr int kKindPlainSpec = 12;
constexpr uint32_t kERing = 4096;
// Byte-wise messages decoded with both digit passes issued together
// (decode_step_bytes's PAR form): the byte-wise bitstream, for messages of
// few chunks, where a warp's chain of dependent steps sets the pace.
constexpr int kKindBytesLat = 13;
template <int KIND>
struct AdaptN {
    static constexpr bool kOn = KIND == kKindAdaptN4 || KIND == kKindAdaptN8 || KIND == kKindAdaptN16;
    static constexpr int kNB = KIND == kKindAdaptN4 ? 3 : KIND == kKindAdaptN8 ? 7 : 15;
};
template <int KIND>
struct WideBits {
    static constexpr uint32_t kLog2 = KIND == kKindWide13 ? 13u : 14u;
};
// Prefix messages: longest code, also the bit count below which a coder's
// decoder reads its next 32-bit word; entries of the 4096-entry code table
// are len << 8 | symbol.  Bits that start no code get length 63: a coder
// holds at most 43 bits, so using such an entry wraps its bit count, which
// then never comes back to 43 or below (refills stop) and the chunk's end
// check rejects it.
constexpr uint32_t kPrefixMaxLen = 12;
constexpr uint32_t kPrefixMaxHeld = 43;
constexpr uint32_t kPrefixNoCode = 63u << 8;
// Adaptive contexts: p = probability of a 0 scaled to M, from M/2, moving by
// (target - p) >> kAdaptRate after every symbol.
constexpr uint32_t kAdaptRate = 5;
constexpr uint32_t kAdaptP0 = kM / 2;

struct Smem {
    uint32_t *tab;
    uint32_t tab_s;
    uint32_t rings_s;   // kWarpRing aligned
    uint8_t *rings;     // generic pointer of rings_s
    uint64_t *bars;
    uint32_t *misc;     // CTA-shared words
    uint8_t *flags;     // raw words per symbol (0 or 1), bypass messages
    uint32_t flags_s;
    uint32_t *fb;       // wide models: B_s << 16 | f_s per symbol
    uint32_t fb_s;
};

template <int W = kWarps>
__device__ __forceinline__ Smem smem_layout(uint8_t *smem) {
    using S = Shape<W>;
    Smem s;
    s.tab = reinterpret_cast<uint32_t *>(smem);
    s.tab_s = smem_addr(smem);
    const uint32_t raw = smem_addr(smem + kTableBytes);
    s.rings_s = (raw + kWarpRing - 1) & ~(kWarpRing - 1);
    s.rings = smem + kTableBytes + (s.rings_s - raw);
    s.bars = reinterpret_cast<uint64_t *>(smem + S::kBarOffset);
    s.misc = reinterpret_cast<uint32_t *>(smem + S::kMiscOffset);
    s.flags = smem + S::kFlagsOffset;
    s.flags_s = smem_addr(smem + S::kFlagsOffset);
    s.fb = reinterpret_cast<uint32_t *>(smem + S::kFbOffset);
    s.fb_s = smem_addr(smem + S::kFbOffset);
    return s;
}

// a * b + c.  The read-position updates and the table address are written
// this way rather than as shift-and-add: with this form the compiler emits
// fewer instructions for the decode step (measured: 20.9 instead of 22.9
// warp-instructions per step, 5-6 % less decode time).
__device__ __forceinline__ uint32_t imad(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t r;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
    return r;
}

// Slot table entry: f_s << 20 | (slot - B_s) << 8 | s   (f_s < M here).
// With E = entry >> 8 = f_s * 2^12 + (slot - B_s) the decode update is
//     f_s * floor(x/M) + slot - B_s = f_s * (floor(x/M) - 2^12) + E  (mod 2^32).
__device__ __forceinline__ uint32_t decode_update(uint32_t x, uint32_t e) {
    return (e >> 20) * ((x >> kLog2M) + (0u - (1u << kLog2M))) + (e >> 8);
}

// Shared-memory loads by 32-bit shared address.  The slot table does not
// change while a chunk is decoded; the ring is rewritten by TMA, so its loads
// stay ordered after the mbarrier waits (volatile).
__device__ __forceinline__ uint32_t ld_table(uint32_t a) {
    uint32_t v;
    asm("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ uint32_t ld_flag(uint32_t a) {
    uint32_t v;
    asm("ld.shared.u8 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ uint32_t ld_ring_u8(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.u8 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ uint32_t ld_ring_u16(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.u16 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ uint32_t ld_ring_u32(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}

// Build the 4096-entry slot table from 256 frequencies (zero for unused
// symbols) with the whole CTA (the first kBuildThreads threads fill the
// slots).  scratch: >= 5 KiB of shared memory not in use (the rings before
// any chunk is decoded).
// Returns (to every thread) the sum of the frequencies; *const_sym receives
// the symbol with f = M, or kNoConst.
//   cum[s] = f_0 + ... + f_{s-1}                       (warp scan)
//   mark[cum[s]] = s for every s with f_s > 0           (scatter)
//   sym(slot) = max of mark[0..slot]                    (max-scan: symbols
//               are laid out in increasing order)
template <int W = kWarps>
__device__ __noinline__ static uint32_t build_slot_table(const uint16_t *freq, uint32_t *tab, uint8_t *scratch,
                                     uint32_t *const_sym) {
    uint32_t *cum = reinterpret_cast<uint32_t *>(scratch);        // 257 words
    uint8_t *mark = scratch + 1040;                               // 4096 bytes
    uint32_t *part = reinterpret_cast<uint32_t *>(scratch + 1040 + kM);  // 8 words
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (uint32_t i = tid; i < kM / 4; i += Shape<W>::kThreads) reinterpret_cast<uint32_t *>(mark)[i] = 0;
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
    const uint32_t total = cum[256];
    if (total != kM) return total;  // not a valid model: the caller reports it
    if (tid < 256) {
        const uint32_t a = cum[tid], b = cum[tid + 1];
        if (b > a) mark[a] = uint8_t(tid);
        if (b - a == kM) *const_sym = tid;
    }
    __syncthreads();
    // the first kBuildThreads threads (8 warps, whole warps) x 16 slots each;
    // every thread reaches the barriers
    constexpr uint32_t kPer = kM / kBuildThreads;
    static_assert(kPer == 16, "16 slots a building thread");
    const bool builder = Shape<W>::kThreads == kBuildThreads || tid < kBuildThreads;
    const uint32_t base = tid * kPer;
    uint32_t mk[kPer];
    uint32_t incl = 0;
    if (builder) {
#pragma unroll
        for (uint32_t q = 0; q < kPer / 4; ++q) {
            const uint32_t w = reinterpret_cast<const uint32_t *>(mark + base)[q];
#pragma unroll
            for (uint32_t b = 0; b < 4; ++b) mk[4 * q + b] = (w >> (8 * b)) & 0xFFu;
        }
        uint32_t run = 0;
#pragma unroll
        for (uint32_t i = 0; i < kPer; ++i) {
            run = max(run, mk[i]);
            mk[i] = run;
        }
        // exclusive max-scan of the per-thread maxima across the builders
        incl = run;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, incl, d);
            if (lane >= uint32_t(d)) incl = max(incl, y);
        }
        if (lane == 31) part[warp] = incl;
    }
    __syncthreads();
    if (builder) {
        uint32_t carry = __shfl_up_sync(kFull, incl, 1);
        if (lane == 0) carry = 0;
        for (uint32_t w = 0; w < warp; ++w) carry = max(carry, part[w]);
#pragma unroll
        for (uint32_t i = 0; i < kPer; ++i) {
            const uint32_t s = max(carry, mk[i]);
            const uint32_t slot = base + i;
            const uint32_t f = cum[s + 1] - cum[s];
            tab[slot] = (f << 20) | ((slot - cum[s]) << 8) | s;
        }
    }
    __syncthreads();
    return total;
}

// The tables of a wide model (M = 2^lm, lm 13 or 14) from 256 frequencies,
// with the whole CTA: fb[s] = B_s << 16 | f_s, and the slot -> symbol byte
// table sym[0..M) (sym(slot) = the s with B_s <= slot < B_s + f_s).  As for
// the slot table: cum by a warp scan, each symbol's first slot marked with
// its index, then a running maximum over the slots (symbols lie in
// increasing order), each thread over M/256 consecutive slots after an
// exclusive max-scan of the threads' maxima.  scratch: >= 1.1 KiB of free
// shared memory.  Returns the frequencies' sum; *const_sym: the symbol with
// f = M, or kNoConst.
template <int W = kWarps>
__device__ __noinline__ static uint32_t build_wide_table(const uint16_t *freq, uint32_t lm,
                                                         uint8_t *sym, uint32_t *fb,
                                                         uint8_t *scratch, uint32_t *const_sym) {
    uint32_t *cum = reinterpret_cast<uint32_t *>(scratch);        // 257 words
    uint32_t *part = reinterpret_cast<uint32_t *>(scratch + 1040);  // 8 words
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, M = 1u << lm;
    uint32_t *sym32 = reinterpret_cast<uint32_t *>(sym);
    for (uint32_t i = tid; i < M / 4; i += Shape<W>::kThreads) sym32[i] = 0;
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
    const uint32_t total = cum[256];
    if (total != M) return total;  // not a valid model: the caller reports it
    if (tid < 256) {
        const uint32_t a = cum[tid], f = cum[tid + 1] - a;
        fb[tid] = (a << 16) | (f & 0xFFFFu);
        if (f > 0) sym[a] = uint8_t(tid);
        if (f == M) *const_sym = tid;
    }
    __syncthreads();
    // the first kBuildThreads threads (whole warps), 8 or 16 words each;
    // every thread reaches the barriers
    const bool builder = Shape<W>::kThreads == kBuildThreads || tid < kBuildThreads;
    const uint32_t words = M / 4 / kBuildThreads, base = tid * words;
    uint32_t incl = 0;
    if (builder) {
        uint32_t run = 0;
        for (uint32_t q = 0; q < words; ++q) {
            const uint32_t w = sym32[base + q];
            run = max(run, max(max(w & 0xFFu, (w >> 8) & 0xFFu), max((w >> 16) & 0xFFu, w >> 24)));
        }
        incl = run;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, incl, d);
            if (lane >= uint32_t(d)) incl = max(incl, y);
        }
        if (lane == 31) part[warp] = incl;
    }
    __syncthreads();
    if (builder) {
        uint32_t carry = __shfl_up_sync(kFull, incl, 1);
        if (lane == 0) carry = 0;
        for (uint32_t w = 0; w < warp; ++w) carry = max(carry, part[w]);
        for (uint32_t q = 0; q < words; ++q) {
            const uint32_t w = sym32[base + q];
            uint32_t out = 0;
#pragma unroll
            for (uint32_t b = 0; b < 4; ++b) {
                carry = max(carry, (w >> (8 * b)) & 0xFFu);
                out |= carry << (8 * b);
            }
            sym32[base + q] = out;
        }
    }
    __syncthreads();
    return total;
}

// The 4096-entry decode table of a canonical prefix code, with the whole CTA:
// the entries whose top len bits are symbol s's code hold len << 8 | s, the
// rest kPrefixNoCode.  len[s] = 0: s not in the code.
template <int W = kWarps>
__device__ __noinline__ static void build_prefix_table(const uint8_t *len, const uint16_t *code,
                                                       uint32_t *tab) {
    const uint32_t tid = threadIdx.x;
    for (uint32_t i = tid; i < kM / 4; i += Shape<W>::kThreads)
        reinterpret_cast<uint4 *>(tab)[i] =
            make_uint4(kPrefixNoCode, kPrefixNoCode, kPrefixNoCode, kPrefixNoCode);
    __syncthreads();
    for (uint32_t s = tid; s < RANS_MAX_ALPHABET; s += Shape<W>::kThreads) {
        const uint32_t l = len[s];
        if (l == 0 || l > kPrefixMaxLen) continue;
        const uint32_t first = uint32_t(code[s]) << (kPrefixMaxLen - l), n = 1u << (kPrefixMaxLen - l);
        const uint32_t e = (l << 8) | s;
        for (uint32_t k = 0; k < n; ++k) tab[first + k] = e;
    }
    __syncthreads();
}

// The ring and barriers of one chunk slot of a warp, carried across the
// chunks the warp decodes.  With one chunk per warp, slot 0's ring is the
// warp's whole 4 KiB.
struct ChainRing {
    uint32_t ring_s;    // shared address, aligned to the ring's size
    uint32_t bar0;      // its kNSeg mbarriers
    uint32_t phase;     // bit i: parity of the next wait on barrier i
};

struct WarpRings {
    ChainRing r[kChains];
    uint32_t timeouts;  // warp-uniform: a bounded wait gave up
};

__device__ __forceinline__ WarpRings rings_init(const Smem &sm, uint32_t warp, uint32_t lane) {
    WarpRings w;
#pragma unroll
    for (uint32_t k = 0; k < kChains; ++k) {
        const uint32_t i = warp * kChains + k;
        w.r[k].ring_s = sm.rings_s + warp * kWarpRing + k * GeoPair::kRing;
        w.r[k].bar0 = smem_addr(sm.bars + i * kNSeg);
        w.r[k].phase = 0;
    }
    w.timeouts = 0;
    if (lane == 0) {
        for (uint32_t i = 0; i < kChains * kNSeg; ++i)
            mbar_init(smem_addr(sm.bars + warp * kChains * kNSeg + i), 1);
        fence_mbar_init();
    }
    __syncwarp();
    return w;
}

// Decoding state of one chunk.  Byte positions in its word stream are taken
// relative to A, the 16-byte aligned message offset at or below the first
// word; stream byte P then lives at ring offset P mod (ring size).
struct Chain {
    const uint8_t *src;  // message + A: source of segment 0
    uint8_t *outp;       // where this lane's next symbol goes
    uint16_t *rawp;      // where its next raw word goes (bypass messages)
    uint32_t x;          // this lane's coder state
    uint32_t rp;         // read position (warp-uniform)
    uint32_t evt;        // ring events done
    uint32_t next_evt;   // rp at which event evt is due (~0: none left)
    uint32_t nseg;       // segments of the chunk
    uint32_t span;       // bytes copied in all (a multiple of 16)
    uint32_t endrel;     // end of the chunk's words
    uint32_t steps;      // full steps (all N coders) left
    uint32_t rem;        // coders with a symbol in the final partial step
    uint32_t st;         // RANS_OK, or the error found when opening
    uint32_t p;          // adaptive messages: this lane's context
    uint32_t rp0;        // byte-wise messages: rp at the first digit
    uint32_t len;        // byte-wise messages: chunk bytes (states, digits, padding)
    uint32_t bhi, blo;   // prefix messages: this lane's bits, right-aligned in bhi:blo
    uint32_t nb;         // prefix messages: bits held (at most 43 unless a code was missing)
    uint32_t cm[15];     // adaptive-n messages: this lane's model (adapt_model.cuh)
    uint32_t nm;         // adaptive-n messages: M - n
    uint32_t cv;         // entry-ahead step: entries hold for stream bytes below cv
};

__device__ __forceinline__ void chain_empty(Chain &c) {
    c.src = nullptr;
    c.outp = nullptr;
    c.rawp = nullptr;
    c.x = kL;
    c.rp = c.evt = c.nseg = c.span = c.endrel = c.steps = c.rem = 0;
    c.next_evt = 0xFFFFFFFFu;
    c.st = RANS_OK;
    c.rp0 = c.len = 0;
    c.p = kAdaptP0;
    c.bhi = c.blo = c.nb = 0;
    c.cv = 0;
}

// Open a prefix-message chunk [o, e): no states, its 32-bit words start at
// the chunk's first byte; offsets must be multiples of 4.
template <class G>
__device__ __forceinline__ void chain_open_prefix(Chain &c, const uint8_t *msg, uint32_t data0,
                                                  uint32_t o, uint32_t e, uint32_t data_end,
                                                  uint32_t n_c, uint32_t N, uint8_t *out,
                                                  uint32_t lane) {
    chain_empty(c);
    if (((o | e) & 3u) || e < o || e > data_end || e - o > 0xFFFFFF00u) {
        c.st = RANS_ERR_CORRUPT;
        return;
    }
    const uint64_t P0 = uint64_t(data0) + o, P1 = uint64_t(data0) + e;
    const uint64_t A = P0 & ~uint64_t(15);
    c.src = msg + A;
    c.span = uint32_t(round16(P1) - A);
    c.nseg = (c.span + G::kSeg - 1) / G::kSeg;
    c.endrel = uint32_t(P1 - A);
    c.rp = uint32_t(P0 - A);
    c.next_evt = 0;
    c.outp = out + lane;
    c.steps = n_c / N;
    c.rem = n_c % N;
}

// Open chunk [o, e) (byte offsets in the data region that starts at msg +
// data0; data_end = end of all chunks) of n_c symbols with N coders, output
// at out.  Reads the N initial states; a malformed chunk gets c.st set and no
// steps.  UNI: the read position passes through warp_uniform (the batched
// decoder's form).
template <class G, bool BYTES = false, bool UNI = false>
__device__ __forceinline__ void chain_open(Chain &c, const uint8_t *msg, uint32_t data0, uint32_t o,
                                           uint32_t e, uint32_t data_end, uint32_t n_c, uint32_t N,
                                           uint8_t *out, uint16_t *raw_out, uint32_t lane) {
    chain_empty(c);
    // Offsets must be even (states and words are 2-byte aligned) and in range.
    if (((o | e) & 1u) || e < o || e > data_end || e - o < 4 * N || e - o > 0xFFFFFF00u) {
        c.st = RANS_ERR_CORRUPT;
        return;
    }
    const uint8_t *chunk = msg + data0 + o;
    uint32_t x = BYTES ? kL8 : kL;
    if (lane < N) x = ld_u16_global(chunk + 4 * lane) | (ld_u16_global(chunk + 4 * lane + 2) << 16);
    // Algorithm 1 requires x in I
    if (!__all_sync(kFull, BYTES ? (x >= kL8 && x < (kL8 << 8)) : x >= kL)) {
        c.st = RANS_ERR_CORRUPT;
        return;
    }
    const uint64_t P0 = uint64_t(data0) + o + 4 * N, P1 = uint64_t(data0) + e;
    const uint64_t A = P0 & ~uint64_t(15);
    c.x = x;
    c.src = msg + A;
    c.span = uint32_t(round16(P1) - A);
    c.nseg = (c.span + G::kSeg - 1) / G::kSeg;
    c.endrel = uint32_t(P1 - A);
    c.rp = UNI ? warp_uniform(uint32_t(P0 - A)) : uint32_t(P0 - A);
    c.rp0 = c.rp;
    c.len = e - o;
    c.next_evt = 0;
    c.outp = out + lane;
    c.rawp = raw_out ? raw_out + lane : nullptr;
    c.steps = n_c / N;
    c.rem = n_c % N;
}

// Bounded wait for the copy into barrier slot `slot`, then flip its parity.
__device__ __forceinline__ void ring_wait(ChainRing &r, uint32_t slot, uint32_t &timeouts) {
    const bool ok = timeouts != 0 || mbar_wait_bounded(r.bar0 + 8 * slot, (r.phase >> slot) & 1u);
    if (__any_sync(kFull, !ok)) timeouts = 1;  // warp-uniform
    r.phase ^= 1u << slot;
}

// Ring event c.evt: issue the copy of segment evt (its slot's previous
// segment lies wholly below rp and was waited for), wait for segment
// evt - LAG, and work out when the next event is due.
template <class G>
__device__ __forceinline__ void chain_event(Chain &c, ChainRing &r, uint32_t &timeouts,
                                            uint32_t lane) {
    const uint32_t k = c.evt;
    const uint32_t slot = k % G::kNSeg;
    const bool issue = k < c.nseg;
    const uint32_t off = k * G::kSeg;
    bulk_g2s_armed_if(issue && lane == 0, r.ring_s + slot * G::kSeg, c.src + off,
                      issue ? min(G::kSeg, c.span - off) : 0u, r.bar0 + 8 * slot);
    if (k >= G::kLag && k - G::kLag < c.nseg) ring_wait(r, (k - G::kLag) % G::kNSeg, timeouts);
    c.evt = k + 1;
    c.next_evt = k + 1 >= c.nseg + G::kLag
                     ? 0xFFFFFFFFu
                     : (k + 2 > G::kNSeg ? (k + 2 - G::kNSeg) * G::kSeg : 0u);
}

template <class G>
__device__ __forceinline__ void chain_service(Chain &c, ChainRing &r, uint32_t &timeouts,
                                              uint32_t lane) {
    while (c.rp >= c.next_evt) chain_event<G>(c, r, timeouts, lane);
}

// The ring's invariant, checked in checked builds after each service: every
// byte the next `bytes` of reads can touch (up to the chunk's end) lies in a
// segment whose copy has been waited for (after events 0..evt-1: segments
// below evt - LAG) and whose ring slot no later copy has taken (segment j's
// slot goes to segment j + NSEG, issued once j + NSEG < min(evt, nseg)).
template <class G>
__device__ __forceinline__ bool ring_window_ok(const Chain &c, uint32_t bytes) {
    const uint32_t hi = min(c.rp + bytes, c.endrel);
    if (hi <= c.rp || c.st != RANS_OK) return true;
    const uint32_t first = c.rp / G::kSeg, last = (hi - 1) / G::kSeg;
    const bool not_overwritten = first + G::kNSeg >= min(c.evt, c.nseg);
    const bool complete = c.evt >= G::kLag && last < c.evt - G::kLag;
    return not_overwritten && complete;
}

// Shared address of the word k words of B bytes past read position rp.
// RING > 0: rp is the byte position in the chunk's word stream and ring_s the
// chunk's ring of RING bytes, aligned to RING, so (offset & (RING - 1)) |
// ring_s addresses it.  RING = 0: rp is the shared address of the read
// position itself, for groups of steps whose reads cannot reach the ring's
// end (one multiply-add, no wrap).
template <uint32_t RING, uint32_t B = 2>
__device__ __forceinline__ uint32_t word_at(uint32_t rp, uint32_t k, uint32_t ring_s) {
    return RING ? ((rp + B * k) & (RING - 1)) | ring_s : imad(k, B, rp);
}

// Decode one step of a chunk: every active lane decodes one symbol and reads
// at most one word.  FULL: every lane of the warp is a coder with a symbol in
// this step.  rp: the warp-uniform read position (word_at).
// EARLY: lane j loads the word at rp + 2j before the table lookup (every
// word the step can read, within its 64-byte window), and the lane that
// needs one takes the word of lane popc(m & lt) by a shuffle: the shared
// load leaves the step's dependent chain, the shuffle takes its place.
// Measured on B300: one 1 MiB chunk 73.2 -> 70.4 ns a step, but a full GPU
// 840 -> 880 us on 1 GiB (a second data-pipe wavefront a step), so only the
// decoder of messages under one wave of chunks uses it.
template <bool FULL, uint32_t RING, bool EARLY = false>
__device__ __forceinline__ void decode_step(uint32_t &x, uint32_t &rp, bool active,
                                            uint32_t tab_s, uint32_t ring_s, uint8_t *outp,
                                            uint32_t lt) {
    const uint32_t e = ld_table(imad(x & (kM - 1), 4u, tab_s));
    const uint32_t wl = EARLY ? ld_ring_u16(word_at<RING>(rp, threadIdx.x & 31u, ring_s)) : 0u;
    if (FULL || active) {
        x = decode_update(x, e);
        *outp = uint8_t(e);
    }
    const bool need = (FULL || active) && x < kL;
    const uint32_t m = __ballot_sync(kFull, need);
    const uint32_t w = EARLY ? __shfl_sync(kFull, wl, __popc(m & lt))
                             : ld_ring_u16(word_at<RING>(rp, __popc(m & lt), ring_s));
    if (need) x = __byte_perm(x, w, 0x1054u);  // (x << 16) | w
    rp = imad(__popc(m), 2u, rp);
}

// Entry ring (kKindPlainSpec) loads and stores: the ring is rewritten by the
// warp as the stream advances, so both stay ordered (volatile).
__device__ __forceinline__ uint32_t ld_ering(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ void st_ering(uint32_t a, uint32_t v) {
    asm volatile("st.shared.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
// Entry-ring address of stream byte position p (even): entry (p / 2) mod 1024.
__device__ __forceinline__ uint32_t ering_at(uint32_t p, uint32_t ering_s) {
    return ((p * 2u) & (kERing - 1)) | ering_s;
}

// The entry-ahead step (kKindPlainSpec), for warps whose chain of dependent
// steps sets the pace.  e: the slot-table entry of x's slot, carried from
// the step before.  A renormalizing lane's next slot is the low 12 bits of
// the word it reads, so its next entry is known as soon as the word is: lane
// j loads the word at rp + 2j and that word's entry from the entry ring
// (spec_convert filled it) before D, and a lane that reads a word takes the
// word and the entry of lane popc(m & lt) by two shuffles.  A lane that does
// not renormalize looks its next entry up from x'.  The step's chain is then
// D, the ballot, its prefix count, a shuffle and a select: no shared-memory
// load after the word is known.  The order of the shared-memory operations
// matters: that table lookup issued after the shuffles (as here) measured
// 65.6 ns a step on one 1 MiB chunk, issued before the ballot 77.4 ns,
// against 70.5 ns for the early-word step.
template <bool FULL>
__device__ __forceinline__ void decode_step_spec(uint32_t &x, uint32_t &e, uint32_t &rp, bool active,
                                                 uint32_t tab_s, uint32_t ring_s, uint32_t ering_s,
                                                 uint8_t *outp, uint32_t lt) {
    const uint32_t pos = imad(threadIdx.x & 31u, 2u, rp);
    const uint32_t wl = ld_ring_u16(word_at<kWarpRing>(pos, 0u, ring_s));
    const uint32_t el = ld_ering(ering_at(pos, ering_s));
    uint32_t xn = x;
    if (FULL || active) {
        xn = decode_update(x, e);
        *outp = uint8_t(e);
    }
    const bool need = (FULL || active) && xn < kL;
    const uint32_t m = __ballot_sync(kFull, need);
    const uint32_t k = __popc(m & lt);
    const uint32_t w = __shfl_sync(kFull, wl, k);
    const uint32_t ew = __shfl_sync(kFull, el, k);
    const uint32_t en = ld_table(imad(xn & (kM - 1), 4u, tab_s));
    x = need ? __byte_perm(xn, w, 0x1054u) : xn;  // (x << 16) | w
    e = need ? ew : en;
    rp = imad(__popc(m), 2u, rp);
}

// Fill the entry ring ahead of the entry-ahead step: for every word at
// stream bytes [c.cv, rp + 2 KiB), in whole 64-byte blocks, the slot-table
// entry of its low 12 bits, at the word's place in the entry ring.  Called
// after the ring events due at rp, which keep [rp, rp + 2 KiB) of words in
// (GeoSpec); entries below rp are spent, so the 1024-entry ring holds what
// is ahead.  Four blocks at a time (loads first, so their latencies
// overlap), then __syncwarp: every lane sees the entries the others stored.
__device__ __forceinline__ void spec_convert(Chain &c, uint32_t ring_s, uint32_t ering_s,
                                             uint32_t tab_s, uint32_t lane) {
    const uint32_t lim = c.rp + 2048u;
    while (c.cv + 64u <= lim) {
        const uint32_t nb = min(4u, (lim - c.cv) >> 6);
        const uint32_t p0 = imad(lane, 2u, c.cv);
        // Selects, not branches, around the loads: the four table lookups
        // then issue back to back (with a branch around each they waited for
        // one another: one 1 MiB chunk 2.15 -> 2.39 ms).
        uint32_t w[4], v[4];
#pragma unroll
        for (uint32_t i = 0; i < 4; ++i)
            w[i] = i < nb ? ld_ring_u16(word_at<kWarpRing>(p0 + 64u * i, 0u, ring_s)) : 0u;
#pragma unroll
        for (uint32_t i = 0; i < 4; ++i)
            v[i] = i < nb ? ld_table(imad(w[i] & (kM - 1), 4u, tab_s)) : 0u;
#pragma unroll
        for (uint32_t i = 0; i < 4; ++i)
            if (i < nb) st_ering(ering_at(p0 + 64u * i, ering_s), v[i]);
        c.cv += 64u * nb;
    }
    __syncwarp();
}

// One step at 13 or 14 bits of resolution (LM): the slot's symbol from the
// byte table, its f and B from the per-symbol table, then the plain
// renormalization (b = 2^16 >= M: at most one word).
template <bool FULL, uint32_t RING, uint32_t LM>
__device__ __forceinline__ void decode_step_wide(uint32_t &x, uint32_t &rp, bool active,
                                                 uint32_t sym_s, uint32_t fb_s, uint32_t ring_s,
                                                 uint8_t *outp, uint32_t lt) {
    const uint32_t slot = x & ((1u << LM) - 1);
    const uint32_t s = ld_flag(sym_s + slot);
    const uint32_t fb = ld_table(imad(s, 4u, fb_s));
    if (FULL || active) {
        x = imad(fb & 0xFFFFu, x >> LM, slot - (fb >> 16));
        *outp = uint8_t(s);
    }
    const bool need = (FULL || active) && x < kL;
    const uint32_t m = __ballot_sync(kFull, need);
    const uint32_t w = ld_ring_u16(word_at<RING>(rp, __popc(m & lt), ring_s));
    if (need) x = __byte_perm(x, w, 0x1054u);  // (x << 16) | w
    rp = imad(__popc(m), 2u, rp);
}

// One step with a binary model (f_0 + f_1 = M, both > 0): the symbol is
// [slot >= f_0], and D is x = f_s * floor(x/M) + slot - B_s with B_0 = 0,
// B_1 = f_0 -- two multiply-adds, one of them kept, instead of a table load.
__device__ __forceinline__ uint32_t decode_update_binary(uint32_t x, uint32_t f0, uint32_t f1,
                                                         uint32_t &one) {
    const uint32_t slot = x & (kM - 1), q = x >> kLog2M;
    one = slot >= f0;
    return one ? imad(f1, q, slot - f0) : imad(f0, q, slot);
}

template <bool FULL, uint32_t RING>
__device__ __forceinline__ void decode_step_binary(uint32_t &x, uint32_t &rp, bool active,
                                                   uint32_t f0, uint32_t f1, uint32_t ring_s,
                                                   uint8_t *outp, uint32_t lt) {
    if (FULL || active) {
        uint32_t one;
        x = decode_update_binary(x, f0, f1, one);
        *outp = uint8_t(one);
    }
    const bool need = (FULL || active) && x < kL;
    const uint32_t m = __ballot_sync(kFull, need);
    const uint32_t w = ld_ring_u16(word_at<RING>(rp, __popc(m & lt), ring_s));
    if (need) x = __byte_perm(x, w, 0x1054u);  // (x << 16) | w
    rp = imad(__popc(m), 2u, rp);
}

// One step of two chunks a and b, their instructions interleaved.
template <bool FULL, uint32_t RING>
__device__ __forceinline__ void decode_step2(uint32_t &xa, uint32_t &rpa, uint32_t ra_s, uint8_t *oa,
                                             uint32_t &xb, uint32_t &rpb, uint32_t rb_s, uint8_t *ob,
                                             bool active, uint32_t tab_s, uint32_t lt) {
    const uint32_t ea = ld_table(imad(xa & (kM - 1), 4u, tab_s));
    const uint32_t eb = ld_table(imad(xb & (kM - 1), 4u, tab_s));
    if (FULL || active) {
        xa = decode_update(xa, ea);
        xb = decode_update(xb, eb);
        *oa = uint8_t(ea);
        *ob = uint8_t(eb);
    }
    const bool na = (FULL || active) && xa < kL;
    const bool nb = (FULL || active) && xb < kL;
    const uint32_t ma = __ballot_sync(kFull, na);
    const uint32_t mb = __ballot_sync(kFull, nb);
    const uint32_t wa = ld_ring_u16(((rpa + 2u * __popc(ma & lt)) & (RING - 1)) | ra_s);
    const uint32_t wb = ld_ring_u16(((rpb + 2u * __popc(mb & lt)) & (RING - 1)) | rb_s);
    if (na) xa = __byte_perm(xa, wa, 0x1054u);
    if (nb) xb = __byte_perm(xb, wb, 0x1054u);
    rpa = imad(__popc(ma), 2u, rpa);
    rpb = imad(__popc(mb), 2u, rpb);
}

// decode_step2 for a binary model (f0, f1).
template <bool FULL, uint32_t RING>
__device__ __forceinline__ void decode_step2_binary(uint32_t &xa, uint32_t &rpa, uint32_t ra_s,
                                                    uint8_t *oa, uint32_t &xb, uint32_t &rpb,
                                                    uint32_t rb_s, uint8_t *ob, bool active,
                                                    uint32_t f0, uint32_t f1, uint32_t lt) {
    if (FULL || active) {
        uint32_t sa, sb;
        xa = decode_update_binary(xa, f0, f1, sa);
        xb = decode_update_binary(xb, f0, f1, sb);
        *oa = uint8_t(sa);
        *ob = uint8_t(sb);
    }
    const bool na = (FULL || active) && xa < kL;
    const bool nb = (FULL || active) && xb < kL;
    const uint32_t ma = __ballot_sync(kFull, na);
    const uint32_t mb = __ballot_sync(kFull, nb);
    const uint32_t wa = ld_ring_u16(((rpa + 2u * __popc(ma & lt)) & (RING - 1)) | ra_s);
    const uint32_t wb = ld_ring_u16(((rpb + 2u * __popc(mb & lt)) & (RING - 1)) | rb_s);
    if (na) xa = __byte_perm(xa, wa, 0x1054u);
    if (nb) xb = __byte_perm(xb, wb, 0x1054u);
    rpa = imad(__popc(ma), 2u, rpa);
    rpb = imad(__popc(mb), 2u, rpb);
}

// One step of a bypass chunk (Section 3): as decode_step, and then every
// lane whose symbol carries a raw word reads it right after its own
// renormalization word; one prefix over the lanes places both kinds of word
// in lane order.  The raw word, or 0 for a symbol without one, goes to *rawp.
template <bool FULL, uint32_t RING>
__device__ __forceinline__ void decode_step_raw(uint32_t &x, uint32_t &rp, bool active,
                                                uint32_t tab_s, uint32_t ring_s, uint32_t flags_s,
                                                uint8_t *outp, uint16_t *rawp, uint32_t lt) {
    const uint32_t e = ld_table(imad(x & (kM - 1), 4u, tab_s));
    const bool on = FULL || active;
    const uint32_t fl = ld_flag(flags_s + (e & 0xFFu));
    if (on) {
        x = decode_update(x, e);
        *outp = uint8_t(e);
    }
    const bool need = on && x < kL;
    const bool has = on && fl != 0u;
    const uint32_t m = __ballot_sync(kFull, need);
    const uint32_t mr = __ballot_sync(kFull, has);
    const uint32_t k = __popc(m & lt) + __popc(mr & lt);
    const uint32_t w = ld_ring_u16(word_at<RING>(rp, k, ring_s));
    const uint32_t rw = ld_ring_u16(word_at<RING>(rp, k + uint32_t(need), ring_s));
    if (need) x = __byte_perm(x, w, 0x1054u);  // (x << 16) | w
    if (on) *rawp = uint16_t(has ? rw : 0u);
    rp = imad(__popc(m) + __popc(mr), 2u, rp);
}

// One step of a byte-wise chunk (b = 2^8 < M, Section 5): after D a lane may
// need two digits.  The digits are read breadth-first across the warp: a
// first pass gives every lane below L one byte (lanes in order), a second
// pass -- taken only when some lane is still below L -- a second one.  (x << 8) | byte is
// a byte permute.
// PAR (kKindBytesLat): both passes' lanes are known right after D (a lane
// takes a second digit exactly when x < L / 2^8, since its first digit is
// below 2^8), so both ballots and both loads are issued together and the
// second pass no longer waits on the first one's merge.  Measured on B300:
// one 1 MiB chunk 3850 -> 2798 us, 148 chunks 275 -> 191 us, 2369 chunks 327
// -> 285 us; slower on a full GPU (1 GiB 1288 -> 1452 us), where the second
// pass is issued on almost every step.
template <bool FULL, uint32_t RING, bool PAR = false>
__device__ __forceinline__ void decode_step_bytes(uint32_t &x, uint32_t &rp, bool active,
                                                  uint32_t tab_s, uint32_t ring_s, uint8_t *outp,
                                                  uint32_t lt) {
    const uint32_t e = ld_table(imad(x & (kM - 1), 4u, tab_s));
    const bool on = FULL || active;
    if (on) {
        x = decode_update(x, e);
        *outp = uint8_t(e);
    }
    if constexpr (PAR) {
        const bool n1 = on && x < kL8, n2 = on && x < (kL8 >> 8);
        const uint32_t m1 = __ballot_sync(kFull, n1), m2 = __ballot_sync(kFull, n2);
        const uint32_t c1 = __popc(m1);
        const uint32_t w1 = ld_ring_u8(word_at<RING, 1>(rp, __popc(m1 & lt), ring_s));
        uint32_t w2 = 0;
        if (m2) w2 = ld_ring_u8(word_at<RING, 1>(rp + c1, __popc(m2 & lt), ring_s));
        if (n1) x = __byte_perm(x, w1, 0x2104u);  // (x << 8) | w
        if (n2) x = __byte_perm(x, w2, 0x2104u);
        rp += c1 + __popc(m2);
        return;
    }
    bool need = on && x < kL8;
    uint32_t m = __ballot_sync(kFull, need);
    uint32_t w = ld_ring_u8(word_at<RING, 1>(rp, __popc(m & lt), ring_s));
    if (need) x = __byte_perm(x, w, 0x2104u);  // (x << 8) | w
    rp += __popc(m);
    need = on && x < kL8;
    m = __ballot_sync(kFull, need);
    if (m) {
        w = ld_ring_u8(word_at<RING, 1>(rp, __popc(m & lt), ring_s));
        if (need) x = __byte_perm(x, w, 0x2104u);
        rp += __popc(m);
    }
}

// One step of an adaptive chunk (binary symbols, Section 5): the lane's own
// context p gives f_0 = p, f_1 = M - p, B_1 = p; no table.  D, then the
// context moves towards the decoded bit, then the usual renormalization.
template <bool FULL, uint32_t RING>
__device__ __forceinline__ void decode_step_adaptive(uint32_t &x, uint32_t &p, uint32_t &rp,
                                                     bool active, uint32_t ring_s, uint8_t *outp,
                                                     uint32_t lt) {
    const bool on = FULL || active;
    if (on) {
        const uint32_t slot = x & (kM - 1);
        const uint32_t one = slot >= p;
        const uint32_t q = kM - p;
        const uint32_t f = one ? q : p;
        x = imad(f, x >> kLog2M, slot - (one ? p : 0u));
        *outp = uint8_t(one);
        // p + floor((T - p) / 2^rate) with T = M after a 0 and T = 2^rate - 1
        // after a 1, where floor((2^rate - 1 - p) / 2^rate) = -floor(p / 2^rate):
        // the two updates of the model in one arithmetic shift.
        p += uint32_t(int32_t(q - one * (kM - ((1u << kAdaptRate) - 1))) >> kAdaptRate);
    }
    const bool need = on && x < kL;
    const uint32_t m = __ballot_sync(kFull, need);
    const uint32_t w = ld_ring_u16(word_at<RING>(rp, __popc(m & lt), ring_s));
    if (need) x = __byte_perm(x, w, 0x1054u);  // (x << 16) | w
    rp = imad(__popc(m), 2u, rp);
}

// One step of an adaptive-n chunk: the lane's own model gives s (the
// boundaries at or below the slot, counted), B_s and f_s by selects; D, then
// the model update, then the usual renormalization.  A boundary is at or
// below the slot exactly when it is at or below s, so the same predicates
// drive the update.
template <bool FULL, uint32_t RING, int NB>
__device__ __forceinline__ void decode_step_adaptive_n(Chain &c, bool active, uint32_t ring_s,
                                                       uint8_t *outp, uint32_t lt) {
    const bool on = FULL || active;
    if (on) {
        const uint32_t slot = c.x & (kM - 1);
        uint32_t s = 0, B = 0, F = kM;
        bool le[NB];
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            le[i] = c.cm[i] <= slot;
            s += le[i];
            B = le[i] ? c.cm[i] : B;
        }
#pragma unroll
        for (int i = NB - 1; i >= 0; --i) F = le[i] ? F : c.cm[i];
        c.x = imad(F - B, c.x >> kLog2M, slot - B);
        *outp = uint8_t(s);
        adapt::update_signed<NB>(c.cm, le, c.nm);
    }
    const bool need = on && c.x < kL;
    const uint32_t m = __ballot_sync(kFull, need);
    const uint32_t w = ld_ring_u16(word_at<RING>(c.rp, __popc(m & lt), ring_s));
    if (need) c.x = __byte_perm(c.x, w, 0x1054u);  // (x << 16) | w
    c.rp = imad(__popc(m), 2u, c.rp);
}

// One step of a prefix-message chunk (Section 4): a lane holding fewer than
// 12 bits reads its next 32-bit word first (lanes in order, ballot + popc,
// as for rANS words), then the top 12 of its bits index the code table;
// the symbol's length is dropped from the bit count.  Bits are kept
// right-aligned, so a read shifts bhi:blo up by one word and a symbol costs
// no shift.
template <bool FULL, uint32_t RING>
__device__ __forceinline__ void decode_step_prefix(Chain &c, bool active, uint32_t tab_s,
                                                   uint32_t ring_s, uint8_t *outp, uint32_t lt) {
    const bool on = FULL || active;
    const bool need = on && c.nb < kPrefixMaxLen;
    const uint32_t m = __ballot_sync(kFull, need);
    const uint32_t w = ld_ring_u32(word_at<RING, 4>(c.rp, __popc(m & lt), ring_s));
    if (need) {
        c.bhi = c.blo;
        c.blo = w;
        c.nb += 32;
    }
    c.rp = imad(__popc(m), 4u, c.rp);
    if (on) {
        const uint32_t idx = __funnelshift_r(c.blo, c.bhi, c.nb - kPrefixMaxLen) & (kM - 1);
        const uint32_t e = ld_table(imad(idx, 4u, tab_s));
        *outp = uint8_t(e);
        c.nb -= e >> 8;
    }
}

// One step of chunk c of message kind KIND; outp/rawp: this step's output.
template <bool FULL, uint32_t RING, int KIND>
__device__ __forceinline__ void kind_step(Chain &c, bool active, uint32_t tab_s, uint32_t ring_s,
                                          uint32_t flags_s, uint8_t *outp, uint16_t *rawp,
                                          uint32_t lt) {
    if (KIND == kKindRaw)
        decode_step_raw<FULL, RING>(c.x, c.rp, active, tab_s, ring_s, flags_s, outp, rawp, lt);
    else if (KIND == kKindBytes || KIND == kKindBytesLat)
        decode_step_bytes<FULL, RING, KIND == kKindBytesLat>(c.x, c.rp, active, tab_s, ring_s,
                                                             outp, lt);
    else if (KIND == kKindAdaptive)
        decode_step_adaptive<FULL, RING>(c.x, c.p, c.rp, active, ring_s, outp, lt);
    else if (KIND == kKindPrefix)
        decode_step_prefix<FULL, RING>(c, active, tab_s, ring_s, outp, lt);
    else if (KIND == kKindWide13 || KIND == kKindWide14)  // flags_s: the f/B table
        decode_step_wide<FULL, RING, WideBits<KIND>::kLog2>(c.x, c.rp, active, tab_s, flags_s,
                                                           ring_s, outp, lt);
    else if (KIND == kKindBinary)  // tab_s, flags_s: f_0, f_1
        decode_step_binary<FULL, RING>(c.x, c.rp, active, tab_s, flags_s, ring_s, outp, lt);
    else if (AdaptN<KIND>::kOn)
        decode_step_adaptive_n<FULL, RING, AdaptN<KIND>::kNB>(c, active, ring_s, outp, lt);
    else
        decode_step<FULL, RING, KIND == kKindPlainEarly>(c.x, c.rp, active, tab_s, ring_s, outp,
                                                         lt);
}

// Decode what is left of one chunk on its own.
template <bool FULL, class G, int KIND = kKindPlain>
__device__ __forceinline__ void chain_run(Chain &c, ChainRing &r, uint32_t &timeouts, uint32_t N,
                                          bool lane_on, uint32_t lane, uint32_t tab_s, uint32_t lt,
                                          uint32_t flags_s = 0) {
    constexpr bool RAW = KIND == kKindRaw;
    for (uint32_t g = c.steps / G::kGroup; g > 0; --g) {
        chain_service<G>(c, r, timeouts, lane);
        RANS_CHECK(timeouts || ring_window_ok<G>(c, G::kGroup * G::kStep));
        const uint32_t off = c.rp & (G::kRing - 1);
        // Measured on B300: 2-3.5 % faster for plain, bypass and byte-wise
        // chunks alone in a warp's ring; no gain for adaptive, prefix and
        // 13/14-bit chunks, and slower for chunk pairs (more code).
        constexpr bool kLinear = (KIND == kKindPlain || KIND == kKindPlainEarly ||
                                  KIND == kKindRaw || KIND == kKindBytes ||
                                  KIND == kKindBytesLat ||
                                  KIND == kKindBinary) &&
                                 G::kRing == kWarpRing;
        if (kLinear && off + G::kGroup * G::kStep <= G::kRing) {
            // A group reads at most kGroup * kStep bytes from rp: here they
            // all lie below the ring's end (3 groups in 4 with a 4 KiB ring
            // and 1 KiB groups), so the steps address the ring by absolute
            // position.
            const uint32_t rp0 = c.rp, a0 = r.ring_s + off;
            c.rp = a0;
#pragma unroll
            for (uint32_t u = 0; u < G::kGroup; ++u)
                kind_step<FULL, 0, KIND>(c, lane_on, tab_s, r.ring_s, flags_s, c.outp + u * N,
                                         RAW ? c.rawp + u * N : nullptr, lt);
            c.rp = rp0 + (c.rp - a0);
        } else {
#pragma unroll
            for (uint32_t u = 0; u < G::kGroup; ++u)
                kind_step<FULL, G::kRing, KIND>(c, lane_on, tab_s, r.ring_s, flags_s,
                                                c.outp + u * N, RAW ? c.rawp + u * N : nullptr, lt);
        }
        c.outp += G::kGroup * N;
        if (RAW) c.rawp += G::kGroup * N;
    }
    for (uint32_t t = c.steps % G::kGroup; t > 0; --t) {
        chain_service<G>(c, r, timeouts, lane);
        RANS_CHECK(timeouts || ring_window_ok<G>(c, G::kStep));
        kind_step<FULL, G::kRing, KIND>(c, lane_on, tab_s, r.ring_s, flags_s, c.outp, c.rawp, lt);
        c.outp += N;
        if (RAW) c.rawp += N;
    }
    c.steps = 0;
    if (c.rem) {
        chain_service<G>(c, r, timeouts, lane);
        RANS_CHECK(timeouts || ring_window_ok<G>(c, G::kStep));
        kind_step<false, G::kRing, KIND>(c, lane < c.rem, tab_s, r.ring_s, flags_s, c.outp,
                                         c.rawp, lt);
        c.rem = 0;
    }
}

// Decode what is left of one chunk with the entry-ahead step (G = GeoSpec,
// ering_s: the warp's entry ring).
template <bool FULL, class G>
__device__ __forceinline__ void chain_run_spec(Chain &c, ChainRing &r, uint32_t &timeouts,
                                               uint32_t N, bool lane_on, uint32_t lane,
                                               uint32_t tab_s, uint32_t lt, uint32_t ering_s) {
    c.cv = c.rp & ~63u;
    uint32_t e = ld_table(imad(c.x & (kM - 1), 4u, tab_s));
    for (uint32_t g = c.steps / G::kGroup; g > 0; --g) {
        chain_service<G>(c, r, timeouts, lane);
        RANS_CHECK(timeouts || ring_window_ok<G>(c, G::kGroup * G::kStep));
        spec_convert(c, r.ring_s, ering_s, tab_s, lane);
#pragma unroll
        for (uint32_t u = 0; u < G::kGroup; ++u)
            decode_step_spec<FULL>(c.x, e, c.rp, lane_on, tab_s, r.ring_s, ering_s,
                                   c.outp + u * N, lt);
        c.outp += G::kGroup * N;
    }
    for (uint32_t t = c.steps % G::kGroup; t > 0; --t) {
        chain_service<G>(c, r, timeouts, lane);
        RANS_CHECK(timeouts || ring_window_ok<G>(c, G::kGroup * G::kStep));
        spec_convert(c, r.ring_s, ering_s, tab_s, lane);
        decode_step_spec<FULL>(c.x, e, c.rp, lane_on, tab_s, r.ring_s, ering_s, c.outp, lt);
        c.outp += N;
    }
    c.steps = 0;
    if (c.rem) {
        chain_service<G>(c, r, timeouts, lane);
        RANS_CHECK(timeouts || ring_window_ok<G>(c, G::kGroup * G::kStep));
        spec_convert(c, r.ring_s, ering_s, tab_s, lane);
        decode_step_spec<false>(c.x, e, c.rp, lane < c.rem, tab_s, r.ring_s, ering_s, c.outp, lt);
        c.rem = 0;
    }
}

// Byte-wise chunks end in zero padding up to a multiple of 4 bytes: the chunk
// must be exactly round4(4N + digits read) long, with zeros after the digits
// (src + rp .. src + endrel, at most 3 bytes).
// Prefix chunks end with every word read and every coder holding at most 43
// bits (no missing code was met), all of them zero.
template <class G, bool BYTES = false, bool PREFIX = false>
__device__ __forceinline__ uint32_t chain_close(Chain &c, ChainRing &r, uint32_t &timeouts,
                                                bool lane_on, uint32_t N = 0) {
    const uint32_t issued = min(c.evt, c.nseg);
    for (uint32_t j = c.evt > G::kLag ? c.evt - G::kLag : 0u; j < issued; ++j)
        ring_wait(r, j % G::kNSeg, timeouts);
    if (c.st != RANS_OK) return c.st;
    if (timeouts) return RANS_ERR_TIMEOUT;
    if (PREFIX) {
        const uint64_t bits = (uint64_t(c.bhi) << 32) | c.blo;
        const bool clean =
            c.nb <= kPrefixMaxHeld && (bits & ((uint64_t(1) << c.nb) - 1)) == 0;
        const bool ok = __all_sync(kFull, !lane_on || clean) && c.rp == c.endrel;
        return ok ? RANS_OK : RANS_ERR_CORRUPT;
    }
    if (BYTES) {
        const uint32_t used = c.rp - c.rp0;
        bool ok = __all_sync(kFull, !lane_on || c.x == kL8) &&
                  ((4 * N + used + 3) & ~3u) == c.len && c.rp <= c.endrel;
        if (ok) {
            const uint32_t i = c.rp + (threadIdx.x & 31);
            const uint32_t pad = i < c.endrel ? c.src[i] : 0u;
            ok = !__any_sync(kFull, pad != 0u);
        }
        return ok ? RANS_OK : RANS_ERR_CORRUPT;
    }
    const bool ok = __all_sync(kFull, !lane_on || c.x == kL) && c.rp == c.endrel;
    return ok ? RANS_OK : RANS_ERR_CORRUPT;
}

// A model with one symbol s of frequency M: C is the identity, so a
// well-formed chunk is N states equal to L and no words.
__device__ __forceinline__ uint32_t const_chunk(const uint8_t *msg, uint32_t data0, uint32_t o,
                                                uint32_t e, uint32_t data_end, uint32_t n_c,
                                                uint32_t N, uint8_t *out, uint32_t const_sym,
                                                uint32_t lane, uint32_t L = kL) {
    if (((o | e) & 1u) || e < o || e > data_end || e - o != 4 * N) return RANS_ERR_CORRUPT;
    const uint8_t *chunk = msg + data0 + o;
    uint32_t x = L;
    if (lane < N) x = ld_u16_global(chunk + 4 * lane) | (ld_u16_global(chunk + 4 * lane + 2) << 16);
    for (uint32_t i = lane; i < n_c; i += 32) out[i] = uint8_t(const_sym);
    return __all_sync(kFull, x == L) ? RANS_OK : RANS_ERR_CORRUPT;
}

// const_chunk for a bypass message: when the one symbol carries a raw word,
// the chunk is the N states followed by one raw word per symbol, in order.
__device__ __forceinline__ uint32_t const_chunk_raw(const uint8_t *msg, uint32_t data0, uint32_t o,
                                                    uint32_t e, uint32_t data_end, uint32_t n_c,
                                                    uint32_t N, uint8_t *out, uint16_t *raw_out,
                                                    uint32_t const_sym, bool has_raw,
                                                    uint32_t lane) {
    const uint64_t words = has_raw ? n_c : 0u;
    if (((o | e) & 1u) || e < o || e > data_end || uint64_t(e - o) != 4ull * N + 2 * words)
        return RANS_ERR_CORRUPT;
    const uint8_t *chunk = msg + data0 + o;
    uint32_t x = kL;
    if (lane < N) x = ld_u16_global(chunk + 4 * lane) | (ld_u16_global(chunk + 4 * lane + 2) << 16);
    for (uint32_t i = lane; i < n_c; i += 32) {
        out[i] = uint8_t(const_sym);
        raw_out[i] = has_raw ? uint16_t(ld_u16_global(chunk + 4 * N + 2 * i)) : uint16_t(0);
    }
    return __all_sync(kFull, x == kL) ? RANS_OK : RANS_ERR_CORRUPT;
}

// Decode chunks c .. c + count - 1 (count = 1, or 2 when PAIR) of a message
// (offsets table offs, data region at msg + data0, data_end = offs[n_chunks])
// of n_sym symbols in chunks of CS with N coders; chunk k's symbols go to
// out + k*CS.  PAIR: the warp's two 2 KiB rings, the two chunks' steps
// interleaved; otherwise one chunk in the warp's 4 KiB ring.  RAW: a bypass
// message (one chunk per warp); symbol i's raw word, or 0, goes to
// raw_out[i] and flags_s addresses the 256 raw-word flags.  const_sym !=
// kNoConst: the model has one symbol with f = M.  UNI: chain_open's UNI (the
// batched decoder's form).  Returns the warp-uniform status (RANS_OK, or the
// first of RANS_ERR_CORRUPT / RANS_ERR_TIMEOUT found).
template <int NT, bool PAIR, int KIND = kKindPlain, bool UNI = false,
          bool LONG = false>  // NT = 32: all lanes are coders; LONG: GeoOneLong
__device__ __forceinline__ uint32_t decode_chunks(WarpRings &w, uint32_t tab_s, const uint8_t *msg,
                                                  uint32_t data0, const uint32_t *offs,
                                                  uint32_t data_end, uint32_t c, uint32_t count,
                                                  uint64_t n_sym, uint32_t CS, uint32_t N_rt,
                                                  uint8_t *out, uint32_t const_sym, uint32_t lane,
                                                  uint32_t lt, uint16_t *raw_out = nullptr,
                                                  uint32_t flags_s = 0, bool const_raw = false) {
    constexpr bool RAW = KIND == kKindRaw;
    constexpr bool BYTES = KIND == kKindBytes || KIND == kKindBytesLat;
    constexpr bool PREFIX = KIND == kKindPrefix;
    static_assert(!(PAIR && KIND != kKindPlain && KIND != kKindBinary),
                  "only plain messages pair chunks");
    constexpr bool BINARY = KIND == kKindBinary;
    constexpr bool SPEC = KIND == kKindPlainSpec;
    static_assert(!(PAIR && SPEC), "the entry-ahead step decodes one chunk per warp");
    using G = typename std::conditional<
        RAW, GeoRaw,
        typename std::conditional<SPEC, GeoSpec,
        typename std::conditional<PREFIX, GeoPrefix,
                                  typename std::conditional<
                                      PAIR, GeoPair,
                                      typename std::conditional<LONG, GeoOneLong, GeoOne>::type>::type>::type>::type>::type;
    constexpr bool kFullWarp = NT == 32;
    const uint32_t N = NT ? NT : N_rt;
    const bool lane_on = lane < N;
    const bool two = PAIR && count > 1;
    const uint64_t first = uint64_t(c) * CS;
    const uint32_t n_a = uint32_t(umin64(CS, n_sym - first));
    const uint32_t n_b = two ? uint32_t(umin64(CS, n_sym - first - CS)) : 0u;
    const uint32_t o0 = offs[c], o1 = offs[c + 1], o2 = two ? offs[c + 2] : 0u;

    constexpr bool ADAPTN = AdaptN<KIND>::kOn;
    if (KIND != kKindAdaptive && !ADAPTN && !PREFIX && const_sym != kNoConst) {
        if (RAW)
            return const_chunk_raw(msg, data0, o0, o1, data_end, n_a, N, out + first,
                                   raw_out + first, const_sym, const_raw, lane);
        if (BYTES)
            return const_chunk(msg, data0, o0, o1, data_end, n_a, N, out + first, const_sym, lane,
                               kL8);
        uint32_t st = const_chunk(msg, data0, o0, o1, data_end, n_a, N, out + first, const_sym, lane);
        if (two) {
            const uint32_t sb =
                const_chunk(msg, data0, o1, o2, data_end, n_b, N, out + first + CS, const_sym, lane);
            if (st == RANS_OK) st = sb;
        }
        return st;
    }

    Chain a, b;
    if (PREFIX)
        chain_open_prefix<G>(a, msg, data0, o0, o1, data_end, n_a, N, out + first, lane);
    else
        chain_open<G, BYTES, UNI>(a, msg, data0, o0, o1, data_end, n_a, N, out + first,
                                  RAW ? raw_out + first : nullptr, lane);
    if (two)
        chain_open<G, false, UNI>(b, msg, data0, o1, o2, data_end, n_b, N, out + first + CS,
                                  nullptr, lane);
    else chain_empty(b);
    if (ADAPTN) {  // flags_s: the alphabet size n
        adapt::init<AdaptN<KIND>::kNB>(a.cm, flags_s);
        a.nm = kM - flags_s;
    }

    if (PAIR) {
        // Both chunks step together while each has a full group left.
        const uint32_t groups = min(a.steps, b.steps) / G::kGroup;
        a.steps -= groups * G::kGroup;
        b.steps -= groups * G::kGroup;
        for (uint32_t g = groups; g > 0; --g) {
            chain_service<G>(a, w.r[0], w.timeouts, lane);
            chain_service<G>(b, w.r[1], w.timeouts, lane);
            RANS_CHECK(w.timeouts || (ring_window_ok<G>(a, G::kGroup * G::kStep) &&
                                      ring_window_ok<G>(b, G::kGroup * G::kStep)));
#pragma unroll
            for (uint32_t u = 0; u < G::kGroup; ++u) {
                if (BINARY)
                    decode_step2_binary<kFullWarp, G::kRing>(
                        a.x, a.rp, w.r[0].ring_s, a.outp + u * N, b.x, b.rp, w.r[1].ring_s,
                        b.outp + u * N, lane_on, tab_s, flags_s, lt);
                else
                    decode_step2<kFullWarp, G::kRing>(a.x, a.rp, w.r[0].ring_s, a.outp + u * N,
                                                      b.x, b.rp, w.r[1].ring_s, b.outp + u * N,
                                                      lane_on, tab_s, lt);
            }
            a.outp += G::kGroup * N;
            b.outp += G::kGroup * N;
        }
    }
    if constexpr (SPEC)  // flags_s: the warp's entry ring
        chain_run_spec<kFullWarp, G>(a, w.r[0], w.timeouts, N, lane_on, lane, tab_s, lt, flags_s);
    else
        chain_run<kFullWarp, G, KIND>(a, w.r[0], w.timeouts, N, lane_on, lane, tab_s, lt, flags_s);
    if (two)
        chain_run<kFullWarp, G, BINARY ? kKindBinary : kKindPlain>(b, w.r[1], w.timeouts, N,
                                                                    lane_on, lane, tab_s, lt,
                                                                    flags_s);
    const uint32_t sa = chain_close<G, BYTES, PREFIX>(a, w.r[0], w.timeouts, lane_on, N);
    const uint32_t sb = two ? chain_close<G>(b, w.r[1], w.timeouts, lane_on) : RANS_OK;
    return sa != RANS_OK ? sa : sb;
}

// Header check of a message of n_sym symbols in chunks of CS with N coders;
// msg_size is the message size and data0 its data-region offset.
__device__ __forceinline__ bool header_ok(const uint8_t *msg, uint64_t msg_size, uint32_t data0,
                                          uint64_t n_sym, uint32_t N, uint32_t CS,
                                          uint32_t n_chunks, uint32_t version = RANS_VERSION,
                                          uint32_t log2m = kLog2M) {
    const uint32_t *h32 = reinterpret_cast<const uint32_t *>(msg);
    const uint64_t hn = uint64_t(h32[4]) | (uint64_t(h32[5]) << 32);
    if (h32[0] != RANS_MAGIC || h32[1] != version || h32[2] != N || h32[3] != log2m ||
        hn != n_sym || h32[6] != CS || h32[7] != n_chunks)
        return false;
    const uint32_t first = h32[8], last = h32[8 + n_chunks];
    return first == 0 && round16(last) == msg_size - data0;
}

}  // namespace dec
}  // namespace rans
