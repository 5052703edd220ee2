// decode_core.cuh -- the decoder's building blocks, shared by the single-message
// kernel (rans_decode.cu) and the batched persistent kernel (rans_batch.cu).
//
// One warp decodes one chunk; lane j is coder j of the chunk's N interleaved
// rANS coders.  Per step every lane decodes one symbol (Algorithm 1 Decode,
// Section 2):
//     slot = x mod M;  (s, f_s, slot - B_s) from a slot table in shared memory
//     x    = f_s * floor(x / M) + slot - B_s
// and then renormalizes at most once (b = 2^16 >= M, Section 5): the lanes
// with x < L form renorm_mask = ballot(x < L); a lane reads the word at
// read_pos + popc(renorm_mask & lanes_below_me) and read_pos advances by
// popc(renorm_mask) -- the packed load of Section 6.
//
// Compressed words stream into a per-warp shared-memory ring through 512-byte
// bulk copies (TMA, cp.async.bulk) completed on mbarriers; decoded bytes go
// out as one coalesced 32-byte store per warp and step.
#pragma once

#include <cstdint>

#include "device_util.cuh"
#include "host_util.h"

namespace rans {
namespace dec {

constexpr int kWarps = 8;                 // warps (chunks in flight) per CTA
constexpr uint32_t kThreads = kWarps * 32;
constexpr uint32_t kSeg = 512;            // bytes per bulk copy
constexpr uint32_t kNSeg = 8;             // ring segments per warp
constexpr uint32_t kRing = kSeg * kNSeg;  // 4 KiB per warp, aligned to 4 KiB in shared space
constexpr uint32_t kGroup = 16;           // steps between ring checks
// A step reads at most 32 words = 64 bytes, so a group reads at most 1 KiB:
// two segments, while the ring holds eight.
static_assert(kGroup * 64 <= 2 * kSeg, "a group must fit in two segments");
constexpr uint32_t kTableBytes = kM * 4;
// Shared memory: [slot table 16 KiB][alignment slack 4 KiB][one ring per
// warp][mbarriers][a few words of CTA state].
constexpr uint32_t kBarOffset = kTableBytes + kRing + kWarps * kRing;
constexpr uint32_t kMiscOffset = kBarOffset + kWarps * kNSeg * 8;
constexpr uint32_t kSmemBytes = kMiscOffset + 64;
constexpr uint32_t kNoConst = 0xFFFFFFFFu;

struct Smem {
    uint32_t *tab;
    uint32_t tab_s;
    uint32_t rings_s;   // 4 KiB aligned
    uint8_t *rings;     // generic pointer of rings_s
    uint64_t *bars;
    uint32_t *misc;     // CTA-shared words
};

__device__ __forceinline__ Smem smem_layout(uint8_t *smem) {
    Smem s;
    s.tab = reinterpret_cast<uint32_t *>(smem);
    s.tab_s = smem_addr(smem);
    const uint32_t raw = smem_addr(smem + kTableBytes);
    s.rings_s = (raw + kRing - 1) & ~(kRing - 1);
    s.rings = smem + kTableBytes + (s.rings_s - raw);
    s.bars = reinterpret_cast<uint64_t *>(smem + kBarOffset);
    s.misc = reinterpret_cast<uint32_t *>(smem + kMiscOffset);
    return s;
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
__device__ __forceinline__ uint32_t ld_ring_u16(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.u16 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}

// Build the 4096-entry slot table from 256 frequencies (zero for unused
// symbols) with the whole CTA (kThreads threads).  scratch: >= 5 KiB of
// shared memory not in use (the rings before any chunk is decoded).
// Returns (to every thread) the sum of the frequencies; *const_sym receives
// the symbol with f = M, or kNoConst.
//   cum[s] = f_0 + ... + f_{s-1}                       (warp scan)
//   mark[cum[s]] = s for every s with f_s > 0           (scatter)
//   sym(slot) = max of mark[0..slot]                    (max-scan: symbols
//               are laid out in increasing order)
__device__ __noinline__ static uint32_t build_slot_table(const uint16_t *freq, uint32_t *tab, uint8_t *scratch,
                                     uint32_t *const_sym) {
    uint32_t *cum = reinterpret_cast<uint32_t *>(scratch);        // 257 words
    uint8_t *mark = scratch + 1040;                               // 4096 bytes
    uint32_t *part = reinterpret_cast<uint32_t *>(scratch + 1040 + kM);  // 8 words
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (uint32_t i = tid; i < kM / 4; i += kThreads) reinterpret_cast<uint32_t *>(mark)[i] = 0;
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
    // kThreads threads x 16 slots each
    constexpr uint32_t kPer = kM / kThreads;
    static_assert(kPer == 16, "slot table build assumes 256 threads");
    const uint32_t base = tid * kPer;
    uint32_t mk[kPer];
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
    // exclusive max-scan of the per-thread maxima across the CTA
    uint32_t incl = run;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, d);
        if (lane >= uint32_t(d)) incl = max(incl, y);
    }
    if (lane == 31) part[warp] = incl;
    __syncthreads();
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
    __syncthreads();
    return total;
}

// Per-warp ring state, carried across the chunks a warp decodes.
struct WarpRing {
    uint32_t ring_s;    // this warp's ring (4 KiB aligned shared address)
    uint32_t bar0;      // its kNSeg mbarriers
    uint32_t phase;     // bit i: parity of the next wait on barrier i
    uint32_t timeouts;  // warp-uniform: a bounded wait gave up
};

__device__ __forceinline__ WarpRing ring_init(const Smem &sm, uint32_t warp, uint32_t lane) {
    WarpRing r;
    r.ring_s = sm.rings_s + warp * kRing;
    r.bar0 = smem_addr(sm.bars + warp * kNSeg);
    r.phase = 0;
    r.timeouts = 0;
    if (lane == 0) {
        for (uint32_t i = 0; i < kNSeg; ++i) mbar_init(r.bar0 + 8 * i, 1);
        fence_mbar_init();
    }
    __syncwarp();
    return r;
}

// Decode one step of a chunk: every active lane decodes one symbol and reads
// at most one word.  FULL: every lane of the warp is a coder with a symbol in
// this step.  rp is the byte position in the word stream (warp-uniform);
// ring_s is the warp's 4 KiB-aligned ring, so (offset & 4095) | ring_s
// addresses it.
template <bool FULL>
__device__ __forceinline__ void decode_step(uint32_t &x, uint32_t &rp, bool active,
                                            uint32_t tab_s, uint32_t ring_s, uint8_t *outp,
                                            uint32_t lt) {
    const uint32_t e = ld_table(tab_s + ((x & (kM - 1)) << 2));
    if (FULL || active) {
        x = decode_update(x, e);
        *outp = uint8_t(e);
    }
    const bool need = (FULL || active) && x < kL;
    const uint32_t m = __ballot_sync(kFull, need);
    const uint32_t w = ld_ring_u16(((rp + 2u * __popc(m & lt)) & (kRing - 1)) | ring_s);
    if (need) x = __byte_perm(x, w, 0x1054u);  // (x << 16) | w
    rp += 2u * __popc(m);
}

// Decode chunk [o, e) (byte offsets in the data region that starts at msg +
// data0; data_end = end of all chunks) of n_c symbols with N coders into out.
// const_sym != kNoConst: the model has one symbol with f = M.  Returns the
// warp-uniform status (RANS_OK, RANS_ERR_CORRUPT or RANS_ERR_TIMEOUT).
template <int NT>  // NT = 32: all 32 lanes are coders; NT = 0: runtime N
__device__ __forceinline__ uint32_t decode_chunk(WarpRing &wr, uint32_t tab_s, const uint8_t *msg,
                                                 uint32_t data0, uint32_t o, uint32_t e,
                                                 uint32_t data_end, uint32_t n_c, uint32_t N_rt,
                                                 uint8_t *out, uint32_t const_sym,
                                                 uint32_t lane, uint32_t lt) {
    const uint32_t N = NT ? NT : N_rt;
    // Offsets must be even (states and words are 2-byte aligned) and in range.
    if (((o | e) & 1u) || e < o || e > data_end || e - o < 4 * N) return RANS_ERR_CORRUPT;
    const uint8_t *chunk = msg + data0 + o;
    uint32_t x = kL;
    if (lane < N) x = ld_u16_global(chunk + 4 * lane) | (ld_u16_global(chunk + 4 * lane + 2) << 16);
    if (!__all_sync(kFull, x >= kL)) return RANS_ERR_CORRUPT;  // Algorithm 1 requires x in I
    uint8_t *outp = out + lane;

    if (const_sym != kNoConst) {
        // f = M: C is the identity; the chunk is N states equal to L.
        for (uint32_t i = lane; i < n_c; i += 32) out[i] = uint8_t(const_sym);
        return (e - o == 4 * N && __all_sync(kFull, x == kL)) ? RANS_OK : RANS_ERR_CORRUPT;
    }

    // Word stream: bytes [P0, P1) of the message, loaded in 512-byte segments
    // starting at the 16-byte aligned A <= P0; stream byte P lives at ring
    // offset (P - A) mod 4096.
    const uint64_t P0 = uint64_t(data0) + o + 4 * N, P1 = uint64_t(data0) + e;
    const uint64_t A = P0 & ~uint64_t(15);
    const uint64_t end16 = round16(P1);
    const uint32_t nseg = uint32_t((end16 - A + kSeg - 1) / kSeg);
    const uint32_t endrel = uint32_t(P1 - A);
    uint32_t rp = uint32_t(P0 - A);
    uint32_t issued = 0, ready = 0, recheck = 0;

    // Issue every segment whose ring slot is free (its previous segment lies
    // wholly below rp), wait until the next group's bytes [rp, rp + 1 KiB)
    // are in, and compute the read position at which either can change again.
    auto service = [&]() {
        const uint32_t limit = min(nseg, kNSeg + rp / kSeg);
        for (; issued < limit; ++issued) {
            if (lane == 0) {
                const uint32_t slot = issued % kNSeg;
                const uint64_t src = A + uint64_t(issued) * kSeg;
                const uint32_t bytes = uint32_t(umin64(kSeg, end16 - src));
                mbar_arrive_expect_tx(wr.bar0 + 8 * slot, bytes);
                bulk_g2s(wr.ring_s + slot * kSeg, msg + src, bytes, wr.bar0 + 8 * slot);
            }
        }
        const uint32_t need = min(nseg, (rp + kGroup * 64 + kSeg - 1) / kSeg);
        for (; ready < need; ++ready) {
            const uint32_t slot = ready % kNSeg;
            const bool ok =
                wr.timeouts != 0 || mbar_wait_bounded(wr.bar0 + 8 * slot, (wr.phase >> slot) & 1u);
            if (__any_sync(kFull, !ok)) wr.timeouts = 1;  // warp-uniform
            wr.phase ^= 1u << slot;
        }
        const uint32_t r_ready =
            ready >= nseg ? 0xFFFFFFFFu
                          : (ready * kSeg >= kGroup * 64 ? ready * kSeg - kGroup * 64 + 1 : 0u);
        const uint32_t r_issue =
            issued >= nseg ? 0xFFFFFFFFu : (issued + 1 >= kNSeg ? (issued + 1 - kNSeg) * kSeg : 0u);
        recheck = min(r_ready, r_issue);
    };

    const uint32_t T_full = n_c / N, rem = n_c % N;
    const bool lane_on = lane < N;
    uint32_t t = 0;
    for (; t + kGroup <= T_full; t += kGroup) {
        if (rp >= recheck) service();
#pragma unroll
        for (uint32_t u = 0; u < kGroup; ++u)
            decode_step<NT == 32>(x, rp, lane_on, tab_s, wr.ring_s, outp + u * N, lt);
        outp += kGroup * N;
    }
    for (; t < T_full; ++t) {
        service();
        decode_step<NT == 32>(x, rp, lane_on, tab_s, wr.ring_s, outp, lt);
        outp += N;
    }
    if (rem) {
        service();
        decode_step<false>(x, rp, lane < rem, tab_s, wr.ring_s, outp, lt);
    }
    // Drain the copies still in flight so that the ring and the barrier
    // phases are clean for the next chunk.
    for (; ready < issued; ++ready) {
        const uint32_t slot = ready % kNSeg;
        const bool ok =
            wr.timeouts != 0 || mbar_wait_bounded(wr.bar0 + 8 * slot, (wr.phase >> slot) & 1u);
        if (__any_sync(kFull, !ok)) wr.timeouts = 1;
        wr.phase ^= 1u << slot;
    }
    if (wr.timeouts) return RANS_ERR_TIMEOUT;
    // A well-formed chunk ends with every coder back at x0 = L and every word
    // read exactly once (decoder and encoder in lockstep, Section 3).
    const bool ok = __all_sync(kFull, !lane_on || x == kL) && rp == endrel;
    return ok ? RANS_OK : RANS_ERR_CORRUPT;
}

// Header check of a message of n_sym symbols in chunks of CS with N coders;
// msg_size is the message size and data0 its data-region offset.
__device__ __forceinline__ bool header_ok(const uint8_t *msg, uint64_t msg_size, uint32_t data0,
                                          uint64_t n_sym, uint32_t N, uint32_t CS,
                                          uint32_t n_chunks) {
    const uint32_t *h32 = reinterpret_cast<const uint32_t *>(msg);
    const uint64_t hn = uint64_t(h32[4]) | (uint64_t(h32[5]) << 32);
    if (h32[0] != RANS_MAGIC || h32[1] != RANS_VERSION || h32[2] != N || h32[3] != kLog2M ||
        hn != n_sym || h32[6] != CS || h32[7] != n_chunks)
        return false;
    const uint32_t first = h32[8], last = h32[8 + n_chunks];
    return first == 0 && round16(last) == msg_size - data0;
}

}  // namespace dec
}  // namespace rans
