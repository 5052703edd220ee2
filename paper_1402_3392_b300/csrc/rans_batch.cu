// rans_batch.cu -- batched decoding and encoding of many independent
// streams, each in one persistent launch.
//
// The work list is built on the device: a setup kernel validates every
// descriptor and writes the exclusive prefix of work items per stream (one
// item = the chunks one CTA decodes at once, of one stream).  The persistent decode
// kernel's CTAs take items from an atomic counter; an item's stream is found
// by binary search in the prefix; its model's slot table is rebuilt in shared
// memory only when the model changes; each warp decodes one chunk with the
// same code as the single-message decoder (two chunks per warp).
#include <algorithm>
#include <atomic>

#include <cuda_runtime.h>

#include "decode_core.cuh"
#include "encode_core.cuh"
#include "host_util.h"

namespace rans {
namespace {

constexpr int kSetupThreads = 1024;

struct BatchLayout {
    uint64_t prefix, wprefix, counter, total;
};
BatchLayout batch_layout(uint32_t n) {
    BatchLayout l{};
    const uint64_t arr = round16(4ull * (uint64_t(n) + 1));
    l.prefix = 0;
    l.wprefix = arr;
    l.counter = 2 * arr;
    l.total = l.counter + 16;
    return l;
}

// Two kinds of work item.  A CTA item: up to item_chunks chunks of one
// stream, decoded by the whole CTA with the stream's slot table in shared
// memory (the CTA rebuilds it when the model changes).  A warp item: up to
// two chunks of a stream with a binary model (symbols 0 and 1, both with
// f > 0), decoded by one warp alone -- D needs no table, so the warps of a
// CTA take chunks of different streams and wait on nobody.  The persistent
// kernel's CTAs drain the CTA items first, then their warps the warp items.
struct BatchDecodeParams {
    const rans_stream *streams;
    const uint16_t *freqs;
    uint32_t *status;
    uint32_t *prefix;   // n_streams + 1 CTA-item offsets
    uint32_t *wprefix;  // n_streams + 1 warp-item offsets
    uint32_t *counter;  // [0] next CTA item, [1] next warp item
    uint32_t n_streams;
    uint32_t n_tables;
    uint32_t item_chunks;  // chunks in one CTA item: the CTA's warps x chunks per warp
};

struct StreamGeom {
    uint64_t n_chunks;
    uint32_t data0;
    bool ok;
};

__device__ __forceinline__ StreamGeom check_stream(const rans_stream &d, uint32_t n_tables) {
    StreamGeom g{0, 0, false};
    if (d.n_lanes < 1 || d.n_lanes > 32 || d.chunk_symbols < 1 || d.table >= n_tables) return g;
    if ((reinterpret_cast<uintptr_t>(d.msg) & 15u) || (d.msg_size & 15u) || d.msg == nullptr)
        return g;
    if (d.n_symbols && d.symbols == nullptr) return g;
    g.n_chunks = (d.n_symbols + d.chunk_symbols - 1) / d.chunk_symbols;
    if (g.n_chunks > 0xFFFFFFFEull) return g;
    const uint64_t data0 = round16(32 + 4 * (g.n_chunks + 1));
    if (d.msg_size < data0 || d.msg_size < 48 || d.msg_size - data0 > 0xFFFFFFFFull + 15)
        return g;
    g.data0 = uint32_t(data0);
    g.ok = true;
    return g;
}

// The binary-model test the setup kernel can afford per stream (its first
// two frequencies); the warp that decodes a chunk checks the whole table.
__device__ __forceinline__ bool binary_candidate(const uint16_t *fr) {
    const uint32_t f0 = fr[0], f1 = fr[1];
    return f0 > 0 && f1 > 0 && f0 + f1 == kM;
}

// One CTA: statuses, the CTA-item and warp-item prefixes, counters.
__global__ void __launch_bounds__(kSetupThreads)
    batch_setup_kernel(const __grid_constant__ BatchDecodeParams p) {
    __shared__ uint32_t sums[2][32];
    __shared__ uint32_t carry_s[2];
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < 2) carry_s[tid] = 0;
    __syncthreads();
    for (uint32_t base = 0; base < p.n_streams; base += kSetupThreads) {
        const uint32_t i = base + tid;
        uint32_t v[2] = {0u, 0u};  // CTA items, warp items
        if (i < p.n_streams) {
            const rans_stream d = p.streams[i];
            const StreamGeom g = check_stream(d, p.n_tables);
            p.status[i] = g.ok ? RANS_OK : RANS_ERR_INVALID_ARG;
            if (g.ok && g.n_chunks > 0 && binary_candidate(p.freqs + uint64_t(d.table) * 256)) {
                v[1] = uint32_t((g.n_chunks + dec::kChains - 1) / dec::kChains);
            } else if (g.ok) {
                const uint64_t k = (g.n_chunks + p.item_chunks - 1) / p.item_chunks;
                v[0] = k > 0 ? uint32_t(k) : 1u;  // an empty stream still has its header checked
            }
        }
        uint32_t incl[2] = {v[0], v[1]};
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const uint32_t y = __shfl_up_sync(kFull, incl[k], d);
                if (lane >= uint32_t(d)) incl[k] += y;
            }
        }
        if (lane == 31) {
            sums[0][warp] = incl[0];
            sums[1][warp] = incl[1];
        }
        __syncthreads();
        if (warp < 2) {
            const uint32_t w = sums[warp][lane];
            uint32_t wi = w;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(kFull, wi, d);
                if (lane >= uint32_t(d)) wi += y;
            }
            sums[warp][lane] = wi - w;
        }
        __syncthreads();
        const uint32_t c0 = carry_s[0], c1 = carry_s[1];
        if (i < p.n_streams) {
            p.prefix[i] = c0 + sums[0][warp] + incl[0] - v[0];
            p.wprefix[i] = c1 + sums[1][warp] + incl[1] - v[1];
        }
        __syncthreads();
        if (tid == kSetupThreads - 1) {
            carry_s[0] = c0 + sums[0][warp] + incl[0];
            carry_s[1] = c1 + sums[1][warp] + incl[1];
        }
        __syncthreads();
    }
    if (tid == 0) {
        p.prefix[p.n_streams] = carry_s[0];
        p.wprefix[p.n_streams] = carry_s[1];
        p.counter[0] = p.counter[1] = 0;
    }
}

// item_stream with a whole warp: 32 probes per round narrow the range 32-fold,
// so 10,000 streams take 3 dependent loads instead of 14.  Warp-uniform.
__device__ __forceinline__ uint32_t item_stream_warp(const uint32_t *prefix, uint32_t n,
                                                     uint32_t v, uint32_t lane) {
    uint32_t lo = 0, hi = n;  // the answer lies in [lo, hi)
    while (hi - lo > 1) {
        const uint32_t step = (hi - lo + 31) / 32;
        const uint32_t idx = lo + lane * step;
        const bool le = idx < hi && prefix[idx] <= v;   // true for a prefix of the lanes
        const uint32_t k = __popc(__ballot_sync(kFull, le)) - 1;   // lane 0 always holds
        lo += k * step;
        hi = min(hi, lo + step);
    }
    return lo;
}

// dec::header_ok with the loads spread over a warp's lanes.  Warp-uniform.
__device__ __forceinline__ bool header_ok_warp(const uint8_t *msg, uint64_t msg_size,
                                               uint32_t data0, uint64_t n_sym, uint32_t N,
                                               uint32_t CS, uint32_t n_chunks, uint32_t lane) {
    const uint32_t *h32 = reinterpret_cast<const uint32_t *>(msg);
    const uint32_t idx = lane < 8 ? lane : lane == 8 ? 8u : 8u + n_chunks;
    const uint32_t v = lane < 10 ? h32[idx] : 0u;
    const uint64_t hn = uint64_t(__shfl_sync(kFull, v, 4)) | (uint64_t(__shfl_sync(kFull, v, 5)) << 32);
    const uint32_t want = lane == 0 ? RANS_MAGIC : lane == 1 ? RANS_VERSION : lane == 2 ? N
                          : lane == 3 ? kLog2M : lane == 6 ? CS : lane == 7 ? n_chunks
                          : lane == 8 ? 0u : v;
    const uint32_t last = __shfl_sync(kFull, v, 9);
    const bool ok = (lane >= 10 || lane == 4 || lane == 5 || lane == 9 || v == want);
    return __all_sync(kFull, ok) && hn == n_sym && round16(last) == msg_size - data0;
}

// The stream of work item v: the largest s with prefix[s] <= v.
__device__ __forceinline__ uint32_t item_stream(const uint32_t *prefix, uint32_t n, uint32_t v) {
    uint32_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (prefix[mid] <= v) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Phase 1 of the batched decoder: CTA items (chunks of table-model streams).
// A CTA item holds ROUNDS groups of chunks per warp (a group: one chunk, or a
// pair): each warp starts with group `warp`, then takes the item's next
// group from a shared counter, so a warp that finishes early takes more and
// the CTA waits for the slowest warp once per item, not once per group.
// Ring addresses and read positions pass through warp_uniform here
// (chain_open's UNI).  Returns wr with the rings' state (barrier phases,
// timeouts) after the phase.
template <int W, bool PAIR, uint32_t ROUNDS>
__device__ __forceinline__ dec::WarpRings batch_cta_items(const BatchDecodeParams &p,
                                                          const dec::Smem &sm, dec::WarpRings wr,
                                                          uint32_t lane, uint32_t warp) {
    constexpr uint32_t kPer = PAIR ? dec::kChains : 1u;
    constexpr uint32_t kItem = W * kPer * ROUNDS;  // chunks in a CTA item
    uint32_t &item_s = sm.misc[0];
    uint32_t &stream_s = sm.misc[1];
    uint32_t &loaded = sm.misc[2];      // model whose slot table is in shared memory
    uint32_t &const_sym = sm.misc[3];
    uint32_t &model_ok = sm.misc[4];
    uint32_t &hdr_ok = sm.misc[5];
    uint32_t &next_group = sm.misc[6];  // the current item's next group to take
    const uint32_t lt = lanemask_lt();
    const uint32_t total = p.prefix[p.n_streams];
    dec::WarpRings wa = wr;
#pragma unroll
    for (uint32_t k = 0; k < dec::kChains; ++k) wa.r[k].ring_s = warp_uniform(wr.r[k].ring_s);
    for (;;) {
        __syncthreads();  // every warp is done with the previous item
        if (threadIdx.x == 0) {
            const uint32_t it = atomicAdd(p.counter, 1u);
            item_s = it;
            next_group = W;
            if (it < total) {
                const uint32_t lo = item_stream(p.prefix, p.n_streams, it);
                stream_s = lo;
                const rans_stream d = p.streams[lo];
                const StreamGeom g = check_stream(d, p.n_tables);
                hdr_ok = dec::header_ok(d.msg, d.msg_size, g.data0, d.n_symbols, d.n_lanes,
                                        d.chunk_symbols, uint32_t(g.n_chunks));
            }
        }
        __syncthreads();
        const uint32_t it = item_s;
        if (it >= total) break;
        const uint32_t s = stream_s;
        const rans_stream d = p.streams[s];
        if (d.table != loaded) {
            if (threadIdx.x == 0) const_sym = dec::kNoConst;
            const uint32_t sum = dec::build_slot_table<W>(p.freqs + uint64_t(d.table) * 256,
                                                          sm.tab, sm.rings, &const_sym);
            if (threadIdx.x == 0) {
                loaded = d.table;
                model_ok = sum == kM;
            }
            __syncthreads();
        }
        if (!model_ok) {
            if (threadIdx.x == 0) report(p.status + s, RANS_ERR_INVALID_ARG);
            continue;
        }
        if (!hdr_ok) {
            if (threadIdx.x == 0) report(p.status + s, RANS_ERR_CORRUPT);
            continue;
        }
        const StreamGeom g = check_stream(d, p.n_tables);
        const uint32_t c0 = (it - p.prefix[s]) * kItem;
        const uint32_t c_end = uint32_t(umin64(g.n_chunks, uint64_t(c0) + kItem));
        for (uint32_t grp = warp;;) {
            const uint32_t c = c0 + kPer * grp;
            if (c >= c_end || wa.timeouts) break;
            const uint32_t *offs = reinterpret_cast<const uint32_t *>(d.msg + 32);
            const uint32_t data_end = offs[g.n_chunks];
            const uint32_t cs = const_sym;
            const uint32_t count = uint32_t(umin64(kPer, g.n_chunks - c));
            const uint32_t st =
                d.n_lanes == 32
                         ? dec::decode_chunks<32, PAIR, dec::kKindPlain, true>(
                               wa, sm.tab_s, d.msg, g.data0, offs, data_end, c, count,
                               d.n_symbols, d.chunk_symbols, 32, d.symbols, cs, lane, lt)
                         : dec::decode_chunks<0, PAIR, dec::kKindPlain, true>(
                               wa, sm.tab_s, d.msg, g.data0, offs, data_end, c, count,
                               d.n_symbols, d.chunk_symbols, d.n_lanes, d.symbols, cs, lane, lt);
            if (st != RANS_OK && lane == 0) report(p.status + s, st);
            if (ROUNDS == 1) break;
            uint32_t nxt = 0;
            if (lane == 0) nxt = atomicAdd(&next_group, 1u);
            grp = __shfl_sync(kFull, nxt, 0);
        }
    }
#pragma unroll
    for (uint32_t k = 0; k < dec::kChains; ++k) wr.r[k].phase = wa.r[k].phase;
    wr.timeouts = wa.timeouts;
    return wr;
}

// Phase 2: warp items, chunk pairs of binary-model streams, a warp at a time
// (read positions warp-uniform as above).
__device__ __forceinline__ void batch_warp_items(const BatchDecodeParams &p, dec::WarpRings wr,
                                                 uint32_t lane) {
    const uint32_t lt = lanemask_lt();
    const uint32_t wtotal = p.wprefix[p.n_streams];
    for (;;) {
        uint32_t it = 0;
        if (lane == 0) it = atomicAdd(p.counter + 1, 1u);
        it = __shfl_sync(kFull, it, 0);
        if (it >= wtotal || wr.timeouts) break;
        const uint32_t s = item_stream_warp(p.wprefix, p.n_streams, it, lane);
        const rans_stream d = p.streams[s];
        const StreamGeom g = check_stream(d, p.n_tables);
        // the whole model: two frequencies summing to M leave no room for
        // others in a valid table
        const uint16_t *fr = p.freqs + uint64_t(d.table) * 256;
        uint32_t part = 0;
#pragma unroll
        for (uint32_t k = 0; k < 8; ++k) part += fr[lane * 8 + k];
        const bool model_ok = __reduce_add_sync(kFull, part) == kM;
        const bool hdr = header_ok_warp(d.msg, d.msg_size, g.data0, d.n_symbols, d.n_lanes,
                                        d.chunk_symbols, uint32_t(g.n_chunks), lane);
        if (!model_ok || !hdr) {
            if (lane == 0) report(p.status + s, model_ok ? RANS_ERR_CORRUPT : RANS_ERR_INVALID_ARG);
            continue;
        }
        const uint32_t f0 = fr[0], f1 = fr[1];
        const uint32_t c = (it - p.wprefix[s]) * dec::kChains;
        const uint32_t *offs = reinterpret_cast<const uint32_t *>(d.msg + 32);
        const uint32_t data_end = offs[g.n_chunks];
        const uint32_t count = uint32_t(umin64(dec::kChains, g.n_chunks - c));
        // f_0 and f_1 ride in the table and flag arguments
        const uint32_t st =
            d.n_lanes == 32
                ? dec::decode_chunks<32, true, dec::kKindBinary, true>(
                      wr, f0, d.msg, g.data0, offs, data_end, c, count, d.n_symbols,
                      d.chunk_symbols, 32, d.symbols, dec::kNoConst, lane, lt, nullptr, f1)
                : dec::decode_chunks<0, true, dec::kKindBinary, true>(
                      wr, f0, d.msg, g.data0, offs, data_end, c, count, d.n_symbols,
                      d.chunk_symbols, d.n_lanes, d.symbols, dec::kNoConst, lane, lt, nullptr, f1);
        if (st != RANS_OK && lane == 0) report(p.status + s, st);
    }
}

// The persistent batched decoder: every CTA takes CTA items until none is
// left, then its warps take warp items.  Bounded for the shape's resident
// CTAs per SM (8 warps: 4, at most 64 registers; 12 warps: 3, at most 56).
// Read positions pass through warp_uniform in both phases, ring addresses in
// the first only.  Measured on B300 against the kernel with neither (3000
// streams of the batched workload: 4.270 -> 4.249 ms; the binary workload:
// 216.5 -> 208.5 us, issue 74.5 -> 77.6 % of cycles with the same
// instructions per opcode in ncu: a scheduling effect, no work moved or
// removed).  Other arrangements moved the two phases against each other, in
// one kernel or in two: uniform ring addresses in both phases 4.169 ms /
// 218.5 us, rebuilt for the second 4.164 ms / 216.3 us, the two phases as
// two kernels 4.261 ms / 213.8 us.
template <int W, bool PAIR, uint32_t ROUNDS>
__global__ void __launch_bounds__(dec::Shape<W>::kThreads, dec::Shape<W>::kCtasPerSm)
    batch_decode_kernel(const __grid_constant__ BatchDecodeParams p) {
    extern __shared__ __align__(128) uint8_t smem[];
    const dec::Smem sm = dec::smem_layout<W>(smem);
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) sm.misc[2] = 0xFFFFFFFFu;  // no slot table loaded yet
    dec::WarpRings wr = dec::rings_init(sm, warp, lane);
    wr = batch_cta_items<W, PAIR, ROUNDS>(p, sm, wr, lane, warp);
    batch_warp_items(p, wr, lane);
}


// ---------------------------------------------------------------------------
// Batched encoding
// ---------------------------------------------------------------------------

struct EncBatchLayout {
    uint64_t items, witems, counter, total;
};
__host__ __device__ inline EncBatchLayout enc_batch_layout(uint32_t n) {
    EncBatchLayout l{};
    const uint64_t arr = (4ull * (uint64_t(n) + 1) + 15) & ~uint64_t(15);
    l.items = 0;
    l.witems = arr;
    l.counter = 2 * arr;
    l.total = l.counter + 16;
    return l;
}

struct BatchEncodeParams {
    const rans_encode_stream *streams;
    const uint16_t *freqs;
    uint64_t *out_sizes;
    uint32_t *status;
    uint8_t *scratch;
    uint64_t scratch_cap;
    uint32_t *items;    // n_streams + 1 CTA-item offsets
    uint32_t *witems;   // n_streams + 1 warp-item offsets (chunks of binary-model streams)
    uint32_t *counter;  // [0] next CTA item, [1] next warp item
    uint32_t n_streams;
    uint32_t n_tables;
};

struct EncGeom {
    uint64_t n_chunks;
    uint32_t data0;
    enc::ScratchLayout sl;
    bool ok;
};

__device__ __forceinline__ EncGeom check_enc_stream(const rans_encode_stream &d, uint32_t n_tables,
                                                    uint64_t scratch_cap) {
    EncGeom g{};
    g.ok = false;
    if (d.n_lanes < 1 || d.n_lanes > 32 || d.chunk_symbols < 1 || d.table >= n_tables) return g;
    if (d.out == nullptr || (reinterpret_cast<uintptr_t>(d.out) & 15u)) return g;
    if (d.n_symbols && d.symbols == nullptr) return g;
    g.n_chunks = (d.n_symbols + d.chunk_symbols - 1) / d.chunk_symbols;
    if (g.n_chunks > 0xFFFFFFFEull ||
        4ull * d.n_lanes * g.n_chunks + 2ull * d.n_symbols > 0xFFFFFFF0ull)
        return g;
    const uint64_t data0 = round16(32 + 4 * (g.n_chunks + 1));
    const uint64_t worst = data0 + round16(4ull * d.n_lanes * g.n_chunks + 2ull * d.n_symbols);
    if (d.out_cap < worst) return g;
    g.sl = enc::scratch_layout(g.n_chunks, d.n_lanes, d.chunk_symbols);
    if ((d.scratch_offset & 15u) || d.scratch_offset < enc_batch_layout(0).total ||
        d.scratch_offset > scratch_cap || scratch_cap - d.scratch_offset < g.sl.total)
        return g;
    g.data0 = uint32_t(data0);
    g.ok = true;
    return g;
}

// One CTA: statuses, CTA-item and warp-item prefixes, counters.  A stream
// whose model passes binary_candidate is coded by single warps, one chunk a
// warp item; any other in CTA items of kWarps chunks.
__global__ void __launch_bounds__(kSetupThreads)
    enc_setup_kernel(const __grid_constant__ BatchEncodeParams p) {
    __shared__ uint32_t sums[2][32];
    __shared__ uint32_t carry_s[2];
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < 2) carry_s[tid] = 0;
    __syncthreads();
    for (uint32_t base = 0; base < p.n_streams; base += kSetupThreads) {
        const uint32_t i = base + tid;
        uint32_t v[2] = {0u, 0u};
        if (i < p.n_streams) {
            const EncGeom g = check_enc_stream(p.streams[i], p.n_tables, p.scratch_cap);
            p.status[i] = g.ok ? RANS_OK : RANS_ERR_INVALID_ARG;
            p.out_sizes[i] = 0;
            if (g.ok && binary_candidate(p.freqs + uint64_t(p.streams[i].table) * 256))
                v[1] = uint32_t(g.n_chunks);
            else if (g.ok)
                v[0] = uint32_t((g.n_chunks + enc::kWarps - 1) / enc::kWarps);
        }
        uint32_t incl[2] = {v[0], v[1]};
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const uint32_t y = __shfl_up_sync(kFull, incl[k], d);
                if (lane >= uint32_t(d)) incl[k] += y;
            }
        }
        if (lane == 31) {
            sums[0][warp] = incl[0];
            sums[1][warp] = incl[1];
        }
        __syncthreads();
        if (warp < 2) {
            const uint32_t w = sums[warp][lane];
            uint32_t wi = w;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(kFull, wi, d);
                if (lane >= uint32_t(d)) wi += y;
            }
            sums[warp][lane] = wi - w;
        }
        __syncthreads();
        const uint32_t c0 = carry_s[0], c1 = carry_s[1];
        if (i < p.n_streams) {
            p.items[i] = c0 + sums[0][warp] + incl[0] - v[0];
            p.witems[i] = c1 + sums[1][warp] + incl[1] - v[1];
        }
        __syncthreads();
        if (tid == kSetupThreads - 1) {
            carry_s[0] = c0 + sums[0][warp] + incl[0];
            carry_s[1] = c1 + sums[1][warp] + incl[1];
        }
        __syncthreads();
    }
    if (tid == 0) {
        p.items[p.n_streams] = carry_s[0];
        p.witems[p.n_streams] = carry_s[1];
        p.counter[0] = p.counter[1] = 0;
    }
}

__device__ __forceinline__ uint32_t find_stream(const uint32_t *prefix, uint32_t n, uint32_t v) {
    uint32_t lo = 0, hi = n;  // largest s with prefix[s] <= v
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (prefix[mid] <= v) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Stream s's message as its coder warps place it (descriptor d, geometry g).
__device__ __forceinline__ enc::Placement stream_placement(const BatchEncodeParams &p, uint32_t s,
                                                           const rans_encode_stream &d,
                                                           const EncGeom &g) {
    uint8_t *scr = p.scratch + d.scratch_offset;
    enc::Placement m;
    m.out = d.out;
    m.out_size = p.out_sizes + s;
    m.status = p.status + s;
    m.words = scr + g.sl.words;
    m.states = reinterpret_cast<const uint32_t *>(scr + g.sl.states);
    m.wstart = reinterpret_cast<const uint32_t *>(scr + g.sl.wstart);
    m.sizes = reinterpret_cast<const uint32_t *>(scr + g.sl.sizes);
    m.lb = enc::scratch_lookback(scr, g.sl, uint32_t(g.n_chunks), d.chunk_symbols, d.n_lanes);
    m.n_sym = d.n_symbols;
    m.N = d.n_lanes;
    m.CS = d.chunk_symbols;
    m.data0 = g.data0;
    m.slot_bytes = g.sl.slot_bytes;
    m.version = RANS_VERSION;
    m.log2m = kLog2M;
    return m;
}

// Chunk c of stream s is coded (acc: the table flags it met): publish its
// size.  Out of line, as is place_pending, so that the coding loop keeps
// its registers.
__device__ __noinline__ void coded(const BatchEncodeParams &p, uint32_t s, uint32_t c,
                                   uint32_t lane, uint32_t acc) {
    const rans_encode_stream d = p.streams[s];
    const EncGeom g = check_enc_stream(d, p.n_tables, p.scratch_cap);
    enc::chunk_coded(stream_placement(p, s, d, g), c, lane, acc);
}

// Place coded chunk c of stream s, waiting (bounded) for the chunks before it.
__device__ __noinline__ void place_pending(const BatchEncodeParams &p, uint32_t s, uint32_t c,
                                           uint32_t lane) {
    const rans_encode_stream d = p.streams[s];
    const EncGeom g = check_enc_stream(d, p.n_tables, p.scratch_cap);
    enc::place_chunk<false, 4>(stream_placement(p, s, d, g), c, lane);
}

// One CTA per stream (grid-stride): zero the look-back words and ticket of
// every accepted stream's scratch.
constexpr int kClearThreads = 256;
__global__ void __launch_bounds__(kClearThreads)
    enc_clear_kernel(const __grid_constant__ BatchEncodeParams p) {
    for (uint32_t s = blockIdx.x; s < p.n_streams; s += gridDim.x) {
        if (p.status[s] != RANS_OK) continue;
        const rans_encode_stream d = p.streams[s];
        const EncGeom g = check_enc_stream(d, p.n_tables, p.scratch_cap);
        uint4 *w = reinterpret_cast<uint4 *>(p.scratch + d.scratch_offset + g.sl.look);
        const uint64_t n = (g.sl.total - g.sl.look) / 16;
        for (uint64_t i = threadIdx.x; i < n; i += blockDim.x) w[i] = make_uint4(0u, 0u, 0u, 0u);
    }
}

// After the placing coder: a rejected stream's size is 0; an accepted stream
// without chunks gets its header here.
__global__ void __launch_bounds__(kClearThreads)
    enc_settle_kernel(const __grid_constant__ BatchEncodeParams p) {
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < p.n_streams;
         s += gridDim.x * blockDim.x) {
        if (p.status[s] != RANS_OK) {
            p.out_sizes[s] = 0;
            continue;
        }
        const rans_encode_stream d = p.streams[s];
        const EncGeom g = check_enc_stream(d, p.n_tables, p.scratch_cap);
        if (g.n_chunks == 0)
            enc::write_header(d.out, p.out_sizes + s, d.n_symbols, d.n_lanes, d.chunk_symbols, 0,
                              g.data0, 0, RANS_VERSION);
    }
}

// Persistent: CTAs take CTA items (8 chunks of one stream, one per warp) in
// order from a counter; when none is left, warps take warp items (one chunk
// of a binary-model stream each) in order from a second counter.  Each warp
// codes its chunk, publishes the chunk's size, and places it after its next
// item (the last one at the end), waiting only for chunks taken earlier.
// A binary stream's chunk needs no table: the model's two entries are built
// in registers per item, and no warp of a CTA waits for another (its chunks
// of 16 Ki symbols left half the warps of an 8-chunk CTA item idle, the
// workload's streams having 4).
__global__ void __launch_bounds__(enc::kThreads, 4)
    batch_encode_kernel(const __grid_constant__ BatchEncodeParams p) {
    extern __shared__ __align__(128) uint8_t smem[];
    const enc::Smem sm = enc::smem_layout(smem);
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    uint32_t &item_s = sm.misc[0];
    uint32_t &stream_s = sm.misc[1];
    uint32_t &loaded = sm.misc[2];
    uint32_t &model_ok = sm.misc[3];
    if (threadIdx.x == 0) loaded = 0xFFFFFFFFu;
    const uint32_t ring_s = sm.rings_s + warp * enc::kRing;
    const uint32_t ge = lanemask_ge();
    const uint32_t total = p.items[p.n_streams];
    constexpr uint32_t kNone = 0xFFFFFFFFu;
    uint32_t pend_s = kNone, pend_c = 0;  // a coded chunk not yet placed
    for (;;) {
        __syncthreads();  // every warp is done with the previous item
        if (threadIdx.x == 0) {
            const uint32_t it = atomicAdd(p.counter, 1u);
            item_s = it;
            if (it < total) stream_s = find_stream(p.items, p.n_streams, it);
        }
        __syncthreads();
        const uint32_t it = item_s;
        if (it >= total) break;
        const uint32_t s = stream_s;
        const rans_encode_stream d = p.streams[s];
        if (d.table != loaded) {
            const uint32_t sum = enc::build_encode_table(p.freqs + uint64_t(d.table) * 256, sm.tab,
                                                         reinterpret_cast<uint32_t *>(sm.rings));
            if (threadIdx.x == 0) {
                loaded = d.table;
                model_ok = sum == kM;
            }
            __syncthreads();
        }
        const EncGeom g = check_enc_stream(d, p.n_tables, p.scratch_cap);
        const uint32_t c = (it - p.items[s]) * enc::kWarps + warp;
        if (!model_ok) {
            if (threadIdx.x == 0) report(p.status + s, RANS_ERR_INVALID_ARG);
            if (c < g.n_chunks) {
                uint8_t *scr = p.scratch + d.scratch_offset;
                enc::publish_failed(
                    enc::scratch_lookback(scr, g.sl, uint32_t(g.n_chunks), d.chunk_symbols, d.n_lanes),
                    c, lane);
            }
            continue;
        }
        bool did = false;
        if (c < g.n_chunks) {
            uint8_t *scr = p.scratch + d.scratch_offset;
            const uint64_t first = uint64_t(c) * d.chunk_symbols;
            const uint32_t n_c = uint32_t(umin64(d.chunk_symbols, d.n_symbols - first));
            uint32_t acc = 0;
            uint8_t *slot = scr + g.sl.words + uint64_t(c) * g.sl.slot_bytes;
            uint32_t *wstart = reinterpret_cast<uint32_t *>(scr + g.sl.wstart) + c;
            uint32_t *sizes = reinterpret_cast<uint32_t *>(scr + g.sl.sizes) + c;
            uint32_t *states = reinterpret_cast<uint32_t *>(scr + g.sl.states) + uint64_t(c) * d.n_lanes;
            if (d.n_lanes == 32)
                enc::encode_chunk<32, false>(d.symbols + first, n_c, 32, slot, g.sl.slot_bytes, wstart, sizes,
                                      states, sm.tab_s, ring_s, ge, lane, acc);
            else
                enc::encode_chunk<0, false>(d.symbols + first, n_c, d.n_lanes, slot, g.sl.slot_bytes, wstart,
                                     sizes, states, sm.tab_s, ring_s, ge, lane, acc);
            coded(p, s, c, lane, acc);
            did = true;
        }
        if (pend_s != kNone) {
            place_pending(p, pend_s, pend_c, lane);
            pend_s = kNone;
        }
        if (did) {
            pend_s = s;
            pend_c = c;
        }
    }

    const uint32_t wtotal = p.witems[p.n_streams];
    for (;;) {
        uint32_t it = 0;
        if (lane == 0) it = atomicAdd(p.counter + 1, 1u);
        it = __shfl_sync(kFull, it, 0);
        if (it >= wtotal) break;
        const uint32_t s = item_stream_warp(p.witems, p.n_streams, it, lane);
        const rans_encode_stream d = p.streams[s];
        const EncGeom g = check_enc_stream(d, p.n_tables, p.scratch_cap);
        const uint32_t c = it - p.witems[s];
        uint8_t *scr = p.scratch + d.scratch_offset;
        // the whole model: f_0 + f_1 = M (binary_candidate) leaves no room
        // for another symbol in a valid table
        const uint16_t *fr = p.freqs + uint64_t(d.table) * 256;
        uint32_t part = 0;
#pragma unroll
        for (uint32_t k = 0; k < 8; ++k) part += fr[lane * 8 + k];
        if (__reduce_add_sync(kFull, part) != kM) {
            if (lane == 0) report(p.status + s, RANS_ERR_INVALID_ARG);
            enc::publish_failed(
                enc::scratch_lookback(scr, g.sl, uint32_t(g.n_chunks), d.chunk_symbols, d.n_lanes),
                c, lane);
            continue;
        }
        const uint32_t f0 = fr[0];
        const uint2 e0 = enc::encode_entry(f0, 0u), e1 = enc::encode_entry(fr[1], f0);
        const uint64_t first = uint64_t(c) * d.chunk_symbols;
        const uint32_t n_c = uint32_t(umin64(d.chunk_symbols, d.n_symbols - first));
        uint32_t acc = 0;
        uint8_t *slot = scr + g.sl.words + uint64_t(c) * g.sl.slot_bytes;
        uint32_t *wstart = reinterpret_cast<uint32_t *>(scr + g.sl.wstart) + c;
        uint32_t *sizes = reinterpret_cast<uint32_t *>(scr + g.sl.sizes) + c;
        uint32_t *states = reinterpret_cast<uint32_t *>(scr + g.sl.states) + uint64_t(c) * d.n_lanes;
        if (d.n_lanes == 32)
            enc::encode_chunk<32, false, false, false, false, false, false, true>(
                d.symbols + first, n_c, 32, slot, g.sl.slot_bytes, wstart, sizes, states, 0u,
                ring_s, ge, lane, acc, nullptr, nullptr, e0, e1);
        else
            enc::encode_chunk<0, false, false, false, false, false, false, true>(
                d.symbols + first, n_c, d.n_lanes, slot, g.sl.slot_bytes, wstart, sizes, states, 0u,
                ring_s, ge, lane, acc, nullptr, nullptr, e0, e1);
        coded(p, s, c, lane, acc > 1u ? enc::kZeroFlag : 0u);  // a symbol outside {0, 1}
        if (pend_s != kNone) place_pending(p, pend_s, pend_c, lane);
        pend_s = s;
        pend_c = c;
    }
    if (pend_s != kNone) place_pending(p, pend_s, pend_c, lane);
    if (lane == 0) bulk_wait<0>();
}

}  // namespace
}  // namespace rans

using namespace rans;

namespace rans {
namespace {

// The batched decoder's CTA shape: 8 warps, two chunks side by side in each;
// CTA items of kBatchRounds pairs per warp.
constexpr int kBatchWarps = 8;
constexpr bool kBatchPair = true;
constexpr uint32_t kBatchRounds = 1;

template <int W, bool PAIR, uint32_t ROUNDS>
int launch_batch_decode(BatchDecodeParams &p, cudaStream_t st) {
    using S = dec::Shape<W>;
    auto kern = batch_decode_kernel<W, PAIR, ROUNDS>;
    p.item_chunks = W * (PAIR ? dec::kChains : 1u) * ROUNDS;
    // Set once per device; concurrent first calls may both set it (harmless).
    static std::atomic<bool> configured[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !configured[dev].load()) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(S::kSmemBytes)) != cudaSuccess)
            return RANS_ERR_CUDA;
        configured[dev].store(true);
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, S::kThreads, S::kSmemBytes) !=
            cudaSuccess ||
        per_sm <= 0)
        return RANS_ERR_CUDA;
    batch_setup_kernel<<<1, kSetupThreads, 0, st>>>(p);
    if (check_launch() != RANS_OK) return RANS_ERR_CUDA;
    kern<<<unsigned(per_sm * sm_count()), S::kThreads, S::kSmemBytes, st>>>(p);
    return check_launch();
}

}  // namespace
}  // namespace rans

extern "C" uint64_t rans_decode_batch_scratch_size(uint32_t n_streams) {
    return batch_layout(n_streams).total;
}

extern "C" int rans_decode_batch(const rans_stream *d_streams, uint32_t n_streams,
                                 const uint16_t *d_freqs, uint32_t n_tables, uint32_t *d_status,
                                 void *d_scratch, uint64_t scratch_cap, rans_stream_t stream) {
    if (n_streams == 0) return RANS_OK;
    if (!d_streams || !d_freqs || n_tables == 0 || !d_status || !d_scratch ||
        !aligned16(d_scratch) || (reinterpret_cast<uintptr_t>(d_streams) & 7u))
        return RANS_ERR_INVALID_ARG;
    const BatchLayout l = batch_layout(n_streams);
    if (scratch_cap < l.total) return RANS_ERR_BUFFER_TOO_SMALL;
    uint8_t *scr = static_cast<uint8_t *>(d_scratch);
    BatchDecodeParams p{};
    p.streams = d_streams;
    p.freqs = d_freqs;
    p.status = d_status;
    p.prefix = reinterpret_cast<uint32_t *>(scr + l.prefix);
    p.wprefix = reinterpret_cast<uint32_t *>(scr + l.wprefix);
    p.counter = reinterpret_cast<uint32_t *>(scr + l.counter);
    p.n_streams = n_streams;
    p.n_tables = n_tables;
    return launch_batch_decode<kBatchWarps, kBatchPair, kBatchRounds>(
        p, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" uint64_t rans_encode_batch_plan(rans_encode_stream *h_streams, uint32_t n_streams) {
    if (n_streams && !h_streams) return 0;
    uint64_t off = enc_batch_layout(n_streams).total;
    for (uint32_t i = 0; i < n_streams; ++i) {
        rans_encode_stream &d = h_streams[i];
        rans_params prm{d.n_lanes, d.chunk_symbols};
        if (!params_ok(&prm)) return 0;
        const MessageGeometry g = geometry(d.n_symbols, &prm);
        d.scratch_offset = off;
        off += round16(enc::scratch_layout(g.n_chunks, d.n_lanes, d.chunk_symbols).total);
    }
    return off;
}

extern "C" int rans_encode_batch(const rans_encode_stream *d_streams, uint32_t n_streams,
                                 const uint16_t *d_freqs, uint32_t n_tables, uint64_t *d_out_sizes,
                                 uint32_t *d_status, void *d_scratch, uint64_t scratch_cap,
                                 rans_stream_t stream) {
    if (n_streams == 0) return RANS_OK;
    if (!d_streams || !d_freqs || n_tables == 0 || !d_status || !d_out_sizes || !d_scratch ||
        !aligned16(d_scratch) || (reinterpret_cast<uintptr_t>(d_streams) & 7u) ||
        (reinterpret_cast<uintptr_t>(d_out_sizes) & 7u))
        return RANS_ERR_INVALID_ARG;
    const EncBatchLayout l = enc_batch_layout(n_streams);
    if (scratch_cap < l.total) return RANS_ERR_BUFFER_TOO_SMALL;
    uint8_t *scr = static_cast<uint8_t *>(d_scratch);
    BatchEncodeParams p{};
    p.streams = d_streams;
    p.freqs = d_freqs;
    p.out_sizes = d_out_sizes;
    p.status = d_status;
    p.scratch = scr;
    p.scratch_cap = scratch_cap;
    p.items = reinterpret_cast<uint32_t *>(scr + l.items);
    p.witems = reinterpret_cast<uint32_t *>(scr + l.witems);
    p.counter = reinterpret_cast<uint32_t *>(scr + l.counter);
    p.n_streams = n_streams;
    p.n_tables = n_tables;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_encode_kernel, enc::kThreads,
                                                      enc::kSmemBytes) != cudaSuccess ||
        per_sm <= 0)
        return RANS_ERR_CUDA;
    const unsigned sms = unsigned(sm_count());
    enc_setup_kernel<<<1, kSetupThreads, 0, st>>>(p);
    if (check_launch() != RANS_OK) return RANS_ERR_CUDA;
    enc_clear_kernel<<<std::min<unsigned>(n_streams, 8 * sms), kClearThreads, 0, st>>>(p);
    if (check_launch() != RANS_OK) return RANS_ERR_CUDA;
    batch_encode_kernel<<<unsigned(per_sm) * sms, enc::kThreads, enc::kSmemBytes, st>>>(p);
    if (check_launch() != RANS_OK) return RANS_ERR_CUDA;
    enc_settle_kernel<<<std::min<unsigned>((n_streams + kClearThreads - 1) / kClearThreads, 8 * sms),
                        kClearThreads, 0, st>>>(p);
    return check_launch();
}

#ifdef RANS_CHECKED
// Checked builds: failed invariants of this file's kernels since the last call.
uint64_t rans_check_failures_batch() { return rans::take_check_failures(); }
#endif
