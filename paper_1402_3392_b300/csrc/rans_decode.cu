// rans_decode.cu -- GPU decoder: one warp decodes one chunk, one lane is one
// of the chunk's N interleaved rANS coders.
//
// Per step every lane decodes one symbol (Algorithm 1 Decode, Section 2):
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
#include <algorithm>

#include <cuda_runtime.h>

#include "device_util.cuh"
#include "host_util.h"

namespace rans {
namespace {

constexpr int kWarps = 8;               // warps (chunks in flight) per CTA
constexpr uint32_t kSeg = 512;          // bytes per bulk copy
constexpr uint32_t kNSeg = 8;           // ring segments per warp
constexpr uint32_t kRing = kSeg * kNSeg;  // 4 KiB per warp, aligned to 4 KiB in shared space
constexpr uint32_t kGroup = 16;         // steps between ring checks
// A step reads at most 32 words = 64 bytes, so a group reads at most 1 KiB:
// two segments, while the ring holds eight.
static_assert(kGroup * 64 <= 2 * kSeg, "a group must fit in two segments");
constexpr uint32_t kTableBytes = kM * 4;
// layout: [slot table 16 KiB][alignment slack][ring per warp][mbarriers][flag]
constexpr uint32_t kSmemBytes = kTableBytes + kRing + kWarps * kRing + kWarps * kNSeg * 8 + 16;

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
    uint32_t const_sym;  // symbol with f = M (decode is a fill), else 0xFFFFFFFF
    uint16_t freq[RANS_MAX_ALPHABET];
};

// Slot table entry: f_s << 20 | (slot - B_s) << 8 | s   (f_s < M here).
// With E = entry >> 8 = f_s * 2^12 + (slot - B_s) the decode update is
//     f_s * floor(x/M) + slot - B_s = f_s * (floor(x/M) - 2^12) + E  (mod 2^32).
__device__ __forceinline__ uint32_t decode_update(uint32_t x, uint32_t e) {
    return (e >> 20) * ((x >> kLog2M) + (0u - (1u << kLog2M))) + (e >> 8);
}

// Shared-memory loads by 32-bit shared address.  The slot table does not
// change after it is built; the ring is rewritten by TMA, so its loads stay
// ordered after the mbarrier waits (volatile).
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

__device__ void build_slot_table(const DecodeParams &p, uint32_t *tab, uint32_t *cum) {
    const uint32_t tid = threadIdx.x;
    if (tid < 32) {
        // cum[s] = f_0 + ... + f_{s-1}: 8 symbols per lane, then a warp scan.
        uint32_t v[8], run = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            v[k] = run;
            run += p.freq[tid * 8 + k];
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
    for (uint32_t slot = tid; slot < kM; slot += blockDim.x) {
        // largest s with cum[s] <= slot (symbols with f = 0 have cum[s] = cum[s+1])
        uint32_t lo = 0, hi = 256;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (cum[mid] <= slot) lo = mid;
            else hi = mid;
        }
        const uint32_t f = cum[lo + 1] - cum[lo];
        tab[slot] = (f << 20) | ((slot - cum[lo]) << 8) | lo;
    }
    __syncthreads();
}

__device__ bool header_ok(const DecodeParams &p) {
    const uint8_t *h = p.msg;
    const uint32_t *h32 = reinterpret_cast<const uint32_t *>(h);
    const uint64_t n_sym = uint64_t(h32[4]) | (uint64_t(h32[5]) << 32);
    if (h32[0] != RANS_MAGIC || h32[1] != RANS_VERSION || h32[2] != p.N || h32[3] != kLog2M ||
        n_sym != p.n_sym || h32[6] != p.CS || h32[7] != p.n_chunks)
        return false;
    const uint32_t first = h32[8], last = h32[8 + p.n_chunks];
    return first == 0 && round16(last) == p.msg_size - p.data0;
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

template <int NT>  // NT = 32: every chunk uses all 32 lanes; NT = 0: runtime N
__global__ void __launch_bounds__(kWarps * 32)
    decode_kernel(const __grid_constant__ DecodeParams p) {
    extern __shared__ __align__(128) uint8_t smem[];
    uint32_t *tab = reinterpret_cast<uint32_t *>(smem);
    const uint32_t raw = smem_addr(smem + kTableBytes);
    const uint32_t rings_s = (raw + kRing - 1) & ~(kRing - 1);
    uint8_t *rings = smem + kTableBytes + (rings_s - raw);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kTableBytes + kRing + kWarps * kRing);
    uint32_t &hdr_ok = *reinterpret_cast<uint32_t *>(bars + kWarps * kNSeg);

    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    const uint32_t N = NT ? NT : p.N;

    if (threadIdx.x == 0) hdr_ok = header_ok(p) ? 1u : 0u;
    if (p.const_sym == 0xFFFFFFFFu)
        build_slot_table(p, tab, reinterpret_cast<uint32_t *>(rings));  // rings unused yet
    else
        __syncthreads();
    if (!hdr_ok) {
        if (threadIdx.x == 0) report(p.status, RANS_ERR_CORRUPT);
        return;
    }

    const uint32_t ring_s = rings_s + warp * kRing;
    const uint32_t tab_s = smem_addr(tab);
    const uint32_t bar0 = smem_addr(bars + warp * kNSeg);
    if (lane == 0) {
        for (uint32_t i = 0; i < kNSeg; ++i) mbar_init(bar0 + 8 * i, 1);
        fence_mbar_init();
    }
    __syncwarp();

    const uint32_t *offs = reinterpret_cast<const uint32_t *>(p.msg + 32);
    const uint32_t data_end = offs[p.n_chunks];
    const uint32_t lt = lanemask_lt();
    uint32_t phase = 0;  // bit i: parity of the next wait on barrier i
    uint32_t timeouts = 0;

    for (uint32_t c = blockIdx.x * kWarps + warp; c < p.n_chunks; c += gridDim.x * kWarps) {
        const uint32_t o = offs[c], e = offs[c + 1];
        const uint64_t first = uint64_t(c) * p.CS;
        const uint32_t n_c = uint32_t(umin64(p.CS, p.n_sym - first));
        // Offsets must be even (states and words are 2-byte aligned) and in range.
        if (((o | e) & 1u) || e < o || e > data_end || e - o < 4 * N) {
            if (lane == 0) report(p.status, RANS_ERR_CORRUPT);
            continue;
        }
        const uint8_t *chunk = p.msg + p.data0 + o;
        uint32_t x = kL;
        if (lane < N)
            x = ld_u16_global(chunk + 4 * lane) | (ld_u16_global(chunk + 4 * lane + 2) << 16);
        if (!__all_sync(kFull, x >= kL)) {  // Algorithm 1 requires x in I
            if (lane == 0) report(p.status, RANS_ERR_CORRUPT);
            continue;
        }
        uint8_t *outp = p.out + first + lane;

        if (p.const_sym != 0xFFFFFFFFu) {
            // f = M: C is the identity; the chunk is N states equal to L.
            if (e - o != 4 * N || !__all_sync(kFull, x == kL)) {
                if (lane == 0) report(p.status, RANS_ERR_CORRUPT);
            }
            for (uint32_t i = lane; i < n_c; i += 32) p.out[first + i] = uint8_t(p.const_sym);
            continue;
        }

        // Word stream: bytes [P0, P1) of the message, loaded in 512-byte
        // segments starting at the 16-byte aligned A <= P0; byte P of the
        // stream lives at ring offset (P - A) mod 4096.
        const uint64_t P0 = uint64_t(p.data0) + o + 4 * N, P1 = uint64_t(p.data0) + e;
        const uint64_t A = P0 & ~uint64_t(15);
        const uint64_t end16 = round16(P1);
        const uint32_t nseg = uint32_t((end16 - A + kSeg - 1) / kSeg);
        const uint32_t endrel = uint32_t(P1 - A);
        uint32_t rp = uint32_t(P0 - A);
        uint32_t issued = 0, ready = 0, recheck = 0;

        // Issue every segment whose ring slot is free (its previous segment
        // lies wholly below rp), wait until the next group's bytes
        // [rp, rp + 1 KiB) are in, and compute the read position at which
        // either can change again.
        auto service = [&]() {
            const uint32_t limit = min(nseg, kNSeg + rp / kSeg);
            for (; issued < limit; ++issued) {
                if (lane == 0) {
                    const uint32_t slot = issued % kNSeg;
                    const uint64_t src = A + uint64_t(issued) * kSeg;
                    const uint32_t bytes = uint32_t(umin64(kSeg, end16 - src));
                    mbar_arrive_expect_tx(bar0 + 8 * slot, bytes);
                    bulk_g2s(ring_s + slot * kSeg, p.msg + src, bytes, bar0 + 8 * slot);
                }
            }
            const uint32_t need = min(nseg, (rp + kGroup * 64 + kSeg - 1) / kSeg);
            for (; ready < need; ++ready) {
                const uint32_t slot = ready % kNSeg;
                const bool ok =
                    timeouts != 0 || mbar_wait_bounded(bar0 + 8 * slot, (phase >> slot) & 1u);
                if (__any_sync(kFull, !ok)) timeouts = 1;  // warp-uniform
                phase ^= 1u << slot;
            }
            const uint32_t r_ready =
                ready >= nseg ? 0xFFFFFFFFu
                              : (ready * kSeg >= kGroup * 64 ? ready * kSeg - kGroup * 64 + 1 : 0u);
            const uint32_t r_issue =
                issued >= nseg ? 0xFFFFFFFFu
                               : (issued + 1 >= kNSeg ? (issued + 1 - kNSeg) * kSeg : 0u);
            recheck = min(r_ready, r_issue);
        };

        const uint32_t T_full = n_c / N, rem = n_c % N;
        const bool lane_on = lane < N;
        uint32_t t = 0;
        for (; t + kGroup <= T_full; t += kGroup) {
            if (rp >= recheck) service();
#pragma unroll
            for (uint32_t u = 0; u < kGroup; ++u)
                decode_step<NT == 32>(x, rp, lane_on, tab_s, ring_s, outp + u * N, lt);
            outp += kGroup * N;
        }
        for (; t < T_full; ++t) {
            service();
            decode_step<NT == 32>(x, rp, lane_on, tab_s, ring_s, outp, lt);
            outp += N;
        }
        if (rem) {
            service();
            decode_step<false>(x, rp, lane < rem, tab_s, ring_s, outp, lt);
        }
        // Drain the copies still in flight so that the ring and the barrier
        // phases are clean for the next chunk.
        for (; ready < issued; ++ready) {
            const uint32_t slot = ready % kNSeg;
            const bool ok =
                timeouts != 0 || mbar_wait_bounded(bar0 + 8 * slot, (phase >> slot) & 1u);
            if (__any_sync(kFull, !ok)) timeouts = 1;
            phase ^= 1u << slot;
        }
        // A well-formed chunk ends with every coder back at x0 = L and every
        // word read exactly once (decoder and encoder in lockstep, Section 3).
        const bool ok = __all_sync(kFull, !lane_on || x == kL) && rp == endrel;
        if (!ok && lane == 0) report(p.status, RANS_ERR_CORRUPT);
        if (timeouts) break;
    }
    if (timeouts && lane == 0) report(p.status, RANS_ERR_TIMEOUT);
}

template <int NT>
int launch_decode(const DecodeParams &p, cudaStream_t stream) {
    static bool configured[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !configured[dev]) {
        if (cudaFuncSetAttribute(decode_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(kSmemBytes)) != cudaSuccess)
            return RANS_ERR_CUDA;
        configured[dev] = true;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, decode_kernel<NT>, kWarps * 32,
                                                      kSmemBytes) != cudaSuccess ||
        per_sm <= 0)
        return RANS_ERR_CUDA;
    const uint64_t want = ceil_div(p.n_chunks, kWarps);
    const uint64_t cap = uint64_t(per_sm) * sm_count();
    const unsigned grid = unsigned(std::max<uint64_t>(1, std::min(want, cap)));
    decode_kernel<NT><<<grid, kWarps * 32, kSmemBytes, stream>>>(p);
    return check_launch();
}

}  // namespace
}  // namespace rans

using namespace rans;

extern "C" int rans_decode(const uint8_t *d_msg, uint64_t msg_size, const uint16_t *h_freq,
                           uint32_t n_alpha, const rans_params *params, uint8_t *d_symbols,
                           uint64_t n_symbols, uint32_t *d_status, rans_stream_t stream) {
    uint32_t const_sym = 0xFFFFFFFFu;
    if (!d_msg || !d_status || !params_ok(params) || !table_ok(h_freq, n_alpha, &const_sym))
        return RANS_ERR_INVALID_ARG;
    if (n_symbols && !d_symbols) return RANS_ERR_INVALID_ARG;
    const MessageGeometry g = geometry(n_symbols, params);
    if (g.n_chunks > 0xFFFFFFFEull) return RANS_ERR_INVALID_ARG;
    if (msg_size < g.data0 || (msg_size & 15u) || !aligned16(d_msg) || msg_size < 48 ||
        msg_size - g.data0 > 0xFFFFFFFFull + 15)
        return RANS_ERR_INVALID_ARG;

    DecodeParams p{};
    p.msg = d_msg;
    p.out = d_symbols;
    p.status = d_status;
    p.msg_size = msg_size;
    p.n_sym = n_symbols;
    p.N = params->n_lanes;
    p.CS = params->chunk_symbols;
    p.n_chunks = uint32_t(g.n_chunks);
    p.data0 = uint32_t(g.data0);
    p.const_sym = const_sym;
    for (uint32_t s = 0; s < n_alpha; ++s) p.freq[s] = h_freq[s];

    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(d_status, 0, sizeof(uint32_t), st) != cudaSuccess) return RANS_ERR_CUDA;
    return p.N == 32 ? launch_decode<32>(p, st) : launch_decode<0>(p, st);
}
