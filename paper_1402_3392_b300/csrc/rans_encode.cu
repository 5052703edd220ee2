// rans_encode.cu -- GPU encoder: one warp encodes one chunk, one lane is one
// of the chunk's N interleaved rANS coders; then the chunks are packed into
// one message behind an offset table.
//
// The encoder runs over the chunk backwards, step T-1 down to 0 (Section 2:
// the encoder processes the message from last to first and writes backwards).
// Per step every lane with a symbol renormalizes at most once (b = 2^16 >= M,
// Section 5) and then applies C (Algorithm 1 Encode):
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
// stores (TMA) into a worst-case scratch slot per chunk.  A single-CTA kernel
// then scans the chunk sizes into the offset table and writes the header, and
// a copy kernel packs every chunk behind it.
#include <algorithm>
#include <mutex>

#include <cuda_runtime.h>

#include "device_util.cuh"
#include "host_util.h"

namespace rans {
namespace {

constexpr int kWarps = 8;
constexpr uint32_t kSeg = 512;
constexpr uint32_t kNSeg = 8;
constexpr uint32_t kRing = kSeg * kNSeg;  // 4 KiB per warp, aligned to 4 KiB in shared space
constexpr uint32_t kGroup = 16;
// A step writes at most 32 words = 64 bytes, so a group writes at most 1 KiB
// and touches at most three segments.
static_assert(kGroup * 64 <= 2 * kSeg, "a group must fit in two segments");
// layout: [encode table 2 KiB][alignment slack][ring per warp]
constexpr uint32_t kSmemBytes = 256 * 8 + kRing + kWarps * kRing;
constexpr uint32_t kZeroFlag = 1u << 19;  // encode-table bit marking f_s = 0

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
    uint16_t freq[RANS_MAX_ALPHABET];
};

// Scratch layout, all sections 16-byte aligned.
struct ScratchLayout {
    uint64_t words, states, wstart, sizes, total;
    uint32_t slot_bytes;
};

ScratchLayout scratch_layout(uint64_t n_chunks, uint32_t N, uint32_t CS) {
    ScratchLayout s{};
    s.slot_bytes = uint32_t(ceil_div(2ull * CS, kSeg) * kSeg);
    s.words = 0;
    s.states = round16(n_chunks * s.slot_bytes + 16);
    s.wstart = s.states + round16(n_chunks * N * 4);
    s.sizes = s.wstart + round16(n_chunks * 4);
    s.total = s.sizes + round16(n_chunks * 4);
    return s;
}

// Encode-table entry for symbol s with frequency f (1 <= f <= M):
//   .x = m_lo = ceil(2^(32+k) / f) - 2^32,  k = ceil(log2 f)   (0 <= m_lo < 2^32)
//   .y = (M - f) << 20 | k << 12 | B_s
// floor(x/f) = (x + umulhi(x, m_lo)) >> k for every x < 2^32: with
// m = 2^(32+k)/f + e, 0 <= e < 1, the error x*e/2^(32+k) < 2^-k <= 1/f never
// carries x/f past the next integer.
// Emit test: x >= f * 2^20  <=>  x > f * 2^20 - 1 = ~((M - f) << 20)  (u32).
__device__ void build_encode_table(const EncodeParams &p, uint2 *tab, uint32_t *cum) {
    const uint32_t tid = threadIdx.x;
    if (tid < 32) {
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
    }
    __syncthreads();
    for (uint32_t s = tid; s < 256; s += blockDim.x) {
        const uint32_t f = p.freq[s];
        uint2 t;
        if (f == 0) {
            t = make_uint2(0u, kZeroFlag);  // never emits, leaves x unchanged
        } else {
            const uint32_t k = 32u - __clz(f - 1u);
            const uint64_t m = ((1ull << (32 + k)) + f - 1) / f;
            t.x = uint32_t(m - (1ull << 32));
            t.y = ((kM - f) << 20) | (k << 12) | cum[s];
        }
        tab[s] = t;
    }
    __syncthreads();
}

__device__ __forceinline__ uint2 ld_enc_table(uint32_t a) {
    uint2 v;
    asm("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a));
    return v;
}
__device__ __forceinline__ void st_ring_u16(uint32_t a, uint32_t v) {
    asm volatile("st.shared.u16 [%0], %1;" ::"r"(a), "h"(uint16_t(v)) : "memory");
}

// Encode one step: renormalize (emit the low 16 bits if x >= f_s * 2^20), then
// x = C(s, x).  wp is the warp-uniform write position (bytes, counting down);
// ring_s is the warp's 4 KiB-aligned ring.
template <bool FULL>
__device__ __forceinline__ void encode_step(uint32_t &x, uint32_t &wp, uint32_t &acc, bool active,
                                            uint32_t s, uint32_t tab_s, uint32_t ring_s,
                                            uint32_t ge) {
    const uint2 t = ld_enc_table(tab_s + (s << 3));
    const bool on = FULL || active;
    if (on) acc |= t.y;
    const bool emit = on && (x > ~(t.y & 0xFFF00000u));
    const uint32_t m = __ballot_sync(kFull, emit);
    if (emit) {
        st_ring_u16(((wp - 2u * __popc(m & ge)) & (kRing - 1)) | ring_s, x);
        x >>= 16;
    }
    wp -= 2u * __popc(m);
    if (on) {
        // floor(x / f) = (x + umulhi(x, m_lo)) >> k with a 33-bit sum
        const uint64_t sum = uint64_t(x) + __umulhi(x, t.x);
        const uint32_t q = __funnelshift_r(uint32_t(sum), uint32_t(sum >> 32), t.y >> 12);
        x = x + q * (t.y >> 20) + (t.y & 0xFFFu);
    }
}

template <int NT>
__global__ void __launch_bounds__(kWarps * 32)
    encode_kernel(const __grid_constant__ EncodeParams p) {
    extern __shared__ __align__(128) uint8_t smem[];
    uint2 *tab = reinterpret_cast<uint2 *>(smem);
    const uint32_t raw = smem_addr(smem + 256 * 8);
    const uint32_t rings_s = (raw + kRing - 1) & ~(kRing - 1);
    uint8_t *rings = smem + 256 * 8 + (rings_s - raw);

    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    const uint32_t N = NT ? NT : p.N;
    build_encode_table(p, tab, reinterpret_cast<uint32_t *>(rings));

    const uint32_t ring_s = rings_s + warp * kRing;
    const uint32_t tab_s = smem_addr(tab);
    const uint32_t ge = lanemask_ge();
    uint32_t acc = 0;

    for (uint32_t c = blockIdx.x * kWarps + warp; c < p.n_chunks; c += gridDim.x * kWarps) {
        const uint64_t first = uint64_t(c) * p.CS;
        const uint32_t n_c = uint32_t(umin64(p.CS, p.n_sym - first));
        const uint8_t *symp = p.sym + first + lane;
        uint8_t *slot_base = p.words + uint64_t(c) * p.slot_bytes;
        uint32_t x = kL;
        uint32_t wp = p.slot_bytes;                 // words occupy [wp, slot_bytes)
        uint32_t flushed = p.slot_bytes / kSeg;     // segments >= flushed are stored

        // Store every segment that lies entirely at or above wp.  The next
        // group writes into the segments holding wp-1 .. wp-1024, whose ring
        // slots last held segments at least five newer stores back.  wp and
        // flushed are warp-uniform; only lane 0 issues and waits.
        auto service = [&]() {
            const uint32_t done = (wp + kSeg - 1) / kSeg;
            if (flushed > done) {
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) {
                    for (uint32_t sg = flushed; sg > done;) {
                        --sg;
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
        const bool lane_on = lane < N;
        if (rem) {
            const bool act = lane < rem;
            const uint32_t s = act ? symp[uint64_t(T_full) * N] : 0u;
            encode_step<false>(x, wp, acc, act, s, tab_s, ring_s, ge);
        }
        int64_t t = int64_t(T_full) - 1;
        for (uint32_t r = T_full % kGroup; r > 0; --r, --t) {
            service();
            const uint32_t s = lane_on ? symp[uint64_t(t) * N] : 0u;
            encode_step<NT == 32>(x, wp, acc, lane_on, s, tab_s, ring_s, ge);
        }
        // Groups of kGroup steps, symbols of the next group loaded ahead.
        uint32_t cur[kGroup], nxt[kGroup];
        if (t >= 0) {
#pragma unroll
            for (uint32_t u = 0; u < kGroup; ++u)
                cur[u] = lane_on ? symp[uint64_t(t - u) * N] : 0u;
        }
        for (; t >= 0; t -= kGroup) {
            const int64_t tn = t - int64_t(kGroup);
#pragma unroll
            for (uint32_t u = 0; u < kGroup; ++u)
                nxt[u] = (tn >= 0 && lane_on) ? symp[uint64_t(tn - u) * N] : 0u;
            service();
#pragma unroll
            for (uint32_t u = 0; u < kGroup; ++u)
                encode_step<NT == 32>(x, wp, acc, lane_on, cur[u], tab_s, ring_s, ge);
#pragma unroll
            for (uint32_t u = 0; u < kGroup; ++u) cur[u] = nxt[u];
        }

        // Store what is left: complete segments, then the partial one rounded
        // down to 16 bytes (bytes below wp are scratch garbage nobody reads).
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
            const uint32_t done = (wp + kSeg - 1) / kSeg;
            for (uint32_t sg = flushed; sg > done;) {
                --sg;
                bulk_s2g(slot_base + uint64_t(sg) * kSeg, ring_s + (sg % kNSeg) * kSeg, kSeg);
            }
            const uint32_t lo = wp & ~15u, hi = done * kSeg;
            if (lo < hi) bulk_s2g(slot_base + lo, ring_s + (lo & (kRing - 1)), hi - lo);
            bulk_commit();
            bulk_wait_read<0>();
            p.wstart[c] = wp;
            p.sizes[c] = 4 * N + (p.slot_bytes - wp);
        }
        __syncwarp();
        if (lane < N) p.states[uint64_t(c) * N + lane] = x;
    }
    // Symbols with f_s = 0 leave the table's flag bit in acc.
    if (__any_sync(kFull, acc & kZeroFlag) && lane == 0) report(p.status, RANS_ERR_ZERO_FREQ);
    if (lane == 0) bulk_wait<0>();
}

struct FinalizeParams {
    uint8_t *out;
    uint64_t *out_size;
    const uint32_t *sizes;
    const uint32_t *status;
    uint64_t n_sym;
    uint32_t N, CS, n_chunks, data0;
};

// One CTA: exclusive scan of the chunk sizes into the offset table, header,
// zero padding, and the message size.
constexpr int kScanThreads = 1024;
__global__ void __launch_bounds__(kScanThreads)
    finalize_kernel(const __grid_constant__ FinalizeParams p) {
    __shared__ uint32_t warp_sums[32];
    __shared__ uint32_t carry_s;
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (*p.status != RANS_OK) {
        if (tid == 0) *p.out_size = 0;
        return;
    }
    uint32_t *offs = reinterpret_cast<uint32_t *>(p.out + 32);
    if (tid == 0) carry_s = 0;
    __syncthreads();
    for (uint64_t base = 0; base < p.n_chunks; base += kScanThreads) {
        const uint64_t i = base + tid;
        const uint32_t v = i < p.n_chunks ? p.sizes[i] : 0u;
        uint32_t incl = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, incl, d);
            if (lane >= uint32_t(d)) incl += y;
        }
        if (lane == 31) warp_sums[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = warp_sums[lane], wi = w;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(kFull, wi, d);
                if (lane >= uint32_t(d)) wi += y;
            }
            warp_sums[lane] = wi - w;  // exclusive prefix of warp totals
        }
        __syncthreads();
        const uint32_t carry = carry_s;
        if (i < p.n_chunks) offs[i] = carry + warp_sums[warp] + incl - v;
        __syncthreads();
        if (tid == kScanThreads - 1) carry_s = carry + warp_sums[warp] + incl;
        __syncthreads();
    }
    if (tid == 0) {
        const uint32_t total = carry_s;
        uint32_t *h = reinterpret_cast<uint32_t *>(p.out);
        h[0] = RANS_MAGIC;
        h[1] = RANS_VERSION;
        h[2] = p.N;
        h[3] = kLog2M;
        h[4] = uint32_t(p.n_sym);
        h[5] = uint32_t(p.n_sym >> 32);
        h[6] = p.CS;
        h[7] = p.n_chunks;
        offs[p.n_chunks] = total;
        for (uint32_t b = 32 + 4 * (p.n_chunks + 1); b < p.data0; ++b) p.out[b] = 0;
        const uint64_t end = uint64_t(p.data0) + total;
        for (uint64_t b = end; b < round16(end); ++b) p.out[b] = 0;
        *p.out_size = round16(end);
    }
}

struct PackParams {
    uint8_t *out;
    const uint8_t *words;
    const uint32_t *states;
    const uint32_t *wstart;
    const uint32_t *status;
    uint32_t N, n_chunks, data0, slot_bytes;
};

// Copy chunk c (states, then words) to its place in the message.  The
// destination is only 2-byte aligned, so whole 16-byte destination blocks are
// assembled from two aligned 16-byte source loads and a funnel shift (the
// source-to-destination shift is the same for every block of a chunk); the
// partial blocks at both ends are written in 16-bit units.
constexpr int kPackThreads = 256;

template <int K>  // K = (source shift in bytes) / 4; rs = 8 * (shift mod 4)
__device__ __forceinline__ void pack_blocks(uint8_t *out, const uint8_t *src, uint64_t B0,
                                            uint64_t B1, uint64_t s_minus_d, uint32_t rs) {
    const bool need_hi = K > 0 || rs != 0;
    for (uint64_t B = B0 + 16ull * threadIdx.x; B < B1; B += 16ull * blockDim.x) {
        const uint64_t sa = (B + s_minus_d) & ~uint64_t(15);
        const uint4 v0 = *reinterpret_cast<const uint4 *>(src + sa);
        const uint4 v1 = need_hi ? *reinterpret_cast<const uint4 *>(src + sa + 16)
                                 : make_uint4(0u, 0u, 0u, 0u);
        const uint32_t w[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
        uint4 r;
        r.x = __funnelshift_r(w[K + 0], w[K + 1], rs);
        r.y = __funnelshift_r(w[K + 1], w[K + 2], rs);
        r.z = __funnelshift_r(w[K + 2], w[K + 3], rs);
        r.w = __funnelshift_r(w[K + 3], w[K + 4], rs);
        *reinterpret_cast<uint4 *>(out + B) = r;
    }
}

__global__ void __launch_bounds__(kPackThreads) pack_kernel(const __grid_constant__ PackParams p) {
    if (*p.status != RANS_OK) return;
    const uint32_t *offs = reinterpret_cast<const uint32_t *>(p.out + 32);
    for (uint32_t c = blockIdx.x; c < p.n_chunks; c += gridDim.x) {
        const uint64_t D = uint64_t(p.data0) + offs[c];
        uint16_t *dst16 = reinterpret_cast<uint16_t *>(p.out + D);
        const uint32_t *st = p.states + uint64_t(c) * p.N;
        for (uint32_t i = threadIdx.x; i < 2 * p.N; i += blockDim.x)
            dst16[i] = uint16_t(st[i >> 1] >> ((i & 1) * 16));
        // words: destination bytes [d0, d1), source bytes from s0 in p.words
        const uint64_t d0 = D + 4ull * p.N;
        const uint64_t s0 = uint64_t(c) * p.slot_bytes + p.wstart[c];
        const uint64_t d1 = d0 + (p.slot_bytes - p.wstart[c]);
        const uint64_t B0 = round16(d0), B1 = d1 & ~uint64_t(15);
        const uint64_t head_end = B0 < d1 ? B0 : d1;
        for (uint64_t b = d0 + 2ull * threadIdx.x; b < head_end; b += 2ull * blockDim.x)
            *reinterpret_cast<uint16_t *>(p.out + b) =
                *reinterpret_cast<const uint16_t *>(p.words + s0 + (b - d0));
        if (B0 < B1) {
            const uint64_t s_minus_d = s0 - d0;  // modulo 2^64
            const uint32_t sh = uint32_t(s_minus_d & 15u);
            const uint32_t rs = 8u * (sh & 3u);
            switch (sh >> 2) {
                case 0: pack_blocks<0>(p.out, p.words, B0, B1, s_minus_d, rs); break;
                case 1: pack_blocks<1>(p.out, p.words, B0, B1, s_minus_d, rs); break;
                case 2: pack_blocks<2>(p.out, p.words, B0, B1, s_minus_d, rs); break;
                default: pack_blocks<3>(p.out, p.words, B0, B1, s_minus_d, rs); break;
            }
        }
        const uint64_t tail_start = B1 > head_end ? B1 : head_end;
        for (uint64_t b = tail_start + 2ull * threadIdx.x; b < d1; b += 2ull * blockDim.x)
            *reinterpret_cast<uint16_t *>(p.out + b) =
                *reinterpret_cast<const uint16_t *>(p.words + s0 + (b - d0));
    }
}

template <int NT>
int launch_encode(const EncodeParams &p, cudaStream_t stream) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, encode_kernel<NT>, kWarps * 32,
                                                      kSmemBytes) != cudaSuccess ||
        per_sm <= 0)
        return RANS_ERR_CUDA;
    const uint64_t want = ceil_div(p.n_chunks, kWarps);
    const uint64_t cap = uint64_t(per_sm) * sm_count();
    const unsigned grid = unsigned(std::max<uint64_t>(1, std::min(want, cap)));
    encode_kernel<NT><<<grid, kWarps * 32, kSmemBytes, stream>>>(p);
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

extern "C" int rans_encode(const uint8_t *d_symbols, uint64_t n_symbols, const uint16_t *h_freq,
                           uint32_t n_alpha, const rans_params *params, uint8_t *d_out,
                           uint64_t out_cap, uint64_t *d_out_size, uint32_t *d_status,
                           void *d_scratch, uint64_t scratch_cap, rans_stream_t stream) {
    if (!params_ok(params) || !table_ok(h_freq, n_alpha, nullptr) || !d_out || !d_out_size ||
        !d_status || !d_scratch || !aligned16(d_out) || !aligned16(d_scratch))
        return RANS_ERR_INVALID_ARG;
    if (n_symbols && !d_symbols) return RANS_ERR_INVALID_ARG;
    const MessageGeometry g = geometry(n_symbols, params);
    // Offsets are u32: the worst-case data region must fit.
    if (g.n_chunks > 0xFFFFFFFEull ||
        4ull * params->n_lanes * g.n_chunks + 2ull * n_symbols > 0xFFFFFFF0ull)
        return RANS_ERR_INVALID_ARG;
    const ScratchLayout sl = scratch_layout(g.n_chunks, params->n_lanes, params->chunk_symbols);
    if (out_cap < rans_max_encoded_size(n_symbols, params) || scratch_cap < sl.total)
        return RANS_ERR_BUFFER_TOO_SMALL;

    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(d_status, 0, sizeof(uint32_t), st) != cudaSuccess) return RANS_ERR_CUDA;
    uint8_t *scr = static_cast<uint8_t *>(d_scratch);

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
    for (uint32_t s = 0; s < n_alpha; ++s) ep.freq[s] = h_freq[s];

    if (g.n_chunks > 0) {
        const int rc = ep.N == 32 ? launch_encode<32>(ep, st) : launch_encode<0>(ep, st);
        if (rc != RANS_OK) return rc;
    }
    FinalizeParams fp{};
    fp.out = d_out;
    fp.out_size = d_out_size;
    fp.sizes = ep.sizes;
    fp.status = d_status;
    fp.n_sym = n_symbols;
    fp.N = ep.N;
    fp.CS = ep.CS;
    fp.n_chunks = ep.n_chunks;
    fp.data0 = uint32_t(g.data0);
    finalize_kernel<<<1, kScanThreads, 0, st>>>(fp);
    if (check_launch() != RANS_OK) return RANS_ERR_CUDA;
    if (g.n_chunks > 0) {
        PackParams pp{};
        pp.out = d_out;
        pp.words = ep.words;
        pp.states = ep.states;
        pp.wstart = ep.wstart;
        pp.status = d_status;
        pp.N = ep.N;
        pp.n_chunks = ep.n_chunks;
        pp.data0 = fp.data0;
        pp.slot_bytes = ep.slot_bytes;
        const unsigned grid = unsigned(std::min<uint64_t>(g.n_chunks, 65535ull * 8));
        pack_kernel<<<grid, kPackThreads, 0, st>>>(pp);
        if (check_launch() != RANS_OK) return RANS_ERR_CUDA;
    }
    return RANS_OK;
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
// kernel.
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
    if (!params_ok(params) || !table_ok(h_freq, n_alpha, nullptr) || !d_out || !d_out_size ||
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

    // Nothing in the scratch has to start at zero: the coder writes every
    // word, state, size and offset before the later kernels read them.
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
    for (uint32_t s = 0; s < n_alpha; ++s) ep.freq[s] = h_freq[s];
    if (g.n_chunks > 0) {
        const int rc = ep.N == 32 ? launch_encode<32>(ep, st) : launch_encode<0>(ep, st);
        if (rc != RANS_OK) return rc;
    }
    FinalizeParams fp{};
    fp.out = d_out;
    fp.out_size = d_out_size;
    fp.sizes = ep.sizes;
    fp.status = d_status;
    fp.n_sym = n_symbols;
    fp.N = ep.N;
    fp.CS = ep.CS;
    fp.n_chunks = ep.n_chunks;
    fp.data0 = uint32_t(g.data0);
    finalize_kernel<<<1, kScanThreads, 0, st>>>(fp);
    if (check_launch() != RANS_OK) return RANS_ERR_CUDA;
    if (g.n_chunks > 0) {
        PackParams pp{};
        pp.out = d_out;
        pp.words = ep.words;
        pp.states = ep.states;
        pp.wstart = ep.wstart;
        pp.status = d_status;
        pp.N = ep.N;
        pp.n_chunks = ep.n_chunks;
        pp.data0 = fp.data0;
        pp.slot_bytes = ep.slot_bytes;
        const unsigned grid = unsigned(std::min<uint64_t>(g.n_chunks, 65535ull * 8));
        pack_kernel<<<grid, kPackThreads, 0, st>>>(pp);
        if (check_launch() != RANS_OK) return RANS_ERR_CUDA;
    }
    return RANS_OK;
}
