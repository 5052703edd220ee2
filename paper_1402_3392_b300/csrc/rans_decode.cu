// rans_decode.cu -- single-message GPU decoder: one warp per chunk or per
// pair of consecutive chunks (chosen per launch from the chunk count), each
// chunk's N interleaved coders on the warp's lanes (decode_core.cuh), one
// slot table per CTA built from the message's model.
#include <algorithm>

#include <cuda_runtime.h>

#include "decode_core.cuh"
#include "host_util.h"

namespace rans {
namespace {

using dec::kSmemBytes;
using dec::kWarps;

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
    uint32_t per_warp;  // chunks a warp decodes side by side: 1 or dec::kChains
    uint16_t freq[RANS_MAX_ALPHABET];
};

template <int NT>  // NT = 32: every chunk uses all 32 lanes; NT = 0: runtime N
__global__ void __launch_bounds__(dec::kThreads)
    decode_kernel(const __grid_constant__ DecodeParams p) {
    extern __shared__ __align__(128) uint8_t smem[];
    const dec::Smem sm = dec::smem_layout(smem);
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    uint32_t &hdr_ok = sm.misc[0];
    uint32_t &const_sym = sm.misc[1];

    if (threadIdx.x == 0) {
        hdr_ok = dec::header_ok(p.msg, p.msg_size, p.data0, p.n_sym, p.N, p.CS, p.n_chunks);
        const_sym = dec::kNoConst;
    }
    dec::build_slot_table(p.freq, sm.tab, sm.rings, &const_sym);  // rings unused yet
    if (!hdr_ok) {
        if (threadIdx.x == 0) report(p.status, RANS_ERR_CORRUPT);
        return;
    }
    dec::WarpRings wr = dec::rings_init(sm, warp, lane);
    const uint32_t cs = const_sym;
    const uint32_t *offs = reinterpret_cast<const uint32_t *>(p.msg + 32);
    const uint32_t data_end = offs[p.n_chunks];
    const uint32_t lt = lanemask_lt();
    const uint32_t per = p.per_warp;
    const uint32_t n_units = (p.n_chunks + per - 1) / per;

    for (uint32_t q = blockIdx.x * kWarps + warp; q < n_units; q += gridDim.x * kWarps) {
        const uint32_t c = q * per;
        const uint32_t count = min(per, p.n_chunks - c);
        const uint32_t st =
            per > 1 ? dec::decode_chunks<NT, true>(wr, sm.tab_s, p.msg, p.data0, offs, data_end, c,
                                                   count, p.n_sym, p.CS, p.N, p.out, cs, lane, lt)
                    : dec::decode_chunks<NT, false>(wr, sm.tab_s, p.msg, p.data0, offs, data_end,
                                                    c, 1, p.n_sym, p.CS, p.N, p.out, cs, lane, lt);
        if (st != RANS_OK && lane == 0) report(p.status, st);
        if (wr.timeouts) break;
    }
}

// Chunks per warp for a message of n_chunks chunks when `warps` warps are
// resident.  A chunk is one chain of dependent steps, so a launch lasts at
// least one chunk's latency and its last wave leaves warps idle.  One chunk
// per warp streams through the warp's whole 4 KiB ring in 1 KiB copies; two
// chunks per warp overlap two chains but have 2 KiB rings (512-byte copies)
// and half the chains in flight.  Measured on a B300 (64 KiB chunks, N = 32;
// w = n_chunks / resident warps; times in us):
//   w      0.4  1.0  1.3  1.7  2.0  2.3  2.6  3.0  3.5  3.8   4.3   5.2
//   one    202  292  430  562  561  654  722  833  958  1102  1175  1448
//   two    271  331  431  561  560  658  758  905  1098 1100  1203  1384
uint32_t chunks_per_warp(uint64_t n_chunks, uint64_t warps) {
    return double(n_chunks) >= 5.0 * double(warps) ? dec::kChains : 1u;
}

template <int NT>
int launch_decode(DecodeParams &p, cudaStream_t stream) {
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
    const uint64_t cap = uint64_t(per_sm) * sm_count();
    p.per_warp = chunks_per_warp(p.n_chunks, cap * kWarps);
    const uint64_t want = ceil_div(p.n_chunks, uint64_t(kWarps) * p.per_warp);
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
    if (!d_msg || !d_status || !params_ok(params) || !table_ok(h_freq, n_alpha, nullptr))
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
    for (uint32_t s = 0; s < n_alpha; ++s) p.freq[s] = h_freq[s];

    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(d_status, 0, sizeof(uint32_t), st) != cudaSuccess) return RANS_ERR_CUDA;
    return p.N == 32 ? launch_decode<32>(p, st) : launch_decode<0>(p, st);
}
