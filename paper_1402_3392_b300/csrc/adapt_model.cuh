// adapt_model.cuh -- the adaptive model over n symbols (2 <= n <= 16) that
// each coder of an adaptive-n message keeps for itself (Section 5: adaptive
// models vectorize as long as every lane updates only its own model).  Used
// by the encoder's forward pass (encode_core.cuh) and the decoder's step
// (decode_core.cuh).
//
// The model is the coder's cumulative frequencies C_1 < ... < C_{n-1}
// (C_0 = 0, C_n = M), held in registers as cm[0..NB) with cm[i] = C_{i+1}
// and every boundary at or above n pinned at M; f_s = C_{s+1} - C_s and
// B_s = C_s.  It starts at C_i = floor(i M / n) and, after symbol s, each
// boundary i moves towards i (i <= s) or towards M - n + i (i > s) by its
// distance >> kRate.  The map d -> d - (d >> kRate) is non-decreasing, so
// the gaps keep their order and every f_s stays >= 1; boundaries pinned at M
// stay there, their upward distance i - n being below 2^kRate.  NB (3, 7 or
// 15) is the register room: n <= NB + 1.
#pragma once

#include <cstdint>

#include "device_util.cuh"

namespace rans {
namespace adapt {

constexpr uint32_t kRate = 5;
constexpr uint32_t kNMax = 16;

template <int NB>
__device__ __forceinline__ void init(uint32_t *cm, uint32_t n) {
#pragma unroll
    for (int i = 0; i < NB; ++i) cm[i] = uint32_t(i + 1) < n ? (uint32_t(i + 1) * kM) / n : kM;
}

// le[i]: boundary i + 1 is at or below the coded symbol (it moves down).
// nm = M - n.  Two forms of the same update (equal over every model the
// update can reach: C_i in [i, M - n + i], boundaries at or above n at M).
// update: the distance to the target chosen by le, shifted, then added or
// subtracted.
template <int NB>
__device__ __forceinline__ void update(uint32_t *cm, const bool *le, uint32_t nm) {
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        const uint32_t b = uint32_t(i + 1);
        const uint32_t d = (le[i] ? cm[i] - b : nm + b - cm[i]) >> kRate;
        cm[i] = le[i] ? cm[i] - d : cm[i] + d;
    }
}
// update_signed: one signed difference v = C_i - t_i and an arithmetic shift.
// A boundary moving down has v = C_i - i >= 0 and C_i' = C_i - (v >> R).  A
// boundary moving up has u = M - n + i - C_i >= 0; with 2^R - 1 added, v = 2^R
// - 1 - u and v >> R (rounding down) = -(u >> R), so C_i' = C_i + (u >> R).
// Four operations a boundary instead of about seven.  Measured on B300 (256
// Mi symbols, n = 16): the decoder 2976 -> 1989 us; the encoder's forward
// pass was slower with it (2406 -> 2620 us), so it keeps update.
template <int NB>
__device__ __forceinline__ void update_signed(uint32_t *cm, const bool *le, uint32_t nm) {
    const uint32_t up = nm - ((1u << kRate) - 1u);
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        const uint32_t b = uint32_t(i + 1);
        const int32_t v = int32_t(cm[i] - b - (le[i] ? 0u : up));
        cm[i] = uint32_t(int32_t(cm[i]) - (v >> kRate));
    }
}

}  // namespace adapt
}  // namespace rans
