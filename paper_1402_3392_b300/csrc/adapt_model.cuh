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
// nm = M - n.
template <int NB>
__device__ __forceinline__ void update(uint32_t *cm, const bool *le, uint32_t nm) {
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        const uint32_t b = uint32_t(i + 1);
        const uint32_t d = (le[i] ? cm[i] - b : nm + b - cm[i]) >> kRate;
        cm[i] = le[i] ? cm[i] - d : cm[i] + d;
    }
}

}  // namespace adapt
}  // namespace rans
