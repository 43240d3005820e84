// fht_packed.cuh -- the first pass of a sum transform over a uint8 image
// (levels 0..m, m <= 6, into a uint16 level) on packed uint16 pairs.
//
// Every value of such a pass is a sum of at most 2^6 bytes (<= 16320), so two
// of them fit one 32-bit register and one 32-bit add adds both with no carry
// between the halves. A lane's 8 buffer columns are then 4 words, word j =
// columns 2j (low half) and 2j + 1 (high half). A shift by an even number of
// columns is a choice of words; by an odd number, one byte permute per word.
// This halves the adds and the warp shuffles of the butterfly, and the
// values go from the image bytes to the shared tile and on to the uint16
// level without being widened and narrowed again. The results are the
// integer sums of the recursion, identical to the generic item code's.
#pragma once

#include <cstdint>

namespace fht {

// Word j of a row shifted by s columns: ext holds the row's 4 words and then
// the next lane's (those a shift reaches).
template <int S>
__device__ __forceinline__ uint32_t shifted_word(const uint32_t (&ext)[8], int j) {
    constexpr int e = S >> 1;
    if constexpr ((S & 1) == 0) return ext[j + e];
    else return __byte_perm(ext[j + e], ext[j + e + 1], 0x5432u);
}

// MR levels on 2^MR rows x 4 packed words held by this lane (the packed form
// of reg_butterfly: the bottom row of a pair is read shifted by u and u + 1
// columns; columns past this lane's 8 come from lane + 1).
template <int MR>
__device__ __forceinline__ void reg_butterfly_u16x2(uint32_t (&v)[1 << MR][4]) {
    constexpr int R = 1 << MR;
#pragma unroll
    for (int half = 1; half < R; half *= 2) {
        uint32_t nv[R][4];
#pragma unroll
        for (int s0 = 0; s0 < R; s0 += 2 * half) {
#pragma unroll
            for (int u = 0; u < half; ++u) {
                const uint32_t *top = v[s0 + u];
                const uint32_t *bot = v[s0 + half + u];
                // highest extended word the shift by u + 1 reads, minus 3
                const int need = ((u + 1) >> 1) + ((u + 1) & 1);
                uint32_t ext[8];
#pragma unroll
                for (int j = 0; j < 4; ++j) ext[j] = bot[j];
#pragma unroll
                for (int j = 0; j < 4; ++j) ext[4 + j] = j < need ? shfl_next(bot[j]) : 0u;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    uint32_t b0, b1;
                    switch (u) {   // u is a compile-time constant after unrolling
                    case 0: b0 = shifted_word<0>(ext, j); b1 = shifted_word<1>(ext, j); break;
                    case 1: b0 = shifted_word<1>(ext, j); b1 = shifted_word<2>(ext, j); break;
                    case 2: b0 = shifted_word<2>(ext, j); b1 = shifted_word<3>(ext, j); break;
                    default: b0 = shifted_word<3>(ext, j); b1 = shifted_word<4>(ext, j); break;
                    }
                    nv[s0 + 2 * u][j] = top[j] + b0;
                    nv[s0 + 2 * u + 1][j] = top[j] + b1;
                }
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int j = 0; j < 4; ++j) v[r][j] = nv[r][j];
    }
}

}  // namespace fht
