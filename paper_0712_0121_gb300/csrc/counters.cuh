// Bit-sliced column counters shared by the packed tile and the RLE
// between-line pass.
#pragma once

#include "morph_internal.cuh"

namespace morph {

// Bit-sliced counter of consecutive 1-rows; push returns "count >= sh".
// KMAX == 2 is only used for sh == 3 and keeps the last two rows instead:
// the AND of the window directly (c[0] = previous row, c[1] = the one before).
template <int KMAX>
struct ColCounter {
    uint32_t c[KMAX];
    uint32_t sat;
    __device__ __forceinline__ void reset() {
#pragma unroll
        for (int k = 0; k < KMAX; ++k) c[k] = 0;
        sat = 0;
    }
    __device__ __forceinline__ uint32_t push(uint32_t v, int K, const uint32_t (&eqm)[KMAX]) {
        if (KMAX == 2) {
            const uint32_t e = v & c[0] & c[1];
            c[1] = c[0];
            c[0] = v;
            return e;
        }
        uint32_t carry = v, eq = ONES;
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            if (k < K || KMAX <= 6) {  // planes above K stay zero and never match
                const uint32_t ck = c[k];
                const uint32_t nk = (ck ^ carry) & v;
                carry = ck & carry;
                c[k] = nk;
                eq &= nk ^ eqm[k];
            }
        }
        sat = v & (sat | eq);
        return sat;
    }
};

}  // namespace morph
