// Skewing packed rows (section "Scaling, Skewing, and Rotation": a skew moves
// every line by its own offset) for morphology with sheared line elements
// (section "Morphology with Lines at Arbitrary Orientations": skew, erode by
// an axis-parallel line, skew back).  One warp per piece of an output row
// (SHIFT_PIECE words), a lane per output word: the word is a funnel shift
// of the two source words it straddles, source positions outside the source
// row take the fill value, bits past the output width are 0.
#include "morph_internal.cuh"

namespace morph {
namespace {

constexpr int SHIFT_PIECE = 256;  // output words per warp item (long rows split)

// valid-bit mask of an output word whose bit b reads source position q0 + b:
// the bits with 0 <= q0 + b < n
__device__ __forceinline__ uint32_t src_range_mask(int64_t q0, int n) {
    const int64_t lo = q0 < 0 ? -q0 : 0;
    const int64_t hi = (int64_t)n - q0 < 32 ? (int64_t)n - q0 : 32;
    if (hi <= lo) return 0u;
    const uint32_t upto = hi >= 32 ? ONES : ((1u << hi) - 1u);
    return upto & ~((lo >= 32) ? ONES : ((1u << lo) - 1u));
}

// Skew into (sign > 0) or out of (sign < 0) a stack of band canvases: band b
// holds image lines b*band - halo .. b*band + band + halo - 1 (lines outside
// the image are rows of fill), each moved right by shift[y] - base[b].
//   skew:   dst = canvas rows (nb * (band + 2 halo)), src = the image;
//   unskew: dst = image lines, src = canvas rows (line y at its band's
//           interior row).
// Output pixel p of a row reads source pixel p - a of its source row.
__global__ void __launch_bounds__(256) k_shift_rows(const uint32_t *src, int64_t sstride, int src_bits,
                                                    uint32_t *dst, int64_t dstride, int dst_bits, int nw_dst,
                                                    int rows, int H, const int32_t *shift, const int32_t *base,
                                                    int band, int halo, int sign, uint32_t fill) {
    const int nw_src = (src_bits + 31) / 32;
    const int brows = band + 2 * halo;
    const int lane = threadIdx.x & 31;
    const int warps = (int)((gridDim.x * blockDim.x) >> 5);
    // one warp per piece of SHIFT_PIECE words of an output row, its lanes
    // over the piece's words
    const int pieces = (nw_dst + SHIFT_PIECE - 1) / SHIFT_PIECE;
    const int64_t items = (int64_t)rows * pieces;
    for (int64_t item = (int64_t)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); item < items; item += warps) {
        const int row = (int)(item / pieces);
        const int k0 = (int)(item - (int64_t)row * pieces) * SHIFT_PIECE;
        const int k1 = min(nw_dst, k0 + SHIFT_PIECE);
        int srow, a;
        if (sign > 0) {
            const int b = row / brows, y = b * band - halo + (row - b * brows);
            if (y < 0 || y >= H) {
                for (int k = k0 + lane; k < k1; k += 32)
                    dst[(int64_t)row * dstride + k] = fill & word_mask(k, dst_bits);
                continue;
            }
            srow = y;
            a = shift[y] - base[b];
        } else {
            const int b = row / band;
            srow = b * brows + halo + (row - b * band);
            a = base[b] - shift[row];
        }
        const uint32_t *rp = src + (int64_t)srow * sstride;
        uint32_t *dp = dst + (int64_t)row * dstride;
        for (int k = k0 + lane; k < k1; k += 32) {
            const int64_t q0 = 32 * (int64_t)k - a;
            const int64_t wi = q0 >> 5;  // floor(q0 / 32): arithmetic shift
            const int r = (int)(q0 & 31);
            const uint32_t w0 = (wi >= 0 && wi < nw_src) ? rp[wi] : 0u;
            const uint32_t w1 = (wi + 1 >= 0 && wi + 1 < nw_src) ? rp[wi + 1] : 0u;
            const uint32_t v = r ? ((w0 >> r) | (w1 << (32 - r))) : w0;
            const uint32_t m = src_range_mask(q0, src_bits);
            dp[k] = ((v & m) | (fill & ~m)) & word_mask(k, dst_bits);
        }
    }
}

}  // namespace

cudaError_t launch_shift_rows(const uint32_t *src, int64_t sstride, int src_bits, uint32_t *dst,
                              int64_t dstride, int dst_bits, int nw_dst, int rows, int H, const int32_t *shift,
                              const int32_t *base, int band, int halo, int sign, uint32_t fill,
                              cudaStream_t s) {
    const int64_t items = (int64_t)rows * ((nw_dst + SHIFT_PIECE - 1) / SHIFT_PIECE);
    int64_t g = (items + 7) / 8;  // 8 warps per CTA, one piece each
    if (g > 152 * 16) g = 152 * 16;
    if (g < 1) g = 1;
    k_shift_rows<<<(int)g, 256, 0, s>>>(src, sstride, src_bits, dst, dstride, dst_bits, nw_dst, rows, H, shift,
                                        base, band, halo, sign, fill);
    return cudaGetLastError();
}

}  // namespace morph
