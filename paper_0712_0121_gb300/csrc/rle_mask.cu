// Erosion and dilation of RLE images by an arbitrary structuring element
// (section "Morphology with Arbitrary Masks", applied run at a time to the
// run-length form).  The element is a list of horizontal runs; a run of the
// element is a within-line erosion / dilation by a segment, shifted to the
// element row's line, and the operation is the union (dilation) or the
// intersection (erosion) of those over the element's runs.
//
// Both are computed as a union of painted intervals:
//  * dilation: element run j, columns [i0, i1): the image line y - j + oy
//    contributes, for each of its runs [s, e), the pixels
//    [s + i0 - ox, e + i1 - 1 - ox) of output line y;
//  * erosion (clipped window, outside = 1): by duality the complement of
//    the dilation of the complement by the reflected element — each GAP
//    [s, e) between the runs of line y + j - oy (and the gaps at either end
//    of the line; outside the image is not a gap) contributes
//    [s - (i1 - 1) + ox, e - i0 + ox), and the output line is the
//    complement of that union.
// The host turns both cases into (dy, lo, hi): source line y + dy, paint
// [a + lo, b + hi) for each interval [a, b) (runs, or gaps for an erosion).
//
// One warp per output line: the line's words in shared memory start empty,
// the lanes take the intervals of each source line and OR them in (end words
// with atomicOr, inner words stored whole — every writer of a word then
// leaves it all ones, in any order; long stretches of inner words are
// stored by the whole warp, so a near-blank line's one long gap costs its
// words / 32 per lane), and the line leaves as packed words (complemented
// for an erosion, padding bits 0); the caller encodes the bitmap into runs.
#include "mask.cuh"

namespace morph {
namespace {

constexpr int RM_THREADS = 256;
constexpr int RM_MAX_WORDS = 12288;  // shared words of one CTA (48 KB)

__global__ void __launch_bounds__(RM_THREADS) k_rle_mask(const __grid_constant__ RleMaskArgs a) {
    extern __shared__ uint32_t rsm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wpc = blockDim.x >> 5;
    const int nw = a.nw;
    uint32_t *row = rsm + (size_t)warp * nw;
    const bool gaps = a.erode != 0;
    for (int y = blockIdx.x * wpc + warp; y < a.H; y += gridDim.x * wpc) {
        for (int k = lane; k < nw; k += 32) row[k] = 0u;
        __syncwarp();
        for (int u = 0; u < a.nruns; ++u) {
            const RleMaskRun run = a.runs[u];
            const int r = y + run.dy;
            if (r < 0 || r >= a.H) continue;  // no pixel of the element's line there
            const int k0 = a.row_ptr[r], n = a.row_ptr[r + 1] - k0;
            const int nint = gaps ? n + 1 : n;
            // the same trip count for every lane (the warp votes below)
            for (int base = 0; base < nint; base += 32) {
                const int k = base + lane;
                int fw0 = 0, fw1 = 0;  // the interval's inner (whole) words
                if (k < nint) {
                    int lo, hi;
                    if (gaps) {
                        lo = k == 0 ? 0 : (int)a.runs_u16[2 * (k0 + k - 1) + 1];
                        hi = k == n ? a.W : (int)a.runs_u16[2 * (k0 + k)];
                    } else {
                        lo = a.runs_u16[2 * (k0 + k)];
                        hi = a.runs_u16[2 * (k0 + k) + 1];
                    }
                    int p = lo + run.lo, q = hi + run.hi;  // an empty gap gives p >= q
                    p = p < 0 ? 0 : p;
                    q = q > a.W ? a.W : q;
                    if (lo < hi && p < q) {
                        // pixels [p, q): the end words by this lane
                        const int w0 = p >> 5, w1 = (q - 1) >> 5;
                        const uint32_t m0 = ONES << (p & 31), m1 = ONES >> (31 - ((q - 1) & 31));
                        if (w0 == w1) {
                            atomicOr(row + w0, m0 & m1);
                        } else {
                            atomicOr(row + w0, m0);
                            atomicOr(row + w1, m1);
                            fw0 = w0 + 1;
                            fw1 = w1;
                        }
                    }
                }
                // inner words: a few by the lane, long stretches by the warp
                if (fw1 - fw0 <= 4) {
                    for (int w = fw0; w < fw1; ++w) row[w] = ONES;
                    fw1 = fw0;
                }
                unsigned long_ones = __ballot_sync(0xffffffffu, fw1 > fw0);
                while (long_ones) {
                    const int src = __ffs(long_ones) - 1;
                    long_ones &= long_ones - 1;
                    const int b0 = __shfl_sync(0xffffffffu, fw0, src), b1 = __shfl_sync(0xffffffffu, fw1, src);
                    for (int w = b0 + lane; w < b1; w += 32) row[w] = ONES;
                }
            }
        }
        __syncwarp();
        const uint32_t inv = gaps ? ONES : 0u;
        uint32_t *out = a.dst + (int64_t)y * a.dstride;
        for (int k = lane; k < nw; k += 32) out[k] = (row[k] ^ inv) & word_mask(k, a.W);
        __syncwarp();
    }
}

}  // namespace

int rle_mask_warps(int nw) {
    int w = RM_MAX_WORDS / (nw > 0 ? nw : 1);
    if (w > RM_THREADS / 32) w = RM_THREADS / 32;
    return w;
}

cudaError_t launch_rle_mask_stage(const RleMaskArgs &a, cudaStream_t s) {
    const int wpc = rle_mask_warps(a.nw);
    if (wpc < 1) return cudaErrorInvalidValue;  // a line longer than the shared memory
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const size_t smem = (size_t)wpc * a.nw * sizeof(uint32_t);
    int grid = (a.H + wpc - 1) / wpc;
    const int cap = sms * 8;  // a few waves of resident CTAs; CTAs stride over the lines
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    k_rle_mask<<<grid, wpc * 32, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace morph
