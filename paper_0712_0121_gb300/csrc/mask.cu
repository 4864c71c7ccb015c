// Erosion by an arbitrary structuring element on packed images (section
// "Morphology with Arbitrary Masks"): run at a time with doubling
// accumulation.  The element is a list of horizontal runs.  For the longest
// run width w_max, doubling levels A_1 = I', A_2s(p) = A_s(p) AND A_s(p + s)
// are built once per image (A_2^m(p) = AND of the 2^m pixels from p on);
// a run of width w at element row j and columns [x0, x0 + w) then
// contributes the AND of the image's pixels under it,
// A_2^m(x + dx1) AND A_2^m(x + dx2) with m = floor(log2 w), dx1 = x0 - ox
// and dx2 = dx1 + w - 2^m, taken on image row y + j - oy; the result is the
// AND of all runs' contributions.  I' is the stage input: the image
// (complemented for a dilation by duality) with 1 outside the image (the
// clipped window), so rows outside contribute nothing; a level word is all
// ones right of the row and far enough left of it (see lvl_word).
#include "morph_internal.cuh"

namespace morph {
namespace {

__device__ __forceinline__ int floor_div32(int v) { return v >= 0 ? v >> 5 : -((31 - v) >> 5); }

// Words of a level row: the level looks right (A(p) covers p .. p+2^m-1),
// so positions left of the image still see its first pixels: a level row
// keeps mask_pad_words(nlev) words left of word 0; further left, and right of
// the row, every word is all ones.
__device__ __forceinline__ int64_t lvl_index(const MaskArgs &a, int m, int r, int k) {
    const int pad = mask_pad_words(a.nlev);
    return ((int64_t)(m - 1) * a.H + r) * (a.nw_valid + pad) + pad + k;
}

// Word k of doubling level m, row r (m = 0: the stage input itself).
__device__ __forceinline__ uint32_t lvl_word(const MaskArgs &a, int m, int r, int k) {
    if (m == 0) {
        if (k < 0 || k >= a.nw_valid) return ONES;
        const uint32_t x = a.src[(int64_t)r * a.sstride + k];
        return (x ^ (a.inv_in ? ONES : 0u)) | ~word_mask(k, a.W);
    }
    if (k < -mask_pad_words(a.nlev) || k >= a.nw_valid) return ONES;
    return a.levels[lvl_index(a, m, r, k)];
}

// Bits [32k + off, 32k + off + 32) of level m, row r.
__device__ __forceinline__ uint32_t lvl_ext(const MaskArgs &a, int m, int r, int k, int off) {
    const int q = floor_div32(off), s = off - 32 * q;
    const uint32_t lo = lvl_word(a, m, r, k + q);
    if (s == 0) return lo;
    return __funnelshift_r(lo, lvl_word(a, m, r, k + q + 1), s);
}

// Level m from level m - 1: A_2s(p) = A_s(p) AND A_s(p + s), s = 2^(m-1),
// for the row's words and its left pad.
__global__ void __launch_bounds__(256) k_mask_level(const __grid_constant__ MaskArgs a, int m) {
    const int pad = mask_pad_words(a.nlev), lw = a.nw_valid + pad;
    const int64_t n = (int64_t)a.H * lw;
    const int s = 1 << (m - 1);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / lw), k = (int)(i - (int64_t)r * lw) - pad;
        a.levels[lvl_index(a, m, r, k)] = lvl_word(a, m - 1, r, k) & lvl_ext(a, m - 1, r, k, s);
    }
}

// Output word k of row y: AND over the runs; words past the row's pixels 0.
__global__ void __launch_bounds__(256) k_mask_acc(const __grid_constant__ MaskArgs a) {
    const int64_t n = (int64_t)a.H * a.nw_cover;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / a.nw_cover), k = (int)(i - (int64_t)y * a.nw_cover);
        uint32_t acc = ONES;
        if (k < a.nw_valid) {
            for (int t = 0; t < a.nruns && acc; ++t) {
                const MaskRun u = a.runs[t];
                const int r = y + u.dy;
                if (r < 0 || r >= a.H) continue;
                acc &= lvl_ext(a, u.m, r, k, u.dx1) & lvl_ext(a, u.m, r, k, u.dx2);
            }
        }
        const uint32_t mask = k < a.nw_valid ? word_mask(k, a.W) : 0u;
        a.dst[(int64_t)y * a.dstride + k] = (acc ^ (a.inv_out ? ONES : 0u)) & mask;
    }
}

int grid_for(int64_t n) {
    int64_t b = (n + 255) / 256;
    if (b > 152 * 8) b = 152 * 8;
    return b < 1 ? 1 : (int)b;
}

}  // namespace

size_t mask_levels_bytes(int W, int H, int nlev) {
    return (size_t)nlev * H * ((W + 31) / 32 + mask_pad_words(nlev)) * sizeof(uint32_t);
}

cudaError_t launch_mask_erode(const MaskArgs &a, cudaStream_t s) {
    for (int m = 1; m <= a.nlev; ++m) {
        k_mask_level<<<grid_for((int64_t)a.H * (a.nw_valid + mask_pad_words(a.nlev))), 256, 0, s>>>(a, m);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    k_mask_acc<<<grid_for((int64_t)a.H * a.nw_cover), 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace morph
