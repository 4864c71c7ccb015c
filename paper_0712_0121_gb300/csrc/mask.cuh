// Arbitrary structuring elements on packed images (see mask.cu).
#pragma once

#include "morph_internal.cuh"

namespace morph {

// One stage = an erosion (AND form) by the element or a dilation (OR form)
// by the reflected element, given as horizontal runs.  A run of width w at
// element row j, columns [x0, x0 + w), origin (ox, oy): dy = j - oy,
// m = floor(log2 w), dx1 = x0 - ox, dx2 = dx1 + w - 2^m.
constexpr int MASK_MAX_RUNS = 1024;
constexpr int MASK_MAX_SIDE = 4096;   // element width and height limit
struct MaskRun {
    int16_t dy, dx1, dx2, m;
};
struct MaskArgs {
    const uint32_t *src;
    int64_t sstride;          // u32 words between source rows
    uint32_t *dst;
    int64_t dstride;          // u32 words between destination rows
    int nw_cover;             // u32 words written per destination row
    int W, H, nw_valid;
    int use_or;               // 0: erosion (AND, 1 outside), 1: dilation (OR, 0 outside)
    uint32_t *levels;         // doubling levels 1..nlev, rows of nw_valid + pad words
    int nlev, nruns;
    MaskRun runs[MASK_MAX_RUNS];
};
// Words kept left of a level row: a level looks right (A_2^m(p) covers
// p .. p+2^m-1), so positions down to -(2^m - 1) still reach the image.
__host__ __device__ inline int mask_pad_words(int nlev) { return ((1 << nlev) - 1 + 31) / 32; }
size_t mask_levels_bytes(int W, int H, int nlev);
cudaError_t launch_mask_stage(const MaskArgs &a, cudaStream_t s);

// One stage on an RLE image (rle_mask.cu): for each element run, source
// line y + dy, every interval [a, b) of that line (its runs, or for an
// erosion its gaps) paints [a + lo, b + hi) of output line y.
struct RleMaskRun {
    int32_t dy, lo, hi;
};
struct RleMaskArgs {
    const int32_t *row_ptr;   // source RLE
    const uint16_t *runs_u16;
    int W, H;
    uint32_t *dst;            // packed output lines (u32 words)
    int64_t dstride;
    int nw;                   // u32 words per line: (W + 31) / 32
    int erode;                // 1: paint the gaps, output the complement
    int nruns;
    RleMaskRun runs[MASK_MAX_RUNS];
};
// Warps (output lines) per CTA for lines of nw words; 0 when one line does
// not fit the CTA's shared memory.
int rle_mask_warps(int nw);
cudaError_t launch_rle_mask_stage(const RleMaskArgs &a, cudaStream_t s);

}  // namespace morph
