// Internal declarations shared by the translation units of libmorph.so.
// Device helpers for 32-bit bit strings, the argument blocks of each kernel
// family and the host-side launchers.  Nothing here is part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "morph.h"

namespace morph {

constexpr uint32_t ONES = 0xFFFFFFFFu;
constexpr int MAX_THREADS = 256;   // CTA size of the tile kernels

// Device-side status latch (first non-OK code wins), see abi.cu.
int *device_status_ptr();          // host: address of the status word on the current device

__device__ __forceinline__ void latch_status(int *st, int code) {
    if (st) atomicCAS(st, 0, code);
}

// Bits of a 32-bit word at positions >= n set (n in [0, 32]): the "padding"
// part of the last word of a row.
__host__ __device__ __forceinline__ uint32_t high_mask_from(int n) {
    return n >= 32 ? 0u : (ONES << n);
}
// Valid-pixel mask of u32 word k of a row of W pixels.
__host__ __device__ __forceinline__ uint32_t word_mask(int k, int W) {
    int rem = W - 32 * k;
    return rem >= 32 ? ONES : (rem <= 0 ? 0u : (ONES >> (32 - rem)));
}

// Inclusive prefix XOR of the bits of x from bit 0 upward: bit b of the
// result is the parity of bits 0..b of x.
__device__ __forceinline__ uint32_t prefix_xor(uint32_t x) {
    x ^= x << 1;
    x ^= x << 2;
    x ^= x << 4;
    x ^= x << 8;
    x ^= x << 16;
    return x;
}

// ------------------------------------------------------------- packed ---
// Parameters of the fused packed tile kernel.  Rows are read and written as
// 32-bit words (a PACKED64 row is the same little-endian bit string).
struct PackedArgs {
    const uint32_t *src;
    int64_t sstride;      // u32 words between source rows
    uint32_t *dst;
    int64_t dstride;      // u32 words between destination rows
    int W, H;
    int nw_valid;         // u32 words holding pixels: ceil(W / 32)
    int nw_cover;         // u32 words written per destination row (>= nw_valid)
    int sw, sh;           // rectangle
    int nst;              // 1 (erode / dilate) or 2 (open / close)
    int ex[2], ey[2];     // origin of the erosion in each stage
    int inv_in, inv_out;  // complement input / output (dilation by duality)
    int K;                // bit planes of the column counters
    uint32_t eqm[16];     // per plane: ONES where bit k of sh is 0, else 0
    int hmode;            // 0 none, 1 direct shifts, 2 doubling
    int m;                // doubling levels: floor(log2(sw))
    // tiling
    int tpr;              // threads per row group
    int groups;           // row groups per CTA
    int band;             // output rows per group
    int rb;               // rows per smem exchange chunk
    int strip_words;      // output words per column strip
    int halo_words;       // extra computed words on each side of a strip
    int nstrips;
    int slot_words;       // smem words per group row slot
};

int packed_halo(int sw, int ex);   // smem / register halo words of the H stage
cudaError_t launch_packed(PackedArgs &a, cudaStream_t s, int band_rows_hint);
int packed_plan(PackedArgs &a, int op, int sw, int sh, int ox, int oy, int band_rows_hint,
                int block_threads_hint);

// ----------------------------------------------------------------- RLE ---
struct RleIn {             // read-only view of an RLE image
    const int32_t *row_ptr;
    const uint16_t *runs;
    int W, H;
};

struct RleOut {
    int32_t *row_ptr;
    uint16_t *runs;
    int64_t capacity;
    int64_t *n_runs;
};

cudaError_t launch_rle_from_bitmap(const uint32_t *src, int64_t sstride, int W, int H,
                                   RleOut out, int32_t *counts, int *status, cudaStream_t s);
cudaError_t launch_rle_to_bitmap(RleIn in, uint32_t *dst, int64_t dstride, int nw_cover,
                                 cudaStream_t s);
// One erode (dilate=0) or dilate (dilate=1) of an RLE image by a sw x sh
// rectangle with origin (ox, oy).  counts: int32[H] scratch.
cudaError_t launch_rle_rect(RleIn in, RleOut out, int dilate, int sw, int sh, int ox, int oy,
                            int32_t *counts, int *status, cudaStream_t s);

}  // namespace morph
