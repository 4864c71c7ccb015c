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

// Message for morph_last_error() (printf-style), see abi.cu.
void set_error(const char *fmt, ...);

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

// Argument checks of the rectangle entry points (abi.cu), shared by every
// entry point that takes an operation, two images and a rectangle.
struct Se {
    int sw, sh, ox, oy;
};
// The rectangle clipped to what can reach inside a W x H image.
Se clip_se(int W, int H, int sw, int sh, int ox, int oy);
// Images valid, same size, both packed or both RLE, not overlapping; op a
// morph_op; rectangle 1..65535 on each side with the origin inside.  Sets
// the error message on failure.
morph_status check_op_args(int op, const morph_image *dst, const morph_image *src, int se_w, int se_h,
                           int ox, int oy);

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
    int nwt;              // u32 words per thread
    int ring;             // 1: ring tile (cp.async row slots), 0: register-prefetch tile
    int vec;              // vector loads / stores of a thread's words allowed (aligned bases and strides)
};

int packed_halo(int sw, int ex);   // register-window halo words of the H stage (0: too wide)
// kmax_class: the column-counter planes of the kernel set that will run the
// plan (the batch kernel instantiates fewer classes); -1 = packed_kmax().
// ring2: open / close use the ring tile (the batch kernel, with two CTAs
// per SM, runs them faster on the register-prefetch tile).
int packed_plan(PackedArgs &a, int op, int sw, int sh, int ox, int oy, int band_rows_hint,
                int block_threads_hint, int kmax_class = -1, bool ring2 = true);
size_t packed_smem_bytes(const PackedArgs &a);
int packed_kmax(const PackedArgs &a);
int packed_threads(const PackedArgs &a);
dim3 packed_grid(const PackedArgs &a);
cudaError_t launch_packed(PackedArgs &a, cudaStream_t s);

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

// Within-line run pass: erosion (dilate = 0, o = erosion origin) or dilation
// (dilate = 1, o = dilation origin) of every run by a width-sw segment.
struct RowOp {
    int dilate, sw, o, W;
};

// Between-line pass over an RLE image (see rle_tile.cuh).
struct VArgs {
    RleIn in;
    RowOp op;
    int inv;                 // complement before and after (dilation)
    int sh, ey, K;
    uint32_t eqm[16];
    int nw_ext;              // words covering positions 0..W
    int nwt;                 // words per thread (2 or 8)
    int tpr, groups, band, rb, slot_words;
    // Output, one of two modes:
    //  bitmap mode (bmp != nullptr): every output row is stored as packed
    //    words (bmp_words per row, stride bmp_stride, padding zero) and, when
    //    counts != nullptr, its run count goes to counts[y];
    //  run mode (bmp == nullptr): write == 0 counts runs into counts[y];
    //    write == 1 encodes the runs at out_row_ptr[y] into out.
    uint32_t *bmp;
    int64_t bmp_stride;
    int bmp_words;
    int write;
    int32_t *counts;
    const int32_t *out_row_ptr;
    int64_t capacity;
    uint16_t *out;
};

// Fill the tiling of the between-line pass for an image of width W, height
// H and window height sh (block size up to MAX_THREADS).
void vpass_plan(VArgs &a, int W, int H, int sh);
size_t vpass_smem_bytes(const VArgs &a);
// Band-tile variant (bitmap output only): tiling for a shared-memory budget;
// false if one tile cannot hold the rows it needs (then use vpass_plan).
bool vband_plan(VArgs &a, int W, int H, int sh, size_t smem_budget);
size_t vband_smem_bytes(const VArgs &a);
int vband_grid(const VArgs &a);
constexpr size_t VBAND_SMEM_BUDGET = 96 * 1024;
// Runs per staging buffer of the band tile (two buffers).
constexpr int VBAND_RUN_CHUNK = 2048;
int vpass_threads(const VArgs &a);
int vpass_grid(const VArgs &a);
int vpass_kmax(int sh);  // counter width for a window of sh rows
// rows handled by one work item of the row-wise RLE kernels
constexpr int RLE_ROWS_PER_ITEM = 64;

// Exclusive prefix sum of counts[0..H) into row_ptr[0..H] (row_ptr[H] =
// total, also stored to *n_runs when not NULL); a total above capacity
// latches MORPH_ECAPACITY.  One launch up to 8192 entries, three above.
void launch_scan_rows(const int32_t *counts, int H, int32_t *row_ptr, int64_t *n_runs,
                      int64_t capacity, int *status, cudaStream_t s);

// Connected components of an RLE image (cc.cu).  labels: int32[runs];
// counts: int32[H], rootptr: int32[H+1], rank: int32[runs] scratch.
struct MorphCC {
    int32_t *labels;
    morph_component *stats;
    int64_t max_components;
    int64_t *n_components;
    int32_t *counts, *rootptr, *rank;
};
cudaError_t launch_rle_components(RleIn in, int conn, MorphCC c, int *status, cudaStream_t s);
cudaError_t launch_run_length_hist(RleIn in, int64_t *black, int64_t *white, cudaStream_t s);

// Transposition (transpose.cu): packed src (H rows, pixels x < W) -> packed
// dst (W rows, nw_out words per row written, words past ceil(H/32) zero).
cudaError_t launch_transpose(const uint32_t *src, int64_t sstride, int W, int H, uint32_t *dst,
                             int64_t dstride, int nw_out, cudaStream_t s);
// RLE transpose through two bitmaps in ws (rle_transpose_ws_bytes(W, H)
// bytes, 256-byte aligned); out has width H and height W.
size_t rle_transpose_ws_bytes(int W, int H);
cudaError_t launch_rle_transpose(RleIn in, RleOut out, void *ws, int *status, cudaStream_t s);

// Skew into / out of a stack of band canvases (skew.cu).  Band b of `band`
// image lines has `halo` extra lines above and below (fill rows outside the
// image) and moves line y right by shift[y] - base[b] (device arrays).
// sign > 0: image (src) -> canvases (dst, `rows` = bands * (band + 2 halo));
// sign < 0: canvases (src) -> image (dst, `rows` = H).  Source positions
// outside [0, src_bits) read as fill; dst bits at p >= dst_bits written 0.
cudaError_t launch_shift_rows(const uint32_t *src, int64_t sstride, int src_bits, uint32_t *dst,
                              int64_t dstride, int dst_bits, int nw_dst, int rows, int H, const int32_t *shift,
                              const int32_t *base, int band, int halo, int sign, uint32_t fill,
                              cudaStream_t s);

cudaError_t launch_rle_from_bitmap(const uint32_t *src, int64_t sstride, int W, int H,
                                   RleOut out, int32_t *counts, int *status, cudaStream_t s);
cudaError_t launch_rle_to_bitmap(RleIn in, uint32_t *dst, int64_t dstride, int nw_cover,
                                 cudaStream_t s);
// One erode (dilate=0) or dilate (dilate=1) of an RLE image by a sw x sh
// rectangle with origin (ox, oy).  counts: int32[H] scratch.
// bmp_scratch: W*H/8 bytes (rows of ceil(W/32) u32 words) for the bitmap
// mode of the between-line pass; nullptr runs it in run mode (count pass,
// then a write pass that recomputes the rows and encodes them).
cudaError_t launch_rle_rect(RleIn in, RleOut out, int dilate, int sw, int sh, int ox, int oy,
                            int32_t *counts, uint32_t *bmp_scratch, int *status, cudaStream_t s);

}  // namespace morph
