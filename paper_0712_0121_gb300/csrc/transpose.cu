// Transposition of packed bitmaps and of RLE images (section "Efficient
// Transpose").  The paper sweeps a list of open vertical intervals down the
// lines, which is inherently sequential per column; here the RLE transpose
// goes through the bitmap: runs painted into packed rows, a bit-matrix
// transpose, runs extracted again — three passes that each move about the
// page's packed size.
//
// Bit-matrix transpose: a CTA takes a tile of 256 rows x 8 words (256 pixel
// columns), staged in shared memory with rows padded to 9 words so that a
// warp reading one word column of 32 consecutive rows hits 32 banks.  Each
// warp transposes 32x32 blocks in registers: lane i holds row i of the
// block, and five butterfly steps (exchange with lane i ^ s, s = 16 .. 1,
// swapping the off-diagonal s x s sub-blocks under a mask) leave column j in
// lane j.  The transposed words go to a second padded tile and are stored
// as 32-byte output row segments.
#include "morph_internal.cuh"

namespace morph {
namespace {

constexpr int XT_W = 8;                 // input words per tile (= output 32-row blocks)
constexpr int XT_Y = 8;                 // 32-row input blocks per tile (= output words per row)
constexpr int XT_ROWS = 32 * XT_Y;      // input rows per tile
constexpr int XT_PADI = XT_W + 1;       // input tile row stride in words
constexpr int XT_PADO = XT_Y + 1;       // output tile row stride in words
constexpr int XT_THREADS = 256;
constexpr int XT_TPO = XT_THREADS / (32 * XT_W);  // threads per output row
constexpr int XT_WPO = XT_Y / XT_TPO;              // output words per thread
static_assert(XT_W % 4 == 0 && XT_WPO % 4 == 0 && XT_ROWS % XT_THREADS == 0, "tile shape");

__device__ __forceinline__ uint32_t warp_transpose32(uint32_t v, int lane) {
    const uint32_t masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const int s = 16 >> q;
        const uint32_t m = masks[q];
        const uint32_t o = __shfl_xor_sync(0xFFFFFFFFu, v, s);
        v = (lane & s) ? ((v & ~m) | ((o >> s) & m)) : ((v & m) | ((o & m) << s));
    }
    return v;
}

// src: H rows of nw_in words (stride sstride), pixels x < W; dst: W rows of
// nw_out words (stride dstride), pixels y < H, words past ceil(H/32) zero.
// A tile is XT_ROWS input rows x XT_W words; its transpose is 32 * XT_W
// output rows x XT_Y words.
__global__ void __launch_bounds__(XT_THREADS) k_transpose(const uint32_t *src, int64_t sstride, int W,
                                                          int H, int nw_in, uint32_t *dst,
                                                          int64_t dstride, int nw_out, int vec) {
    __shared__ uint32_t ti[XT_ROWS * XT_PADI];
    __shared__ uint32_t to[32 * XT_W * XT_PADO];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int X0w = blockIdx.x * XT_W;    // first input word column
    const int Y0 = blockIdx.y * XT_ROWS;  // first input row
    uint32_t wm[XT_W];
#pragma unroll
    for (int w = 0; w < XT_W; ++w) wm[w] = word_mask(X0w + w, W);
    const bool full_w = X0w + XT_W <= nw_in;
    // thread t loads input rows Y0 + t + 256 i, words X0w .. X0w + XT_W - 1
#pragma unroll
    for (int i = 0; i < XT_ROWS / XT_THREADS; ++i) {
        const int r = t + XT_THREADS * i, y = Y0 + r;
        uint32_t v[XT_W];
        if (y < H && vec && full_w) {
            const uint4 *pv = reinterpret_cast<const uint4 *>(src + (int64_t)y * sstride + X0w);
#pragma unroll
            for (int c = 0; c < XT_W / 4; ++c) {
                const uint4 a = pv[c];
                v[4 * c] = a.x;
                v[4 * c + 1] = a.y;
                v[4 * c + 2] = a.z;
                v[4 * c + 3] = a.w;
            }
        } else {
#pragma unroll
            for (int w = 0; w < XT_W; ++w)
                v[w] = (y < H && X0w + w < nw_in) ? src[(int64_t)y * sstride + X0w + w] : 0u;
        }
#pragma unroll
        for (int w = 0; w < XT_W; ++w) ti[r * XT_PADI + w] = v[w] & wm[w];
    }
    __syncthreads();
    // block (bx, by): input word column bx, input rows by*32 .. +31 -> output
    // rows (X0w + bx) * 32 + lane, output word Y0 / 32 + by
#pragma unroll 4
    for (int q = warp; q < XT_W * XT_Y; q += XT_THREADS / 32) {
        const int bx = q % XT_W, by = q / XT_W;
        const uint32_t v = warp_transpose32(ti[(by * 32 + lane) * XT_PADI + bx], lane);
        to[(bx * 32 + lane) * XT_PADO + by] = v;
    }
    __syncthreads();
    // XT_TPO threads per output row, XT_WPO words each
    const int orow = t / XT_TPO, part = t % XT_TPO;
    const int x = X0w * 32 + orow;
    const int ow0 = Y0 / 32 + part * XT_WPO;
    if (x < W) {
        uint32_t *p = dst + (int64_t)x * dstride + ow0;
        const uint32_t *q = to + orow * XT_PADO + part * XT_WPO;
        if (vec && ow0 + XT_WPO <= nw_out) {
#pragma unroll
            for (int w = 0; w < XT_WPO; w += 4)
                *reinterpret_cast<uint4 *>(p + w) = make_uint4(q[w], q[w + 1], q[w + 2], q[w + 3]);
        } else {
#pragma unroll
            for (int w = 0; w < XT_WPO; ++w)
                if (ow0 + w < nw_out) p[w] = q[w];
        }
    }
}

}  // namespace

cudaError_t launch_transpose(const uint32_t *src, int64_t sstride, int W, int H, uint32_t *dst,
                             int64_t dstride, int nw_out, cudaStream_t s) {
    const int nw_in = (W + 31) / 32;
    // 16-byte vector access: aligned bases and strides (tile columns and
    // output segments start at multiples of 4 words)
    const int vec = ((uintptr_t)src % 16 == 0) && (sstride % 4 == 0) && ((uintptr_t)dst % 16 == 0) &&
                    (dstride % 4 == 0);
    const dim3 grid((nw_in + XT_W - 1) / XT_W, (nw_out + XT_Y - 1) / XT_Y);
    k_transpose<<<grid, XT_THREADS, 0, s>>>(src, sstride, W, H, nw_in, dst, dstride, nw_out, vec);
    return cudaGetLastError();
}

size_t rle_transpose_ws_bytes(int W, int H) {
    auto a256 = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t nwa = (size_t)(W + 31) / 32, nwb = (size_t)(H + 31) / 32;
    return a256((size_t)H * nwa * 4) + a256((size_t)W * nwb * 4) + a256((size_t)W * 4);
}

cudaError_t launch_rle_transpose(RleIn in, RleOut out, void *ws, int *status, cudaStream_t s) {
    auto a256 = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const int W = in.W, H = in.H;
    const int nwa = (W + 31) / 32, nwb = (H + 31) / 32;
    uint32_t *a = (uint32_t *)ws;
    uint32_t *b = (uint32_t *)((char *)ws + a256((size_t)H * nwa * 4));
    int32_t *counts = (int32_t *)((char *)b + a256((size_t)W * nwb * 4));
    cudaError_t e = launch_rle_to_bitmap(in, a, nwa, nwa, s);
    if (e == cudaSuccess) e = launch_transpose(a, nwa, W, H, b, nwb, nwb, s);
    if (e == cudaSuccess) e = launch_rle_from_bitmap(b, nwb, H, W, out, counts, status, s);
    return e;
}

}  // namespace morph
