// Erosion and dilation by an arbitrary structuring element on packed images
// (section "Morphology with Arbitrary Masks"): run at a time with doubling
// accumulation.  The element is a list of horizontal runs.  For the longest
// run width w_max, doubling levels A_1 = I, A_2s(p) = A_s(p) op A_s(p + s)
// are built once per image (A_2^m(p) = op over the 2^m pixels from p on);
// a run of width w at element row j, columns [x0, x0 + w) then contributes
// op over the image's pixels under it, A_2^m(x + dx1) op A_2^m(x + dx2) with
// m = floor(log2 w), dx1 = x0 - ox and dx2 = dx1 + w - 2^m, taken on image
// row y + j - oy; the result is op over all runs' contributions.  op is AND
// for an erosion (1 outside the image: the clipped window) and OR for a
// dilation by the reflected element (0 outside), so rows outside contribute
// nothing, and a level word is the identity right of the row and far enough
// left of it.  Each thread produces four consecutive output words: one
// five-word load per run end serves all four, and a thread stops once its
// words can no longer change (all 0 for AND, all 1 for OR).
#include "mask.cuh"

namespace morph {
namespace {

constexpr int MW = 4;  // output words per thread

__device__ __forceinline__ int floor_div32(int v) { return v >= 0 ? v >> 5 : -((31 - v) >> 5); }

__device__ __forceinline__ int64_t lvl_index(const MaskArgs &a, int m, int r, int k) {
    const int pad = mask_pad_words(a.nlev);
    return ((int64_t)(m - 1) * a.H + r) * (a.nw_valid + pad) + pad + k;
}

// Word k of doubling level m, row r (m = 0: the image itself, its padding
// bits set to the identity of op).
__device__ __forceinline__ uint32_t lvl_word(const MaskArgs &a, int m, int r, int k) {
    const uint32_t idv = a.use_or ? 0u : ONES;
    if (m == 0) {
        if (k < 0 || k >= a.nw_valid) return idv;
        const uint32_t x = a.src[(int64_t)r * a.sstride + k], vm = word_mask(k, a.W);
        return a.use_or ? (x & vm) : (x | ~vm);
    }
    if (k < -mask_pad_words(a.nlev) || k >= a.nw_valid) return idv;
    return a.levels[lvl_index(a, m, r, k)];
}

// Bits [32k + off, 32k + off + 32) of level m, row r.
__device__ __forceinline__ uint32_t lvl_ext(const MaskArgs &a, int m, int r, int k, int off) {
    const int q = floor_div32(off), s = off - 32 * q;
    const uint32_t lo = lvl_word(a, m, r, k + q);
    if (s == 0) return lo;
    return __funnelshift_r(lo, lvl_word(a, m, r, k + q + 1), s);
}

// MW consecutive words of level m, row r, starting at bit 32k + off.
__device__ __forceinline__ void lvl_ext4(const MaskArgs &a, int m, int r, int k, int off,
                                         uint32_t (&out)[MW]) {
    const int q = floor_div32(off), s = off - 32 * q;
    uint32_t w[MW + 1];
#pragma unroll
    for (int t = 0; t <= MW; ++t) w[t] = lvl_word(a, m, r, k + q + t);
#pragma unroll
    for (int t = 0; t < MW; ++t) out[t] = s ? __funnelshift_r(w[t], w[t + 1], s) : w[t];
}

// Level m from level m - 1: A_2s(p) = A_s(p) op A_s(p + s), s = 2^(m-1),
// for the row's words and its left pad.
// A CTA of 256 threads covers rpb = max(1, 256 / width) rows of `width`
// units (one unit per thread; wider rows loop); CTAs step over row blocks.
struct RowTiling {
    int width, rpb, ry, u0;
    __device__ RowTiling(int w) : width(w) {
        rpb = w <= (int)blockDim.x ? (int)blockDim.x / w : 1;
        ry = w <= (int)blockDim.x ? (int)threadIdx.x / w : 0;
        u0 = w <= (int)blockDim.x ? (int)threadIdx.x - ry * w : (int)threadIdx.x;
    }
    __device__ int ustep() const { return width <= (int)blockDim.x ? width : (int)blockDim.x; }
};

// Level m from level m - 1: A_2s(p) = A_s(p) op A_s(p + s), s = 2^(m-1),
// for the row's words and its left pad.
__global__ void __launch_bounds__(256) k_mask_level(const __grid_constant__ MaskArgs a, int m) {
    const int pad = mask_pad_words(a.nlev), lw = a.nw_valid + pad;
    const int s = 1 << (m - 1);
    const RowTiling t(lw);
    if (t.ry >= t.rpb) return;
    for (int r = blockIdx.x * t.rpb + t.ry; r < a.H; r += gridDim.x * t.rpb)
        for (int kk = t.u0; kk < lw; kk += t.ustep()) {
            const int k = kk - pad;
            const uint32_t x = lvl_word(a, m - 1, r, k), y = lvl_ext(a, m - 1, r, k, s);
            a.levels[lvl_index(a, m, r, k)] = a.use_or ? (x | y) : (x & y);
        }
}

// All levels of a block of rows in one launch: each row's level m-1 stays in
// shared memory (two buffers per row, ping-pong) while level m is computed
// from it and written out.  A row buffer holds the row's words, its left pad
// and MASK_RPAD words of the identity on the right (the farthest a level
// reaches: 2^(nlev-1) <= 2048 pixels).  Used while the buffers fit.
constexpr int MASK_RPAD = 66;

__global__ void __launch_bounds__(256) k_mask_levels(const __grid_constant__ MaskArgs a) {
    extern __shared__ uint32_t lsm[];
    const int pad = mask_pad_words(a.nlev), lw = a.nw_valid + pad, bw = lw + MASK_RPAD;
    const uint32_t idv = a.use_or ? 0u : ONES;
    const RowTiling t(lw);
    const bool act = t.ry < t.rpb;
    uint32_t *b0 = lsm + (size_t)(act ? t.ry : 0) * 2 * bw, *b1 = b0 + bw;
    for (int rb = blockIdx.x * t.rpb; rb < a.H; rb += gridDim.x * t.rpb) {
        const int r = rb + t.ry;
        const bool live = act && r < a.H;
        if (live)
            for (int u = t.u0; u < bw; u += t.ustep()) {
                const int k = u - pad;
                b0[u] = k < a.nw_valid ? lvl_word(a, 0, r, k) : idv;  // k < 0: identity
                b1[u] = idv;
            }
        __syncthreads();
        uint32_t *cur = b0, *nxt = b1;
        for (int m = 1; m <= a.nlev; ++m) {
            const int s = 1 << (m - 1), q = s >> 5, sh = s & 31;
            if (live)
                for (int u = t.u0; u < lw; u += t.ustep()) {
                    const uint32_t x = cur[u], lo = cur[u + q];
                    const uint32_t y = sh ? __funnelshift_r(lo, cur[u + q + 1], sh) : lo;
                    const uint32_t v = a.use_or ? (x | y) : (x & y);
                    nxt[u] = v;
                    a.levels[lvl_index(a, m, r, u - pad)] = v;
                }
            __syncthreads();
            uint32_t *tmp = cur;
            cur = nxt;
            nxt = tmp;
        }
    }
}

// Output words [MW g, MW g + MW) of row y: op over the runs; words past the
// row's pixels are written 0.
__global__ void __launch_bounds__(256) k_mask_acc(const __grid_constant__ MaskArgs a) {
    const int ng = (a.nw_cover + MW - 1) / MW;
    const bool use_or = a.use_or != 0;
    const uint32_t idv = use_or ? 0u : ONES, done = use_or ? ONES : 0u;
    const RowTiling tl(ng);
    if (tl.ry >= tl.rpb) return;
    for (int y = blockIdx.x * tl.rpb + tl.ry; y < a.H; y += gridDim.x * tl.rpb)
    for (int g = tl.u0; g < ng; g += tl.ustep()) {
        const int k0 = g * MW;
        uint32_t acc[MW];
#pragma unroll
        for (int t = 0; t < MW; ++t) acc[t] = idv;
        if (k0 < a.nw_valid) {
            for (int u = 0; u < a.nruns; ++u) {
                const MaskRun run = a.runs[u];
                const int r = y + run.dy;
                if (r < 0 || r >= a.H) continue;
                uint32_t e1[MW], e2[MW];
                lvl_ext4(a, run.m, r, k0, run.dx1, e1);
                lvl_ext4(a, run.m, r, k0, run.dx2, e2);
                bool fin = true;
#pragma unroll
                for (int t = 0; t < MW; ++t) {
                    acc[t] = use_or ? (acc[t] | e1[t] | e2[t]) : (acc[t] & e1[t] & e2[t]);
                    fin = fin && acc[t] == done;
                }
                if (fin) break;
            }
        }
        uint32_t *p = a.dst + (int64_t)y * a.dstride;
#pragma unroll
        for (int t = 0; t < MW; ++t) {
            const int k = k0 + t;
            if (k < a.nw_cover) p[k] = acc[t] & (k < a.nw_valid ? word_mask(k, a.W) : 0u);
        }
    }
}

// CTAs of 256 threads for rows of `width` units (see RowTiling)
int grid_rows(int width, int H) {
    const int rpb = width <= 256 ? 256 / width : 1;
    int64_t b = (H + rpb - 1) / rpb;
    if (b > 152 * 16) b = 152 * 16;
    return b < 1 ? 1 : (int)b;
}

}  // namespace

size_t mask_levels_bytes(int W, int H, int nlev) {
    return (size_t)nlev * H * ((W + 31) / 32 + mask_pad_words(nlev)) * sizeof(uint32_t);
}

cudaError_t launch_mask_stage(const MaskArgs &a, cudaStream_t s) {
    const int lw = a.nw_valid + mask_pad_words(a.nlev);
    const int rpb = lw <= 256 ? 256 / lw : 1;
    const size_t lsmem = (size_t)rpb * 2 * (lw + MASK_RPAD) * sizeof(uint32_t);
    if (a.nlev > 0 && lsmem <= 48 * 1024) {
        k_mask_levels<<<grid_rows(lw, a.H), 256, lsmem, s>>>(a);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    for (int m = 1; m <= a.nlev && !(lsmem <= 48 * 1024); ++m) {
        k_mask_level<<<grid_rows(a.nw_valid + mask_pad_words(a.nlev), a.H), 256, 0, s>>>(a, m);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    k_mask_acc<<<grid_rows((a.nw_cover + MW - 1) / MW, a.H), 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace morph
