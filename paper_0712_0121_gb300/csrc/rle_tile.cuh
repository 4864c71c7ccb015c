// Device bodies of the run-length kernels, written over explicit row ranges
// (or band indices) so that both the single-image launches and the
// persistent batch kernel run them.
//
// RLE image: row_ptr[H+1] and uint16 runs (start, end) with end exclusive
// (section "Run Length Image Coding").  Seen as a uint16 array, the runs of a
// row are exactly the ascending list of its transitions (0->1 at a start,
// 1->0 at an end); the kernels read and write them that way — the paper's
// TransitionSource / TransitionSink abstraction (section "Between Line
// Boolean Operations") in array form.  Variable-size outputs go through
// count -> exclusive prefix sum over rows -> write.
#pragma once

#include "counters.cuh"
#include "cp_async.cuh"
#include "morph_internal.cuh"

namespace morph {

constexpr unsigned FULL_MASK = 0xFFFFFFFFu;

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ int warp_excl_scan(int v, int lane, int &total) {
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL_MASK, x, o);
        if (lane >= o) x += y;
    }
    total = __shfl_sync(FULL_MASK, x, 31);
    return x - v;
}

// ------------------------------------------------------ bitmap -> RLE (K6)
// Transition word k: bit b set iff pixel 32k+b differs from pixel 32k+b-1
// (pixel -1 and pixels >= W are 0).  Words 0 .. W/32 cover positions 0..W.
// Rows [r0, r1); a warp takes B2R_RPW rows at once (rows warp, warp+nwarps,
// ...) and issues the loads of all of them before using any, so one memory
// round trip serves B2R_RPW rows.  Word k-1's top bit comes from lane k-1
// (lane 0: the previous chunk's lane 31).  Plain loads, not the read-only
// path: in the batch kernel the bitmap may have been written earlier in the
// same launch.
constexpr int B2R_RPW = 8;

__device__ __forceinline__ void b2r_load(const uint32_t *src, int64_t sstride, int W, int nw_valid,
                                         int yb, int ystep, int r1, int k,
                                         uint32_t (&w)[B2R_RPW]) {
    const bool kin = k < nw_valid;
    const uint32_t m = kin ? word_mask(k, W) : 0u;
#pragma unroll
    for (int j = 0; j < B2R_RPW; ++j) {
        const int y = yb + j * ystep;
        w[j] = (kin && y < r1) ? (src[(int64_t)y * sstride + k] & m) : 0u;
    }
}

__device__ __forceinline__ uint32_t b2r_trans(uint32_t w, uint32_t &carry, int lane) {
    uint32_t p = __shfl_up_sync(FULL_MASK, w, 1);
    if (lane == 0) p = carry;
    carry = __shfl_sync(FULL_MASK, w, 31);
    return w ^ ((w << 1) | (p >> 31));
}

__device__ __forceinline__ void b2r_count_rows(const uint32_t *src, int64_t sstride, int W, int r0,
                                               int r1, int32_t *counts) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int nw_valid = (W + 31) >> 5, nw_ext = (W >> 5) + 1;
    for (int yb = r0 + warp; yb < r1; yb += nwarps * B2R_RPW) {
        int cnt[B2R_RPW];
        uint32_t carry[B2R_RPW];
#pragma unroll
        for (int j = 0; j < B2R_RPW; ++j) cnt[j] = 0, carry[j] = 0u;
        for (int k0 = 0; k0 < nw_ext; k0 += 32) {
            uint32_t w[B2R_RPW];
            b2r_load(src, sstride, W, nw_valid, yb, nwarps, r1, k0 + lane, w);
#pragma unroll
            for (int j = 0; j < B2R_RPW; ++j) cnt[j] += __popc(b2r_trans(w[j], carry[j], lane));
        }
#pragma unroll
        for (int j = 0; j < B2R_RPW; ++j) {
            int c = cnt[j];
#pragma unroll
            for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(FULL_MASK, c, o);
            const int y = yb + j * nwarps;
            if (lane == 0 && y < r1) counts[y] = c >> 1;
        }
    }
}

// NCH 32-word chunks of the rows are loaded together (3 measured faster in
// the batch kernel, 1 in the single-image kernel with its higher occupancy).
// Chunks at or past word W/32 + 1 hold no transition (their words are 0 and
// the word before has a top bit of 0 unless W is a multiple of 32, in which
// case word W/32 is still inside), so they are skipped.
template <int NCH>
__device__ __forceinline__ void b2r_write_rows(const uint32_t *src, int64_t sstride, int W, int r0,
                                               int r1, const int32_t *row_ptr, uint16_t *runs) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int nw_valid = (W + 31) >> 5, nw_ext = (W >> 5) + 1;
    for (int yb = r0 + warp; yb < r1; yb += nwarps * B2R_RPW) {
        int64_t pos[B2R_RPW];
        uint32_t carry[B2R_RPW];
#pragma unroll
        for (int j = 0; j < B2R_RPW; ++j) {
            const int y = yb + j * nwarps;
            pos[j] = y < r1 ? 2 * (int64_t)row_ptr[y] : 0;
            carry[j] = 0u;
        }
        for (int k00 = 0; k00 < nw_ext; k00 += 32 * NCH) {
            uint32_t w[NCH][B2R_RPW];
#pragma unroll
            for (int c = 0; c < NCH; ++c)
                b2r_load(src, sstride, W, nw_valid, yb, nwarps, r1, k00 + 32 * c + lane, w[c]);
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
                const int k0 = k00 + 32 * c;
                if (k0 >= nw_ext) break;
                const int k = k0 + lane;
                uint32_t t[B2R_RPW];
                int ex[B2R_RPW], tot[B2R_RPW];
                // the rows' transition words and offsets first (independent,
                // so their shuffle chains overlap), then the data-dependent
                // stores
#pragma unroll
                for (int j = 0; j < B2R_RPW; ++j) t[j] = b2r_trans(w[c][j], carry[j], lane);
#pragma unroll
                for (int j = 0; j < B2R_RPW; ++j) ex[j] = __popc(t[j]);
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
                    for (int j = 0; j < B2R_RPW; ++j) {
                        const int y = __shfl_up_sync(FULL_MASK, ex[j], o);
                        if (lane >= o) ex[j] += y;
                    }
                }
#pragma unroll
                for (int j = 0; j < B2R_RPW; ++j) {
                    tot[j] = __shfl_sync(FULL_MASK, ex[j], 31);
                    ex[j] -= __popc(t[j]);
                }
#pragma unroll
                for (int j = 0; j < B2R_RPW; ++j) {
                    uint32_t tj = t[j];
                    int64_t q = pos[j] + ex[j];
                    while (tj) {
                        const int b = __ffs(tj) - 1;
                        runs[q++] = (uint16_t)(32 * k + b);
                        tj &= tj - 1;
                    }
                    pos[j] += tot[j];
                }
            }
        }
    }
}

// Exclusive prefix sum, by one CTA (any size that is a multiple of 32, up to
// 1024), of in[0], in[istride], ... (n values) plus `base` into out[0],
// out[ostride], ...; returns base + the sum to every thread.  Every read of
// a pass happens before its writes, so in == out works in place.
__device__ __forceinline__ int64_t scan_block(const int32_t *in, int64_t istride, int n,
                                              int32_t *out, int64_t ostride, int64_t base0) {
    constexpr int ITEMS = 4;
    __shared__ int64_t wsum[32];
    __shared__ int64_t base_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int nthreads = blockDim.x;
    if (tid == 0) base_s = base0;
    __syncthreads();
    for (int start = 0; start < n; start += nthreads * ITEMS) {
        int64_t v[ITEMS], loc = 0;
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            const int idx = start + tid * ITEMS + j;
            v[j] = idx < n ? in[idx * istride] : 0;
            loc += v[j];
        }
        int64_t x = loc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(FULL_MASK, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int64_t s = lane < nwarps ? wsum[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t y = __shfl_up_sync(FULL_MASK, s, o);
                if (lane >= o) s += y;
            }
            wsum[lane] = s;  // inclusive over warps
        }
        __syncthreads();
        const int64_t base = base_s;
        int64_t run = base + (warp ? wsum[warp - 1] : 0) + x - loc;
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            const int idx = start + tid * ITEMS + j;
            if (idx < n) out[idx * ostride] = (int32_t)run;
            run += v[j];
        }
        __syncthreads();
        if (tid == 0) base_s = base + wsum[nwarps - 1];
        __syncthreads();
    }
    const int64_t total = base_s;
    __syncthreads();  // base_s is reused by the next call
    return total;
}

// Exclusive prefix sum of counts[0..H) into row_ptr[0..H], the total into
// row_ptr[H] and *n_runs; latches MORPH_ECAPACITY when total > capacity.
// One CTA (any size that is a multiple of 32, up to 1024).
__device__ __forceinline__ void scan_rows_block(const int32_t *counts, int H, int32_t *row_ptr,
                                                int64_t *n_runs, int64_t capacity, int *status) {
    const int64_t total = scan_block(counts, 1, H, row_ptr, 1, 0);
    if (threadIdx.x == 0) {
        row_ptr[H] = (int32_t)total;
        if (n_runs) *n_runs = total;
        if (total > capacity) latch_status(status, MORPH_ECAPACITY);
    }
    __syncthreads();
}

// ------------------------------------------------------ RLE -> bitmap (K7)
// Each run XORs its two transition bits into a per-warp row buffer in shared
// memory; a prefix XOR across the row (within words, then a ballot parity
// scan across words) turns transitions back into pixels.  sm: nwarps *
// nw_cover words.
__device__ __forceinline__ void r2b_rows(const RleIn &in, uint32_t *dst, int64_t dstride,
                                         int nw_cover, int r0, int r1, uint32_t *sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    uint32_t *buf = sm + (size_t)warp * nw_cover;
    const int nbits = 32 * nw_cover;
    for (int y = r0 + warp; y < r1; y += nwarps) {
        for (int k = lane; k < nw_cover; k += 32) buf[k] = 0;
        __syncwarp();
        const int a = in.row_ptr[y], b = in.row_ptr[y + 1];
        for (int i = a + lane; i < b; i += 32) {
            const int s = in.runs[2 * (int64_t)i], e = in.runs[2 * (int64_t)i + 1];
            if (s < nbits) atomicXor(buf + (s >> 5), 1u << (s & 31));
            if (e < nbits) atomicXor(buf + (e >> 5), 1u << (e & 31));
        }
        __syncwarp();
        uint32_t carry = 0;
        for (int k0 = 0; k0 < nw_cover; k0 += 32) {
            const int k = k0 + lane;
            const uint32_t T = k < nw_cover ? buf[k] : 0u;
            const unsigned bal = __ballot_sync(FULL_MASK, __popc(T) & 1);
            const uint32_t pre = (__popc(bal & lanemask_lt()) & 1) ^ carry;
            const uint32_t bits = prefix_xor(T) ^ (pre ? ONES : 0u);
            if (k < nw_cover) dst[(int64_t)y * dstride + k] = bits & word_mask(k, in.W);
            carry ^= __popc(bal) & 1;
        }
        __syncwarp();
    }
}

// --------------------------------------------------- within-line pass (K4)
// 1D erosion of a run [s, e) by a width-sw segment with origin ex (clipped
// window): [s + ex, e - (sw-1-ex)), except that a run touching the left
// (right) border keeps that end; dropped when empty.  1D dilation: every run
// grows to [s - ox, e + sw-1-ox) clipped to [0, W); consecutive grown runs
// overlap or touch exactly when the gap between the original runs is
// <= sw - 1, and then merge (their inner transitions are dropped).  This is
// the paper's erode1d / dilate1d (section "Within-Line Morphological
// Operations") with the shrink amounts of the rectangle's origin.
struct RunT {
    int s, e;      // transformed run
    bool ks, ke;   // keep its start / end transition
};

__device__ __forceinline__ RunT row_op(const uint16_t *runs, int64_t i, int64_t a, int64_t b,
                                       const RowOp &op) {
    RunT r;
    const int s = runs[2 * i], e = runs[2 * i + 1];
    if (!op.dilate) {
        r.s = (s == 0) ? 0 : s + op.o;
        r.e = (e >= op.W) ? op.W : e - (op.sw - 1 - op.o);
        r.ks = r.ke = r.s < r.e;
    } else {
        r.s = s - op.o < 0 ? 0 : s - op.o;
        r.e = e + op.sw - 1 - op.o > op.W ? op.W : e + op.sw - 1 - op.o;
        r.ks = (i == a) || (s - (int)runs[2 * i - 1] > op.sw - 1);
        r.ke = (i == b - 1) || ((int)runs[2 * i + 2] - e > op.sw - 1);
    }
    return r;
}

// The run [s, e) after the row pass, as an interval (empty when s2 >= e2).
// Dilated runs may overlap their neighbours: painting them with OR merges
// them, so no neighbour test is needed where the result is a bitmap row.
__device__ __forceinline__ void run_interval(uint32_t pair, const RowOp &op, int &s2, int &e2) {
    const int s = (int)(pair & 0xFFFFu), e = (int)(pair >> 16);
    if (!op.dilate) {
        s2 = (s == 0) ? 0 : s + op.o;
        e2 = (e >= op.W) ? op.W : e - (op.sw - 1 - op.o);
    } else {
        s2 = s - op.o < 0 ? 0 : s - op.o;
        e2 = e + op.sw - 1 - op.o > op.W ? op.W : e + op.sw - 1 - op.o;
    }
}

// OR the pixels [s, e) (0 <= s < e) into a shared-memory row.  The partial
// end words are shared with other runs (atomic OR); the words in between
// belong to this run alone, or end up all ones whatever the order.
__device__ __forceinline__ void paint_run(uint32_t *rowp, int s, int e) {
    const int ws = s >> 5, we = (e - 1) >> 5;
    const uint32_t ms = ONES << (s & 31), me = ONES >> (31 - ((e - 1) & 31));
    if (ws == we) {
        atomicOr(rowp + ws, ms & me);
    } else {
        atomicOr(rowp + ws, ms);
        for (int w = ws + 1; w < we; ++w) rowp[w] = ONES;
        atomicOr(rowp + we, me);
    }
}

// One warp per row; rows [r0, r1).  Count pass (write == 0) or write pass.
__device__ __forceinline__ void rowpass_rows(const RleIn &in, const RowOp &op, int write,
                                             int32_t *counts, const int32_t *out_row_ptr,
                                             uint16_t *out, int r0, int r1) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int y = r0 + warp; y < r1; y += nwarps) {
        const int64_t a = in.row_ptr[y], b = in.row_ptr[y + 1];
        int64_t grp = write ? (int64_t)out_row_ptr[y] : 0;  // run index of the next output
        int cnt = 0;
        for (int64_t i0 = a; i0 < b; i0 += 32) {
            const int64_t i = i0 + lane;
            RunT r = {0, 0, false, false};
            if (i < b) r = row_op(in.runs, i, a, b, op);
            const unsigned bs = __ballot_sync(FULL_MASK, r.ks);
            if (write) {
                // group index of run i = number of kept starts up to i, minus one
                const int incl = __popc(bs & (lanemask_lt() | (1u << lane)));
                const int64_t gi = grp + incl - 1;
                if (r.ks) out[2 * gi] = (uint16_t)r.s;
                if (r.ke) out[2 * gi + 1] = (uint16_t)r.e;
            }
            grp += __popc(bs);
            cnt += __popc(bs);
        }
        if (!write && lane == 0) counts[y] = cnt;
    }
}

// --------------------------------------------------- between-line pass (K5)
// Vertical erosion of the row-pass result by an sh-row window [y-ey, y-ey+sh-1]
// (dilation: the same on the complement).  A tile owns `groups` bands of rows
// across the full width; each thread owns NWT 32-pixel words of every row.
// Per chunk of rb rows:
//   P1 clear the transition slots; P2 every run of an input row (after the
//   row pass) XORs its kept transitions into the slot; P3 one warp per slot
//   turns transitions into pixels (prefix XOR); P4 every thread pushes its
//   words into bit-sliced counters of consecutive covered rows — the "count
//   reached sh" plane is the output row, i.e. the intersection of the sh
//   neighbouring rows' intervals; P5 one warp per output row either stores
//   the row as packed words (bitmap mode, with its run count if asked) or
//   finds its transitions and counts them (count pass) or writes them at
//   row_ptr (write pass).  sm: 2 * rb * groups * slot_words words.
template <int NWT, int KMAX>
__device__ __forceinline__ void vpass_tile(const VArgs &a, int bx, uint32_t *sm) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwarps = blockDim.x >> 5;
    const int g = tid / a.tpr, lt = tid - g * a.tpr;
    const bool act = g < a.groups;
    const int W = a.in.W, H = a.in.H;
    const int nw_valid = (W + 31) >> 5;
    const int slot = a.slot_words, nslot = a.rb * a.groups;
    uint32_t *T = sm;                          // [rb][groups][slot]
    uint32_t *O = sm + (size_t)nslot * slot;   // [rb][groups][slot]
    const int Ybase = bx * a.groups * a.band;
    const int iters = a.band + a.sh - 1;

    uint32_t vmask[NWT], eqm[KMAX];
    ColCounter<KMAX> cc[NWT];
#pragma unroll
    for (int k = 0; k < KMAX; ++k) eqm[k] = a.eqm[k];
#pragma unroll
    for (int t = 0; t < NWT; ++t) {
        const int w = lt * NWT + t;
        vmask[t] = (act && w < nw_valid) ? word_mask(w, W) : 0u;
        cc[t].reset();
    }
    const uint32_t invm = a.inv ? ONES : 0u;
    // run ranges of the chunk's input rows: start and exclusive prefix of counts
    int *sA = reinterpret_cast<int *>(O + (size_t)nslot * slot);
    int *sP = sA + nslot + 1;

    for (int c0 = 0; c0 < iters; c0 += a.rb) {
        // P1: clear transition slots; read the run range of every slot's row
        for (int q = tid; q < nslot * slot; q += blockDim.x) T[q] = 0;
        for (int q = tid; q < nslot; q += blockDim.x) {
            const int i = q / a.groups, gq = q - i * a.groups;
            const int r = Ybase + gq * a.band - a.ey + c0 + i;
            int r0 = 0, n = 0;
            if (r >= 0 && r < H) {
                r0 = a.in.row_ptr[r];
                n = a.in.row_ptr[r + 1] - r0;
            }
            sA[q] = r0;
            sP[q] = n;
        }
        __syncthreads();
        if (warp == 0) {
            int carry = 0;
            for (int q0 = 0; q0 < nslot; q0 += 32) {
                const int q = q0 + lane;
                const int n = q < nslot ? sP[q] : 0;
                int tot;
                const int ex = warp_excl_scan(n, lane, tot);
                if (q < nslot) sP[q] = carry + ex;
                carry += tot;
            }
            if (lane == 0) sP[nslot] = carry;
        }
        __syncthreads();
        // P2: every run of the chunk is an independent item: its kept
        // transitions (after the within-line pass) are XORed into its slot
        {
            const int total = sP[nslot];
            const int nbits = 32 * slot;
            for (int gi = tid; gi < total; gi += blockDim.x) {
                int lo = 0, hi = nslot;  // sP[lo] <= gi < sP[hi]
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (sP[mid] <= gi) lo = mid;
                    else hi = mid;
                }
                const int64_t ra = sA[lo], rb_ = ra + (sP[lo + 1] - sP[lo]);
                const RunT rt = row_op(a.in.runs, ra + (gi - sP[lo]), ra, rb_, a.op);
                uint32_t *slotp = T + (size_t)lo * slot;
                // the bounds guards only matter for a non-canonical input list
                if (rt.ks && rt.s >= 0 && rt.s < nbits) atomicXor(slotp + (rt.s >> 5), 1u << (rt.s & 31));
                if (rt.ke && rt.e >= 0 && rt.e < nbits) atomicXor(slotp + (rt.e >> 5), 1u << (rt.e & 31));
            }
        }
        __syncthreads();
        // P3: transitions -> pixels, one warp per slot row
        for (int q = warp; q < nslot; q += nwarps) {
            uint32_t *slotp = T + (size_t)q * slot;
            uint32_t carry = 0;
            for (int k0 = 0; k0 < a.nw_ext; k0 += 32) {
                const int k = k0 + lane;
                const uint32_t x = k < a.nw_ext ? slotp[k] : 0u;
                const unsigned bal = __ballot_sync(FULL_MASK, __popc(x) & 1);
                const uint32_t pre = (__popc(bal & lanemask_lt()) & 1) ^ carry;
                if (k < a.nw_ext) slotp[k] = prefix_xor(x) ^ (pre ? ONES : 0u);
                carry ^= __popc(bal) & 1;
            }
        }
        __syncthreads();
        // P4: column counters -> output rows
        if (act) {
            for (int i = 0; i < a.rb; ++i) {
                const int r = Ybase + g * a.band - a.ey + c0 + i;
                const bool rin = r >= 0 && r < H;
                const uint32_t *tp = T + (size_t)(i * a.groups + g) * slot + lt * NWT;
                uint32_t *op = O + (size_t)(i * a.groups + g) * slot + lt * NWT;
#pragma unroll
                for (int t = 0; t < NWT; ++t) {
                    const uint32_t v = rin ? ((tp[t] ^ invm) | ~vmask[t]) : ONES;
                    op[t] = (cc[t].push(v, a.K, eqm) ^ invm) & vmask[t];
                }
            }
        }
        __syncthreads();
        // P5: encode output rows
        for (int q = warp; q < nslot; q += nwarps) {
            const int i = q / a.groups, gq = q - i * a.groups;
            const int it = c0 + i;
            const int y0 = Ybase + gq * a.band;
            const int y = y0 + it - (a.sh - 1);
            if (it < a.sh - 1 || y >= y0 + a.band || y >= H) continue;
            const uint32_t *op = O + (size_t)q * slot;
            if (a.bmp) {
                // bitmap mode: store the row's words, count its runs if asked
                uint32_t *row = a.bmp + (int64_t)y * a.bmp_stride;
                const int kmax = a.nw_ext > a.bmp_words ? a.nw_ext : a.bmp_words;
                int cnt = 0;
                for (int k0 = 0; k0 < kmax; k0 += 32) {
                    const int k = k0 + lane;
                    const uint32_t w = k < a.nw_ext ? op[k] : 0u;
                    if (k < a.bmp_words) row[k] = k < nw_valid ? w : 0u;
                    if (a.counts && k < a.nw_ext) {
                        const uint32_t p = k > 0 ? op[k - 1] : 0u;
                        cnt += __popc(w ^ ((w << 1) | (p >> 31)));
                    }
                }
                if (a.counts) {
#pragma unroll
                    for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(FULL_MASK, cnt, o);
                    if (lane == 0) a.counts[y] = cnt >> 1;
                }
                continue;
            }
            int64_t pos0 = a.write ? 2 * (int64_t)a.out_row_ptr[y] : 0;
            int cnt = 0;
            for (int k0 = 0; k0 < a.nw_ext; k0 += 32) {
                const int k = k0 + lane;
                uint32_t t = 0;
                if (k < a.nw_ext) {
                    const uint32_t w = op[k];
                    const uint32_t p = k > 0 ? op[k - 1] : 0u;
                    t = w ^ ((w << 1) | (p >> 31));
                }
                if (a.write) {
                    int tot;
                    const int ex = warp_excl_scan(__popc(t), lane, tot);
                    int64_t pos = pos0 + ex;
                    while (t) {
                        const int b = __ffs(t) - 1;
                        a.out[pos++] = (uint16_t)(32 * k + b);
                        t &= t - 1;
                    }
                    pos0 += tot;
                } else {
                    cnt += __popc(t);
                }
            }
            if (!a.write) {
#pragma unroll
                for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(FULL_MASK, cnt, o);
                if (lane == 0) a.counts[y] = cnt >> 1;
            }
        }
    }
    __syncthreads();
}

// Band tile of the between-line pass (bitmap output).  A tile owns the
// output rows [Y0, Y0 + groups*band); every input row it needs (those rows
// shifted by -ey, plus sh-1 more) is built ONCE as pixels in shared memory:
//   P1 clear the rows and read each row's run offset; P2 stage the tile's
//   runs (one contiguous range of the run array) chunk by chunk, double
//   buffered with asynchronous copies, and paint
//   every run, after the within-line pass, into its row with OR — the union
//   of the row's intervals, overlapping dilated runs included;
//   P4 each thread walks its words down one of `groups` segments of the band
//   (a segment starts sh-1 rows early to warm its counters) reading the rows
//   from shared memory, and stores every output word straight to the bitmap.
// Two barriers per run chunk, none per row.  sm: vband_smem_bytes().
template <int NWT, int KMAX>
__device__ __forceinline__ void vband_tile(const VArgs &a, int bx, uint32_t *sm) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwarps = blockDim.x >> 5;
    const int g = tid / a.tpr, lt = tid - g * a.tpr;
    const bool act = g < a.groups;
    const int W = a.in.W, H = a.in.H;
    const int nw_valid = (W + 31) >> 5;
    const int stride = a.slot_words;               // words per tile row (>= nw_ext)
    const int S = a.band, sh = a.sh;
    const int Y0 = bx * a.groups * S;              // first output row of the tile
    const int R = a.groups * S + sh - 1;           // tile rows
    const int r0 = Y0 - a.ey;                      // input row of tile row 0
    uint32_t *T = sm;
    int *sP = reinterpret_cast<int *>(T + (size_t)R * stride);
    uint32_t *sR = T + ((((size_t)R * stride + R + 1) * 4 + 15) & ~(size_t)15) / 4;
    const uint32_t *runs32 = reinterpret_cast<const uint32_t *>(a.in.runs);

    // P1: clear the rows; sP[i] = index of the first run of tile row i (rows
    // outside the image have none: their offsets clamp to rows 0 and H)
    {
        const int n = R * stride, n4 = n >> 2;
        uint4 *T4 = reinterpret_cast<uint4 *>(T);
        for (int q = tid; q < n4; q += blockDim.x) T4[q] = make_uint4(0u, 0u, 0u, 0u);
        for (int q = 4 * n4 + tid; q < n; q += blockDim.x) T[q] = 0u;
    }
    for (int i = tid; i <= R; i += blockDim.x) {
        const int r = min(max(r0 + i, 0), H);
        sP[i] = a.in.row_ptr[r];
    }
    __syncthreads();
    // P2: the tile's runs are one contiguous range of the run array.  Stage
    // it chunk by chunk with asynchronous copies into two buffers (chunk c+1
    // is in flight while chunk c is painted) and paint every run, after the
    // row pass, into its row
    {
        const int qb = sP[0], qe = sP[R];
        const int nch = (qe - qb + VBAND_RUN_CHUNK - 1) / VBAND_RUN_CHUNK;
        auto issue = [&](int c) {
            const int c0 = qb + c * VBAND_RUN_CHUNK, ns = min(qe - c0, VBAND_RUN_CHUNK);
            uint32_t *buf = sR + (c & 1) * VBAND_RUN_CHUNK;
            for (int k = tid; k < ns; k += blockDim.x) cp_async4(buf + k, runs32 + c0 + k);
            cp_async_commit();
        };
        if (nch > 0) issue(0);
        for (int c = 0; c < nch; ++c) {
            if (c + 1 < nch) {
                issue(c + 1);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncthreads();
            const int c0 = qb + c * VBAND_RUN_CHUNK, c1 = min(qe, c0 + VBAND_RUN_CHUNK);
            const uint32_t *buf = sR + (c & 1) * VBAND_RUN_CHUNK;
            // each warp paints a contiguous share of the chunk's runs; a
            // lane finds its run's row by walking forward from the row of
            // the warp's previous 32 runs (empty rows are skipped)
            const int per = ((c1 - c0 + nwarps - 1) / nwarps + 31) & ~31;
            const int w0 = c0 + warp * per, w1 = min(c1, w0 + per);
            if (w0 < w1) {
                int lo = 0, hi = R;  // sP[lo] <= w0 < sP[hi]
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (sP[mid] <= w0) lo = mid;
                    else hi = mid;
                }
                int r = lo;
                for (int q0 = w0; q0 < w1; q0 += 32) {
                    const int q = min(q0 + lane, w1 - 1);
                    int rr = r;
                    while (sP[rr + 1] <= q) ++rr;
                    if (q0 + lane < w1) {
                        int s2, e2;
                        run_interval(buf[q - c0], a.op, s2, e2);
                        // the clamps only matter for a non-canonical input list
                        s2 = max(s2, 0);
                        e2 = min(e2, W);
                        if (s2 < e2) paint_run(T + (size_t)rr * stride, s2, e2);
                    }
                    r = __shfl_sync(FULL_MASK, rr, 31);
                }
            }
            __syncthreads();  // buffer c & 1 is refilled by the next issue
        }
    }
    // P4: column counters down each segment, output words straight to global
    if (!act) return;
    uint32_t vmask[NWT], eqm[KMAX];
    bool st_ok[NWT];
    ColCounter<KMAX> cc[NWT];
#pragma unroll
    for (int k = 0; k < KMAX; ++k) eqm[k] = a.eqm[k];
#pragma unroll
    for (int t = 0; t < NWT; ++t) {
        const int w = lt * NWT + t;
        vmask[t] = w < nw_valid ? word_mask(w, W) : 0u;
        st_ok[t] = w < a.bmp_words;
        cc[t].reset();
    }
    const uint32_t invm = a.inv ? ONES : 0u;
    const int i0 = g * S;                          // first tile row of the segment
    // NWT == 2: one 64-bit shared load per row (rows start at even words) and
    // one 64-bit store when the output rows allow it
    const bool vec_st = NWT == 2 && st_ok[NWT - 1] && (a.bmp_stride & 1) == 0 &&
                        ((uintptr_t)a.bmp & 7) == 0;
    for (int it = 0; it < S + sh - 1; ++it) {
        const int i = i0 + it;
        const int r = r0 + i;
        const bool rin = r >= 0 && r < H;
        const uint32_t *tp = T + (size_t)i * stride + lt * NWT;
        uint32_t x[NWT], o[NWT];
        if constexpr (NWT == 2) {
            const uint2 v2 = *reinterpret_cast<const uint2 *>(tp);
            x[0] = v2.x;
            x[1] = v2.y;
        } else {
#pragma unroll
            for (int t = 0; t < NWT; ++t) x[t] = tp[t];
        }
#pragma unroll
        for (int t = 0; t < NWT; ++t) {
            const uint32_t v = rin ? ((x[t] ^ invm) | ~vmask[t]) : ONES;
            o[t] = (cc[t].push(v, a.K, eqm) ^ invm) & vmask[t];
        }
        const int y = Y0 + i0 + it - (sh - 1);
        if (it >= sh - 1 && y < H) {
            uint32_t *p = a.bmp + (int64_t)y * a.bmp_stride + lt * NWT;
            if (vec_st) {
                *reinterpret_cast<uint2 *>(p) = make_uint2(o[0], o[NWT - 1]);
            } else {
#pragma unroll
                for (int t = 0; t < NWT; ++t)
                    if (st_ok[t]) p[t] = o[t];
            }
        }
    }
}

}  // namespace morph
