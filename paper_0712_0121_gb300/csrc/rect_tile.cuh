// Device body of the packed rectangle tile: erosion, dilation, opening and
// closing of packed bitmaps by a rectangle, one or two erosion stages in one
// pass over the page (dilation by duality: complement in, erode with the
// reflected rectangle, complement out; outside the image every stage sees 1,
// the clipped-window reading).
//
// Each stage is separable (section "Morphological Operations": erode2d =
// erode1d along one axis, then along the other) and runs its between-line
// (vertical) pass FIRST, then its within-line (horizontal) pass, so that the
// expensive horizontal pass runs once per output row and only the cheap
// vertical pass sees the window's extra rows.
//
//  * Vertical pass (window of sh rows), per thread down its own word column,
//    no exchange between threads:
//      sh == 1      nothing;
//      sh <= 3      the AND of a register window of the last rows;
//      sh >= 4      van Herk / Gil-Werman (below), or, where its rings would
//                   take too much shared memory, bit-sliced counters of
//                   consecutive 1-rows in registers (6 planes, about 20
//                   logic operations per word);
//                   van Herk / Gil-Werman: rows are taken in blocks of sh;
//                   g = prefix AND within the current block (one AND per
//                   row), s = suffix AND within the previous block (computed
//                   once per block by a backward sweep over that block's rows,
//                   kept in a per-thread shared-memory ring of sh entries);
//                   the window ending at a row of the current block is
//                   s[position + 1] AND g — three ANDs per word whatever sh.
//  * Horizontal pass on the rows of the vertical result, exchanged through
//    shared memory (a thread reads its words and HALO words on each side):
//      reach <= 1 or 2 on both sides: direct funnel shifts;
//      otherwise the doubling of section "Efficient Binary Decompositions"
//      done one-sided: A_2s(x) = A_s(x) AND A_s(x+s) for s = 1, 2, ...,
//      2^(m-1) (2^m <= sw < 2^(m+1)), then
//      E(x) = A_2^m(x - L) AND A_2^m(x + R + 1 - 2^m)
//      with L / R the reach left / right of the origin.  About 2 log2(sw)
//      logic operations per word.  Words outside the image are all ones at
//      every level (AND of ones), so the border needs no special case.
//
// Tiling: a group of `tpr` threads covers a full row (or a column strip with
// halo words when a row is wider than one CTA) and walks down a band of
// `band` output rows; a CTA holds `groups` groups.  Input rows arrive through
// a rolling register queue RB rows deep (each thread loads only its own
// words).  One barrier per chunk of RB rows: iteration c runs the vertical
// pass of chunk c into an exchange buffer and the horizontal pass of the
// chunk c-1 rows exchanged before the previous barrier (two stages: also the
// second stage's passes, one chunk later), with two buffers per stage.
// Per-row work avoids index arithmetic: row pointers advance by a stride,
// each stage's lag is rounded up to whole chunks so that a chunk is all
// warm-up or all output, and rows are checked against the image only in the
// chunks at its top and bottom.
#pragma once

#include <type_traits>

#include "counters.cuh"
#include "morph_internal.cuh"

namespace morph {

// RV_CNT: counters of 6 bit planes (sh < 64); RV_CNT4 / RV_CNT5: 4 or 5
// planes for sh < 16 / sh < 32 (two stages, two words per thread only)
enum RectVMode { RV_NONE = 0, RV_W3 = 1, RV_VHGW = 2, RV_CNT = 3, RV_CNT4 = 4, RV_CNT5 = 5 };
__host__ __device__ constexpr bool rv_cnt(int vm) { return vm == RV_CNT || vm == RV_CNT4 || vm == RV_CNT5; }
__host__ __device__ constexpr int rv_planes(int vm) { return vm == RV_CNT4 ? 4 : (vm == RV_CNT5 ? 5 : 6); }
enum RectHMode { RH_NONE = 0, RH_D1 = 1, RH_D2 = 2, RH_LOG = 3 };

struct RectArgs {
    const uint32_t *src;
    int64_t sstride;      // u32 words between source rows
    uint32_t *dst;
    int64_t dstride;      // u32 words between destination rows
    int W, H;
    int nw_valid;         // u32 words holding pixels
    int nw_cover;         // u32 words written per destination row
    int sw, sh;           // clipped rectangle
    int nst;              // stages: 1 erode / dilate, 2 open / close
    int L[2], R[2];       // per stage: horizontal reach left / right of the origin
    int up[2];            // per stage: window rows above the output row (origin row)
    int m;                // floor(log2(sw))
    int inv_in, inv_out;  // complement input / output
    // tiling (rect_plan)
    int nwt;              // u32 words per thread
    int threads;          // CTA size
    int tpr;              // threads per row group
    int groups;           // row groups per CTA
    int band;             // output rows per group
    int strip_words, halo_words, nstrips;
    int pad;              // all-ones words on each side of an exchange slot
    int slot_words;       // exchange slot: pad + row_words + pad
    int vec;              // aligned bases and strides: vector loads / stores
    int vec_rows;         // vec, and every thread's words lie inside the rows
    int vmode, hmode, halo;  // kernel variant (must match the template)
    int band_auto;        // band chosen at launch from the resident CTAs
    int row_words;        // words of a row in an exchange slot: tpr * nwt rounded up to RECT_NWH
    int tph;              // horizontal tasks per row: row_words / RECT_NWH
    int ktasks;           // horizontal tasks per thread and chunk (at most RECT_KT)
    int nw_full;          // words holding 32 pixels: W / 32
    int vec16;            // dst 16-byte aligned and dstride a multiple of 4 words
    int vec_tasks;        // every horizontal task stores 8 whole aligned words inside the row
};

constexpr int RECT_RB = 8;  // bands are whole multiples of this many rows
// Rows per chunk (one barrier per chunk): 8, or 4 for two stages, whose four
// exchange buffers would otherwise crowd out the CTAs of an SM.
__host__ __device__ constexpr int rect_rb(int nst) { return nst == 2 ? 4 : 8; }
constexpr int RECT_CNT_SH = 63;  // tallest window of the counter mode (6 bit planes)
constexpr int RECT_NWH = 8;      // words of one horizontal-pass task
constexpr int RECT_KT = 8;       // horizontal tasks per thread and chunk, at most
constexpr size_t RECT_SMEM_MAX = 200 * 1024;  // shared memory of one tile at most

template <int NWT>
struct RectVec;
template <>
struct RectVec<2> {
    using V = uint2;
    __device__ static V ld(const uint32_t *p) { return *reinterpret_cast<const uint2 *>(p); }
    __device__ static void st(uint32_t *p, const uint32_t (&x)[2]) {
        *reinterpret_cast<uint2 *>(p) = make_uint2(x[0], x[1]);
    }
    __device__ static void get(const V &v, uint32_t (&x)[2]) {
        x[0] = v.x;
        x[1] = v.y;
    }
};
template <>
struct RectVec<4> {
    using V = uint4;
    __device__ static V ld(const uint32_t *p) { return *reinterpret_cast<const uint4 *>(p); }
    __device__ static void st(uint32_t *p, const uint32_t (&x)[4]) {
        *reinterpret_cast<uint4 *>(p) = make_uint4(x[0], x[1], x[2], x[3]);
    }
    __device__ static void get(const V &v, uint32_t (&x)[4]) {
        x[0] = v.x;
        x[1] = v.y;
        x[2] = v.z;
        x[3] = v.w;
    }
};

template <>
struct RectVec<8> {
    struct V {
        uint4 a, b;
    };
    __device__ static V ld(const uint32_t *p) {
        return V{*reinterpret_cast<const uint4 *>(p), *reinterpret_cast<const uint4 *>(p + 4)};
    }
    __device__ static void st(uint32_t *p, const uint32_t (&x)[8]) {
        *reinterpret_cast<uint4 *>(p) = make_uint4(x[0], x[1], x[2], x[3]);
        *reinterpret_cast<uint4 *>(p + 4) = make_uint4(x[4], x[5], x[6], x[7]);
    }
    __device__ static void get(const V &v, uint32_t (&x)[8]) {
        x[0] = v.a.x; x[1] = v.a.y; x[2] = v.a.z; x[3] = v.a.w;
        x[4] = v.b.x; x[5] = v.b.y; x[6] = v.b.z; x[7] = v.b.w;
    }
};

// Shared-memory words of one thread, NWT words at p (NWT-word aligned).
template <int NWT>
__device__ __forceinline__ void lds_own(const uint32_t *p, uint32_t (&x)[NWT]) {
    RectVec<NWT>::get(RectVec<NWT>::ld(p), x);
}

// The H-pass window: HALO words, the thread's NWT words at `own` (aligned to
// NWT words), HALO words; widest aligned vector loads.
template <int NWT, int HALO>
__device__ __forceinline__ void lds_win(const uint32_t *own, uint32_t (&v)[NWT + 2 * HALO]) {
    constexpr int NWIN = NWT + 2 * HALO;
    uint32_t mid[NWT];
    lds_own<NWT>(own, mid);
#pragma unroll
    for (int t = 0; t < NWT; ++t) v[HALO + t] = mid[t];
    if constexpr (HALO % 4 == 0 && NWT == 4) {
#pragma unroll
        for (int j = 0; j < HALO; j += 4) {
            uint32_t a[4], b[4];
            lds_own<4>(own - HALO + j, a);
            lds_own<4>(own + NWT + j, b);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                v[j + q] = a[q];
                v[HALO + NWT + j + q] = b[q];
            }
        }
    } else if constexpr (HALO % 2 == 0) {
#pragma unroll
        for (int j = 0; j < HALO; j += 2) {
            uint32_t a[2], b[2];
            lds_own<2>(own - HALO + j, a);
            lds_own<2>(own + NWT + j, b);
            v[j] = a[0];
            v[j + 1] = a[1];
            v[HALO + NWT + j] = b[0];
            v[HALO + NWT + j + 1] = b[1];
        }
    } else {
#pragma unroll
        for (int j = 0; j < HALO; ++j) {
            v[j] = own[j - HALO];
            v[HALO + NWT + j] = own[NWT + j];
        }
    }
    (void)NWIN;
}

// o[t] = bits [32 (HALO + t) + 32 OFF + r, +32) of the window A (words past
// the window's right end read as ones).
template <int NWT, int NWIN, int OFF>
__device__ __forceinline__ void shift_words(const uint32_t (&A)[NWIN], int r, uint32_t (&o)[NWT]) {
    constexpr int HALO = (NWIN - NWT) / 2;
#pragma unroll
    for (int t = 0; t < NWT; ++t) {
        constexpr int base = HALO + OFF;
        const int q = base + t;
        const uint32_t lo = A[q];
        const uint32_t hi = (q + 1 < NWIN) ? A[q + 1] : ONES;
        o[t] = __funnelshift_r(lo, hi, r);
    }
}

// o = the window shifted by d bits (pixel x of o is pixel x + d of A),
// -32 HALO <= d <= 32 HALO; d is the same for every thread of the CTA.
template <int NWT, int HALO>
__device__ __forceinline__ void shifted(const uint32_t (&A)[NWT + 2 * HALO], int d, uint32_t (&o)[NWT]) {
    constexpr int NWIN = NWT + 2 * HALO;
    const int q = d >> 5, r = d & 31;
    switch (q) {
    case -4: if constexpr (HALO >= 4) shift_words<NWT, NWIN, -4>(A, r, o); break;
    case -3: if constexpr (HALO >= 3) shift_words<NWT, NWIN, -3>(A, r, o); break;
    case -2: if constexpr (HALO >= 2) shift_words<NWT, NWIN, -2>(A, r, o); break;
    case -1: shift_words<NWT, NWIN, -1>(A, r, o); break;
    case 0: shift_words<NWT, NWIN, 0>(A, r, o); break;
    case 1: shift_words<NWT, NWIN, 1>(A, r, o); break;
    case 2: if constexpr (HALO >= 2) shift_words<NWT, NWIN, 2>(A, r, o); break;
    case 3: if constexpr (HALO >= 3) shift_words<NWT, NWIN, 3>(A, r, o); break;
    default: if constexpr (HALO >= 4) shift_words<NWT, NWIN, 4>(A, r, o); break;
    }
}

// Horizontal erosion of one row: window [x - L, x + R] of the stage input
// held in `win` (shared memory, the thread's own words at `own`), XORed with
// inm (the complement of a dilation or of the next stage's input, folded
// into the last logic operation).
template <int NWT, int HM, int HALO>
__device__ __forceinline__ void rect_hpass(const uint32_t *own, int L, int R, int m, uint32_t inm,
                                           uint32_t (&out)[NWT]) {
    if constexpr (HM == RH_NONE) {
        lds_own<NWT>(own, out);
#pragma unroll
        for (int t = 0; t < NWT; ++t) out[t] ^= inm;
    } else if constexpr (HM == RH_D1 || HM == RH_D2) {
        uint32_t v[NWT + 2];
        lds_win<NWT, 1>(own, v);
        // shift amounts clamped to the reach: a zero shift ANDs a word with
        // itself, so no per-side predicate is needed
        const int r1 = R < 1 ? R : 1, l1 = L < 1 ? L : 1;
#pragma unroll
        for (int t = 0; t < NWT; ++t) {
            const uint32_t c = v[1 + t], nx = v[2 + t], pv = v[t];
            uint32_t e = c & __funnelshift_r(c, nx, r1) & __funnelshift_l(pv, c, l1);
            if constexpr (HM == RH_D2) {
                const int r2 = R < 2 ? R : 2, l2 = L < 2 ? L : 2;
                e &= __funnelshift_r(c, nx, r2) & __funnelshift_l(pv, c, l2);
            }
            out[t] = e ^ inm;
        }
    } else {
        constexpr int NWIN = NWT + 2 * HALO;
        constexpr int LMAX = HALO == 1 ? 6 : (HALO == 2 ? 7 : 8);
        uint32_t A[NWIN];
        lds_win<NWT, HALO>(own, A);
#pragma unroll
        for (int l = 0; l < LMAX; ++l) {
            if (l < m) {
                const int s = 1 << l;
                if (s < 32) {
#pragma unroll
                    for (int j = 0; j < NWIN; ++j) A[j] &= __funnelshift_r(A[j], j + 1 < NWIN ? A[j + 1] : ONES, s);
                } else {
                    const int qw = s >> 5;
#pragma unroll
                    for (int j = 0; j < NWIN; ++j) A[j] &= (j + qw < NWIN) ? A[j + qw] : ONES;
                }
            }
        }
        uint32_t lo[NWT], hi[NWT];
        shifted<NWT, HALO>(A, -L, lo);
        shifted<NWT, HALO>(A, R + 1 - (1 << m), hi);
#pragma unroll
        for (int t = 0; t < NWT; ++t) out[t] = (lo[t] & hi[t]) ^ inm;
    }
}


// Vertical pass state of one stage.
template <int NWT, int VM>
struct RectV {
    uint32_t g[NWT];   // VHGW: prefix AND of the current block; W3: previous row
    uint32_t p2[NWT];  // W3: the row before the previous one (ones when sh == 2)
    uint32_t keep2;    // W3: ones when sh == 2
    int j;             // VHGW: position in the block
    uint32_t *ring;    // VHGW: this thread's column of the ring, entries rstride words apart
    uint32_t *rp;      // VHGW: entry j
    int rstride;
    static constexpr int KP = rv_planes(VM);
    ColCounter<KP> cnt[NWT];  // CNT: run counters
    uint32_t eqm[KP];         // CNT: per plane, ones where that bit of sh is 0
    int K;                    // CNT: bit length of sh

    __device__ __forceinline__ void init(uint32_t *ring_base, int tid, int threads, int sh) {
#pragma unroll
        for (int t = 0; t < NWT; ++t) {
            g[t] = ONES;
            p2[t] = ONES;
        }
        keep2 = sh == 3 ? 0u : ONES;
        if constexpr (rv_cnt(VM)) {
#pragma unroll
            for (int t = 0; t < NWT; ++t) cnt[t].reset();
            K = 0;
            for (int v = sh; v; v >>= 1) ++K;
#pragma unroll
            for (int k = 0; k < KP; ++k) eqm[k] = ((sh >> k) & 1) ? 0u : ONES;
        }
        j = 0;
        ring = ring_base + tid * NWT;
        rstride = threads * NWT;
        rp = ring;
        if constexpr (VM == RV_VHGW) {
            // entry sh is a permanent all-ones sentinel: the suffix "after"
            // the last row of a block, read when the window is the block
            uint32_t ones[NWT];
#pragma unroll
            for (int t = 0; t < NWT; ++t) ones[t] = ONES;
            RectVec<NWT>::st(ring + sh * rstride, ones);
        }
    }

    // Push the next row of the stage input; out = AND of the last sh rows
    // (meaningful once sh rows have been pushed).
    __device__ __forceinline__ void push(const uint32_t (&in)[NWT], uint32_t (&out)[NWT], int sh) {
        if constexpr (VM == RV_NONE) {
#pragma unroll
            for (int t = 0; t < NWT; ++t) out[t] = in[t];
        } else if constexpr (VM == RV_W3) {
#pragma unroll
            for (int t = 0; t < NWT; ++t) {
                out[t] = in[t] & g[t] & p2[t];
                p2[t] = g[t] | keep2;
                g[t] = in[t];
            }
        } else if constexpr (rv_cnt(VM)) {
#pragma unroll
            for (int t = 0; t < NWT; ++t) out[t] = cnt[t].push(in[t], K, eqm);
        } else {
            using RV = RectVec<NWT>;
            uint32_t s[NWT];
            RV::get(RV::ld(rp + rstride), s);  // suffix of the previous block at j + 1
#pragma unroll
            for (int t = 0; t < NWT; ++t) {
                g[t] &= in[t];
                out[t] = s[t] & g[t];
            }
            RV::st(rp, in);
            rp += rstride;
            if (++j == sh) {
                // suffix ANDs of the block just completed, in place; entry 0
                // is never read (the window starting there is the full
                // block).  Entries are read in small groups before any of them
                // is written back, so that the loads overlap.
                uint32_t acc[NWT];
                RV::get(RV::ld(ring + (sh - 1) * rstride), acc);
                constexpr int BB = NWT >= 4 ? 2 : 4;  // entries per group (registers)
                for (int q0 = sh - 2; q0 >= 1; q0 -= BB) {
                    uint32_t x[BB][NWT];
#pragma unroll
                    for (int e = 0; e < BB; ++e)
                        if (q0 - e >= 1) RV::get(RV::ld(ring + (q0 - e) * rstride), x[e]);
#pragma unroll
                    for (int e = 0; e < BB; ++e) {
                        if (q0 - e >= 1) {
#pragma unroll
                            for (int t = 0; t < NWT; ++t) acc[t] &= x[e][t];
                            RV::st(ring + (q0 - e) * rstride, acc);
                        }
                    }
                }
                j = 0;
                rp = ring;
#pragma unroll
                for (int t = 0; t < NWT; ++t) g[t] = ONES;
            }
        }
    }
};

// Shared memory of the tile in u32 words.  Exchange buffers (when there is a
// horizontal pass): one set for one stage; for two stages three sets — the
// stage-1 vertical result, the stage-1 horizontal result handed back to the
// stage-2 vertical pass, and the stage-2 vertical result.  A set is two
// chunks of rows, a row slot per group.  Then the van Herk / Gil-Werman ring
// of sh + 1 entries per thread and stage.
__host__ __device__ inline size_t rect_xbuf_words(const RectArgs &a) {
    return (size_t)2 * rect_rb(a.nst) * a.groups * a.slot_words;
}
__host__ __device__ inline int rect_xsets(const RectArgs &a) {
    return a.hmode == RH_NONE ? 0 : (a.nst == 2 ? 3 : 1);
}
__host__ __device__ inline size_t rect_ring_words(const RectArgs &a) {
    return a.vmode == RV_VHGW ? (size_t)(a.sh + 1) * a.threads * a.nwt : 0;
}
__host__ __device__ inline size_t rect_smem_words(const RectArgs &a) {
    return (size_t)rect_xsets(a) * rect_xbuf_words(a) + (size_t)a.nst * rect_ring_words(a);
}

// Horizontal-pass tasks: every chunk of RB rows splits into RB x groups x
// tph tasks of RECT_NWH words of one row (task t: row t / (groups tph),
// group, segment).  A thread takes tasks tid, tid + threads, ... in every
// chunk; the decomposition of its first task and of the stride between its
// tasks are worked out once, so the loop only adds and carries.
struct RectTasks {
    int total;          // tasks per chunk
    int i0, g0, s0;     // row, group, segment of task tid
    int di, dg, ds;     // the same of the stride `threads`
    __device__ __forceinline__ void init(int tid, int threads, int rb, int groups, int tph) {
        const int per_row = groups * tph;
        total = rb * per_row;
        i0 = tid / per_row;
        g0 = (tid - i0 * per_row) / tph;
        s0 = tid - i0 * per_row - g0 * tph;
        di = threads / per_row;
        dg = (threads - di * per_row) / tph;
        ds = threads - di * per_row - dg * tph;
    }
};

// Horizontal pass of one chunk of exchanged rows as tasks of RECT_NWH words
// of one row.  LAST: the task's words of output row u0 + i of its group's
// band go to the destination (complemented by inm, padding bits 0);
// otherwise they go, complemented by inm, into `yb` at the same slot
// position.  With the plan's vec_tasks every task is 8 whole, 16-byte
// aligned words inside the row: its store needs no per-word checks.
template <int HM, int HALO, bool LAST>
__device__ __forceinline__ void rect_htasks(const RectArgs &a, const RectTasks &tasks, const uint32_t *xb,
                                            uint32_t *yb, int u0, int L, int R, int bx, int strip0,
                                            int strip_end, uint32_t inm, int row_words) {
    constexpr int NWH = RECT_NWH;
    const int groups = a.groups, band = a.band, H = a.H;
    const int64_t dstride = a.dstride;
    int i = tasks.i0, gq = tasks.g0, sg = tasks.s0;
#pragma unroll 1
    for (int tk = threadIdx.x; tk < tasks.total; tk += blockDim.x) {
        const int off = i * row_words + gq * a.slot_words + a.pad + sg * NWH;
        uint32_t h[NWH];
        rect_hpass<NWH, HM, HALO>(xb + off, L, R, a.m, inm, h);
        if constexpr (LAST) {
            const int y = (bx * groups + gq) * band + u0 + i;
            if (y < H) {
                const int ws = strip0 - a.halo_words + sg * NWH;  // first word of the task
                uint32_t *p = a.dst + (int64_t)y * dstride + ws;
                if (ws + NWH > a.nw_full) {
                    // the row's last words: padding bits and words past the
                    // pixels are written 0
#pragma unroll
                    for (int t = 0; t < NWH; ++t) h[t] &= word_mask(ws + t, a.W);
                }
                if (a.vec_tasks || (a.vec16 && (ws & 3) == 0 && ws >= strip0 && ws + NWH <= strip_end)) {
                    RectVec<NWH>::st(p, h);
                } else {
#pragma unroll
                    for (int t = 0; t < NWH; ++t)
                        if (ws + t >= strip0 && ws + t < strip_end) p[t] = h[t];
                }
            }
        } else {
            RectVec<NWH>::st(yb + off, h);
        }
        sg += tasks.ds;
        gq += tasks.dg;
        i += tasks.di;
        if (sg >= a.tph) {
            sg -= a.tph;
            ++gq;
        }
        if (gq >= groups) {
            gq -= groups;
            ++i;
        }
    }
}

template <int NST, int NWT, int VM, int HM, int HALO>
__device__ __forceinline__ void rect_tile(const RectArgs &a, int bx, int by, uint32_t *sm) {
    constexpr int RB = rect_rb(NST);
    constexpr bool XCH = HM != RH_NONE;  // rows exchanged between threads
    using RV = RectVec<NWT>;
    // a plan made for another variant or CTA size must not run this body
    if (a.nwt != NWT || a.vmode != VM || a.nst != NST || (int)blockDim.x != a.threads || a.hmode != HM ||
        a.halo != HALO)
        return;
    const int tid = threadIdx.x;
    const int tpr = a.tpr, groups = a.groups, band = a.band, H = a.H, sh = a.sh;
    const int g = tid / tpr, lt = tid - g * tpr;
    const bool act = g < groups;
    const int gg = act ? g : 0;
    const int strip0 = by * a.strip_words;
    const int w0 = strip0 - a.halo_words + lt * NWT;
    const int strip_end = strip0 + a.strip_words < a.nw_cover ? strip0 + a.strip_words : a.nw_cover;
    const int Y0 = (bx * groups + gg) * band;
    // Each stage's vertical pass lags sh - 1 rows behind its input; the lag
    // is rounded up to whole chunks (the extra rows are more warm-up), so
    // that every chunk is either all warm-up or all output of its stage.
    const int lagv = (sh - 1 + RB - 1) / RB * RB;
    const int ex = lagv - (sh - 1);
    const int lag = NST * lagv;           // input index of output row 0
    const int n_in = band + lag;          // input rows of the group (band is a multiple of RB)
    const int nch = n_in / RB;
    const int r_first = Y0 - a.up[0] - (NST == 2 ? a.up[1] : 0) - NST * ex;
    const int y1_first = Y0 - (NST == 2 ? a.up[1] + ex : 0);  // stage-1 row of stage-2 input 0

    // per-word masks of this thread (threads past the last group mirror the
    // words of group 0 and store nothing)
    uint32_t nmw[NWT], vmask[NWT];
    bool ld_ok[NWT], st_ok[NWT];
    bool all_ld = true, all_st = true;
#pragma unroll
    for (int t = 0; t < NWT; ++t) {
        const int w = w0 + t;
        ld_ok[t] = w >= 0 && w < a.nw_valid;
        vmask[t] = ld_ok[t] ? word_mask(w, a.W) : 0u;
        nmw[t] = ~vmask[t];
        const bool st_in = w >= strip0 && w < strip0 + a.strip_words && w < a.nw_cover;
        st_ok[t] = act && st_in;
        all_ld = all_ld && ld_ok[t];
        all_st = all_st && st_in;
    }
    // The row loop below is compiled twice: for whole-vector loads and
    // stores of every thread's words, and for the general case.  It holds
    // the barriers, so the choice must be the same for every thread of the
    // CTA: the planner allows the vector copy only when every word of every
    // thread is inside the rows (a.vec_rows).
    const bool vec_path = a.vec_rows != 0;
    (void)all_ld;
    (void)all_st;
    const uint32_t inm_in = a.inv_in ? ONES : 0u, inm_out = a.inv_out ? ONES : 0u;

    // shared memory: exchange sets (the stage-1 vertical result; for two
    // stages also the stage-1 horizontal result and the stage-2 vertical
    // result), then the rings
    const size_t xw = XCH ? rect_xbuf_words(a) : 0;
    uint32_t *X1 = sm, *Y1 = sm + xw, *X2 = sm + 2 * xw;
    uint32_t *ring_base = sm + rect_xsets(a) * xw;
    const int row_words = groups * a.slot_words;  // between rows of a chunk
    const int buf_words = RB * row_words;         // between the two buffers
    const int own_off = gg * a.slot_words + a.pad + lt * NWT;

    RectV<NWT, VM> v1, v2;
    v1.init(ring_base, tid, a.threads, sh);
    if constexpr (NST == 2) v2.init(ring_base + rect_ring_words(a), tid, a.threads, sh);

    if constexpr (XCH) {
        // every word of an exchange slot outside the row (the left pad, and
        // everything right of the row up to the slot's end) is all ones,
        // written once
        const int nslots = rect_xsets(a) * 2 * RB * groups;
        const int row_end = a.pad + tpr * NWT;
        for (int s = tid; s < nslots; s += blockDim.x) {
            uint32_t *p = sm + (size_t)s * a.slot_words;
            for (int j = 0; j < a.pad; ++j) p[j] = ONES;
            for (int j = row_end; j < a.slot_words; ++j) p[j] = ONES;
        }
        __syncthreads();
    }
    RectTasks tasks;
    tasks.init(tid, a.threads, RB, groups, a.tph);

    const int64_t sstride = a.sstride, dstride = a.dstride;
    // Row pointers advance by one stride per row; they are dereferenced only
    // for rows inside the image and words inside the row.
    const uint32_t *lp = a.src + w0 + (int64_t)r_first * sstride;  // next row to load
    uint32_t *sp = a.dst + w0 + (int64_t)Y0 * dstride;              // next output row

    auto body = [&](auto vec_flag) {
        constexpr bool VEC = decltype(vec_flag)::value;
        auto ld_words = [&](const uint32_t *p, uint32_t (&x)[NWT]) {
            if constexpr (VEC) {
                RV::get(RV::ld(p), x);
            } else {
#pragma unroll
                for (int t = 0; t < NWT; ++t) x[t] = ld_ok[t] ? p[t] : 0u;
            }
        };
        auto store = [&](const uint32_t (&h)[NWT], bool ok) {
            uint32_t o[NWT];
#pragma unroll
            for (int t = 0; t < NWT; ++t) o[t] = (h[t] ^ inm_out) & vmask[t];
            if constexpr (VEC) {
                if (act && ok) RV::st(sp, o);
            } else if (ok) {
#pragma unroll
                for (int t = 0; t < NWT; ++t)
                    if (st_ok[t]) sp[t] = o[t];
            }
            sp += dstride;
        };

        // rolling prefetch queue: q[i] holds input row k with k % RB == i
        uint32_t q[RB][NWT];
#pragma unroll
        for (int i = 0; i < RB; ++i) {
            const int r = r_first + i;
            if (r >= 0 && r < H) {
                ld_words(lp, q[i]);
            } else {
#pragma unroll
                for (int t = 0; t < NWT; ++t) q[i][t] = 0u;
            }
            lp += sstride;
        }

        // Stage-1 vertical pass of chunk c (and, for two stages without a
        // horizontal pass, the second stage's vertical pass in registers).
        // FAST: every row of this chunk and of the next one lies inside the image
        // and is needed, so no row needs a check.
        auto vchunk = [&](int c, auto fast) {
            constexpr bool F = decltype(fast)::value;
            const int rc = r_first + c * RB;
            uint32_t *xo = X1 + (c & 1) * buf_words + own_off;
            const bool out1 = c * RB >= lagv;  // the chunk's rows are stage-1 output
            const bool out2 = c * RB >= lag;   // ... and output rows of the tile
            const int u0 = c * RB - lag;       // output row of the chunk's first row
            const bool st_all = Y0 + u0 + RB <= H;
            const int y10 = y1_first + c * RB - lagv;
            const bool f2free = y10 >= 0 && y10 + RB <= H;
#pragma unroll
            for (int i = 0; i < RB; ++i) {
                uint32_t in[NWT], o[NWT];
                if constexpr (F) {
#pragma unroll
                    for (int t = 0; t < NWT; ++t) in[t] = (q[i][t] ^ inm_in) | nmw[t];
                    ld_words(lp, q[i]);
                } else {
                    const int r = rc + i;
                    const uint32_t fill = (r >= 0 && r < H) ? 0u : ONES;
#pragma unroll
                    for (int t = 0; t < NWT; ++t) in[t] = (q[i][t] ^ inm_in) | nmw[t] | fill;
                    const int rn = r + RB;
                    if (rn >= 0 && rn < H && c * RB + i + RB < n_in) {
                        ld_words(lp, q[i]);
                    } else {
#pragma unroll
                        for (int t = 0; t < NWT; ++t) q[i][t] = 0u;
                    }
                }
                lp += sstride;
                v1.push(in, o, sh);
                if constexpr (XCH) {
                    if (act && out1) RV::st(xo + i * row_words, o);
                } else if constexpr (NST == 1) {
                    if (out2) store(o, st_all || Y0 + u0 + i < H);
                } else {
                    if (out1) {
                        const int y1 = y10 + i;
                        const uint32_t fill2 = (f2free || (y1 >= 0 && y1 < H)) ? 0u : ONES;
                        uint32_t in2[NWT], o2[NWT];
#pragma unroll
                        for (int t = 0; t < NWT; ++t) in2[t] = ~o[t] | nmw[t] | fill2;
                        v2.push(in2, o2, sh);
                        if (out2) store(o2, st_all || Y0 + u0 + i < H);
                    }
                }
            }
        };

        // Horizontal pass on an exchanged chunk as tasks of RECT_NWH words
        // (rect_htasks): the last stage stores rows u0 + i of its group's
        // band, stage 1 of two writes its rows into `yb` for the stage-2
        // vertical pass.
        // (stage 1 of two hands its rows back complemented: the stage-2
        // vertical pass erodes the complement)
        auto htasks = [&](const uint32_t *xb, uint32_t *yb, int u0, int L, int R, auto last_flag) {
            constexpr bool LST = decltype(last_flag)::value;
            rect_htasks<HM, HALO, LST>(a, tasks, xb, yb, u0, L, R, bx, strip0, strip_end, LST ? inm_out : ONES,
                                       row_words);
        };

        // Two stages: the stage-2 vertical pass of a chunk of stage-1 rows
        // handed back by the stage-1 horizontal tasks, into the stage-2
        // exchange buffer.
        auto v2chunk = [&](int c2) {
            const uint32_t *yb = Y1 + (c2 & 1) * buf_words + own_off;
            uint32_t *xo = X2 + (c2 & 1) * buf_words + own_off;
            const int y10 = y1_first + c2 * RB - lagv;
            const bool f2free = y10 >= 0 && y10 + RB <= H;
            const bool w2 = c2 * RB >= lag;
#pragma unroll
            for (int i = 0; i < RB; ++i) {
                uint32_t h[NWT], in2[NWT], o2[NWT];
                lds_own<NWT>(yb + i * row_words, h);
                const int y1 = y10 + i;
                const uint32_t fill2 = (f2free || (y1 >= 0 && y1 < H)) ? 0u : ONES;
#pragma unroll
                for (int t = 0; t < NWT; ++t) in2[t] = h[t] | nmw[t] | fill2;  // h: complemented already
                v2.push(in2, o2, sh);
                if (act && w2) RV::st(xo + i * row_words, o2);
            }
        };

        const int last = XCH ? nch + (NST == 2 ? 2 : 0) : nch - 1;
        for (int c = 0; c <= last; ++c) {
            if constexpr (XCH) {
                if constexpr (NST == 2) {
                    const int c3 = c - 3;
                    if (c3 >= 0 && c3 * RB >= lag)
                        htasks(X2 + (c3 & 1) * buf_words, nullptr, c3 * RB - lag, a.L[1], a.R[1], std::true_type{});
                    const int c2 = c - 2;
                    if (c2 >= 0 && c2 < nch && c2 * RB >= lagv) v2chunk(c2);
                    const int c1 = c - 1;
                    if (c1 >= 0 && c1 < nch && c1 * RB >= lagv)
                        htasks(X1 + (c1 & 1) * buf_words, Y1 + (c1 & 1) * buf_words, 0, a.L[0], a.R[0],
                               std::false_type{});
                } else {
                    const int c1 = c - 1;
                    if (c1 >= 0 && c1 * RB >= lag)
                        htasks(X1 + (c1 & 1) * buf_words, nullptr, c1 * RB - lag, a.L[0], a.R[0], std::true_type{});
                }
            }
            if (c < nch) {
                const int rc = r_first + c * RB;
                const bool fast = rc >= 0 && rc + 2 * RB <= H && (c + 2) * RB <= n_in;
                if (fast) vchunk(c, std::true_type{});
                else vchunk(c, std::false_type{});
            }
            if constexpr (XCH) __syncthreads();
        }
    };
    if (vec_path) body(std::true_type{});
    else body(std::false_type{});
}

}  // namespace morph

namespace morph {

// Host side (rect.cu).  rect_plan fills the stage parameters and the tiling
// for op (MORPH_ERODE .. MORPH_CLOSE) by a sw x sh rectangle with origin
// (ox, oy) (already clipped to the image); hints of 0 take the defaults.
// Returns 0, or -1 when the horizontal reach exceeds 128 pixels or the
// window is too tall for the tile's shared memory (RECT_SMEM_MAX).
// rle_src: plan for the run-length-source tile (rle_rect.cuh).
int rect_plan(RectArgs &a, int op, int sw, int sh, int ox, int oy, int band_hint, int threads_hint,
              int nwt_hint, size_t smem_budget, bool rle_src = false);
__host__ __device__ inline dim3 rect_grid(const RectArgs &a) {
    return dim3((a.H + a.groups * a.band - 1) / (a.groups * a.band), a.nstrips);
}
// Several images of one variant in one launch (the batch's independent jobs).
struct RectJobs {
    const RectArgs *jobs;  // device: one plan per image (same variant and CTA size)
    const int *starts;     // device: first CTA of each image, njobs + 1 entries
    int njobs, ctas;
    size_t smem;           // dynamic shared memory: the largest of the images' needs
};
// Image of CTA b: the j with starts[j] <= b < starts[j + 1].
__device__ __forceinline__ int rect_job_of(const int *starts, int njobs, int b) {
    int lo = 0, hi = njobs;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (starts[mid] <= b) lo = mid;
        else hi = mid;
    }
    return lo;
}
// Band height for `slots` resident CTAs: whole waves of CTAs over the image
// when it is tall, else the smallest band that keeps the window's extra rows
// a modest share.
void rect_fit_band(RectArgs &a, int slots);
int rect_sm_count(int dev);
// mj: launch the images of a job table (plans of a's variant) instead of a.
cudaError_t launch_rect(const RectArgs &a, cudaStream_t s, const RectJobs *mj = nullptr);
cudaError_t launch_rect_1_2(const RectArgs &a, cudaStream_t s, const RectJobs *mj);
cudaError_t launch_rect_1_4(const RectArgs &a, cudaStream_t s, const RectJobs *mj);
cudaError_t launch_rect_2_2(const RectArgs &a, cudaStream_t s, const RectJobs *mj);
cudaError_t launch_rect_2_4(const RectArgs &a, cudaStream_t s, const RectJobs *mj);

}  // namespace morph
