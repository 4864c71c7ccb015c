// Device body of the fused packed tile (used by the single-image kernel and
// by the persistent batch kernel).
//
// Every operation is one or two EROSION stages with complement (dilation by
// duality: D_B(I) = NOT E_B'(NOT I), B' the reflected rectangle with origin
// (sw-1-ox, sh-1-oy); outside the image every erosion stage sees 1, which is
// 0 for the dilated image — the clipped-window convention).  Opening = E then
// D, closing = D then E, both stages in one pass over the page (section
// "Within-Line Morphological Operations": opening and closing are not
// separable and are built from erosions and dilations).
//
// A stage is separable (section "Morphological Operations", erode2d =
// erode1d, transpose, erode1d): a between-line (vertical) pass, then a
// within-line (horizontal) pass.
//
//  * Vertical pass: each thread walks down its own word column.  For every
//    bit it keeps a bit-sliced counter of consecutive 1-rows ending at the
//    current row (K planes, K = bit length of sh) and a "count reached sh"
//    plane, which is the erosion of the window ending at this row.  About 3K
//    logic operations per word and row, whatever sh is.
//  * Horizontal pass: rows of the vertical result are exchanged through
//    shared memory.  The window [x-L, x+R] (L = ex, R = sw-1-ex) is the AND of
//    a right-looking part [x, x+R] and a left-looking part [x-L, x]; each part
//    is either direct shifted ANDs (reach <= 3) or a logarithmic
//    decomposition (section "Efficient Binary Decompositions":
//    A_2s(x) = A_s(x) AND A_s(x+s), then A_2^m(x) AND A_2^m(x+f),
//    f = reach+1-2^m), all with compile-time funnel shifts across words.
//    Splitting at the origin keeps every out-of-image word a constant all-ones
//    word at every doubling level (the border problem the paper's shift-free
//    variant addresses).
//
// Tiling: a CTA covers the full row width (or a column strip with halo words
// when a row is wider than one CTA) and `groups` row bands of `band` output
// rows; a band first sweeps nst*(sh-1) warm-up rows.
#pragma once

#include "counters.cuh"
#include "cp_async.cuh"
#include "morph_internal.cuh"

namespace morph {

constexpr int PK_NWT = 2;  // u32 words per thread (4 measured slower: register pressure)

// Shared-memory row slots keep a permanent all-ones pad of pk_pad(HALO)
// words on both sides; the pad is even so that a thread's two words start on
// an 8-byte boundary.
__host__ __device__ constexpr int pk_pad(int halo) { return (halo + 1) & ~1; }

// ---------------------------------------------------------- H pass parts
// Right-looking erosion of the thread's NWT words: AND of V(x..x+R).
// W[0..NWIN) holds words from HALO words left of the thread's first word.
template <int NWT, int HALO>
__device__ __forceinline__ void h_right(const uint32_t (&W)[NWT + 2 * HALO], uint32_t (&out)[NWT],
                                        int R, int m, int f) {
    constexpr int NWIN = NWT + 2 * HALO;
    constexpr int LMAX = (HALO == 1) ? 6 : (HALO == 2 ? 7 : 8);
    if (R <= 3) {
#pragma unroll
        for (int t = 0; t < NWT; ++t) {
            const uint32_t c = W[HALO + t], nx = W[HALO + t + 1];
            const uint32_t s1 = __funnelshift_r(c, nx, 1);
            const uint32_t s2 = R >= 2 ? __funnelshift_r(c, nx, 2) : ONES;
            const uint32_t s3 = R >= 3 ? __funnelshift_r(c, nx, 3) : ONES;
            out[t] = R == 0 ? c : (c & s1 & s2 & s3);
        }
        return;
    }
    uint32_t A[NWIN];
#pragma unroll
    for (int j = 0; j < NWIN; ++j) A[j] = W[j];
#pragma unroll
    for (int l = 0; l < LMAX; ++l) {
        if (l < m) {
            const int s = 1 << l;
            if (s < 32) {
#pragma unroll
                for (int j = HALO; j < NWIN; ++j) {
                    const uint32_t nx = (j + 1 < NWIN) ? A[j + 1] : ONES;
                    A[j] &= __funnelshift_r(A[j], nx, s);
                }
            } else {
                const int q = s >> 5;
#pragma unroll
                for (int j = HALO; j < NWIN; ++j) A[j] &= (j + q < NWIN) ? A[j + q] : ONES;
            }
        }
    }
    const int q = f >> 5, r = f & 31;
#pragma unroll
    for (int t = 0; t < NWT; ++t) {
        uint32_t sh = 0;
#pragma unroll
        for (int qq = 0; qq < HALO; ++qq) {
            if (HALO == 1 || qq == q) {
                const int j = HALO + t + qq;
                sh = __funnelshift_r(A[j], (j + 1 < NWIN) ? A[j + 1] : ONES, r);
            }
        }
        out[t] = A[HALO + t] & sh;
    }
}

// Left-looking erosion of the thread's NWT words: AND of V(x-L..x).
template <int NWT, int HALO>
__device__ __forceinline__ void h_left(const uint32_t (&W)[NWT + 2 * HALO], uint32_t (&out)[NWT],
                                       int L, int m, int f) {
    constexpr int NWIN = NWT + 2 * HALO;
    constexpr int LMAX = (HALO == 1) ? 6 : (HALO == 2 ? 7 : 8);
    if (L <= 3) {
#pragma unroll
        for (int t = 0; t < NWT; ++t) {
            const uint32_t c = W[HALO + t], pv = W[HALO + t - 1];
            const uint32_t s1 = __funnelshift_l(pv, c, 1);
            const uint32_t s2 = L >= 2 ? __funnelshift_l(pv, c, 2) : ONES;
            const uint32_t s3 = L >= 3 ? __funnelshift_l(pv, c, 3) : ONES;
            out[t] = L == 0 ? c : (c & s1 & s2 & s3);
        }
        return;
    }
    uint32_t B[NWIN];
#pragma unroll
    for (int j = 0; j < NWIN; ++j) B[j] = W[j];
#pragma unroll
    for (int l = 0; l < LMAX; ++l) {
        if (l < m) {
            const int s = 1 << l;
            if (s < 32) {
#pragma unroll
                for (int j = HALO + NWT - 1; j >= 0; --j) {
                    const uint32_t pv = (j >= 1) ? B[j - 1] : ONES;
                    B[j] &= __funnelshift_l(pv, B[j], s);
                }
            } else {
                const int q = s >> 5;
#pragma unroll
                for (int j = HALO + NWT - 1; j >= 0; --j) B[j] &= (j - q >= 0) ? B[j - q] : ONES;
            }
        }
    }
    const int q = f >> 5, r = f & 31;
#pragma unroll
    for (int t = 0; t < NWT; ++t) {
        uint32_t sh = 0;
#pragma unroll
        for (int qq = 0; qq < HALO; ++qq) {
            if (HALO == 1 || qq == q) {
                const int j = HALO + t - qq;
                sh = __funnelshift_l((j - 1 >= 0) ? B[j - 1] : ONES, B[j], r);
            }
        }
        out[t] = B[HALO + t] & sh;
    }
}

struct HPlan {  // one horizontal erosion stage
    int L, R, mL, mR, fL, fR;
};

__host__ __device__ inline int ilog2_floor(int v) {
    int k = -1;
    while (v) { ++k; v >>= 1; }
    return k;
}

__host__ __device__ inline HPlan make_hplan(int sw, int ex) {
    HPlan h;
    h.L = ex;
    h.R = sw - 1 - ex;
    h.mL = ilog2_floor(h.L + 1);
    h.mR = ilog2_floor(h.R + 1);
    h.fL = h.L + 1 - (1 << h.mL);
    h.fR = h.R + 1 - (1 << h.mR);
    return h;
}

// HX1: both reaches <= 1 (rectangles up to 3 wide): one funnel shift per side.
// Wn: the thread's words with HALO words on each side, in registers.
template <int NWT, int HALO, bool HX1>
__device__ __forceinline__ void h_stage_win(const uint32_t (&Wn)[NWT + 2 * HALO], uint32_t (&out)[NWT],
                                            const HPlan &h) {
    if (HX1) {
#pragma unroll
        for (int t = 0; t < NWT; ++t) {
            const uint32_t c = Wn[HALO + t];
            out[t] = c & __funnelshift_r(c, Wn[HALO + t + 1], h.R) & __funnelshift_l(Wn[HALO + t - 1], c, h.L);
        }
        return;
    }
    uint32_t r[NWT], l[NWT];
    h_right<NWT, HALO>(Wn, r, h.R, h.mR, h.fR);
    h_left<NWT, HALO>(Wn, l, h.L, h.mL, h.fL);
#pragma unroll
    for (int t = 0; t < NWT; ++t) out[t] = r[t] & l[t];
}

template <int NWT, int HALO, bool HX1>
__device__ __forceinline__ void h_stage(const uint32_t *win_smem, uint32_t (&out)[NWT], const HPlan &h) {
    uint32_t Wn[NWT + 2 * HALO];
#pragma unroll
    for (int j = 0; j < NWT + 2 * HALO; ++j) Wn[j] = win_smem[j];
    h_stage_win<NWT, HALO, HX1>(Wn, out, h);
}

// ------------------------------------------------------------- the tile
// Rows per shared-memory exchange chunk: the chunk's global loads are issued
// together, then consumed.
constexpr int PK_RB = 8;

// One-stage tile (erode / dilate with sw > 1).  Input rows are copied
// asynchronously into a ring of shared-memory row slots, PK_NBUF1 chunks
// deep (chunk c+2 is in flight while chunk c is processed); per row each
// thread reads its NWT words and HALO neighbour words from the slot, runs
// the horizontal pass, then its column counters, and stores its words.  One
// barrier per chunk; no register staging of future rows.  NWT = 4 amortises
// the per-row address and predicate work and the halo words of the
// horizontal doubling over more words; NWT = 2 keeps fewer registers where
// the work per word is small (reach 1) or the counters are deep (sh >= 32).
constexpr int PK_NBUF1 = 3;

__host__ __device__ constexpr int pk1_nwt(bool hx1, int kmax) { return (hx1 || kmax >= 6) ? 2 : 4; }
__host__ __device__ constexpr int pk1_rb(int nwt) { return nwt == 4 ? 4 : 8; }
// slot pad: a multiple of NWT words, so that each thread's words start on
// an NWT*4-byte boundary of the slot
__host__ __device__ constexpr int pk1_pad(int halo, int nwt) { return (halo + nwt - 1) / nwt * nwt; }

template <int NWT>
struct WordsT;
template <>
struct WordsT<2> {
    using V = uint2;
    __device__ static void cp(uint32_t *d, const uint32_t *p) { cp_async8(d, p); }
    __device__ static V make(uint32_t x) { return make_uint2(x, x); }
};
template <>
struct WordsT<4> {
    using V = uint4;
    __device__ static void cp(uint32_t *d, const uint32_t *p) { cp_async16(d, p); }
    __device__ static V make(uint32_t x) { return make_uint4(x, x, x, x); }
};

// The thread's window (HALO words, its NWT words at `own`, HALO words) from
// shared memory with the widest aligned vector loads (own is NWT-word
// aligned).
template <int NWT, int HALO>
__device__ __forceinline__ void lds_window(const uint32_t *own, uint32_t (&v)[NWT + 2 * HALO]) {
    constexpr int NWIN = NWT + 2 * HALO;
    auto ld2 = [&](int j, int o) {
        const uint2 x = *reinterpret_cast<const uint2 *>(own + o);
        v[j] = x.x;
        v[j + 1] = x.y;
    };
    auto ld4 = [&](int j, int o) {
        const uint4 x = *reinterpret_cast<const uint4 *>(own + o);
        v[j] = x.x;
        v[j + 1] = x.y;
        v[j + 2] = x.z;
        v[j + 3] = x.w;
    };
    if constexpr (HALO % NWT == 0) {
#pragma unroll
        for (int j = 0; j < NWIN; j += NWT) {
            if constexpr (NWT == 4) ld4(j, j - HALO);
            else ld2(j, j - HALO);
        }
    } else if constexpr (HALO == 1) {
        v[0] = own[-1];
        if constexpr (NWT == 4) ld4(1, 0);
        else ld2(1, 0);
        v[NWIN - 1] = own[NWT];
    } else {
        static_assert(NWT == 4 && HALO == 2, "window layout");
        ld2(0, -2);
        ld4(2, 0);
        ld2(6, 4);
    }
}

template <int NST, int NWT, int KMAX, int HALO, bool HX1>
__device__ __forceinline__ void packed1_tile(const PackedArgs &a, int bx, int by, uint32_t *sm) {
    constexpr int RB = pk1_rb(NWT), NBUF = PK_NBUF1;
    constexpr int PAD = pk1_pad(HALO, NWT), NWIN = NWT + 2 * HALO;
    constexpr int KC = KMAX > 0 ? KMAX : 1;
    using WT = WordsT<NWT>;
    // the plan's layout (threads per row, slot size, shared memory) is made
    // for a.nwt words per thread; never run this body on another layout
    if (a.nwt != NWT || !a.ring) return;
    const int tid = threadIdx.x;
    const int tpr = a.tpr, groups = a.groups, band = a.band, H = a.H;
    const int g = tid / tpr, lt = tid - g * tpr;
    const bool act = g < groups;
    const int gg = act ? g : 0;
    const int strip0 = by * a.strip_words;
    const int w0 = strip0 - a.halo_words + lt * NWT;
    const int Y0 = (bx * groups + gg) * band;
    const int sh = a.sh;
    const int wup = NST * (sh - 1);
    const int iters = band + wup;
    const int y_end = min(Y0 + band, H);
    const int K = a.K;
    uint32_t eqm[KC];
#pragma unroll
    for (int k = 0; k < KC; ++k) eqm[k] = a.eqm[k];
    const HPlan hp = make_hplan(a.sw, a.ex[0]);
    const HPlan hp2 = make_hplan(a.sw, a.ex[1]);
    const uint32_t inm_in = a.inv_in ? ONES : 0u, inm_out = a.inv_out ? ONES : 0u;

    // stage-input masks of the window words: padding bits and words outside
    // the row become 1 whatever the slot holds there
    uint32_t nmw[NWIN];
#pragma unroll
    for (int j = 0; j < NWIN; ++j) {
        const int w = w0 - HALO + j;
        nmw[j] = (w >= 0 && w < a.nw_valid) ? ~word_mask(w, a.W) : ONES;
    }
    uint32_t vmask[NWT];
    bool st_ok[NWT], ld_ok[NWT];
    bool all_ld = true, all_st = true;
#pragma unroll
    for (int t = 0; t < NWT; ++t) {
        const int w = w0 + t;
        ld_ok[t] = act && w >= 0 && w < a.nw_valid;
        vmask[t] = ld_ok[t] ? word_mask(w, a.W) : 0u;
        st_ok[t] = act && w >= strip0 && w < strip0 + a.strip_words && w < a.nw_cover;
        all_ld = all_ld && ld_ok[t];
        all_st = all_st && st_ok[t];
    }
    // a.vec: bases aligned to NWT words and strides multiples of NWT words
    const bool vec_ld = a.vec && all_ld;
    const bool vec_st = a.vec && all_st;
    ColCounter<KC> cc[NWT], cc2[NWT];
#pragma unroll
    for (int t = 0; t < NWT; ++t) {
        cc[t].reset();
        cc2[t].reset();
    }

    const int r_first = Y0 - (NST == 2 ? a.ey[1] : 0) - a.ey[0];
    const int64_t sstride = a.sstride, dstride = a.dstride;
    const uint32_t *src = a.src + w0;  // dereferenced only for words inside the row
    uint32_t *dst = a.dst + w0;
    const int row_words = groups * a.slot_words;       // between row slots of a chunk
    const int buf_words = RB * row_words;              // between chunks
    uint32_t *my = sm + gg * a.slot_words + PAD + lt * NWT;  // own words, row 0, buffer 0
    // two stages: the first stage's rows are exchanged through RB more slots
    uint32_t *xmy = my + NBUF * buf_words;

    auto issue = [&](int c) {
        if (act) {
            uint32_t *b = my + (c % NBUF) * buf_words;
            const int rb0 = r_first + c * RB;
#pragma unroll
            for (int i = 0; i < RB; ++i) {
                const int r = rb0 + i;
                uint32_t *d = b + i * row_words;
                if (r >= 0 && r < H) {
                    const uint32_t *p = src + (int64_t)r * sstride;
                    if (vec_ld) {
                        WT::cp(d, p);
                    } else {
#pragma unroll
                        for (int t = 0; t < NWT; ++t)
                            if (ld_ok[t]) cp_async4(d + t, p + t);
                    }
                } else {
                    // outside the image: raw words whose stage input is all ones
                    *reinterpret_cast<typename WT::V *>(d) = WT::make(~inm_in);
                }
            }
        }
        cp_async_commit();
    };

    auto store_out = [&](int it, const uint32_t (&h)[NWT]) {
        const int y = Y0 + it - wup;
        if (it >= wup && y < y_end) {
            uint32_t o[NWT];
#pragma unroll
            for (int t = 0; t < NWT; ++t) o[t] = (h[t] ^ inm_out) & vmask[t];
            uint32_t *p = dst + (int64_t)y * dstride;
            if (vec_st) {
                typename WT::V x;
                x.x = o[0];
                x.y = o[1];
                if constexpr (NWT == 4) {
                    x.z = o[2];
                    x.w = o[3];
                }
                *reinterpret_cast<typename WT::V *>(p) = x;
            } else {
#pragma unroll
                for (int t = 0; t < NWT; ++t)
                    if (st_ok[t]) p[t] = o[t];
            }
        }
    };

    const int nch = (iters + RB - 1) / RB;
    issue(0);
    if (nch > 1) issue(1);
    for (int c = 0; c < nch; ++c) {
        if (c + 1 < nch) cp_async_wait<1>();
        else cp_async_wait<0>();
        __syncthreads();
        // buffer (c + 2) % NBUF was last read in chunk c - 1, before the barrier
        if (c + 2 < nch) issue(c + 2);
        const uint32_t *b = my + (c % NBUF) * buf_words;
#pragma unroll
        for (int i = 0; i < RB; ++i) {
            const int it = c * RB + i;
            uint32_t v[NWIN];
            lds_window<NWT, HALO>(b + i * row_words, v);
#pragma unroll
            for (int j = 0; j < NWIN; ++j) v[j] = (v[j] ^ inm_in) | nmw[j];
            uint32_t h[NWT];
            h_stage_win<NWT, HALO, HX1>(v, h, hp);
            if (KMAX > 0) {
#pragma unroll
                for (int t = 0; t < NWT; ++t) h[t] = cc[t].push(h[t], K, eqm);
            }
            if constexpr (NST == 2) {
                // second stage input: the complement of the first stage's row
                // (dilation by duality), 1 outside the image and in padding bits
                const int y1 = Y0 - a.ey[1] + it - (sh - 1);
                const uint32_t fill = (y1 >= 0 && y1 < H) ? 0u : ONES;
                typename WT::V x;
                x.x = ~(h[0] & vmask[0]) | fill;
                x.y = ~(h[1] & vmask[1]) | fill;
                if constexpr (NWT == 4) {
                    x.z = ~(h[2] & vmask[2]) | fill;
                    x.w = ~(h[3] & vmask[3]) | fill;
                }
                if (act) *reinterpret_cast<typename WT::V *>(xmy + i * row_words) = x;
            } else {
                store_out(it, h);
            }
        }
        if constexpr (NST == 2) {
            __syncthreads();
#pragma unroll
            for (int i = 0; i < RB; ++i) {
                const int it = c * RB + i;
                uint32_t v[NWIN];
                lds_window<NWT, HALO>(xmy + i * row_words, v);
#pragma unroll
                for (int j = 0; j < NWIN; ++j) v[j] |= nmw[j];
                uint32_t h[NWT];
                h_stage_win<NWT, HALO, HX1>(v, h, hp2);
                if (KMAX > 0 && it >= sh - 1) {
#pragma unroll
                    for (int t = 0; t < NWT; ++t) h[t] = cc2[t].push(h[t], K, eqm);
                }
                store_out(it, h);
            }
        }
    }
}

// Template parameters: NST stages (1 or 2), HS (horizontal stage present,
// i.e. sw > 1), KMAX (bit planes of the column counters, >= K; 0 when sh ==
// 1; 2 = a two-row shift register for sh <= 3), HALO (words of horizontal
// reach), HX1 (horizontal reach <= 1 on both sides).  bx: row-band block index, by:
// column-strip index.  sm: dynamic shared memory of packed_smem_bytes().
template <int NST, bool HS, int KMAX, int HALO, bool HX1>
__device__ __forceinline__ void packed_tile2(const PackedArgs &a, int bx, int by, uint32_t *sm) {
    constexpr int NWT = PK_NWT;
    if (a.ring || a.nwt != NWT) return;  // a plan made for the ring tile
    constexpr int RB = PK_RB;
    constexpr int PAD = pk_pad(HALO);
    constexpr int KC = KMAX > 0 ? KMAX : 1;
    const int tid = threadIdx.x;
    const int tpr = a.tpr, groups = a.groups, band = a.band, H = a.H, sh = a.sh;
    const int g = tid / tpr;
    const int lt = tid - g * tpr;
    const bool act = g < groups;
    const int gg = act ? g : 0;
    const int strip0 = by * a.strip_words;
    const int w0 = strip0 - a.halo_words + lt * NWT;
    const int Y0 = (bx * groups + gg) * band;
    const int wup = NST * (sh - 1);
    const int iters = band + wup;
    const int y_end = min(Y0 + band, H);
    const int slot = a.slot_words;
    const int K = a.K;
    const bool inv_in = a.inv_in, inv_out = a.inv_out;
    uint32_t eqm[KC];
#pragma unroll
    for (int k = 0; k < KC; ++k) eqm[k] = a.eqm[k];
    const HPlan hp0 = make_hplan(a.sw, a.ex[0]);
    const HPlan hp1 = make_hplan(a.sw, a.ex[1]);

    uint32_t vmask[NWT];
    bool st_ok[NWT];
#pragma unroll
    for (int t = 0; t < NWT; ++t) {
        const int w = w0 + t;
        vmask[t] = (act && w >= 0 && w < a.nw_valid) ? word_mask(w, a.W) : 0u;
        st_ok[t] = act && w >= strip0 && w < strip0 + a.strip_words && w < a.nw_cover;
    }
    const bool vec_ld = a.vec && vmask[0] && vmask[NWT - 1];
    const bool vec_st = a.vec && st_ok[0] && st_ok[NWT - 1];
    const bool any_ld = vmask[0] || vmask[NWT - 1];

    ColCounter<KC> c1[NWT], c2[NWT];
#pragma unroll
    for (int t = 0; t < NWT; ++t) {
        c1[t].reset();
        c2[t].reset();
    }
    const int r_first = Y0 - (NST == 2 ? a.ey[1] : 0) - a.ey[0];
    const int64_t sstride = a.sstride, dstride = a.dstride;
    const uint32_t *src = a.src + w0;
    uint32_t *dst = a.dst + w0;

    const uint32_t inm_in = inv_in ? ONES : 0u, inm_out = inv_out ? ONES : 0u;
    const uint32_t nvm0 = ~vmask[0], nvm1 = ~vmask[1];

    // Raw words of input row r (0 outside the image).  Plain loads: in the
    // batch kernel a job's input can be another job's output written earlier
    // in the same launch, which the read-only path may not see.
    auto load_raw = [&](int r, uint32_t (&raw)[NWT]) {
        raw[0] = raw[1] = 0u;
        if (r >= 0 && r < H && any_ld) {
            const uint32_t *p = src + (int64_t)r * sstride;
            if (vec_ld) {
                const uint2 x = *reinterpret_cast<const uint2 *>(p);
                raw[0] = x.x;
                raw[1] = x.y;
            } else {
                if (vmask[0]) raw[0] = p[0];
                if (vmask[1]) raw[1] = p[1];
            }
        }
    };
    // Stage-1 input from raw words: complement for dilation, padding bits
    // and rows outside the image set to 1.
    auto stage_in = [&](int r, uint32_t (&v)[NWT]) {
        const uint32_t fill = (r >= 0 && r < H) ? 0u : ONES;
        v[0] = (v[0] ^ inm_in) | nvm0 | fill;
        v[1] = (v[1] ^ inm_in) | nvm1 | fill;
    };
    auto store_row = [&](int y, const uint32_t (&h)[NWT]) {
        const uint32_t o0 = (h[0] ^ inm_out) & vmask[0];
        const uint32_t o1 = (h[1] ^ inm_out) & vmask[1];
        uint32_t *p = dst + (int64_t)y * dstride;
        if (vec_st) {
            *reinterpret_cast<uint2 *>(p) = make_uint2(o0, o1);
        } else {
            if (st_ok[0]) p[0] = o0;
            if (st_ok[1]) p[1] = o1;
        }
    };
    auto vpush1 = [&](uint32_t (&v)[NWT]) {
        if (KMAX > 0) {
            v[0] = c1[0].push(v[0], K, eqm) | nvm0;
            v[1] = c1[1].push(v[1], K, eqm) | nvm1;
        }
    };

    // The rows of the next chunk are loaded while the current one is
    // processed (register double buffering).
    uint32_t nxt[RB][NWT];
#pragma unroll
    for (int i = 0; i < RB; ++i) load_raw(r_first + i, nxt[i]);

    if (!HS) {
        // Vertical-only rectangle (sw == 1): no exchange between threads.
        for (int c0 = 0; c0 < iters; c0 += RB) {
            uint32_t v[RB][NWT];
#pragma unroll
            for (int i = 0; i < RB; ++i) {
                v[i][0] = nxt[i][0];
                v[i][1] = nxt[i][1];
            }
            if (c0 + RB < iters) {
#pragma unroll
                for (int i = 0; i < RB; ++i) load_raw(r_first + c0 + RB + i, nxt[i]);
            }
#pragma unroll
            for (int i = 0; i < RB; ++i) {
                const int it = c0 + i;
                stage_in(r_first + it, v[i]);
                vpush1(v[i]);
                if (NST == 2) {
                    const int y1 = Y0 - a.ey[1] + it - (sh - 1);
                    const uint32_t fill = (y1 >= 0 && y1 < H) ? 0u : ONES;
                    v[i][0] = ~(v[i][0] & vmask[0]) | fill;
                    v[i][1] = ~(v[i][1] & vmask[1]) | fill;
                    if (KMAX > 0 && it >= sh - 1) {
                        v[i][0] = c2[0].push(v[i][0], K, eqm);
                        v[i][1] = c2[1].push(v[i][1], K, eqm);
                    }
                }
                const int y = Y0 + it - wup;
                if (it >= wup && y < y_end) store_row(y, v[i]);
            }
        }
        return;
    }

    // Shared memory: [stage][buffer 2][row in chunk][group][slot words]; a
    // slot is PAD all-ones words, the group's row words, PAD all-ones words.
    const int rows_per_buf = RB * groups;
    {
        const int nslots = NST * 2 * rows_per_buf;
        for (int s = tid; s < nslots; s += blockDim.x) {
            uint32_t *p = sm + (size_t)s * slot;
#pragma unroll
            for (int j = 0; j < PAD; ++j) {
                p[j] = ONES;
                p[slot - 1 - j] = ONES;
            }
        }
    }
    __syncthreads();

    for (int c0 = 0, chunk = 0; c0 < iters; c0 += RB, ++chunk) {
        const int buf = chunk & 1;
        uint32_t *s1 = sm + ((size_t)(0 * 2 + buf) * rows_per_buf) * slot;
        uint32_t *s2 = sm + ((size_t)(1 * 2 + buf) * rows_per_buf) * slot;
        // phase A: stage-1 vertical pass on the chunk's rows (loaded during
        // the previous chunk) -> s1, then start loading the next chunk
        {
            uint32_t v[RB][NWT];
#pragma unroll
            for (int i = 0; i < RB; ++i) {
                v[i][0] = nxt[i][0];
                v[i][1] = nxt[i][1];
            }
#pragma unroll
            for (int i = 0; i < RB; ++i) {
                stage_in(r_first + c0 + i, v[i]);
                vpush1(v[i]);
                if (act) {
                    uint32_t *p = s1 + (size_t)(i * groups + g) * slot + PAD + lt * NWT;
                    *reinterpret_cast<uint2 *>(p) = make_uint2(v[i][0], v[i][1]);
                }
            }
            if (c0 + RB < iters) {
#pragma unroll
                for (int i = 0; i < RB; ++i) load_raw(r_first + c0 + RB + i, nxt[i]);
            }
        }
        __syncthreads();
        // phase B: stage-1 horizontal pass; store, or stage-2 vertical -> s2
#pragma unroll 2
        for (int i = 0; i < RB; ++i) {
            const int it = c0 + i;
            uint32_t h[NWT];
            h_stage<NWT, HALO, HX1>(s1 + (size_t)(i * groups + gg) * slot + PAD - HALO + lt * NWT, h, hp0);
            if (NST == 1) {
                const int y = Y0 + it - wup;
                if (it >= wup && y < y_end) store_row(y, h);
            } else {
                const int y1 = Y0 - a.ey[1] + it - (sh - 1);
                const uint32_t fill = (y1 >= 0 && y1 < H) ? 0u : ONES;
                uint32_t v2[NWT];
#pragma unroll
                for (int t = 0; t < NWT; ++t) {
                    v2[t] = ~(h[t] & vmask[t]) | fill;
                    if (KMAX > 0 && it >= sh - 1) v2[t] = c2[t].push(v2[t], K, eqm);
                    v2[t] |= ~vmask[t];
                }
                if (act) {
                    uint32_t *p = s2 + (size_t)(i * groups + g) * slot + PAD + lt * NWT;
                    *reinterpret_cast<uint2 *>(p) = make_uint2(v2[0], v2[1]);
                }
            }
        }
        if (NST == 2) {
            __syncthreads();
            // phase C: stage-2 horizontal pass and store
#pragma unroll 2
            for (int i = 0; i < RB; ++i) {
                const int it = c0 + i;
                uint32_t h[NWT];
                h_stage<NWT, HALO, HX1>(s2 + (size_t)(i * groups + gg) * slot + PAD - HALO + lt * NWT, h, hp1);
                const int y = Y0 + it - wup;
                if (it >= wup && y < y_end) store_row(y, h);
            }
        }
    }
}

// RING2: open / close on the ring tile (else the register-prefetch tile);
// the plan's a.ring must agree.
template <int NST, bool HS, int KMAX, int HALO, bool HX1, bool RING2 = true>
__device__ __forceinline__ void packed_tile(const PackedArgs &a, int bx, int by, uint32_t *sm) {
    if constexpr (HS && (NST == 1 || RING2)) {
        packed1_tile<NST, pk1_nwt(HX1, KMAX), KMAX, HALO, HX1>(a, bx, by, sm);
    } else {
        packed_tile2<NST, HS, KMAX, HALO, HX1>(a, bx, by, sm);
    }
}

}  // namespace morph
