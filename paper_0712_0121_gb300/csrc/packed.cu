// Packed-bitmap rectangular morphology: one fused tile kernel.
//
// Every operation is reduced to one or two EROSION stages with complement
// (dilation by duality: D_B(I) = NOT E_B'(NOT I), B' the reflected rectangle,
// whose origin is (sw-1-ox, sh-1-oy); the outside of the image is 1 for every
// erosion stage, which is 0 for the dilated image — the clipped-window
// boundary convention).  Opening = E then D, closing = D then E, fused in one
// launch (section "Within-Line Morphological Operations": opening and closing
// are not separable and are built from erosions and dilations).
//
// A stage is separable (section "Morphological Operations", erode2d =
// erode1d, transpose, erode1d): a between-line (vertical) pass followed by a
// within-line (horizontal) pass.
//
//  * Vertical pass (K2): each thread walks down its own word column(s).  For
//    every bit it keeps a bit-sliced counter of consecutive 1-rows ending at
//    the current row (K bit planes, K = bit length of sh) plus a "reached sh"
//    plane; the erosion of the window that ends at this row is that plane.
//    Cost: about 3K logic operations per word per row, whatever sh is.
//  * Horizontal pass (K1): the rows of the vertical result are exchanged
//    through shared memory; each thread loads a window of words around its
//    own and erodes it by logarithmic decomposition (section "Efficient
//    Binary Decompositions": A_2s(x) = A_s(x) AND A_s(x+s), then the final
//    AND of two copies shifted by -ox and sw-2^m-ox) using funnel shifts with
//    cross-word carries, or by direct shifted ANDs for sw <= 4.
//
// Tiling (K3): a CTA covers the full row width (or a column strip with halo
// words for very wide rows) and `groups` independent row bands of `band`
// output rows each; a band first sweeps nst*(sh-1) halo rows to warm up its
// counters.  Every page word is read once from DRAM per band (plus the halo
// rows, normally L2 hits) and written once.
#include "morph_internal.cuh"

namespace morph {
namespace {

// Window bits at positions 32*j + b + (32*q + r), b in [0, 32).  j is a
// compile-time index after unrolling; q is runtime, |q| <= HALO.
template <int NWIN, int HALO>
__device__ __forceinline__ uint32_t win_shift(const uint32_t (&A)[NWIN], int j, int q, int r) {
    uint32_t res = ONES;
#pragma unroll
    for (int qq = -HALO; qq <= HALO; ++qq) {
        if (qq == q) {
            const int lo = j + qq, hi = j + qq + 1;
            const uint32_t a = (lo >= 0 && lo < NWIN) ? A[lo] : ONES;
            const uint32_t b = (hi >= 0 && hi < NWIN) ? A[hi] : ONES;
            res = __funnelshift_r(a, b, r);
        }
    }
    return res;
}

// Horizontal erosion of NWT words of a row held in `win` (NWT + 2*HALO words
// starting HALO words to the left of the thread's first word; words outside
// the image are all ones).  Erosion window [x - ex, x + sw - 1 - ex].
template <int NWT, int HALO>
__device__ __forceinline__ void h_erode(const uint32_t *win_smem, uint32_t (&out)[NWT], int hmode,
                                        int sw, int ex, int m) {
    constexpr int NWIN = NWT + 2 * HALO;
    constexpr int LMAX = (HALO == 1) ? 7 : (HALO == 2 ? 8 : 9);
    uint32_t A[NWIN];
#pragma unroll
    for (int j = 0; j < NWIN; ++j) A[j] = win_smem[j];
    if (hmode == 1) {
#pragma unroll
        for (int t = 0; t < NWT; ++t) {
            uint32_t acc = ONES;
            for (int d = -ex; d <= sw - 1 - ex; ++d) acc &= win_shift<NWIN, HALO>(A, HALO + t, d >> 5, d & 31);
            out[t] = acc;
        }
        return;
    }
#pragma unroll
    for (int l = 0; l < LMAX; ++l) {
        if (l < m) {
            const int s = 1 << l;
            if (s < 32) {
#pragma unroll
                for (int j = 0; j < NWIN; ++j) {
                    const uint32_t nx = (j + 1 < NWIN) ? A[j + 1] : ONES;
                    A[j] &= __funnelshift_r(A[j], nx, s);
                }
            } else {
                const int q = s >> 5;
#pragma unroll
                for (int j = 0; j < NWIN; ++j) A[j] &= (j + q < NWIN) ? A[j + q] : ONES;
            }
        }
    }
    const int d1 = -ex, d2 = sw - (1 << m) - ex;
#pragma unroll
    for (int t = 0; t < NWT; ++t)
        out[t] = win_shift<NWIN, HALO>(A, HALO + t, d1 >> 5, d1 & 31) &
                 win_shift<NWIN, HALO>(A, HALO + t, d2 >> 5, d2 & 31);
}

// Bit-sliced counter of consecutive 1-rows; returns the plane "count >= sh".
template <int KMAX>
struct ColCounter {
    uint32_t c[KMAX];
    uint32_t sat;
    __device__ __forceinline__ void reset() {
#pragma unroll
        for (int k = 0; k < KMAX; ++k) c[k] = 0;
        sat = 0;
    }
    __device__ __forceinline__ uint32_t push(uint32_t v, int K, const uint32_t *eqm) {
        uint32_t carry = v, eq = ONES;
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            if (k < K) {
                const uint32_t ck = c[k];
                const uint32_t nk = (ck ^ carry) & v;
                carry = ck & carry;
                c[k] = nk;
                eq &= nk ^ eqm[k];
            }
        }
        sat = v & (sat | eq);
        return sat;
    }
};

template <int NWT, int HALO, int KMAX>
__global__ void __launch_bounds__(MAX_THREADS) k_packed(const PackedArgs a) {
    extern __shared__ uint32_t sm[];
    const int tid = threadIdx.x;
    const int g = tid / a.tpr;
    const int lt = tid - g * a.tpr;
    const bool act = g < a.groups;
    const int gg = act ? g : 0;
    const int strip0 = blockIdx.y * a.strip_words;
    const int w0 = strip0 - a.halo_words + lt * NWT;
    const int Y0 = (blockIdx.x * a.groups + gg) * a.band;
    const int wup = a.nst * (a.sh - 1);
    const int iters = a.band + wup;
    const int slot = a.slot_words;
    const int rows_per_buf = a.rb * a.groups;

    // Shared memory: [stage][buffer 2][row in chunk][group][slot words];
    // the HALO words at both ends of a slot are permanent all-ones padding.
    // Without a horizontal stage (sw == 1) each thread only reads back its
    // own words, so no barrier is needed.
    {
        const int nslots = a.nst * 2 * rows_per_buf;
        for (int s = tid; s < nslots; s += blockDim.x) {
            uint32_t *p = sm + (size_t)s * slot;
#pragma unroll
            for (int j = 0; j < HALO; ++j) {
                p[j] = ONES;
                p[slot - 1 - j] = ONES;
            }
        }
    }

    uint32_t vmask[NWT];
#pragma unroll
    for (int t = 0; t < NWT; ++t) {
        const int w = w0 + t;
        vmask[t] = (act && w >= 0 && w < a.nw_valid) ? word_mask(w, a.W) : 0u;
    }
    ColCounter<KMAX> c1[NWT], c2[NWT];
#pragma unroll
    for (int t = 0; t < NWT; ++t) {
        c1[t].reset();
        c2[t].reset();
    }
    const int r_first = Y0 - (a.nst == 2 ? a.ey[1] : 0) - a.ey[0];
    __syncthreads();

    for (int c0 = 0, chunk = 0; c0 < iters; c0 += a.rb, ++chunk) {
        const int buf = chunk & 1;
        uint32_t *s1 = sm + ((size_t)(0 * 2 + buf) * rows_per_buf) * slot;
        uint32_t *s2 = sm + ((size_t)(1 * 2 + buf) * rows_per_buf) * slot;
        // ---- phase A: stage-1 vertical pass on rb input rows -> s1
        for (int i = 0; i < a.rb; ++i) {
            const int r = r_first + c0 + i;
            const bool rin = (r >= 0 && r < a.H);
            uint32_t v[NWT];
#pragma unroll
            for (int t = 0; t < NWT; ++t) {
                uint32_t raw = 0;
                if (rin && vmask[t]) raw = __ldg(a.src + (int64_t)r * a.sstride + (w0 + t));
                if (a.inv_in) raw = ~raw;
                v[t] = rin ? (raw | ~vmask[t]) : ONES;
                if (a.sh > 1) v[t] = c1[t].push(v[t], a.K, a.eqm) | ~vmask[t];
            }
            if (act) {
                uint32_t *p = s1 + (size_t)(i * a.groups + g) * slot + HALO + lt * NWT;
#pragma unroll
                for (int t = 0; t < NWT; ++t) p[t] = v[t];
            }
        }
        if (a.hmode) __syncthreads();
        // ---- phase B: stage-1 horizontal pass; then store or stage-2 vertical
        for (int i = 0; i < a.rb; ++i) {
            const int it = c0 + i;
            uint32_t h[NWT];
            const uint32_t *row = s1 + (size_t)(i * a.groups + gg) * slot;
            if (a.hmode) {
                h_erode<NWT, HALO>(row + lt * NWT, h, a.hmode, a.sw, a.ex[0], a.m);
            } else {
#pragma unroll
                for (int t = 0; t < NWT; ++t) h[t] = row[HALO + lt * NWT + t];
            }
            if (a.nst == 1) {
                const int y = Y0 + it - wup;
                if (act && it >= wup && y < Y0 + a.band && y < a.H) {
#pragma unroll
                    for (int t = 0; t < NWT; ++t) {
                        const int w = w0 + t;
                        if (w >= strip0 && w < strip0 + a.strip_words && w < a.nw_cover) {
                            const uint32_t o = (a.inv_out ? ~h[t] : h[t]) & vmask[t];
                            a.dst[(int64_t)y * a.dstride + w] = o;
                        }
                    }
                }
            } else {
                const int y1 = Y0 - a.ey[1] + it - (a.sh - 1);
                const bool yin = (y1 >= 0 && y1 < a.H);
                uint32_t v2[NWT];
#pragma unroll
                for (int t = 0; t < NWT; ++t) {
                    v2[t] = yin ? ~(h[t] & vmask[t]) : ONES;
                    if (a.sh > 1 && it >= a.sh - 1) v2[t] = c2[t].push(v2[t], a.K, a.eqm);
                    v2[t] |= ~vmask[t];
                }
                if (act) {
                    uint32_t *p = s2 + (size_t)(i * a.groups + g) * slot + HALO + lt * NWT;
#pragma unroll
                    for (int t = 0; t < NWT; ++t) p[t] = v2[t];
                }
            }
        }
        if (a.nst == 2) {
            if (a.hmode) __syncthreads();
            // ---- phase C: stage-2 horizontal pass and store
            for (int i = 0; i < a.rb; ++i) {
                const int it = c0 + i;
                uint32_t h[NWT];
                const uint32_t *row = s2 + (size_t)(i * a.groups + gg) * slot;
                if (a.hmode) {
                    h_erode<NWT, HALO>(row + lt * NWT, h, a.hmode, a.sw, a.ex[1], a.m);
                } else {
#pragma unroll
                    for (int t = 0; t < NWT; ++t) h[t] = row[HALO + lt * NWT + t];
                }
                const int y = Y0 + it - wup;
                if (act && it >= wup && y < Y0 + a.band && y < a.H) {
#pragma unroll
                    for (int t = 0; t < NWT; ++t) {
                        const int w = w0 + t;
                        if (w >= strip0 && w < strip0 + a.strip_words && w < a.nw_cover) {
                            const uint32_t o = (a.inv_out ? ~h[t] : h[t]) & vmask[t];
                            a.dst[(int64_t)y * a.dstride + w] = o;
                        }
                    }
                }
            }
        }
    }
}

constexpr int NWT = 2;

template <int HALO, int KMAX>
cudaError_t launch_t(const PackedArgs &a, cudaStream_t s) {
    const int threads = ((a.groups * a.tpr + 31) / 32) * 32;
    const size_t smem = (size_t)a.nst * 2 * a.rb * a.groups * a.slot_words * sizeof(uint32_t);
    dim3 grid((a.H + a.groups * a.band - 1) / (a.groups * a.band), a.nstrips);
    auto kern = k_packed<NWT, HALO, KMAX>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<grid, threads, smem, s>>>(a);
    return cudaGetLastError();
}

template <int HALO>
cudaError_t launch_k(const PackedArgs &a, cudaStream_t s) {
    if (a.K <= 3) return launch_t<HALO, 3>(a, s);
    if (a.K <= 6) return launch_t<HALO, 6>(a, s);
    return launch_t<HALO, 16>(a, s);
}

int bit_length(int v) {
    int k = 0;
    while (v) { ++k; v >>= 1; }
    return k;
}

}  // namespace

int packed_halo(int sw, int ex) {
    const int reach = ex > sw - 1 - ex ? ex : sw - 1 - ex;
    const int hw = (reach + 31) / 32;
    if (hw <= 1) return 1;
    if (hw <= 2) return 2;
    if (hw <= 4) return 4;
    return 0;  // wider than the register window supports
}

// Fill the stage / tiling parameters.  Returns 0 on success, -1 if the
// rectangle is too wide for the horizontal register window.
int packed_plan(PackedArgs &a, int op, int sw, int sh, int ox, int oy, int band_hint,
                int threads_hint) {
    const int rx = sw - 1 - ox, ry = sh - 1 - oy;
    a.sw = sw;
    a.sh = sh;
    switch (op) {
    case MORPH_ERODE: a.nst = 1; a.ex[0] = ox; a.ey[0] = oy; a.inv_in = 0; a.inv_out = 0; break;
    case MORPH_DILATE: a.nst = 1; a.ex[0] = rx; a.ey[0] = ry; a.inv_in = 1; a.inv_out = 1; break;
    case MORPH_OPEN:
        a.nst = 2; a.ex[0] = ox; a.ey[0] = oy; a.ex[1] = rx; a.ey[1] = ry;
        a.inv_in = 0; a.inv_out = 1; break;
    default:
        a.nst = 2; a.ex[0] = rx; a.ey[0] = ry; a.ex[1] = ox; a.ey[1] = oy;
        a.inv_in = 1; a.inv_out = 0; break;
    }
    if (a.nst == 1) { a.ex[1] = a.ex[0]; a.ey[1] = a.ey[0]; }
    a.K = bit_length(sh);
    for (int k = 0; k < 16; ++k) a.eqm[k] = ((sh >> k) & 1) ? 0u : ONES;
    a.hmode = sw == 1 ? 0 : (sw <= 4 ? 1 : 2);
    a.m = bit_length(sw) - 1;
    const int halo = packed_halo(sw, ox);
    if (halo == 0) return -1;

    int max_threads = threads_hint > 0 ? threads_hint : MAX_THREADS;
    if (max_threads > MAX_THREADS) max_threads = MAX_THREADS;
    if (max_threads < 32) max_threads = 32;
    const int cover_threads = (a.nw_cover + NWT - 1) / NWT;
    if (cover_threads <= max_threads) {
        a.tpr = cover_threads;
        a.groups = max_threads / cover_threads;
        a.strip_words = a.nw_cover;
        a.halo_words = 0;
        a.nstrips = 1;
    } else {
        a.tpr = max_threads;
        a.groups = 1;
        a.halo_words = ((a.nst * halo + NWT - 1) / NWT) * NWT;
        a.strip_words = max_threads * NWT - 2 * a.halo_words;
        a.nstrips = (a.nw_cover + a.strip_words - 1) / a.strip_words;
    }
    a.rb = 4;
    const int wup = a.nst * (sh - 1);
    int band = band_hint > 0 ? band_hint : 4 * wup;
    if (band < 16) band = 16;
    if (band_hint <= 0 && band > 1024) band = 1024;
    a.band = ((band + a.rb - 1) / a.rb) * a.rb;
    // Never give a group more rows than the image has.
    const int hcap = ((a.H + a.rb - 1) / a.rb) * a.rb;
    if (a.band > hcap) a.band = hcap;
    if (a.groups * a.band > hcap) {
        a.groups = (hcap + a.band - 1) / a.band;
        if (a.groups < 1) a.groups = 1;
    }
    a.slot_words = a.tpr * NWT + 2 * halo;
    return 0;
}

cudaError_t launch_packed(PackedArgs &a, cudaStream_t s, int) {
    switch (packed_halo(a.sw, a.ex[0])) {
    case 1: return launch_k<1>(a, s);
    case 2: return launch_k<2>(a, s);
    case 4: return launch_k<4>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace morph
