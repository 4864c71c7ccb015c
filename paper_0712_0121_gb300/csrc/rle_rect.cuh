// Rectangle tile with a run-length source: erosion, dilation, opening and
// closing of an RLE image into a packed bitmap, both stages of an opening or
// closing in one pass (no intermediate bitmap, no re-encode between stages).
//
// Stage 1's within-line operation is done on the runs (section "Within-Line
// Morphological Operations": erode1d shrinks every run, dilate1d grows it,
// the clipped-window borders keep a run's end at the image side), while the
// runs are painted into shared-memory rows; the rest follows the packed
// rectangle tile (rect_tile.cuh): stage 1's between-line pass down each
// thread's word columns, then, for two stages, the stage-2 between-line pass
// in the same registers and the stage-2 within-line pass as row tasks.
//
// Per chunk of RB rows of every group: the rows' runs are one contiguous
// range of the CSR run array; the group's threads take its runs in turn,
// apply the row operation and OR them into a zeroed row slot (atomic OR on
// the partial end words).  The row slots are triple-buffered — iteration c
// paints chunk c + 1 and reads chunk c, and the readers clear the words they
// read, ready for chunk c + 3 — so one barrier per chunk suffices; the
// chunk's row offsets are staged one iteration earlier in the same way.
#pragma once

#include "rect_tile.cuh"
#include "rle_tile.cuh"

namespace morph {

struct RleSrc {
    const int32_t *row_ptr;   // H + 1 offsets
    const uint32_t *runs32;   // (start | end << 16) per run
    RowOp op1;                // stage-1 within-line operation on the runs
    int64_t cap;              // runs the array holds: offsets past it are never read
};

// Shared memory of the RLE-source tile in u32 words: three sets of painted
// row slots, the chunk row offsets (three sets), for two stages the stage-2
// exchange buffers, then the van Herk / Gil-Werman rings.
__host__ __device__ inline size_t rle_rect_rowset_words(const RectArgs &a) {
    return (size_t)rect_rb(a.nst) * a.groups * a.slot_words;
}
__host__ __device__ inline size_t rle_rect_rp_words(const RectArgs &a) {
    return ((size_t)a.groups * (rect_rb(a.nst) + 1) + 3) & ~(size_t)3;
}
__host__ __device__ inline size_t rle_rect_smem_words(const RectArgs &a) {
    const size_t x2 = a.nst == 2 && a.hmode != RH_NONE ? rect_xbuf_words(a) : 0;
    return 3 * rle_rect_rowset_words(a) + 3 * rle_rect_rp_words(a) + x2 + (size_t)a.nst * rect_ring_words(a);
}

template <int NST, int NWT, int VM, int HM, int HALO>
__device__ __forceinline__ void rle_rect_tile(const RectArgs &a, const RleSrc &src, int bx, uint32_t *sm) {
    constexpr int RB = rect_rb(NST);
    constexpr bool H2 = NST == 2 && HM != RH_NONE;  // stage-2 within-line pass as row tasks
    using RV = RectVec<NWT>;
    if (a.nwt != NWT || a.vmode != VM || a.nst != NST || (int)blockDim.x != a.threads || a.nstrips != 1 ||
        a.hmode != HM || a.halo != HALO)
        return;
    const int tid = threadIdx.x;
    const int tpr = a.tpr, groups = a.groups, band = a.band, H = a.H, W = a.W, sh = a.sh;
    const int g = tid / tpr, lt = tid - g * tpr;
    const bool act = g < groups;
    const int gg = act ? g : 0;
    const int w0 = lt * NWT;
    const int Y0 = (bx * groups + gg) * band;
    const int lagv = (sh - 1 + RB - 1) / RB * RB;
    const int ex = lagv - (sh - 1);
    const int lag = NST * lagv;
    const int n_in = band + lag;
    const int nch = n_in / RB;
    // input row of chunk row 0, for a group
    auto first_row = [&](int gq) {
        return (bx * groups + gq) * band - a.up[0] - (NST == 2 ? a.up[1] : 0) - NST * ex;
    };
    const int r_first = first_row(gg);
    const int y1_first = Y0 - (NST == 2 ? a.up[1] + ex : 0);

    uint32_t nmw[NWT], vmask[NWT];
    bool st_ok[NWT];
#pragma unroll
    for (int t = 0; t < NWT; ++t) {
        const int w = w0 + t;
        vmask[t] = w < a.nw_valid ? word_mask(w, W) : 0u;
        nmw[t] = ~vmask[t];
        st_ok[t] = act && w < a.nw_cover;
    }
    const bool vec_st = a.vec_rows != 0;
    const uint32_t inm_in = a.inv_in ? ONES : 0u, inm_out = a.inv_out ? ONES : 0u;

    const size_t rsw = rle_rect_rowset_words(a), rpw = rle_rect_rp_words(a);
    uint32_t *S = sm;                                              // 3 painted row sets
    int *RP = reinterpret_cast<int *>(sm + 3 * rsw);               // 3 row-offset sets
    uint32_t *X2 = sm + 3 * rsw + 3 * rpw;                         // stage-2 exchange
    uint32_t *ring_base = X2 + (H2 ? rect_xbuf_words(a) : 0);
    const int row_words = groups * a.slot_words;
    const int own_off = gg * a.slot_words + a.pad + lt * NWT;

    RectV<NWT, VM> v1, v2;
    v1.init(ring_base, tid, a.threads, sh);
    if constexpr (NST == 2) v2.init(ring_base + rect_ring_words(a), tid, a.threads, sh);
    RectTasks tasks;
    tasks.init(tid, a.threads, RB, groups, a.tph);

    // zero one painted row set (the pads included: words outside the row
    // become ones only through the stage-input mask, never by painting)
    auto zero_set = [&](int set) {
        uint4 *p = reinterpret_cast<uint4 *>(S + (size_t)set * rsw);
        const int n4 = (int)(rsw >> 2);
        for (int k = tid; k < n4; k += blockDim.x) p[k] = make_uint4(0u, 0u, 0u, 0u);
    };
    // row offsets of chunk c of every group: RP[set][gq][0..RB]
    auto stage_rp = [&](int c, int set) {
        int *rp = RP + (size_t)set * rpw;
        for (int k = tid; k < groups * (RB + 1); k += blockDim.x) {
            const int gq = k / (RB + 1), i = k - gq * (RB + 1);
            int r = first_row(gq) + c * RB + i;
            r = r < 0 ? 0 : (r > H ? H : r);
            rp[k] = src.row_ptr[r];
        }
    };
    // paint the runs of chunk c (offsets in RP[set]) into row set `set`
    // (four runs per thread are loaded before any is painted, so that their
    // global loads overlap)
    auto paint = [&](int c, int set) {
        if (!act) return;
        const int *rp = RP + (size_t)set * rpw + gg * (RB + 1);
        uint32_t *rows = S + (size_t)set * rsw + gg * a.slot_words + a.pad;
        const int q0 = rp[0];
        // an encode that overflowed its buffer (reported by the status
        // latch) leaves offsets past the runs: never read beyond them
        const int q1 = (int64_t)rp[RB] < src.cap ? rp[RB] : (int)src.cap;
        // the chunk's row boundaries in registers: a run's row is the number
        // of boundaries at or below it (offsets never decrease; empty rows
        // are skipped), no walk through shared memory
        int bnd[RB - 1];
#pragma unroll
        for (int i = 0; i < RB - 1; ++i) bnd[i] = rp[i + 1];
        for (int qb = q0 + lt; qb < q1; qb += 4 * tpr) {
            uint32_t pr[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int q = qb + e * tpr;
                pr[e] = q < q1 ? src.runs32[q] : 0u;
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int q = qb + e * tpr;
                if (q < q1) {
                    int row = 0;
#pragma unroll
                    for (int i = 0; i < RB - 1; ++i) row += q >= bnd[i] ? 1 : 0;
                    int s2, e2;
                    run_interval(pr[e], src.op1, s2, e2);
                    s2 = s2 < 0 ? 0 : s2;
                    e2 = e2 > W ? W : e2;
                    if (s2 < e2) paint_run(rows + (size_t)row * row_words, s2, e2);
                }
            }
        }
        (void)c;
    };

    // prologue: the stage-2 exchange slots' words outside the row are all
    // ones; the three painted sets zeroed (afterwards every painted word is
    // cleared by the thread that reads it), chunk 0's offsets staged and
    // painted, chunk 1's offsets staged
    if constexpr (H2) {
        const int nslots = 2 * RB * groups;
        const int row_end = a.pad + tpr * NWT;
        for (int s = tid; s < nslots; s += blockDim.x) {
            uint32_t *p = X2 + (size_t)s * a.slot_words;
            for (int j = 0; j < a.pad; ++j) p[j] = ONES;
            for (int j = row_end; j < a.slot_words; ++j) p[j] = ONES;
        }
    }
    zero_set(0);
    zero_set(1);
    zero_set(2);
    stage_rp(0, 0);
    if (nch > 1) stage_rp(1, 1);
    __syncthreads();
    paint(0, 0);
    __syncthreads();

    const int64_t dstride = a.dstride;
    uint32_t *sp = a.dst + w0 + (int64_t)Y0 * dstride;
    auto store = [&](const uint32_t (&h)[NWT], bool ok) {
        uint32_t o[NWT];
#pragma unroll
        for (int t = 0; t < NWT; ++t) o[t] = (h[t] ^ inm_out) & vmask[t];
        if (ok) {
            if (vec_st) {
                if (act) RV::st(sp, o);
            } else {
#pragma unroll
                for (int t = 0; t < NWT; ++t)
                    if (st_ok[t]) sp[t] = o[t];
            }
        }
        sp += dstride;
    };

    const int last = H2 ? nch : nch - 1;
    for (int c = 0; c <= last; ++c) {
        if (c + 2 < nch) stage_rp(c + 2, (c + 2) % 3);
        if (c + 1 < nch) paint(c + 1, (c + 1) % 3);
        if constexpr (H2) {
            const int c1 = c - 1;
            if (c1 >= 0 && c1 * RB >= lag)
                rect_htasks<HM, HALO, true>(a, tasks, X2 + (c1 & 1) * rect_xbuf_words(a) / 2, nullptr,
                                            c1 * RB - lag, a.L[1], a.R[1], bx, 0, a.nw_cover, inm_out,
                                            row_words);
        }
        if (c < nch) {
            const uint32_t *sb = S + (size_t)(c % 3) * rsw + own_off;
            uint32_t *xo = X2 + (c & 1) * rect_xbuf_words(a) / 2 + own_off;
            const int rc = r_first + c * RB;
            const bool out1 = c * RB >= lagv;
            const bool out2 = c * RB >= lag;
            const int u0 = c * RB - lag;
            const bool st_all = Y0 + u0 + RB <= H;
            const int y10 = y1_first + c * RB - lagv;
            const bool f2free = y10 >= 0 && y10 + RB <= H;
#pragma unroll
            for (int i = 0; i < RB; ++i) {
                uint32_t x[NWT], in[NWT], o[NWT];
                lds_own<NWT>(sb + i * row_words, x);
                if (act) {
                    // the painted words are read once: cleared here for the
                    // chunk painted into this set two iterations later
                    uint32_t z[NWT];
#pragma unroll
                    for (int t = 0; t < NWT; ++t) z[t] = 0u;
                    RV::st(const_cast<uint32_t *>(sb) + i * row_words, z);
                }
                const int r = rc + i;
                const uint32_t fill = (r >= 0 && r < H) ? 0u : ONES;
#pragma unroll
                for (int t = 0; t < NWT; ++t) in[t] = (x[t] ^ inm_in) | nmw[t] | fill;
                v1.push(in, o, sh);
                if constexpr (NST == 1) {
                    if (out2) store(o, st_all || Y0 + u0 + i < H);
                } else {
                    if (out1) {
                        const int y1 = y10 + i;
                        const uint32_t fill2 = (f2free || (y1 >= 0 && y1 < H)) ? 0u : ONES;
                        uint32_t in2[NWT], o2[NWT];
#pragma unroll
                        for (int t = 0; t < NWT; ++t) in2[t] = ~o[t] | nmw[t] | fill2;
                        v2.push(in2, o2, sh);
                        if constexpr (H2) {
                            if (act && out2) RV::st(xo + i * row_words, o2);
                        } else {
                            if (out2) store(o2, st_all || Y0 + u0 + i < H);
                        }
                    }
                }
            }
        }
        __syncthreads();
    }
}

}  // namespace morph

namespace morph {

// Host side (rle_rect_k*.cu): launch the run-length-source tile of a plan
// made by rect_plan(..., rle_src = true) with a.dst / a.dstride the bitmap
// it writes.
// A table entry of several RLE images of one variant in one launch: the
// plan, and the source runs as byte offsets from the launch's base pointer
// (the batch workspace).
struct RleJob {
    RectArgs a;
    int64_t off_row_ptr, off_runs;
    RowOp op1;
    int64_t cap;
};
struct RleJobs {
    const RleJob *jobs;  // device
    const int *starts;   // device: first CTA of each image, njobs + 1 entries
    const uint8_t *base;
    int njobs, ctas;
    size_t smem;
};
cudaError_t launch_rle_rect_tile(const RectArgs &a, const RleSrc &src, cudaStream_t s,
                                 const RleJobs *mj = nullptr);
cudaError_t launch_rle_rect_w2(const RectArgs &a, const RleSrc &src, cudaStream_t s, const RleJobs *mj);
cudaError_t launch_rle_rect_w4(const RectArgs &a, const RleSrc &src, cudaStream_t s, const RleJobs *mj);

}  // namespace morph
