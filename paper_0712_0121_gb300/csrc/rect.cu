// Planner of the packed rectangle tile (rect_tile.cuh): stage parameters
// (dilation by duality), kernel variant and tiling.
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "rle_rect.cuh"
#include "rect_tile.cuh"

namespace morph {
namespace {

int floor_log2(int v) {
    int k = -1;
    while (v) { ++k; v >>= 1; }
    return k;
}

int round_up(int v, int m) { return (v + m - 1) / m * m; }

constexpr int RECT_MAX_GROUPS = 16;

// Optional override of the tiling for tuning runs: MORPH_RECT_TILING =
// "nwt,threads,band,vmode" (0 keeps the default of the first three fields,
// -1 of the last).  Read once.
struct TilingOverride {
    int nwt = 0, threads = 0, band = 0, vmode = -1;
    TilingOverride() {
        const char *e = getenv("MORPH_RECT_TILING");
        if (e) sscanf(e, "%d,%d,%d,%d", &nwt, &threads, &band, &vmode);
    }
};
const TilingOverride &tiling_override() {
    static const TilingOverride t;
    return t;
}

// Horizontal tasks per thread and chunk for the current groups.
int task_count(const RectArgs &a) {
    const int total = rect_rb(a.nst) * a.groups * a.tph;
    return (total + a.threads - 1) / a.threads;
}

void set_band(RectArgs &a, int band) {
    band = round_up(band, RECT_RB);
    const int hcap = round_up(a.H, RECT_RB);
    if (band > hcap) band = hcap;
    const int full = a.threads / a.tpr;  // groups the CTA can hold
    a.groups = full;
    if (a.groups * band > hcap) a.groups = (hcap + band - 1) / band;
    if (a.groups < 1) a.groups = 1;
    a.band = band;
    a.ktasks = task_count(a);
}

// Fill the tiling for nwt words per thread and `threads` threads per CTA.
void tile(RectArgs &a, int nwt, int threads) {
    a.nwt = nwt;
    const int cover = a.nw_cover > a.nw_valid ? a.nw_cover : a.nw_valid;
    const int tpr = (cover + nwt - 1) / nwt;
    // narrow rows: at most RECT_MAX_GROUPS row groups per CTA (each group
    // holds exchange slots), the CTA shrunk to whole warps
    if (tpr * RECT_MAX_GROUPS < threads) threads = round_up(tpr * RECT_MAX_GROUPS, 32);
    a.threads = threads;
    if (tpr <= threads) {
        a.tpr = tpr;
        a.groups = threads / tpr;
        a.strip_words = cover;
        a.halo_words = 0;
        a.nstrips = 1;
    } else {
        a.tpr = threads;
        a.groups = 1;
        a.halo_words = round_up(a.nst * a.halo, nwt);
        a.strip_words = threads * nwt - 2 * a.halo_words;
        a.nstrips = (cover + a.strip_words - 1) / a.strip_words;
    }
    a.pad = round_up(a.halo > 0 ? a.halo : 1, 4);
    // a row of the exchange slot holds whole horizontal tasks of RECT_NWH words
    a.row_words = round_up(a.tpr * nwt, RECT_NWH);
    a.tph = a.row_words / RECT_NWH;
    a.slot_words = 2 * a.pad + a.row_words;
}


}  // namespace

int rect_plan(RectArgs &a, int op, int sw, int sh, int ox, int oy, int band_hint, int threads_hint,
              int nwt_hint, size_t smem_budget, bool rle_src) {
    const int rx = sw - 1 - ox, ry = sh - 1 - oy;
    a.sw = sw;
    a.sh = sh;
    switch (op) {
    case MORPH_ERODE:
        a.nst = 1; a.L[0] = ox; a.R[0] = rx; a.up[0] = oy; a.inv_in = 0; a.inv_out = 0; break;
    case MORPH_DILATE:  // erosion of the complement by the reflected rectangle
        a.nst = 1; a.L[0] = rx; a.R[0] = ox; a.up[0] = ry; a.inv_in = 1; a.inv_out = 1; break;
    case MORPH_OPEN:
        a.nst = 2; a.L[0] = ox; a.R[0] = rx; a.up[0] = oy; a.L[1] = rx; a.R[1] = ox; a.up[1] = ry;
        a.inv_in = 0; a.inv_out = 1; break;
    default:  // MORPH_CLOSE
        a.nst = 2; a.L[0] = rx; a.R[0] = ox; a.up[0] = ry; a.L[1] = ox; a.R[1] = rx; a.up[1] = oy;
        a.inv_in = 1; a.inv_out = 0; break;
    }
    if (a.nst == 1) {
        a.L[1] = a.L[0];
        a.R[1] = a.R[0];
        a.up[1] = a.up[0];
    }
    a.m = floor_log2(sw);
    const int reach = ox > rx ? ox : rx;
    if (reach > 128) return -1;
    if (sw == 1) { a.hmode = RH_NONE; a.halo = 1; }
    else if (reach <= 1) { a.hmode = RH_D1; a.halo = 1; }
    else if (reach <= 2) { a.hmode = RH_D2; a.halo = 1; }
    else {
        a.hmode = RH_LOG;
        const int hw = (reach + 31) / 32;
        a.halo = hw <= 1 ? 1 : (hw <= 2 ? 2 : 4);
    }
    a.vmode = sh == 1 ? RV_NONE : (sh <= 3 ? RV_W3 : RV_VHGW);
    // a run-length source does stage 1's within-line pass on the runs: one
    // stage has no within-line pass in the tile at all
    if (rle_src && a.nst == 1) {
        a.hmode = RH_NONE;
        a.halo = 1;
    }
    auto smem_words = [&](const RectArgs &t) { return rle_src ? rle_rect_smem_words(t) : rect_smem_words(t); };
    const TilingOverride &ov = tiling_override();
    const bool force_v = ov.vmode >= 0 && sh >= 4 && (ov.vmode == RV_VHGW || (ov.vmode == RV_CNT && sh <= RECT_CNT_SH));
    if (force_v) a.vmode = ov.vmode;
    if (!nwt_hint) nwt_hint = ov.nwt;
    if (!threads_hint) threads_hint = ov.threads;
    if (!band_hint) band_hint = ov.band;
    if (!smem_budget) smem_budget = 110 * 1024;
    // words per thread and CTA size: the first candidate whose shared
    // memory (exchange buffers, van Herk / Gil-Werman rings of sh rows)
    // fits the budget, so that two CTAs stay resident per SM.  Two stages
    // whose rings do not fit with 256 threads keep their per-column state
    // in registers instead (counters, two words per thread: four would
    // spill).
    const int cand[4][2] = {{4, 256}, {2, 256}, {4, 128}, {2, 128}};
    const int ncand = (a.nst == 2 && a.vmode == RV_VHGW && !force_v && sh <= RECT_CNT_SH) ? 2 : 4;
    bool done = false;
    for (int i = 0; i < ncand && !done; ++i) {
        const int nwt = nwt_hint ? nwt_hint : cand[i][0];
        const int thr = threads_hint ? threads_hint : cand[i][1];
        tile(a, nwt, thr);
        if (smem_words(a) * 4 <= smem_budget || (nwt_hint && threads_hint)) done = true;
    }
    if (a.nst == 2 && a.vmode == RV_VHGW && !force_v && sh <= RECT_CNT_SH &&
        (!done || smem_words(a) * 4 > smem_budget)) {
        a.vmode = RV_CNT;
        tile(a, nwt_hint ? nwt_hint : 2, threads_hint ? threads_hint : 256);
        done = true;
    }
    // two-stage counters: as many bit planes as sh has bits (the 4- and
    // 5-plane variants are built for two words per thread)
    if (rv_cnt(a.vmode) && a.nst == 2 && a.nwt == 2) a.vmode = sh < 16 ? RV_CNT4 : (sh < 32 ? RV_CNT5 : RV_CNT);
    // the run-length-source tile has counters for two stages and two words
    // per thread only (a forced tiling may ask for others)
    if (rle_src && rv_cnt(a.vmode) && (a.nst != 2 || a.nwt != 2)) return -1;
    if (!done) tile(a, 2, 128);
    // windows too tall for the rings of even the smallest tiling: the caller
    // falls back to the bit-sliced counter tile (O(log sh) state per word)
    if (smem_words(a) * 4 > RECT_SMEM_MAX) return -1;
    if (rle_src && a.nstrips != 1) return -1;  // the run painter covers one strip
    // output rows per group: a few windows' worth, so that the rows read
    // twice (the window's extra rows) stay a small share; without a hint the
    // launch refines it from the resident CTAs (rect_fit_band)
    const int wup = a.nst * (sh - 1);
    int band = band_hint > 0 ? band_hint : 4 * wup;
    if (band < 64) band = 64;
    if (band_hint <= 0 && band > 1024) band = 1024;
    a.band_auto = band_hint <= 0;
    set_band(a, band);
    a.nw_full = a.W / 32;
    a.vec16 = ((uintptr_t)a.dst % 16 == 0) && (a.dstride % 4 == 0);
    // one strip whose 8-word tasks all lie inside the written words: every
    // task stores two aligned 16-byte vectors, no per-word checks
    a.vec_tasks = a.vec16 && a.nstrips == 1 && a.halo_words == 0 && a.row_words <= a.nw_cover;
    // the horizontal tasks of a chunk must fit the threads' task slots (the
    // most groups a launch may give the CTA)
    {
        RectArgs t = a;
        t.groups = t.threads / t.tpr;
        if (task_count(t) > RECT_KT) return -1;
    }
    const int vb = a.nwt * 4;
    a.vec = ((uintptr_t)a.src % vb == 0) && ((uintptr_t)a.dst % vb == 0) && (a.sstride % a.nwt == 0) &&
            (a.dstride % a.nwt == 0);
    // every word of every thread loaded and stored whole: one strip whose
    // threads cover exactly the row's words
    a.vec_rows = a.vec && a.nstrips == 1 && a.tpr * a.nwt == a.nw_valid && a.nw_cover == a.nw_valid;
    return 0;
}

void rect_fit_band(RectArgs &a, int slots) {
    const int wup = a.nst * (a.sh - 1);
    const int full = a.threads / a.tpr;
    int64_t gslots = (int64_t)slots * full / a.nstrips;  // groups running at once per strip
    if (gslots < 1) gslots = 1;
    int base = 2 * wup > 32 ? 2 * wup : 32;        // smallest band worth a group
    int target = 4 * wup > 64 ? 4 * wup : 64;      // band that makes the extra rows small
    int64_t waves = (a.H + gslots * target / 2) / (gslots * target);
    if (waves < 1) waves = 1;
    int band = (int)((a.H + gslots * waves - 1) / (gslots * waves));
    if (band < base) band = base;
    set_band(a, band);
}

int rect_sm_count(int dev) {
    static int n[64] = {};
    if (dev < 0 || dev >= 64) return 148;
    if (!n[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) v = 1;
        n[dev] = v;
    }
    return n[dev];
}


cudaError_t launch_rect(const RectArgs &a, cudaStream_t s, const RectJobs *mj) {
    if (a.nst == 1) return a.nwt == 4 ? launch_rect_1_4(a, s, mj) : launch_rect_1_2(a, s, mj);
    return a.nwt == 4 ? launch_rect_2_4(a, s, mj) : launch_rect_2_2(a, s, mj);
}

}  // namespace morph

namespace morph {
cudaError_t launch_rle_rect_tile(const RectArgs &a, const RleSrc &src, cudaStream_t s, const RleJobs *mj) {
    return a.nwt == 4 ? launch_rle_rect_w4(a, src, s, mj) : launch_rle_rect_w2(a, src, s, mj);
}
}  // namespace morph
