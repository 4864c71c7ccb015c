// C ABI entry points of libmorph.so: argument checks, the choice of kernels
// for each operation and format, workspace layout and the device status latch.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "mask.cuh"
#include <vector>

#include "morph_internal.cuh"
#include "rect_tile.cuh"
#include "rle_rect.cuh"

namespace morph {

// First device-side condition latched since the last morph_sync_status().
__device__ int g_status;

namespace {

thread_local char t_err[512] = "";

morph_status fail(morph_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(t_err, sizeof(t_err), fmt, ap);
    va_end(ap);
    return st;
}

morph_status cuda_fail(cudaError_t e, const char *what) {
    return fail(MORPH_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

int word_bits(int fmt) { return fmt == MORPH_PACKED32 ? 32 : 64; }
bool is_packed(int fmt) { return fmt == MORPH_PACKED32 || fmt == MORPH_PACKED64; }

struct Range {
    uintptr_t lo, hi;  // [lo, hi)
};
bool overlap(Range a, Range b) { return a.lo < b.hi && b.lo < a.hi && a.lo < a.hi && b.lo < b.hi; }

Range packed_range(const morph_image *im) {
    const int64_t bpw = word_bits(im->fmt) / 8;
    const int64_t row_bytes = ((int64_t)im->width + word_bits(im->fmt) - 1) / word_bits(im->fmt) * bpw;
    const uintptr_t lo = (uintptr_t)im->words;
    return {lo, lo + (uintptr_t)(((int64_t)im->height - 1) * im->stride_words * bpw + row_bytes)};
}

morph_status check_image(const morph_image *im, const char *name) {
    if (!im) return fail(MORPH_EINVAL, "%s is NULL", name);
    if (im->reserved != 0) return fail(MORPH_EINVAL, "%s.reserved must be 0", name);
    if (im->width < 1 || im->height < 1)
        return fail(MORPH_EINVAL, "%s: width and height must be >= 1 (got %d x %d)", name,
                    im->width, im->height);
    if (is_packed(im->fmt)) {
        const int B = word_bits(im->fmt);
        if (!im->words) return fail(MORPH_EINVAL, "%s.words is NULL", name);
        if ((uintptr_t)im->words % (B / 8))
            return fail(MORPH_EINVAL, "%s.words is not aligned to %d bytes", name, B / 8);
        if (im->stride_words < ((int64_t)im->width + B - 1) / B)
            return fail(MORPH_EINVAL, "%s.stride_words %lld < ceil(width / %d)", name,
                        (long long)im->stride_words, B);
        return MORPH_OK;
    }
    if (im->fmt == MORPH_RLE) {
        if (im->width > 65535)
            return fail(MORPH_EINVAL, "%s: RLE width %d > 65535 (16-bit run ends)", name, im->width);
        if (!im->row_ptr) return fail(MORPH_EINVAL, "%s.row_ptr is NULL", name);
        if (im->capacity_runs < 0) return fail(MORPH_EINVAL, "%s.capacity_runs < 0", name);
        if (im->capacity_runs > 0 && !im->runs) return fail(MORPH_EINVAL, "%s.runs is NULL", name);
        if ((uintptr_t)im->runs % 4)
            return fail(MORPH_EINVAL, "%s.runs is not aligned to 4 bytes (one (start, end) pair)", name);
        return MORPH_OK;
    }
    return fail(MORPH_EINVAL, "%s.fmt %d is not a morph_format", name, im->fmt);
}


size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct RleWs {
    size_t counts, bmp, tmp_nruns, tmp_rowptr, tmp_runs, total;
    int64_t tmp_capacity;
};

// counts int32[H] | output rows as bitmap words | (open/close) intermediate RLE
RleWs rle_ws(int op, int W, int H) {
    RleWs w;
    w.counts = 0;
    size_t off = align256((size_t)H * sizeof(int32_t));
    w.bmp = off;
    off += align256((size_t)H * ((W + 31) / 32) * sizeof(uint32_t));
    w.tmp_capacity = 0;
    w.tmp_nruns = w.tmp_rowptr = w.tmp_runs = off;
    if (op == MORPH_OPEN || op == MORPH_CLOSE) {
        w.tmp_capacity = (int64_t)H * ((W + 1) / 2);
        w.tmp_nruns = off;
        off += align256(sizeof(int64_t));
        w.tmp_rowptr = off;
        off += align256((size_t)(H + 1) * sizeof(int32_t));
        w.tmp_runs = off;
        off += align256((size_t)w.tmp_capacity * 2 * sizeof(uint16_t));
    }
    w.total = off;
    return w;
}

}  // namespace

// Clip the rectangle to what can reach inside the image: a window side that
// sticks out further than W-1 (H-1) pixels covers the same clipped pixels.
Se clip_se(int W, int H, int sw, int sh, int ox, int oy) {
    int l = ox, r = sw - 1 - ox, u = oy, d = sh - 1 - oy;
    if (l > W - 1) l = W - 1;
    if (r > W - 1) r = W - 1;
    if (u > H - 1) u = H - 1;
    if (d > H - 1) d = H - 1;
    return {l + r + 1, u + d + 1, l, u};
}

morph_status check_op_args(int op, const morph_image *dst, const morph_image *src, int se_w,
                           int se_h, int ox, int oy) {
    morph_status st = check_image(src, "src");
    if (st) return st;
    if ((st = check_image(dst, "dst"))) return st;
    if (op < MORPH_ERODE || op > MORPH_CLOSE) return fail(MORPH_EINVAL, "op %d is not a morph_op", op);
    if (dst->width != src->width || dst->height != src->height)
        return fail(MORPH_EINVAL, "dst is %d x %d but src is %d x %d", dst->width, dst->height,
                    src->width, src->height);
    if (is_packed(src->fmt) != is_packed(dst->fmt))
        return fail(MORPH_EINVAL, "src and dst must both be packed or both be RLE");
    if (se_w < 1 || se_h < 1 || se_w > 65535 || se_h > 65535)
        return fail(MORPH_EINVAL, "structuring element %d x %d outside 1..65535", se_w, se_h);
    if (ox < 0 || ox >= se_w || oy < 0 || oy >= se_h)
        return fail(MORPH_EINVAL, "origin (%d, %d) outside the %d x %d rectangle", ox, oy, se_w, se_h);
    if (is_packed(src->fmt)) {
        if (overlap(packed_range(src), packed_range(dst))) return fail(MORPH_EINVAL, "dst overlaps src");
    } else {
        const Range srp{(uintptr_t)src->row_ptr, (uintptr_t)(src->row_ptr + src->height + 1)};
        const Range drp{(uintptr_t)dst->row_ptr, (uintptr_t)(dst->row_ptr + dst->height + 1)};
        const Range dru{(uintptr_t)dst->runs, (uintptr_t)(dst->runs + 2 * dst->capacity_runs)};
        const Range sru{(uintptr_t)src->runs, (uintptr_t)(src->runs + 2 * src->capacity_runs)};
        if (overlap(srp, drp) || overlap(srp, dru) || overlap(sru, drp) || overlap(sru, dru))
            return fail(MORPH_EINVAL, "dst overlaps src");
    }
    return MORPH_OK;
}

namespace {

// Horizontal reach of one fused launch (register window of 4 words).
constexpr int MAX_REACH = 128;

bool needs_chain(Se se) { return packed_halo(se.sw, se.ox) == 0; }

int chain_passes(Se se) {
    const int l = se.ox, r = se.sw - 1 - se.ox;
    const int nl = (l + MAX_REACH - 1) / MAX_REACH, nr = (r + MAX_REACH - 1) / MAX_REACH;
    return nl > nr ? nl : nr;
}

size_t packed_ws_bytes(int op, int W, int H, Se se) {
    if (!needs_chain(se)) return 0;
    const size_t img = align256((size_t)H * ((W + 31) / 32) * sizeof(uint32_t));
    return (op == MORPH_OPEN || op == MORPH_CLOSE ? 3 : 2) * img;
}

struct PackedBuf {
    const uint32_t *src;
    int64_t sstride;
    uint32_t *dst;
    int64_t dstride;
    int nw_cover;
};

cudaError_t packed_launch(int op, int W, int H, PackedBuf b, Se se, cudaStream_t s) {
    RectArgs a;
    memset(&a, 0, sizeof(a));
    a.src = b.src;
    a.sstride = b.sstride;
    a.dst = b.dst;
    a.dstride = b.dstride;
    a.W = W;
    a.H = H;
    a.nw_valid = (W + 31) / 32;
    a.nw_cover = b.nw_cover;
    // erosion / dilation: the vertical-first tile; opening / closing, and
    // windows taller than its van Herk / Gil-Werman rings hold: the tile with
    // bit-sliced column counters (one stage's ring less in shared memory)
    if (rect_plan(a, op, se.sw, se.sh, se.ox, se.oy, 0, 0, 0, 0) == 0) return launch_rect(a, s);
    PackedArgs p;
    memset(&p, 0, sizeof(p));
    p.src = b.src;
    p.sstride = b.sstride;
    p.dst = b.dst;
    p.dstride = b.dstride;
    p.W = W;
    p.H = H;
    p.nw_valid = (W + 31) / 32;
    p.nw_cover = b.nw_cover;
    if (packed_plan(p, op, se.sw, se.sh, se.ox, se.oy, 0, 0) != 0) return cudaErrorInvalidValue;
    return launch_packed(p, s);
}

// Erosion (or dilation) by a rectangle whose horizontal reach exceeds one
// launch: the segment [-l, r] is the Minkowski sum of segments [-l_k, r_k]
// (each containing 0, reach <= MAX_REACH); erosions by such segments compose
// exactly under the clipped window, so the passes run one after the other
// through scratch images; the vertical part rides on the last pass.
cudaError_t packed_chain(int op, int W, int H, PackedBuf io, Se se, uint32_t *t0, uint32_t *t1,
                         cudaStream_t s) {
    const int n = chain_passes(se);
    const int nwv = (W + 31) / 32;
    int l = se.ox, r = se.sw - 1 - se.ox;
    const uint32_t *in = io.src;
    int64_t in_stride = io.sstride;
    for (int k = 0; k < n; ++k) {
        const int lk = l / (n - k), rk = r / (n - k);
        l -= lk;
        r -= rk;
        const bool last = k == n - 1;
        uint32_t *out = last ? io.dst : (k % 2 == 0 ? t0 : t1);
        PackedBuf b{in, in_stride, out, last ? io.dstride : nwv, last ? io.nw_cover : nwv};
        Se sk{lk + rk + 1, last ? se.sh : 1, lk, last ? se.oy : 0};
        cudaError_t e = packed_launch(op, W, H, b, sk, s);
        if (e != cudaSuccess) return e;
        in = out;
        in_stride = nwv;
    }
    return cudaSuccess;
}

morph_status run_packed(int op, const morph_image *dst, const morph_image *src, Se se, void *ws,
                        size_t ws_bytes, cudaStream_t s) {
    const int W = src->width, H = src->height;
    PackedBuf io{(const uint32_t *)src->words, src->stride_words * (word_bits(src->fmt) / 32),
                 (uint32_t *)dst->words, dst->stride_words * (word_bits(dst->fmt) / 32),
                 dst->fmt == MORPH_PACKED32 ? (W + 31) / 32 : 2 * ((W + 63) / 64)};
    cudaError_t e;
    if (!needs_chain(se)) {
        e = packed_launch(op, W, H, io, se, s);
    } else {
        const size_t need = packed_ws_bytes(op, W, H, se);
        if (!ws || ws_bytes < need)
            return fail(MORPH_ENOMEM, "a %d-pixel-wide rectangle needs %zu bytes of workspace, got %zu",
                        se.sw, need, ws ? ws_bytes : (size_t)0);
        const size_t img = need / (op == MORPH_OPEN || op == MORPH_CLOSE ? 3 : 2);
        uint32_t *t0 = (uint32_t *)ws, *t1 = (uint32_t *)((char *)ws + img);
        if (op == MORPH_ERODE || op == MORPH_DILATE) {
            e = packed_chain(op, W, H, io, se, t0, t1, s);
        } else {
            const int nwv = (W + 31) / 32;
            uint32_t *mid = (uint32_t *)((char *)ws + 2 * img);
            const int first = op == MORPH_OPEN ? MORPH_ERODE : MORPH_DILATE;
            const int second = op == MORPH_OPEN ? MORPH_DILATE : MORPH_ERODE;
            PackedBuf a{io.src, io.sstride, mid, nwv, nwv};
            e = packed_chain(first, W, H, a, se, t0, t1, s);
            if (e == cudaSuccess) {
                PackedBuf b{mid, nwv, io.dst, io.dstride, io.nw_cover};
                e = packed_chain(second, W, H, b, se, t0, t1, s);
            }
        }
    }
    if (e != cudaSuccess) return cuda_fail(e, "packed morphology launch");
    return MORPH_OK;
}

RleIn rle_in(const morph_image *im) {
    return {im->row_ptr, im->runs, im->width, im->height};
}
RleOut rle_out(const morph_image *im) {
    return {im->row_ptr, im->runs, im->capacity_runs, im->n_runs};
}

morph_status run_rle(int op, const morph_image *dst, const morph_image *src, Se se, void *ws,
                     size_t ws_bytes, cudaStream_t s) {
    const int W = src->width, H = src->height;
    const RleWs L = rle_ws(op, W, H);
    if (!ws || ws_bytes < L.total)
        return fail(MORPH_ENOMEM, "workspace of %zu bytes is smaller than the %zu bytes needed",
                    ws ? ws_bytes : (size_t)0, L.total);
    char *base = (char *)ws;
    int32_t *counts = (int32_t *)(base + L.counts);
    uint32_t *bmp = (uint32_t *)(base + L.bmp);
    int *st = device_status_ptr();
    cudaError_t e;
    // windows taller than one row: the run-length-source tile (stage 1's
    // within-line pass on the runs, every between-line pass and stage 2 on
    // painted rows, both stages of an opening / closing in one pass) into
    // the bitmap scratch, then one encode into dst
    if (se.sh > 1) {
        const int nw = (W + 31) / 32;
        RectArgs a;
        memset(&a, 0, sizeof(a));
        a.dst = bmp;
        a.dstride = nw;
        a.W = W;
        a.H = H;
        a.nw_valid = nw;
        a.nw_cover = nw;
        if (rect_plan(a, op, se.sw, se.sh, se.ox, se.oy, 0, 0, 0, 0, true) == 0) {
            const int dil1 = op == MORPH_DILATE || op == MORPH_CLOSE;
            const RleSrc rs{src->row_ptr, reinterpret_cast<const uint32_t *>(src->runs), RowOp{dil1, se.sw, se.ox, W},
                            src->capacity_runs};
            e = launch_rle_rect_tile(a, rs, s);
            if (e == cudaSuccess) e = launch_rle_from_bitmap(bmp, nw, W, H, rle_out(dst), counts, st, s);
            if (e != cudaSuccess) return cuda_fail(e, "RLE morphology launch");
            return MORPH_OK;
        }
    }
    if (op == MORPH_ERODE || op == MORPH_DILATE) {
        e = launch_rle_rect(rle_in(src), rle_out(dst), op == MORPH_DILATE, se.sw, se.sh, se.ox,
                            se.oy, counts, bmp, st, s);
    } else {
        RleOut tmp{(int32_t *)(base + L.tmp_rowptr), (uint16_t *)(base + L.tmp_runs),
                   L.tmp_capacity, (int64_t *)(base + L.tmp_nruns)};
        const int first_dilate = op == MORPH_CLOSE;
        e = launch_rle_rect(rle_in(src), tmp, first_dilate, se.sw, se.sh, se.ox, se.oy, counts,
                            bmp, st, s);
        if (e == cudaSuccess) {
            RleIn tin{tmp.row_ptr, tmp.runs, W, H};
            e = launch_rle_rect(tin, rle_out(dst), !first_dilate, se.sw, se.sh, se.ox, se.oy,
                                counts, bmp, st, s);
        }
    }
    if (e != cudaSuccess) return cuda_fail(e, "RLE morphology launch");
    return MORPH_OK;
}

// ------------------------------------------------------ arbitrary masks
// Runs of the element (reflected for a dilation stage) into a.runs; fills
// a.nruns and a.nlev.  Errors: no pixel, too many runs.
morph_status mask_runs(const uint8_t *mask, int mw, int mh, int ox, int oy, bool reflect,
                       MaskArgs &a) {
    int n = 0, nlev = 0;
    const int rox = reflect ? mw - 1 - ox : ox, roy = reflect ? mh - 1 - oy : oy;
    for (int j = 0; j < mh; ++j) {
        const uint8_t *row = mask + (size_t)(reflect ? mh - 1 - j : j) * mw;
        auto in = [&](int i) { return row[reflect ? mw - 1 - i : i] != 0; };
        for (int i = 0; i < mw;) {
            if (!in(i)) { ++i; continue; }
            const int x0 = i;
            while (i < mw && in(i)) ++i;
            const int w = i - x0;
            if (n == MASK_MAX_RUNS)
                return fail(MORPH_EINVAL, "structuring element has more than %d horizontal runs",
                            MASK_MAX_RUNS);
            int m = 0;
            while ((2 << m) <= w) ++m;
            MaskRun &u = a.runs[n++];
            u.dy = (int16_t)(j - roy);
            u.dx1 = (int16_t)(x0 - rox);
            u.dx2 = (int16_t)(x0 - rox + w - (1 << m));
            u.m = (int16_t)m;
            if (m > nlev) nlev = m;
        }
    }
    if (n == 0) return fail(MORPH_EINVAL, "structuring element has no pixel");
    a.nruns = n;
    a.nlev = nlev;
    return MORPH_OK;
}

morph_status check_mask_args(int op, const morph_image *dst, const morph_image *src,
                             const uint8_t *mask, int mw, int mh, int ox, int oy) {
    morph_status st = check_image(src, "src");
    if (st) return st;
    if ((st = check_image(dst, "dst"))) return st;
    if (op < MORPH_ERODE || op > MORPH_CLOSE) return fail(MORPH_EINVAL, "op %d is not a morph_op", op);
    if (is_packed(src->fmt) != is_packed(dst->fmt))
        return fail(MORPH_EINVAL, "src and dst must both be packed or both be RLE");
    if (dst->width != src->width || dst->height != src->height)
        return fail(MORPH_EINVAL, "dst is %d x %d but src is %d x %d", dst->width, dst->height,
                    src->width, src->height);
    if (is_packed(src->fmt)) {
        if (overlap(packed_range(src), packed_range(dst))) return fail(MORPH_EINVAL, "dst overlaps src");
    } else {
        const Range srp{(uintptr_t)src->row_ptr, (uintptr_t)(src->row_ptr + src->height + 1)};
        const Range drp{(uintptr_t)dst->row_ptr, (uintptr_t)(dst->row_ptr + dst->height + 1)};
        const Range dru{(uintptr_t)dst->runs, (uintptr_t)(dst->runs + 2 * dst->capacity_runs)};
        const Range sru{(uintptr_t)src->runs, (uintptr_t)(src->runs + 2 * src->capacity_runs)};
        if (overlap(srp, drp) || overlap(srp, dru) || overlap(sru, drp) || overlap(sru, dru))
            return fail(MORPH_EINVAL, "dst overlaps src");
    }
    if (!mask) return fail(MORPH_EINVAL, "mask is NULL");
    if (mw < 1 || mh < 1 || mw > MASK_MAX_SIDE || mh > MASK_MAX_SIDE)
        return fail(MORPH_EINVAL, "mask %d x %d outside 1..%d", mw, mh, MASK_MAX_SIDE);
    if (ox < 0 || ox >= mw || oy < 0 || oy >= mh)
        return fail(MORPH_EINVAL, "origin (%d, %d) outside the %d x %d mask", ox, oy, mw, mh);
    return MORPH_OK;
}

// Runs of the element as painted intervals of one RLE stage (rle_mask.cu):
// a dilation paints each run [s, e) of line y - j + oy grown to
// [s + i0 - ox, e + i1 - 1 - ox); an erosion paints each gap of line
// y + j - oy grown to [s - (i1 - 1) + ox, e - i0 + ox) and complements.
morph_status rle_mask_runs(const uint8_t *mask, int mw, int mh, int ox, int oy, bool erode,
                           RleMaskArgs &a) {
    int n = 0;
    for (int j = 0; j < mh; ++j) {
        const uint8_t *row = mask + (size_t)j * mw;
        for (int i = 0; i < mw;) {
            if (!row[i]) { ++i; continue; }
            const int i0 = i;
            while (i < mw && row[i]) ++i;
            const int i1 = i;
            if (n == MASK_MAX_RUNS)
                return fail(MORPH_EINVAL, "structuring element has more than %d horizontal runs",
                            MASK_MAX_RUNS);
            RleMaskRun &u = a.runs[n++];
            if (erode) {
                u.dy = j - oy;
                u.lo = ox - (i1 - 1);
                u.hi = ox - i0;
            } else {
                u.dy = oy - j;
                u.lo = i0 - ox;
                u.hi = i1 - 1 - ox;
            }
        }
    }
    if (n == 0) return fail(MORPH_EINVAL, "structuring element has no pixel");
    a.nruns = n;
    return MORPH_OK;
}

// RLE images: each stage paints into the bitmap scratch and encodes it
// (open / close encode the first stage into the intermediate RLE).
morph_status run_rle_mask(int op, const morph_image *dst, const morph_image *src, const uint8_t *mask,
                          int mw, int mh, int ox, int oy, void *ws, size_t ws_bytes, cudaStream_t s) {
    static thread_local RleMaskArgs a;  // 12 KB: kept off the stack
    const int W = src->width, H = src->height, nw = (W + 31) / 32;
    const RleWs L = rle_ws(op, W, H);
    if (!ws || ws_bytes < L.total)
        return fail(MORPH_ENOMEM, "the mask operation needs %zu bytes of workspace, got %zu", L.total,
                    ws ? ws_bytes : (size_t)0);
    if ((uintptr_t)ws % 256) return fail(MORPH_EINVAL, "workspace is not 256-byte aligned");
    char *base = (char *)ws;
    int32_t *counts = (int32_t *)(base + L.counts);
    uint32_t *bmp = (uint32_t *)(base + L.bmp);
    int *st = device_status_ptr();
    const bool two = op == MORPH_OPEN || op == MORPH_CLOSE;
    const bool erode0 = op == MORPH_ERODE || op == MORPH_OPEN;
    morph_status ms = rle_mask_runs(mask, mw, mh, ox, oy, erode0, a);
    if (ms) return ms;
    a.row_ptr = src->row_ptr;
    a.runs_u16 = src->runs;
    a.W = W;
    a.H = H;
    a.dst = bmp;
    a.dstride = nw;
    a.nw = nw;
    a.erode = erode0;
    cudaError_t e = launch_rle_mask_stage(a, s);
    if (e == cudaSuccess && !two) e = launch_rle_from_bitmap(bmp, nw, W, H, rle_out(dst), counts, st, s);
    if (e == cudaSuccess && two) {
        // the intermediate holds up to ceil(W / 2) runs per line: never full
        const RleOut tmp{(int32_t *)(base + L.tmp_rowptr), (uint16_t *)(base + L.tmp_runs), L.tmp_capacity,
                         (int64_t *)(base + L.tmp_nruns)};
        e = launch_rle_from_bitmap(bmp, nw, W, H, tmp, counts, st, s);
        if (e == cudaSuccess) {
            if ((ms = rle_mask_runs(mask, mw, mh, ox, oy, !erode0, a))) return ms;
            a.row_ptr = tmp.row_ptr;
            a.runs_u16 = tmp.runs;
            a.erode = !erode0;
            e = launch_rle_mask_stage(a, s);
        }
        if (e == cudaSuccess) e = launch_rle_from_bitmap(bmp, nw, W, H, rle_out(dst), counts, st, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "RLE mask morphology launch");
    return MORPH_OK;
}

size_t mask_ws_bytes(int op, int W, int H, int nlev) {
    size_t n = align256(mask_levels_bytes(W, H, nlev));
    if (op == MORPH_OPEN || op == MORPH_CLOSE) n += align256((size_t)H * ((W + 31) / 32) * 4);
    return n;
}

// ---- sheared line elements: skew, vertical line, skew back
// The skew runs per band of lines, each band in its own canvas with its own
// base shift, so a canvas is only as much wider than the image as the
// shifts vary across one band (a skew of the whole image at once would need
// a canvas wider by the shift range of the whole height).  Bands carry
// L - 1 halo lines above and below, enough for either stage's window.
constexpr int LINE_MAX_SPAN = 1 << 20;

struct LinePlan {
    int band, halo, nb, brows, span;
};

LinePlan line_plan(int H, int L, const int32_t *shift, std::vector<int32_t> *base) {
    LinePlan p;
    p.band = 4 * L > 512 ? 4 * L : 512;
    if (p.band > H) p.band = H;
    p.halo = L - 1;
    p.nb = (H + p.band - 1) / p.band;
    p.brows = p.band + 2 * p.halo;
    p.span = 0;
    if (base) base->assign(p.nb, 0);
    for (int b = 0; b < p.nb; ++b) {
        const int y0 = b * p.band - p.halo < 0 ? 0 : b * p.band - p.halo;
        const int y1 = b * p.band + p.band + p.halo > H ? H : b * p.band + p.band + p.halo;
        int lo = shift[y0], hi = shift[y0];
        for (int y = y0 + 1; y < y1; ++y) {
            lo = shift[y] < lo ? shift[y] : lo;
            hi = shift[y] > hi ? shift[y] : hi;
        }
        if (base) (*base)[b] = lo;
        const int64_t sp = (int64_t)hi - lo;
        p.span = sp > LINE_MAX_SPAN ? LINE_MAX_SPAN + 1 : (sp > p.span ? (int)sp : p.span);
    }
    return p;
}

size_t line_ws_vertical(int op, int W, int H, const LinePlan &p) {
    const size_t nwc = ((size_t)W + p.span + 31) / 32, nw = ((size_t)W + 31) / 32;
    const size_t crows = (size_t)p.nb * p.brows;
    size_t n = align256((size_t)H * 4) + align256((size_t)p.nb * 4) + 2 * align256(crows * nwc * 4);
    if (op == MORPH_OPEN || op == MORPH_CLOSE) n += align256((size_t)H * nw * 4);
    return n;
}

// W x H: the image the vertical procedure runs on (the transpose for
// horizontal lines)
size_t line_ws(int op, int W, int H, const LinePlan &p, int horizontal) {
    if (!horizontal) return line_ws_vertical(op, W, H, p);
    const size_t nwt = ((size_t)W + 31) / 32;  // rows of the transposed image
    return 2 * align256((size_t)H * nwt * 4) + line_ws_vertical(op, W, H, p);
}

// One stage (erode or dilate) of u32 rows: skew into the band canvases A
// (fill = the value the clipped window ignores), vertical line A -> B,
// skew back to dst.
cudaError_t line_stage(bool dil, const uint32_t *src, int64_t sst, uint32_t *dst, int64_t dstride,
                       int dst_cover, int W, int H, const int32_t *dshift, const int32_t *dbase,
                       const LinePlan &p, int L, int o, uint32_t *A, uint32_t *B, cudaStream_t s) {
    const int Wc = W + p.span, nwc = (Wc + 31) / 32, crows = p.nb * p.brows;
    cudaError_t e = launch_shift_rows(src, sst, W, A, nwc, Wc, nwc, crows, H, dshift, dbase, p.band, p.halo, 1,
                                      dil ? 0u : ONES, s);
    if (e != cudaSuccess) return e;
    e = packed_launch(dil ? MORPH_DILATE : MORPH_ERODE, Wc, crows, PackedBuf{A, nwc, B, nwc, nwc},
                      clip_se(Wc, crows, 1, L, 0, o), s);
    if (e != cudaSuccess) return e;
    return launch_shift_rows(B, nwc, Wc, dst, dstride, W, dst_cover, H, H, dshift, dbase, p.band, p.halo, -1,
                             0u, s);
}

// The sheared vertical line on a W x H image of u32 rows; ws holds
// line_ws_vertical(op, W, H, p) bytes.
cudaError_t line_vertical(int op, const uint32_t *src, int64_t sst, uint32_t *dst, int64_t dstride,
                          int dst_cover, int W, int H, const int32_t *shift, const LinePlan &p,
                          const std::vector<int32_t> &base, int L, int o, char *ws, cudaStream_t s) {
    const size_t nwc = ((size_t)W + p.span + 31) / 32, nw = ((size_t)W + 31) / 32;
    const size_t crows = (size_t)p.nb * p.brows;
    int32_t *dshift = (int32_t *)ws;
    int32_t *dbase = (int32_t *)(ws + align256((size_t)H * 4));
    uint32_t *A = (uint32_t *)((char *)dbase + align256((size_t)p.nb * 4));
    uint32_t *B = (uint32_t *)((char *)A + align256(crows * nwc * 4));
    uint32_t *T = (uint32_t *)((char *)B + align256(crows * nwc * 4));
    cudaError_t e = cudaMemcpyAsync(dshift, shift, (size_t)H * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dbase, base.data(), (size_t)p.nb * 4, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    if (op == MORPH_ERODE || op == MORPH_DILATE)
        return line_stage(op == MORPH_DILATE, src, sst, dst, dstride, dst_cover, W, H, dshift, dbase, p, L, o,
                          A, B, s);
    const bool dil0 = op == MORPH_CLOSE;
    e = line_stage(dil0, src, sst, T, (int64_t)nw, (int)nw, W, H, dshift, dbase, p, L, o, A, B, s);
    if (e != cudaSuccess) return e;
    return line_stage(!dil0, T, (int64_t)nw, dst, dstride, dst_cover, W, H, dshift, dbase, p, L, o, A, B, s);
}

}  // namespace

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(t_err, sizeof(t_err), fmt, ap);
    va_end(ap);
}

int *device_status_ptr() {
    static std::mutex mu;
    static int *ptrs[128] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!ptrs[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_status) == cudaSuccess) ptrs[dev] = (int *)p;
    }
    return ptrs[dev];
}

}  // namespace morph

using namespace morph;

extern "C" {

morph_status morph_rect(int op, const morph_image *dst, const morph_image *src, int se_w, int se_h,
                        int origin_x, int origin_y, void *workspace, size_t workspace_bytes,
                        void *stream) {
    morph_status st = check_op_args(op, dst, src, se_w, se_h, origin_x, origin_y);
    if (st) return st;
    const Se se = clip_se(src->width, src->height, se_w, se_h, origin_x, origin_y);
    cudaStream_t s = (cudaStream_t)stream;
    if (is_packed(src->fmt)) return run_packed(op, dst, src, se, workspace, workspace_bytes, s);
    return run_rle(op, dst, src, se, workspace, workspace_bytes, s);
}

morph_status morph_erode_rect(const morph_image *dst, const morph_image *src, int se_w, int se_h,
                              int origin_x, int origin_y, void *workspace,
                              size_t workspace_bytes, void *stream) {
    return morph_rect(MORPH_ERODE, dst, src, se_w, se_h, origin_x, origin_y, workspace,
                      workspace_bytes, stream);
}

morph_status morph_dilate_rect(const morph_image *dst, const morph_image *src, int se_w, int se_h,
                               int origin_x, int origin_y, void *workspace,
                               size_t workspace_bytes, void *stream) {
    return morph_rect(MORPH_DILATE, dst, src, se_w, se_h, origin_x, origin_y, workspace,
                      workspace_bytes, stream);
}

morph_status morph_open_rect(const morph_image *dst, const morph_image *src, int se_w, int se_h,
                             int origin_x, int origin_y, void *workspace, size_t workspace_bytes,
                             void *stream) {
    return morph_rect(MORPH_OPEN, dst, src, se_w, se_h, origin_x, origin_y, workspace,
                      workspace_bytes, stream);
}

morph_status morph_close_rect(const morph_image *dst, const morph_image *src, int se_w, int se_h,
                              int origin_x, int origin_y, void *workspace,
                              size_t workspace_bytes, void *stream) {
    return morph_rect(MORPH_CLOSE, dst, src, se_w, se_h, origin_x, origin_y, workspace,
                      workspace_bytes, stream);
}

size_t morph_workspace_size(int op, const morph_image *dst, const morph_image *src, int se_w,
                            int se_h, int origin_x, int origin_y) {
    (void)dst;
    if (!src || src->width < 1 || src->height < 1 || se_w < 1 || se_h < 1 || origin_x < 0 ||
        origin_x >= se_w || origin_y < 0 || origin_y >= se_h)
        return 0;
    if (is_packed(src->fmt)) {
        const Se se = clip_se(src->width, src->height, se_w, se_h, origin_x, origin_y);
        return packed_ws_bytes(op, src->width, src->height, se);
    }
    return rle_ws(op, src->width, src->height).total;
}

size_t morph_mask_workspace_size(int op, const morph_image *dst, const morph_image *src,
                                 const uint8_t *mask, int mask_w, int mask_h, int origin_x,
                                 int origin_y) {
    if (check_mask_args(op, dst, src, mask, mask_w, mask_h, origin_x, origin_y)) return 0;
    if (src->fmt == MORPH_RLE) {
        static thread_local RleMaskArgs r;
        if (rle_mask_runs(mask, mask_w, mask_h, origin_x, origin_y, true, r)) return 0;
        return rle_ws(op, src->width, src->height).total;
    }
    static thread_local MaskArgs a;
    if (mask_runs(mask, mask_w, mask_h, origin_x, origin_y, false, a)) return 0;
    return mask_ws_bytes(op, src->width, src->height, a.nlev);
}

morph_status morph_mask(int op, const morph_image *dst, const morph_image *src, const uint8_t *mask,
                        int mask_w, int mask_h, int origin_x, int origin_y, void *workspace,
                        size_t workspace_bytes, void *stream) {
    morph_status st = check_mask_args(op, dst, src, mask, mask_w, mask_h, origin_x, origin_y);
    if (st) return st;
    if (src->fmt == MORPH_RLE)
        return run_rle_mask(op, dst, src, mask, mask_w, mask_h, origin_x, origin_y, workspace,
                            workspace_bytes, (cudaStream_t)stream);
    static thread_local MaskArgs a;  // 8 KB: kept off the stack
    const int W = src->width, H = src->height, nwv = (W + 31) / 32;
    // stages: erosion by the element (AND) or dilation by the reflected one (OR)
    const bool two = op == MORPH_OPEN || op == MORPH_CLOSE;
    const bool dil0 = op == MORPH_DILATE || op == MORPH_CLOSE;
    if ((st = mask_runs(mask, mask_w, mask_h, origin_x, origin_y, dil0, a))) return st;
    const size_t need = mask_ws_bytes(op, W, H, a.nlev);
    if (need && (!workspace || workspace_bytes < need))
        return fail(MORPH_ENOMEM, "the mask operation needs %zu bytes of workspace, got %zu", need,
                    workspace ? workspace_bytes : (size_t)0);
    if ((uintptr_t)workspace % 256) return fail(MORPH_EINVAL, "workspace is not 256-byte aligned");
    uint32_t *levels = (uint32_t *)workspace;
    uint32_t *mid = two ? (uint32_t *)((char *)workspace + align256(mask_levels_bytes(W, H, a.nlev)))
                        : nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    a.W = W;
    a.H = H;
    a.nw_valid = nwv;
    a.levels = levels;
    a.src = (const uint32_t *)src->words;
    a.sstride = src->stride_words * (word_bits(src->fmt) / 32);
    a.use_or = dil0;
    if (two) {
        a.dst = mid;
        a.dstride = nwv;
        a.nw_cover = nwv;
    } else {
        a.dst = (uint32_t *)dst->words;
        a.dstride = dst->stride_words * (word_bits(dst->fmt) / 32);
        a.nw_cover = dst->fmt == MORPH_PACKED32 ? nwv : 2 * ((W + 63) / 64);
    }
    cudaError_t e = launch_mask_stage(a, s);
    if (e == cudaSuccess && two) {
        if ((st = mask_runs(mask, mask_w, mask_h, origin_x, origin_y, !dil0, a))) return st;
        a.src = mid;
        a.sstride = nwv;
        a.dst = (uint32_t *)dst->words;
        a.dstride = dst->stride_words * (word_bits(dst->fmt) / 32);
        a.nw_cover = dst->fmt == MORPH_PACKED32 ? nwv : 2 * ((W + 63) / 64);
        a.use_or = !dil0;
        e = launch_mask_stage(a, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "mask morphology launch");
    return MORPH_OK;
}

size_t morph_convert_workspace_size(int height) {
    return height < 1 ? 0 : align256((size_t)height * sizeof(int32_t));
}

morph_status rle_from_bitmap(const morph_image *dst_rle, const morph_image *src_packed,
                             void *workspace, size_t workspace_bytes, void *stream) {
    morph_status st = check_image(src_packed, "src");
    if (st) return st;
    if ((st = check_image(dst_rle, "dst"))) return st;
    if (!is_packed(src_packed->fmt) || dst_rle->fmt != MORPH_RLE)
        return fail(MORPH_EINVAL, "rle_from_bitmap needs a packed src and an RLE dst");
    if (dst_rle->width != src_packed->width || dst_rle->height != src_packed->height)
        return fail(MORPH_EINVAL, "dst and src sizes differ");
    const size_t need = morph_convert_workspace_size(src_packed->height);
    if (!workspace || workspace_bytes < need)
        return fail(MORPH_ENOMEM, "workspace of %zu bytes is smaller than the %zu bytes needed",
                    workspace ? workspace_bytes : (size_t)0, need);
    const Range src_r = packed_range(src_packed);
    const Range drp{(uintptr_t)dst_rle->row_ptr, (uintptr_t)(dst_rle->row_ptr + dst_rle->height + 1)};
    const Range dru{(uintptr_t)dst_rle->runs, (uintptr_t)(dst_rle->runs + 2 * dst_rle->capacity_runs)};
    if (overlap(src_r, drp) || overlap(src_r, dru)) return fail(MORPH_EINVAL, "dst overlaps src");
    cudaError_t e = launch_rle_from_bitmap(
        (const uint32_t *)src_packed->words, src_packed->stride_words * (word_bits(src_packed->fmt) / 32),
        src_packed->width, src_packed->height, rle_out(dst_rle), (int32_t *)workspace,
        device_status_ptr(), (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "rle_from_bitmap launch");
    return MORPH_OK;
}

morph_status rle_to_bitmap(const morph_image *dst_packed, const morph_image *src_rle, void *stream) {
    morph_status st = check_image(src_rle, "src");
    if (st) return st;
    if ((st = check_image(dst_packed, "dst"))) return st;
    if (src_rle->fmt != MORPH_RLE || !is_packed(dst_packed->fmt))
        return fail(MORPH_EINVAL, "rle_to_bitmap needs an RLE src and a packed dst");
    if (dst_packed->width != src_rle->width || dst_packed->height != src_rle->height)
        return fail(MORPH_EINVAL, "dst and src sizes differ");
    const Range dst_r = packed_range(dst_packed);
    const Range srp{(uintptr_t)src_rle->row_ptr, (uintptr_t)(src_rle->row_ptr + src_rle->height + 1)};
    const Range sru{(uintptr_t)src_rle->runs, (uintptr_t)(src_rle->runs + 2 * src_rle->capacity_runs)};
    if (overlap(dst_r, srp) || overlap(dst_r, sru)) return fail(MORPH_EINVAL, "dst overlaps src");
    const int W = dst_packed->width;
    const int nw_cover = dst_packed->fmt == MORPH_PACKED32 ? (W + 31) / 32 : 2 * ((W + 63) / 64);
    cudaError_t e = launch_rle_to_bitmap(rle_in(src_rle), (uint32_t *)dst_packed->words,
                                         dst_packed->stride_words * (word_bits(dst_packed->fmt) / 32),
                                         nw_cover, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "rle_to_bitmap launch");
    return MORPH_OK;
}

size_t morph_components_workspace_size(const morph_image *src_rle) {
    if (!src_rle || src_rle->fmt != MORPH_RLE || src_rle->height < 1 || src_rle->capacity_runs < 0 ||
        src_rle->capacity_runs > INT32_MAX)
        return 0;
    const size_t H = (size_t)src_rle->height;
    const size_t cap = src_rle->capacity_runs > 0 ? (size_t)src_rle->capacity_runs : 1;
    return align256(H * 4) + align256((H + 1) * 4) + align256(cap * 4);
}

morph_status morph_rle_components(int32_t *labels, morph_component *stats, int64_t max_components,
                                  int64_t *n_components, const morph_image *src_rle,
                                  int connectivity, void *workspace, size_t workspace_bytes,
                                  void *stream) {
    morph_status st = check_image(src_rle, "src");
    if (st) return st;
    if (src_rle->fmt != MORPH_RLE) return fail(MORPH_EINVAL, "morph_rle_components needs an RLE src");
    if (src_rle->capacity_runs > INT32_MAX)
        return fail(MORPH_EINVAL, "src.capacity_runs above 2^31 - 1 (int32 labels)");
    if (connectivity != 4 && connectivity != 8)
        return fail(MORPH_EINVAL, "connectivity %d is neither 4 nor 8", connectivity);
    if (!labels || !n_components) return fail(MORPH_EINVAL, "labels and n_components must not be NULL");
    if ((uintptr_t)labels % 4 || (uintptr_t)n_components % 8 || (uintptr_t)stats % 8)
        return fail(MORPH_EINVAL, "labels, n_components or stats misaligned");
    if (stats && max_components < 0) return fail(MORPH_EINVAL, "max_components < 0");
    const int H = src_rle->height;
    const int64_t cap = src_rle->capacity_runs;
    const Range srp{(uintptr_t)src_rle->row_ptr, (uintptr_t)(src_rle->row_ptr + H + 1)};
    const Range sru{(uintptr_t)src_rle->runs, (uintptr_t)(src_rle->runs + 2 * cap)};
    const Range lr{(uintptr_t)labels, (uintptr_t)(labels + cap)};
    const Range sr{(uintptr_t)stats, (uintptr_t)(stats ? stats + max_components : stats)};
    const Range nr{(uintptr_t)n_components, (uintptr_t)(n_components + 1)};
    if (overlap(lr, srp) || overlap(lr, sru) || overlap(sr, srp) || overlap(sr, sru) ||
        overlap(lr, sr) || overlap(nr, lr) || overlap(nr, sr) || overlap(nr, srp) || overlap(nr, sru))
        return fail(MORPH_EINVAL, "labels, stats, n_components and src overlap");
    const size_t need = morph_components_workspace_size(src_rle);
    if (!workspace || workspace_bytes < need)
        return fail(MORPH_ENOMEM, "the components need %zu bytes of workspace, got %zu", need,
                    workspace ? workspace_bytes : (size_t)0);
    if ((uintptr_t)workspace % 256) return fail(MORPH_EINVAL, "workspace is not 256-byte aligned");
    char *w = (char *)workspace;
    MorphCC c;
    c.labels = labels;
    c.stats = stats;
    c.max_components = stats ? max_components : 0;
    c.n_components = n_components;
    c.counts = (int32_t *)w;
    c.rootptr = (int32_t *)(w + align256((size_t)H * 4));
    c.rank = (int32_t *)(w + align256((size_t)H * 4) + align256((size_t)(H + 1) * 4));
    cudaError_t e = launch_rle_components(rle_in(src_rle), connectivity, c, device_status_ptr(),
                                          (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "connected components launch");
    return MORPH_OK;
}

morph_status morph_run_length_hist(int64_t *black_hist, int64_t *white_hist,
                                   const morph_image *src_rle, void *stream) {
    morph_status st = check_image(src_rle, "src");
    if (st) return st;
    if (src_rle->fmt != MORPH_RLE) return fail(MORPH_EINVAL, "morph_run_length_hist needs an RLE src");
    if ((uintptr_t)black_hist % 8 || (uintptr_t)white_hist % 8)
        return fail(MORPH_EINVAL, "histograms are not 8-byte aligned");
    const int W = src_rle->width, H = src_rle->height;
    const int64_t cap = src_rle->capacity_runs;
    const Range srp{(uintptr_t)src_rle->row_ptr, (uintptr_t)(src_rle->row_ptr + H + 1)};
    const Range sru{(uintptr_t)src_rle->runs, (uintptr_t)(src_rle->runs + 2 * cap)};
    const Range br{(uintptr_t)black_hist, (uintptr_t)(black_hist ? black_hist + W + 1 : black_hist)};
    const Range wr{(uintptr_t)white_hist, (uintptr_t)(white_hist ? white_hist + W + 1 : white_hist)};
    if (overlap(br, wr) || overlap(br, srp) || overlap(br, sru) || overlap(wr, srp) || overlap(wr, sru))
        return fail(MORPH_EINVAL, "histograms and src overlap");
    if (!black_hist && !white_hist) return MORPH_OK;
    cudaError_t e = launch_run_length_hist(rle_in(src_rle), black_hist, white_hist, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "run-length histogram launch");
    return MORPH_OK;
}

morph_status morph_transpose(const morph_image *dst, const morph_image *src, void *stream) {
    morph_status st = check_image(src, "src");
    if (st) return st;
    if ((st = check_image(dst, "dst"))) return st;
    if (!is_packed(src->fmt) || !is_packed(dst->fmt))
        return fail(MORPH_EINVAL, "morph_transpose needs packed images (morph_rle_transpose for RLE)");
    if (dst->width != src->height || dst->height != src->width)
        return fail(MORPH_EINVAL, "dst is %d x %d, the transpose of %d x %d must be %d x %d", dst->width,
                    dst->height, src->width, src->height, src->height, src->width);
    if (overlap(packed_range(src), packed_range(dst))) return fail(MORPH_EINVAL, "dst overlaps src");
    const int nw_out = dst->fmt == MORPH_PACKED32 ? (dst->width + 31) / 32 : 2 * ((dst->width + 63) / 64);
    cudaError_t e = launch_transpose((const uint32_t *)src->words, src->stride_words * (word_bits(src->fmt) / 32),
                                     src->width, src->height, (uint32_t *)dst->words,
                                     dst->stride_words * (word_bits(dst->fmt) / 32), nw_out,
                                     (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "transpose launch");
    return MORPH_OK;
}

size_t morph_rle_transpose_workspace_size(const morph_image *src_rle) {
    if (!src_rle || src_rle->fmt != MORPH_RLE || src_rle->width < 1 || src_rle->height < 1) return 0;
    return rle_transpose_ws_bytes(src_rle->width, src_rle->height);
}

morph_status morph_rle_transpose(const morph_image *dst_rle, const morph_image *src_rle, void *workspace,
                                 size_t workspace_bytes, void *stream) {
    morph_status st = check_image(src_rle, "src");
    if (st) return st;
    if ((st = check_image(dst_rle, "dst"))) return st;
    if (src_rle->fmt != MORPH_RLE || dst_rle->fmt != MORPH_RLE)
        return fail(MORPH_EINVAL, "morph_rle_transpose needs RLE images (morph_transpose for packed)");
    if (dst_rle->width != src_rle->height || dst_rle->height != src_rle->width)
        return fail(MORPH_EINVAL, "dst is %d x %d, the transpose of %d x %d must be %d x %d",
                    dst_rle->width, dst_rle->height, src_rle->width, src_rle->height,
                    src_rle->height, src_rle->width);
    const Range srp{(uintptr_t)src_rle->row_ptr, (uintptr_t)(src_rle->row_ptr + src_rle->height + 1)};
    const Range sru{(uintptr_t)src_rle->runs, (uintptr_t)(src_rle->runs + 2 * src_rle->capacity_runs)};
    const Range drp{(uintptr_t)dst_rle->row_ptr, (uintptr_t)(dst_rle->row_ptr + dst_rle->height + 1)};
    const Range dru{(uintptr_t)dst_rle->runs, (uintptr_t)(dst_rle->runs + 2 * dst_rle->capacity_runs)};
    if (overlap(drp, srp) || overlap(drp, sru) || overlap(dru, srp) || overlap(dru, sru))
        return fail(MORPH_EINVAL, "dst overlaps src");
    const size_t need = rle_transpose_ws_bytes(src_rle->width, src_rle->height);
    if (!workspace || workspace_bytes < need)
        return fail(MORPH_ENOMEM, "the transpose needs %zu bytes of workspace, got %zu", need,
                    workspace ? workspace_bytes : (size_t)0);
    if ((uintptr_t)workspace % 256) return fail(MORPH_EINVAL, "workspace is not 256-byte aligned");
    cudaError_t e = launch_rle_transpose(rle_in(src_rle), rle_out(dst_rle), workspace, device_status_ptr(),
                                         (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "RLE transpose launch");
    return MORPH_OK;
}

size_t morph_sheared_line_workspace_size(int op, const morph_image *src, const int32_t *shift,
                                         int n_shift, int length, int horizontal) {
    if (!src || src->width < 1 || src->height < 1 || !shift || op < MORPH_ERODE || op > MORPH_CLOSE ||
        length < 1)
        return 0;
    if (n_shift != (horizontal ? src->width : src->height)) return 0;
    // the vertical procedure runs on the transpose for horizontal lines
    const int W = horizontal ? src->height : src->width, H = n_shift;
    const LinePlan p = line_plan(H, length, shift, nullptr);
    if (p.span > LINE_MAX_SPAN) return 0;
    return line_ws(op, W, H, p, horizontal);
}

morph_status morph_sheared_line(int op, const morph_image *dst, const morph_image *src, const int32_t *shift,
                                int n_shift, int length, int origin, int horizontal, void *workspace,
                                size_t workspace_bytes, void *stream) {
    morph_status st = check_image(src, "src");
    if (st) return st;
    if ((st = check_image(dst, "dst"))) return st;
    if (op < MORPH_ERODE || op > MORPH_CLOSE) return fail(MORPH_EINVAL, "op %d is not erode/dilate/open/close", op);
    if (!is_packed(src->fmt) || !is_packed(dst->fmt)) return fail(MORPH_EINVAL, "sheared lines need packed images");
    if (dst->width != src->width || dst->height != src->height) return fail(MORPH_EINVAL, "dst and src sizes differ");
    if (overlap(packed_range(src), packed_range(dst))) return fail(MORPH_EINVAL, "dst overlaps src");
    const int W = src->width, H = src->height;
    if (!shift) return fail(MORPH_EINVAL, "shift is NULL");
    if (n_shift != (horizontal ? W : H))
        return fail(MORPH_EINVAL, "n_shift %d: one shift per %s needed (%d)", n_shift, horizontal ? "column" : "line",
                    horizontal ? W : H);
    if (length < 1 || origin < 0 || origin >= length)
        return fail(MORPH_EINVAL, "line of length %d with origin %d", length, origin);
    // the vertical procedure's image: the transpose for horizontal lines
    const int Wv = horizontal ? H : W, Hv = n_shift;
    std::vector<int32_t> base;
    const LinePlan p = line_plan(Hv, length, shift, &base);
    if (p.span > LINE_MAX_SPAN)
        return fail(MORPH_EINVAL, "shifts vary by more than %d pixels within one band", LINE_MAX_SPAN);
    const size_t need = line_ws(op, Wv, Hv, p, horizontal);
    if (!workspace || workspace_bytes < need)
        return fail(MORPH_ENOMEM, "the sheared line needs %zu bytes of workspace, got %zu", need,
                    workspace ? workspace_bytes : (size_t)0);
    if ((uintptr_t)workspace % 256) return fail(MORPH_EINVAL, "workspace is not 256-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t *sw = (const uint32_t *)src->words;
    const int64_t sst = src->stride_words * (word_bits(src->fmt) / 32);
    uint32_t *dw = (uint32_t *)dst->words;
    const int64_t dstride = dst->stride_words * (word_bits(dst->fmt) / 32);
    const int cover = dst->fmt == MORPH_PACKED32 ? (W + 31) / 32 : 2 * ((W + 63) / 64);
    cudaError_t e;
    if (!horizontal) {
        e = line_vertical(op, sw, sst, dw, dstride, cover, W, H, shift, p, base, length, origin,
                          (char *)workspace, s);
    } else {
        // the transposed case: columns skewed, the line along the rows
        const int nwt = (H + 31) / 32;
        uint32_t *XT = (uint32_t *)workspace;
        uint32_t *XD = (uint32_t *)((char *)workspace + align256((size_t)W * nwt * 4));
        char *rest = (char *)XD + align256((size_t)W * nwt * 4);
        e = launch_transpose(sw, sst, W, H, XT, nwt, nwt, s);
        if (e == cudaSuccess)
            e = line_vertical(op, XT, nwt, XD, nwt, nwt, H, W, shift, p, base, length, origin, rest, s);
        if (e == cudaSuccess) e = launch_transpose(XD, nwt, H, W, dw, dstride, cover, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "sheared line launch");
    return MORPH_OK;
}

morph_status morph_line_element(double angle_deg, int half_length, int width, int height, int32_t *shift,
                                int capacity, int *n_shift, int *length, int *origin, int *horizontal) {
    if (!shift || !n_shift || !length || !origin || !horizontal)
        return fail(MORPH_EINVAL, "morph_line_element: NULL output");
    if (half_length < 0 || width < 1 || height < 1 || !std::isfinite(angle_deg))
        return fail(MORPH_EINVAL, "morph_line_element: half length %d, %d x %d image, angle %g", half_length,
                    width, height, angle_deg);
    // reduce to [-90, 90): the same line a half turn away
    double a = std::fmod(angle_deg + 90.0, 180.0);
    if (a < 0.0) a += 180.0;
    a -= 90.0;
    // within 45 degrees of the x axis the line runs along the rows and the
    // skew moves columns; otherwise it runs along the columns and moves rows
    const bool rows = a >= -45.0 && a <= 45.0;
    const double off = rows ? a : 90.0 - a;  // angle from the nearer axis
    const double rad = off * (M_PI / 180.0);
    const double t = std::tan(rad);
    const int n = rows ? width : height;
    if (capacity < n)
        return fail(MORPH_EINVAL, "morph_line_element: the table needs %d entries, capacity %d", n, capacity);
    for (int i = 0; i < n; ++i) shift[i] = (int32_t)std::floor((double)i * t + 0.5);
    const int c = (int)std::floor((double)half_length * std::fabs(std::cos(rad)) + 0.5);
    *n_shift = n;
    *length = 2 * c + 1;
    *origin = c;
    *horizontal = rows ? 1 : 0;
    return MORPH_OK;
}

morph_status morph_sync_status(void *stream) {
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    int *p = device_status_ptr();
    if (!p) return fail(MORPH_ECUDA, "device status word unavailable");
    int code = 0;
    e = cudaMemcpy(&code, p, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "status read");
    if (code) {
        const int zero = 0;
        e = cudaMemcpy(p, &zero, sizeof(int), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "status clear");
        return fail((morph_status)code, "device reported %s", morph_status_string(code));
    }
    return MORPH_OK;
}

const char *morph_last_error(void) { return t_err; }

const char *morph_status_string(int status) {
    switch (status) {
    case MORPH_OK: return "MORPH_OK";
    case MORPH_EINVAL: return "MORPH_EINVAL";
    case MORPH_ECAPACITY: return "MORPH_ECAPACITY";
    case MORPH_ENOMEM: return "MORPH_ENOMEM";
    case MORPH_ECUDA: return "MORPH_ECUDA";
    case MORPH_ETIMEOUT: return "MORPH_ETIMEOUT";
    default: return "unknown morph_status";
    }
}

int morph_abi_version(void) { return MORPH_ABI_VERSION; }

}  // extern "C"
