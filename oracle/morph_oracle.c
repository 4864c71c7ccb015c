/*
 * Plain CPU oracle for rectangular binary morphology, run-length coding,
 * connected components of RLE images, run-length statistics and
 * transposition.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this code:
 * only tests/, the smoke check in __graft_entry__ and the cpu_baseline leg of
 * bench.py load it.  It shares no source with the CUDA library.
 *
 * Images are unpacked: one byte per pixel, value 0 or 1, row-major, row 0
 * first, W bytes per row, no padding.  Pixel (x, y) is in[y * W + x].
 *
 * Definitions (the paper's set semantics, written out literally):
 *
 *   erosion  (paper, section "Within-Line Morphological Operations", 1D
 *             erosion; section "2D Morphological Operators for Rectangular
 *             Masks", brute force used "for reference and verification"):
 *       E(x,y) = min { I(x+i-ox, y+j-oy) : 0<=i<sw, 0<=j<sh, inside image }
 *   dilation (the reflected structuring element, Minkowski addition):
 *       D(x,y) = max { I(x-i+ox, y-j+oy) : 0<=i<sw, 0<=j<sh, inside image }
 *   opening  = D(E(I)), closing = E(D(I))  (section "Within-Line ...": opening
 *             and closing are not separable and are built from erosions and
 *             dilations).
 *
 * Boundary reading: positions outside the image are simply left out of the
 * min / max ("clipped window").  Erosion therefore behaves as if the outside
 * were 1 and dilation as if it were 0.  The paper's text is not consistent on
 * this point (its 1D erosion shrinks runs at the border, its complement closes
 * the last gap at maxint); the clipped window is the reading under which
 * duality, separability, idempotence and (anti-)extensivity all hold exactly.
 *
 * Run-length coding (section "Run Length Image Coding"): each row is the
 * ascending list of its maximal runs of 1-pixels, each run stored as two
 * 16-bit numbers (start, end) with end exclusive ("half-open" reading of the
 * paper's [s, e]; its complement routine uses half-open intervals).
 *
 * Two evaluation modes for the rectangle operations:
 *   brute force  — the definition above, pixel by pixel;
 *   separable    — a 1D pass along rows then a 1D pass along columns, the
 *                  decomposition erode2d = erode1d, transpose, erode1d given
 *                  in section "Morphological Operations".  Each 1D pass is
 *                  still the plain clipped min / max over its window.
 * The tests check the two modes against each other.
 *
 * Optional threading: `nthreads` > 1 splits the independent output rows over
 * OpenMP threads; it does not change any result.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define EXPORT __attribute__((visibility("default")))

static void set_threads(int nthreads) {
#ifdef _OPENMP
    omp_set_num_threads(nthreads > 0 ? nthreads : 1);
#else
    (void)nthreads;
#endif
}

/* ---------------------------------------------------------------- brute */

/* E(x,y) = min over the clipped window.  Early exit on the first 0 does not
 * change the minimum of 0/1 values. */
EXPORT void oracle_erode_rect(uint8_t *out, const uint8_t *in, int W, int H,
                              int sw, int sh, int ox, int oy, int nthreads) {
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 8) if (nthreads > 1)
    for (int y = 0; y < H; y++) {
        for (int x = 0; x < W; x++) {
            uint8_t v = 1;
            for (int j = 0; j < sh && v; j++) {
                int yy = y + j - oy;
                if (yy < 0 || yy >= H) continue;
                for (int i = 0; i < sw; i++) {
                    int xx = x + i - ox;
                    if (xx < 0 || xx >= W) continue;
                    if (in[(size_t)yy * W + xx] == 0) { v = 0; break; }
                }
            }
            out[(size_t)y * W + x] = v;
        }
    }
}

/* D(x,y) = max over the clipped, reflected window. */
EXPORT void oracle_dilate_rect(uint8_t *out, const uint8_t *in, int W, int H,
                               int sw, int sh, int ox, int oy, int nthreads) {
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 8) if (nthreads > 1)
    for (int y = 0; y < H; y++) {
        for (int x = 0; x < W; x++) {
            uint8_t v = 0;
            for (int j = 0; j < sh && !v; j++) {
                int yy = y - j + oy;
                if (yy < 0 || yy >= H) continue;
                for (int i = 0; i < sw; i++) {
                    int xx = x - i + ox;
                    if (xx < 0 || xx >= W) continue;
                    if (in[(size_t)yy * W + xx] != 0) { v = 1; break; }
                }
            }
            out[(size_t)y * W + x] = v;
        }
    }
}

/* ---------------------------------------------------------------- masks */

/* Section "Morphology with Arbitrary Masks": the structuring element is a
 * bitmap, mask[j * mw + i] != 0 when (i, j) belongs to it, origin (ox, oy).
 * The definitions are the rectangle ones with the window replaced by the
 * element's pixels (same clipped-window reading):
 *   E(x,y) = min { I(x+i-ox, y+j-oy) : mask(i,j), inside image }
 *   D(x,y) = max { I(x-i+ox, y-j+oy) : mask(i,j), inside image }
 * This is the paper's pixel-at-a-time loop, kept as the reference. */
EXPORT void oracle_erode_mask(uint8_t *out, const uint8_t *in, int W, int H,
                              const uint8_t *mask, int mw, int mh, int ox, int oy,
                              int nthreads) {
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 8) if (nthreads > 1)
    for (int y = 0; y < H; y++) {
        for (int x = 0; x < W; x++) {
            uint8_t v = 1;
            for (int j = 0; j < mh && v; j++) {
                int yy = y + j - oy;
                if (yy < 0 || yy >= H) continue;
                for (int i = 0; i < mw; i++) {
                    if (!mask[j * mw + i]) continue;
                    int xx = x + i - ox;
                    if (xx < 0 || xx >= W) continue;
                    if (in[(size_t)yy * W + xx] == 0) { v = 0; break; }
                }
            }
            out[(size_t)y * W + x] = v;
        }
    }
}

EXPORT void oracle_dilate_mask(uint8_t *out, const uint8_t *in, int W, int H,
                               const uint8_t *mask, int mw, int mh, int ox, int oy,
                               int nthreads) {
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 8) if (nthreads > 1)
    for (int y = 0; y < H; y++) {
        for (int x = 0; x < W; x++) {
            uint8_t v = 0;
            for (int j = 0; j < mh && !v; j++) {
                int yy = y - j + oy;
                if (yy < 0 || yy >= H) continue;
                for (int i = 0; i < mw; i++) {
                    if (!mask[j * mw + i]) continue;
                    int xx = x - i + ox;
                    if (xx < 0 || xx >= W) continue;
                    if (in[(size_t)yy * W + xx] != 0) { v = 1; break; }
                }
            }
            out[(size_t)y * W + x] = v;
        }
    }
}

/* ----------------------------------------------------------- separable */

/* 1D pass along rows: window of sw pixels, origin ox; erode = min, dilate =
 * max over the reflected window.  Clipped at the row ends. */
static void pass_rows(uint8_t *out, const uint8_t *in, int W, int H, int sw,
                      int ox, int dilate, int nthreads) {
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 8) if (nthreads > 1)
    for (int y = 0; y < H; y++) {
        const uint8_t *r = in + (size_t)y * W;
        uint8_t *o = out + (size_t)y * W;
        for (int x = 0; x < W; x++) {
            uint8_t v = dilate ? 0 : 1;
            for (int i = 0; i < sw; i++) {
                int xx = dilate ? x - i + ox : x + i - ox;
                if (xx < 0 || xx >= W) continue;
                if (dilate) { if (r[xx]) { v = 1; break; } }
                else        { if (!r[xx]) { v = 0; break; } }
            }
            o[x] = v;
        }
    }
}

/* 1D pass along columns: window of sh rows, origin oy. */
static void pass_cols(uint8_t *out, const uint8_t *in, int W, int H, int sh,
                      int oy, int dilate, int nthreads) {
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 8) if (nthreads > 1)
    for (int y = 0; y < H; y++) {
        uint8_t *o = out + (size_t)y * W;
        for (int x = 0; x < W; x++) {
            uint8_t v = dilate ? 0 : 1;
            for (int j = 0; j < sh; j++) {
                int yy = dilate ? y - j + oy : y + j - oy;
                if (yy < 0 || yy >= H) continue;
                uint8_t p = in[(size_t)yy * W + x];
                if (dilate) { if (p) { v = 1; break; } }
                else        { if (!p) { v = 0; break; } }
            }
            o[x] = v;
        }
    }
}

static int rect_sep(uint8_t *out, const uint8_t *in, int W, int H, int sw,
                    int sh, int ox, int oy, int dilate, int nthreads) {
    uint8_t *tmp = (uint8_t *)malloc((size_t)W * H);
    if (!tmp) return -1;
    pass_rows(tmp, in, W, H, sw, ox, dilate, nthreads);
    pass_cols(out, tmp, W, H, sh, oy, dilate, nthreads);
    free(tmp);
    return 0;
}

EXPORT int oracle_erode_rect_sep(uint8_t *out, const uint8_t *in, int W, int H,
                                 int sw, int sh, int ox, int oy, int nthreads) {
    return rect_sep(out, in, W, H, sw, sh, ox, oy, 0, nthreads);
}

EXPORT int oracle_dilate_rect_sep(uint8_t *out, const uint8_t *in, int W, int H,
                                  int sw, int sh, int ox, int oy, int nthreads) {
    return rect_sep(out, in, W, H, sw, sh, ox, oy, 1, nthreads);
}

/* ------------------------------------------------------------- batches */

/* n independent images of W x H stored back to back (used by the exhaustive
 * tiny-image checks).  op: 0 erode, 1 dilate, 2 open, 3 close. */
EXPORT int oracle_rect_batch(uint8_t *out, const uint8_t *in, int64_t n, int W,
                             int H, int sw, int sh, int ox, int oy, int op) {
    size_t px = (size_t)W * H;
    uint8_t *tmp = (uint8_t *)malloc(px);
    if (!tmp) return -1;
    for (int64_t k = 0; k < n; k++) {
        const uint8_t *a = in + (size_t)k * px;
        uint8_t *b = out + (size_t)k * px;
        switch (op) {
        case 0: oracle_erode_rect(b, a, W, H, sw, sh, ox, oy, 1); break;
        case 1: oracle_dilate_rect(b, a, W, H, sw, sh, ox, oy, 1); break;
        case 2:
            oracle_erode_rect(tmp, a, W, H, sw, sh, ox, oy, 1);
            oracle_dilate_rect(b, tmp, W, H, sw, sh, ox, oy, 1);
            break;
        default:
            oracle_dilate_rect(tmp, a, W, H, sw, sh, ox, oy, 1);
            oracle_erode_rect(b, tmp, W, H, sw, sh, ox, oy, 1);
            break;
        }
    }
    free(tmp);
    return 0;
}

/* ------------------------------------------------------------------ RLE */

/* Number of maximal runs of 1s in each row; returns the total. */
EXPORT int64_t oracle_rle_count(int32_t *row_counts, const uint8_t *in, int W,
                                int H) {
    int64_t total = 0;
    for (int y = 0; y < H; y++) {
        const uint8_t *r = in + (size_t)y * W;
        int32_t c = 0;
        for (int x = 0; x < W; x++)
            if (r[x] && (x == 0 || !r[x - 1])) c++;
        if (row_counts) row_counts[y] = c;
        total += c;
    }
    return total;
}

/* Canonical runs of each row: row_ptr[H+1] (prefix of counts) and runs as
 * uint16 pairs (start, end), end exclusive, ascending, separated by gaps. */
EXPORT void oracle_rle_encode(int32_t *row_ptr, uint16_t *runs,
                              const uint8_t *in, int W, int H) {
    int64_t k = 0;
    row_ptr[0] = 0;
    for (int y = 0; y < H; y++) {
        const uint8_t *r = in + (size_t)y * W;
        int x = 0;
        while (x < W) {
            if (!r[x]) { x++; continue; }
            int s = x;
            while (x < W && r[x]) x++;
            runs[2 * k] = (uint16_t)s;
            runs[2 * k + 1] = (uint16_t)x;
            k++;
        }
        row_ptr[y + 1] = (int32_t)k;
    }
}

/* Paint every run [start, end) of every row; everything else is 0.
 * Returns 0, or -1 if a run is empty, out of range, or not ascending. */
EXPORT int oracle_rle_decode(uint8_t *out, const int32_t *row_ptr,
                             const uint16_t *runs, int W, int H) {
    memset(out, 0, (size_t)W * H);
    for (int y = 0; y < H; y++) {
        uint8_t *r = out + (size_t)y * W;
        int prev_end = -1;
        for (int32_t k = row_ptr[y]; k < row_ptr[y + 1]; k++) {
            int s = runs[2 * k], e = runs[2 * k + 1];
            if (s >= e || e > W || s <= prev_end) return -1;
            for (int x = s; x < e; x++) r[x] = 1;
            prev_end = e;
        }
    }
    return 0;
}

/* ------------------------------------------------- connected components */

/* Section "Connected Component Extraction and Statistics": every run of
 * the RLE image gets a label, each label starts as its own set of a
 * union-find structure, and the lines are visited top to bottom merging
 * every run of the current line with each run of the line above that it
 * touches.  Finally each run is relabelled by its set's representative.
 *
 * Touching (the paper: the runs' intervals overlap, which is the line
 * adjacency graph of section "Other Operations"):
 *   conn == 4: [s, e) and [s', e') share a column: s < e' and s' < e;
 *   conn == 8: they also touch diagonally:         s <= e' and s' <= e.
 * Canonical numbering (the paper leaves the representative open): the
 * components are numbered 0, 1, ... in the order in which their first run
 * appears in raster order (row by row, left to right), so the labels are
 * unique.  Returns the number of components. */
static int32_t uf_find(int32_t *parent, int32_t x) {
    int32_t r = x;
    while (parent[r] != r) r = parent[r];
    while (parent[x] != r) {  /* path compression */
        int32_t n = parent[x];
        parent[x] = r;
        x = n;
    }
    return r;
}

static void uf_union(int32_t *parent, int32_t a, int32_t b) {
    a = uf_find(parent, a);
    b = uf_find(parent, b);
    if (a != b) parent[a > b ? a : b] = a < b ? a : b;
}

EXPORT int64_t oracle_rle_components(int32_t *label, const int32_t *row_ptr,
                                     const uint16_t *runs, int H, int conn) {
    const int32_t n = row_ptr[H];
    const int d = conn == 8 ? 1 : 0;
    int32_t *parent = (int32_t *)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
    int32_t *number = (int32_t *)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
    for (int32_t i = 0; i < n; i++) parent[i] = i;
    for (int y = 1; y < H; y++) {
        /* the runs of both lines are ascending: one linear walk */
        int32_t a = row_ptr[y - 1];
        const int32_t a_end = row_ptr[y];
        for (int32_t k = row_ptr[y]; k < row_ptr[y + 1]; k++) {
            const int s = runs[2 * k], e = runs[2 * k + 1];
            /* runs above that end before this one starts can touch no later run */
            while (a < a_end && runs[2 * a + 1] + d <= s) a++;
            for (int32_t b = a; b < a_end && runs[2 * b] < e + d; b++)
                uf_union(parent, k, b);
        }
    }
    int64_t count = 0;
    for (int32_t i = 0; i < n; i++) number[i] = -1;
    for (int32_t i = 0; i < n; i++) {
        const int32_t r = uf_find(parent, i);
        if (number[r] < 0) number[r] = (int32_t)count++;
        label[i] = number[r];
    }
    free(parent);
    free(number);
    return count;
}

/* Statistics over the labelled runs (same section: iterate through the runs
 * and accumulate into arrays indexed by the label).  Per component c,
 * stats[7 c + .]: x0, y0, x1, y1 (bounding box, half-open), area (pixels),
 * sum of x, sum of y over its pixels.  Pixel by pixel on purpose. */
EXPORT void oracle_rle_component_stats(int64_t *stats, const int32_t *label,
                                       const int32_t *row_ptr, const uint16_t *runs,
                                       int H, int64_t ncomp) {
    for (int64_t c = 0; c < ncomp; c++) {
        int64_t *t = stats + 7 * c;
        t[0] = INT64_MAX; t[1] = INT64_MAX; t[2] = INT64_MIN; t[3] = INT64_MIN;
        t[4] = 0; t[5] = 0; t[6] = 0;
    }
    for (int y = 0; y < H; y++) {
        for (int32_t k = row_ptr[y]; k < row_ptr[y + 1]; k++) {
            int64_t *t = stats + 7 * (int64_t)label[k];
            for (int x = runs[2 * k]; x < runs[2 * k + 1]; x++) {
                if (x < t[0]) t[0] = x;
                if (y < t[1]) t[1] = y;
                if (x + 1 > t[2]) t[2] = x + 1;
                if (y + 1 > t[3]) t[3] = y + 1;
                t[4] += 1;
                t[5] += x;
                t[6] += y;
            }
        }
    }
}

/* Run-length statistics (section "Other Operations"): histograms of the
 * lengths of the black runs (1-pixels) and of the white runs (maximal gaps
 * of 0-pixels in a row, including those at the row's ends; an empty row is
 * one white run of length W), read off the runs of each line.  black[L] and
 * white[L], L = 0..W, count the runs of length L. */
EXPORT void oracle_run_length_hist(int64_t *black, int64_t *white, const int32_t *row_ptr,
                                   const uint16_t *runs, int W, int H) {
    memset(black, 0, sizeof(int64_t) * (W + 1));
    memset(white, 0, sizeof(int64_t) * (W + 1));
    for (int y = 0; y < H; y++) {
        int prev_end = 0;
        for (int32_t k = row_ptr[y]; k < row_ptr[y + 1]; k++) {
            const int s = runs[2 * k], e = runs[2 * k + 1];
            black[e - s]++;
            if (s > prev_end) white[s - prev_end]++;
            prev_end = e;
        }
        if (W > prev_end) white[W - prev_end]++;
    }
}

/* ---------------------------------------------------------- transpose */

/* Section "Efficient Transpose" (the decode-recode and sweep
 * algorithms compute this same image): out is H x W (W bytes per row of
 * the input, H per row of the output), out(y, x) = in(x, y). */
EXPORT void oracle_transpose(uint8_t *out, const uint8_t *in, int W, int H) {
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) out[(size_t)x * H + y] = in[(size_t)y * W + x];
}

/* The sweep of section "Efficient Transpose", for RLE images: instead of an
 * open-run entry per output line, a list of open intervals of columns, each
 * with the line its vertical runs started on.  Line y of the input is merged
 * with the list in one left-to-right walk over the boundaries of both:
 *   columns in an open interval and in a run of line y stay open (same start),
 *   columns in an open interval but in no run close: each column x gets the
 *     vertical run [start, y) in output line x,
 *   columns in a run but in no open interval open with start y.
 * After the last line every open interval closes at H.  Output line x
 * receives its runs in the order they close, which is ascending, and two
 * runs of a column are separated by at least the line that closed the first,
 * so the output is canonical.
 *
 * Two walks over the image: the first counts each output line's runs into
 * out_row_ptr (then turned into offsets), the second writes them.  Input:
 * canonical runs (ascending, non-empty, separated, ends <= W; checked).
 * Returns the number of output runs, -1 for a non-canonical input, -2 when
 * the runs do not fit `cap`, -3 when out of host memory. */
typedef struct { int a, b, s; } SweepIv;

static void sweep_close(int x0, int x1, int start, int y, int32_t *cur, uint16_t *out_runs) {
    for (int x = x0; x < x1; x++) {
        if (out_runs) {
            out_runs[2 * (int64_t)cur[x]] = (uint16_t)start;
            out_runs[2 * (int64_t)cur[x] + 1] = (uint16_t)y;
        }
        cur[x]++;
    }
}

static void sweep_open(SweepIv *nx, int *nn, int a, int b, int s) {
    if (*nn > 0 && nx[*nn - 1].b == a && nx[*nn - 1].s == s) {
        nx[*nn - 1].b = b;
        return;
    }
    nx[*nn].a = a;
    nx[*nn].b = b;
    nx[*nn].s = s;
    (*nn)++;
}

static int sweep_pass(const int32_t *row_ptr, const uint16_t *runs, int W, int H, int32_t *cur,
                      uint16_t *out_runs, SweepIv *op, SweepIv *nx) {
    int no = 0;
    for (int y = 0; y < H; y++) {
        const int64_t r0 = row_ptr[y], r1 = row_ptr[y + 1];
        for (int64_t r = r0; r < r1; r++) {
            const int s = runs[2 * r], e = runs[2 * r + 1];
            if (s >= e || e > W || (r > r0 && s <= runs[2 * r - 1])) return -1;
        }
        int nn = 0, p = 0, x = 0;
        int64_t q = r0;
        while (p < no || q < r1) {
            const int oa = p < no ? op[p].a : INT32_MAX, ob = p < no ? op[p].b : INT32_MAX;
            const int ra = q < r1 ? runs[2 * q] : INT32_MAX, rb = q < r1 ? runs[2 * q + 1] : INT32_MAX;
            if (x < oa && x < ra) x = oa < ra ? oa : ra;
            const int in_o = oa <= x && x < ob, in_r = ra <= x && x < rb;
            int z = INT32_MAX;
            if (in_o) { if (ob < z) z = ob; } else if (oa < z) z = oa;
            if (in_r) { if (rb < z) z = rb; } else if (ra < z) z = ra;
            if (in_o && in_r) sweep_open(nx, &nn, x, z, op[p].s);
            else if (in_o) sweep_close(x, z, op[p].s, y, cur, out_runs);
            else sweep_open(nx, &nn, x, z, y);
            x = z;
            if (p < no && op[p].b <= x) p++;
            if (q < r1 && runs[2 * q + 1] <= x) q++;
        }
        SweepIv *t = op;
        op = nx;
        nx = t;
        no = nn;
    }
    for (int p = 0; p < no; p++) sweep_close(op[p].a, op[p].b, op[p].s, H, cur, out_runs);
    return 0;
}

EXPORT int64_t oracle_rle_transpose_sweep(int32_t *out_row_ptr, uint16_t *out_runs, int64_t cap,
                                          const int32_t *row_ptr, const uint16_t *runs, int W,
                                          int H) {
    /* an interval list never holds more entries than W (they are disjoint,
     * non-empty column ranges) */
    SweepIv *a = (SweepIv *)malloc(sizeof(SweepIv) * (size_t)(W + 1));
    SweepIv *b = (SweepIv *)malloc(sizeof(SweepIv) * (size_t)(W + 1));
    int32_t *cnt = (int32_t *)calloc((size_t)W + 1, sizeof(int32_t));
    int64_t total = -3;
    if (!a || !b || !cnt) goto done;
    total = -1;
    if (sweep_pass(row_ptr, runs, W, H, cnt, NULL, a, b)) goto done;
    out_row_ptr[0] = 0;
    for (int x = 0; x < W; x++) out_row_ptr[x + 1] = out_row_ptr[x] + cnt[x];
    total = out_row_ptr[W];
    if (total > cap) {
        total = -2;
        goto done;
    }
    for (int x = 0; x < W; x++) cnt[x] = out_row_ptr[x];
    sweep_pass(row_ptr, runs, W, H, cnt, out_runs, a, b);
done:
    free(a);
    free(b);
    free(cnt);
    return total;
}

/* --------------------------------------------------- sheared line SEs */

/* Section "Morphology with Lines at Arbitrary Orientations": a line at an
 * angle is eroded by skewing the image perpendicular to the erosion,
 * eroding by an axis-parallel line and skewing back.  Written out: line y
 * is shifted right by shift[y] (the skew), the vertical line of `length`
 * rows with origin o is applied (clipped window, as for the rectangles:
 * positions that hold no image pixel are left out), and the lines are
 * shifted back.  Pixel by pixel that is
 *   E(x,y) = AND over j in [-o, length-1-o] of I(x + shift[y] - shift[y+j], y+j)
 *   D(x,y) = OR  over j in [-(length-1-o), o] of the same,
 * each term only where 0 <= y+j < H and 0 <= x + shift[y] - shift[y+j] < W.
 * dilate = 0 erodes, 1 dilates. */
EXPORT void oracle_sheared_line(uint8_t *out, const uint8_t *in, int W, int H,
                                const int32_t *shift, int length, int o, int dilate) {
    const int j0 = dilate ? -(length - 1 - o) : -o;
    const int j1 = dilate ? o : length - 1 - o;
    for (int y = 0; y < H; y++) {
        for (int x = 0; x < W; x++) {
            int v = dilate ? 0 : 1;
            for (int j = j0; j <= j1; j++) {
                const int yy = y + j;
                if (yy < 0 || yy >= H) continue;
                const long xx = (long)x + shift[y] - shift[yy];
                if (xx < 0 || xx >= W) continue;
                const int p = in[(size_t)yy * W + xx];
                if (dilate ? p : !p) { v = dilate; break; }
            }
            out[(size_t)y * W + x] = (uint8_t)v;
        }
    }
}

/* ---------------------------------------------------- layout analysis */

/* Section "Document Analysis Performance": the spacing of words and of
 * lines is estimated from the lengths of the white runs, but the paper does
 * not give the rule.  Reading: the estimate is the smallest length L in
 * 1 .. lmax such that the white runs of length at most L make up at least
 * pct percent of all white runs of length at most lmax (longer gaps —
 * margins, gutters, blank lines — are left out of both counts); 0 when no
 * white run has a length in 1 .. lmax.  white[L], L = 0 .. lmax, counts the
 * white runs of length L.  Integer arithmetic only. */
EXPORT int oracle_layout_gap(const int64_t *white, int lmax, int pct) {
    int64_t total = 0;
    for (int L = 1; L <= lmax; L++) total += white[L];
    if (total == 0) return 0;
    int64_t upto = 0;
    int L = 1;
    for (;;) {
        upto += white[L];
        if (upto * 100 >= (int64_t)pct * total || L == lmax) return L;
        L++;
    }
}
