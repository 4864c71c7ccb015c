/*
 * Seeded synthetic document pages (host code, deterministic on any host).
 *
 * These pages stand in for the paper's scanned journal pages (300 dpi UW3
 * scans) and its binarised 7000x7000 cadastral map, neither of which is
 * available.  The generator holds no morphology: it only paints rectangles,
 * blurs noise and draws Bernoulli pixels.  Output is one byte per pixel (0/1),
 * row-major, row 0 first.
 *
 * Random numbers: SplitMix64 (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), used both as a sequential
 * stream and as a counter-based hash of (seed, index).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define EXPORT __attribute__((visibility("default")))

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

typedef struct { uint64_t s; } rng_t;

static inline uint64_t rng_next(rng_t *r) {
    r->s += 0x9E3779B97F4A7C15ULL;
    return mix64(r->s);
}
/* uniform in [0, 1) with 53 random bits */
static inline double rng_unif(rng_t *r) { return (double)(rng_next(r) >> 11) * 0x1.0p-53; }
/* uniform integer in [lo, hi] */
static inline int rng_int(rng_t *r, int lo, int hi) {
    if (hi <= lo) return lo;
    return lo + (int)(rng_next(r) % (uint64_t)(hi - lo + 1));
}
/* counter-based uniform for pixel i of stream `seed` */
static inline double hash_unif(uint64_t seed, uint64_t i) {
    return (double)(mix64(seed + (i + 1) * 0x9E3779B97F4A7C15ULL) >> 11) * 0x1.0p-53;
}

static void fill_rect(uint8_t *img, int W, int H, int x0, int y0, int w, int h) {
    int x1 = x0 + w, y1 = y0 + h;
    if (x0 < 0) x0 = 0;
    if (y0 < 0) y0 = 0;
    if (x1 > W) x1 = W;
    if (y1 > H) y1 = H;
    if (x1 <= x0 || y1 <= y0) return;
    for (int y = y0; y < y1; y++) memset(img + (size_t)y * W + x0, 1, (size_t)(x1 - x0));
}

static double ink_fraction(const uint8_t *img, size_t n) {
    size_t c = 0;
    for (size_t i = 0; i < n; i++) c += img[i];
    return n ? (double)c / (double)n : 0.0;
}

#define NCAND 12 /* candidate strokes per glyph */

typedef struct {
    int W, H;
    uint64_t seed;
    int gw_min, gw_max, gh_min, gh_max, gap_min, gap_max, ncols, n_ruled, n_filled;
} text_params;

/* Paint one text page at ink level q in [0, 3]: q <= 1 keeps a fraction q of
 * the text lines with a base stroke probability; 1 < q <= 2 keeps every line
 * and raises the stroke probability; q > 2 thickens the strokes.  All random
 * draws are made whatever q is, so the painted set only grows with q (ink is
 * monotone in q). */
static void paint_text(uint8_t *img, const text_params *p, double q) {
    const int W = p->W, H = p->H;
    const double p0 = 0.3;
    double line_keep = q < 1.0 ? q : 1.0;
    double p_stroke = q <= 1.0 ? p0 : (q <= 2.0 ? p0 + (q - 1.0) * (1.0 - p0) : 1.0);
    double bold = q <= 2.0 ? 1.0 : 1.0 + 2.0 * (q - 2.0);
    memset(img, 0, (size_t)W * H);
    rng_t r = {p->seed};
    int margin = W / 16 > 2 ? W / 16 : 2;
    int vmargin = H / 16 > 2 ? H / 16 : 2;
    int ncols = p->ncols > 0 ? p->ncols : 1;
    int col_gap = W / 30 > 4 ? W / 30 : 4;
    int avail = W - 2 * margin - (ncols - 1) * col_gap;
    if (avail < p->gw_max + 2) { margin = 1; col_gap = 2; ncols = 1; avail = W - 2; }
    int col_w = avail / ncols;
    int pitch = p->gh_max + (p->gh_max + 1) / 2;
    if (pitch < 2) pitch = 2;

    for (int c = 0; c < ncols; c++) {
        int cx0 = margin + c * (col_w + col_gap), cx1 = cx0 + col_w;
        for (int y0 = vmargin; y0 + p->gh_max <= H - vmargin; y0 += pitch) {
            double u_line = rng_unif(&r);
            int para = rng_unif(&r) < 0.08;            /* paragraph break: empty line */
            int keep = (u_line < line_keep) && !para;
            int x = cx0 + (rng_unif(&r) < 0.15 ? 3 * p->gw_max / 2 : 0); /* indent */
            int line_end = cx1 - (rng_unif(&r) < 0.2 ? rng_int(&r, 0, col_w / 2) : 0);
            while (1) {
                int gw = rng_int(&r, p->gw_min, p->gw_max);
                int gh = rng_int(&r, p->gh_min, p->gh_max);
                if (x + gw > line_end) break;
                int gy = y0 + (p->gh_max - gh);          /* glyphs share a baseline */
                int t0 = gh / 6 > 1 ? gh / 6 : 1;
                int t = (int)(t0 * bold);               /* stroke thickness */
                for (int k = 0; k < NCAND; k++) {
                    double u = rng_unif(&r);
                    int kind = rng_int(&r, 0, 3);
                    int a = rng_int(&r, 0, gw - 1), b = rng_int(&r, 0, gh - 1);
                    int len = rng_int(&r, (gh + 1) / 2, gh);
                    if (!keep || u >= p_stroke) continue;
                    switch (kind) {
                    case 0: fill_rect(img, W, H, x + a - t / 2, gy, t, gh); break;          /* stem */
                    case 1: fill_rect(img, W, H, x, gy + b - t / 2, gw, t); break;          /* bar */
                    case 2: fill_rect(img, W, H, x + a - t / 2, gy + gh - len, t, len); break;
                    default: fill_rect(img, W, H, x + a / 2, gy + b - t / 2, (gw + 1) / 2, t); break;
                    }
                }
                int gap = rng_int(&r, p->gap_min, p->gap_max);
                if (rng_unif(&r) < 0.18) gap = 3 * gap + p->gw_min;   /* word space */
                x += gw + gap;
            }
        }
    }
    /* ruled lines (thickness 1-3 px) and filled rectangles, scaled by line_keep */
    for (int k = 0; k < p->n_ruled; k++) {
        double u = rng_unif(&r);
        int c = rng_int(&r, 0, ncols - 1);
        int y = rng_int(&r, vmargin, H - vmargin - 1), th = rng_int(&r, 1, 3);
        if (u < line_keep) fill_rect(img, W, H, margin + c * (col_w + col_gap), y, col_w, th);
    }
    for (int k = 0; k < p->n_filled; k++) {
        double u = rng_unif(&r);
        int w = rng_int(&r, W / 40 + 1, W / 8 + 2), h = rng_int(&r, H / 60 + 1, H / 12 + 2);
        int x = rng_int(&r, 0, W - w > 0 ? W - w : 0), y = rng_int(&r, 0, H - h > 0 ? H - h : 0);
        if (u < line_keep * 0.5) fill_rect(img, W, H, x, y, w, h);
    }
}

/* Text-like page whose ink fraction is within `tol` of `density` when that is
 * reachable (bisection on the monotone ink level).  Returns the ink fraction. */
EXPORT double synth_text(uint8_t *out, int W, int H, uint64_t seed, double density,
                         int gw_min, int gw_max, int gh_min, int gh_max, int gap_min,
                         int gap_max, int ncols, int n_ruled, int n_filled, double tol) {
    if (W <= 0 || H <= 0) return 0.0;
    if (gw_min < 1) gw_min = 1;
    if (gh_min < 1) gh_min = 1;
    if (gw_max < gw_min) gw_max = gw_min;
    if (gh_max < gh_min) gh_max = gh_min;
    if (gap_min < 0) gap_min = 0;
    if (gap_max < gap_min) gap_max = gap_min;
    text_params p = {W, H, seed, gw_min, gw_max, gh_min, gh_max, gap_min, gap_max,
                     ncols, n_ruled, n_filled};
    size_t n = (size_t)W * H;
    double lo = 0.0, hi = 3.0, best_q = 1.0, best_err = 1e9;
    for (int it = 0; it < 24; it++) {
        double q = 0.5 * (lo + hi);
        paint_text(out, &p, q);
        double d = ink_fraction(out, n);
        double err = fabs(d - density);
        if (err < best_err) { best_err = err; best_q = q; }
        if (err <= tol) return d;
        if (d < density) lo = q; else hi = q;
    }
    paint_text(out, &p, best_q);
    return ink_fraction(out, n);
}

/* exp(x) for x <= 0 from its Taylor series after halving the argument k
 * times, then squaring k times: plain IEEE operations in a fixed order, so
 * the result is the same on every host (no libm, no fused multiply-add). */
static double det_exp(double x) {
    int k = 0;
    while (x < -0.125) { x *= 0.5; k++; }
    double term = 1.0, s = 1.0;
    for (int i = 1; i < 20; i++) { term = term * x / (double)i; s += term; }
    while (k-- > 0) s = s * s;
    return s;
}

static int cmp_double(const void *a, const void *b) {
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

static inline int mirror(int i, int n) {
    if (n == 1) return 0;
    while (i < 0 || i >= n) i = i < 0 ? -i - 1 : 2 * n - i - 1;
    return i;
}

/* Clustered "halftone": iid U(0,1) noise blurred by a Gaussian (sigma px,
 * kernel truncated at 3 sigma, mirrored borders, float64), thresholded so that
 * the `density` fraction of largest values is ink (empirical quantile). */
EXPORT double synth_halftone(uint8_t *out, int W, int H, uint64_t seed, double density,
                             double sigma) {
    if (W <= 0 || H <= 0) return 0.0;
    size_t n = (size_t)W * H;
    int R = (int)ceil(3.0 * sigma);
    double *k = (double *)malloc(sizeof(double) * (2 * R + 1));
    double *a = (double *)malloc(sizeof(double) * n);
    double *b = (double *)malloc(sizeof(double) * n);
    if (!k || !a || !b) { free(k); free(a); free(b); return -1.0; }
    double ks = 0.0;
    for (int i = -R; i <= R; i++) { k[i + R] = det_exp(-(double)i * i / (2.0 * sigma * sigma)); ks += k[i + R]; }
    for (int i = 0; i <= 2 * R; i++) k[i] /= ks;
    for (size_t i = 0; i < n; i++) a[i] = hash_unif(seed, i);
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            double s = 0.0;
            for (int d = -R; d <= R; d++) s += k[d + R] * a[(size_t)y * W + mirror(x + d, W)];
            b[(size_t)y * W + x] = s;
        }
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            double s = 0.0;
            for (int d = -R; d <= R; d++) s += k[d + R] * b[(size_t)mirror(y + d, H) * W + x];
            a[(size_t)y * W + x] = s;
        }
    /* exact quantile: histogram to find the bucket holding rank m, sort that bucket */
    size_t m = (size_t)llround((1.0 - density) * (double)n); /* pixels below threshold */
    double thr;
    if (m == 0) thr = -1.0;
    else if (m >= n) thr = 2.0;
    else {
        double mn = a[0], mx = a[0];
        for (size_t i = 1; i < n; i++) { if (a[i] < mn) mn = a[i]; if (a[i] > mx) mx = a[i]; }
        enum { NB = 1 << 16 };
        size_t *hist = (size_t *)calloc(NB, sizeof(size_t));
        double scale = (mx > mn) ? (NB - 1) / (mx - mn) : 0.0;
        for (size_t i = 0; i < n; i++) hist[(size_t)((a[i] - mn) * scale)]++;
        size_t acc = 0; int bk = 0;
        while (acc + hist[bk] < m) acc += hist[bk++];
        size_t cnt = hist[bk];
        double *v = (double *)malloc(sizeof(double) * (cnt ? cnt : 1));
        size_t j = 0;
        for (size_t i = 0; i < n; i++) if ((size_t)((a[i] - mn) * scale) == (size_t)bk) v[j++] = a[i];
        qsort(v, cnt, sizeof(double), cmp_double);
        thr = v[m - acc - 1];  /* the m-th smallest value: pixels <= thr are background */
        free(v); free(hist);
    }
    for (size_t i = 0; i < n; i++) out[i] = a[i] > thr;
    free(k); free(a); free(b);
    return ink_fraction(out, n);
}

/* Salt-and-pepper: every pixel is ink with probability p, independently. */
EXPORT double synth_noise(uint8_t *out, int W, int H, uint64_t seed, double p) {
    size_t n = (size_t)W * H;
    for (size_t i = 0; i < n; i++) out[i] = hash_unif(seed, i) < p;
    return ink_fraction(out, n);
}

/* Uniform random bits with P(1) = p, same as synth_noise (kept separate for
 * the name used by tests on tiny random images). */
EXPORT void synth_bernoulli(uint8_t *out, int64_t n, uint64_t seed, double p) {
    for (int64_t i = 0; i < n; i++) out[i] = hash_unif(seed, (uint64_t)i) < p;
}

/* Sequential integers in [lo, hi] from the SplitMix64 stream (used for
 * seeded choices such as per-page sizes and structuring elements). */
EXPORT void synth_ints(int32_t *out, int64_t n, uint64_t seed, int lo, int hi) {
    rng_t r = {seed};
    for (int64_t i = 0; i < n; i++) out[i] = rng_int(&r, lo, hi);
}

/* Sequential uniforms in [0, 1). */
EXPORT void synth_unif(double *out, int64_t n, uint64_t seed) {
    rng_t r = {seed};
    for (int64_t i = 0; i < n; i++) out[i] = rng_unif(&r);
}
