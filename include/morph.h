/*
 * morph.h — C ABI of the GB300 binary / run-length morphology library.
 *
 * Binary erosion, dilation, opening and closing with rectangular structuring
 * elements (SEs) on packed bitmaps and on row-wise run-length (RLE) images,
 * the conversions between the two formats, arbitrary structuring elements on
 * packed bitmaps, line elements at arbitrary angles, transposition,
 * connected components with per-component statistics and run-length
 * histograms (Breuel, "Efficient Binary and Run
 * Length Morphology and its Application to Document Image Processing").
 *
 * Every buffer named here is DEVICE memory owned by the caller; the library
 * never allocates device memory.  Scratch space, where an operation needs it,
 * is passed in as `workspace` (size from morph_workspace_size).  All work is
 * enqueued asynchronously on the caller's CUDA stream (`stream` is a
 * cudaStream_t; NULL = the legacy default stream).  The returned status covers
 * argument checks and the launches; conditions that only the device can see
 * (an RLE output larger than its capacity, a bounded wait that gave up) are
 * latched in a device-side status word and reported by morph_sync_status().
 *
 * Pixel conventions (identical for every entry point):
 *   - pixel (x, y): x = column 0..W-1, y = row 0..H-1, row 0 first in memory;
 *   - 1 = ink (foreground), 0 = background;
 *   - packed rows are little-endian bit strings: pixel x of a row is bit
 *     (x mod B) of word (x div B), B = 32 (MORPH_PACKED32) or 64
 *     (MORPH_PACKED64).  Bits at x >= W ("padding bits") are ignored on input
 *     and written as 0 on output;
 *   - an RLE row is the ascending list of its maximal runs of 1s, each run a
 *     pair of uint16 (start, end) with end EXCLUSIVE, separated by at least one
 *     0-pixel (section "Run Length Image Coding": runs as pairs of 16-bit
 *     integers, so W <= 65535 for RLE images).  runs[2k], runs[2k+1] are the
 *     start and end of run k; the runs of row y are k in
 *     [row_ptr[y], row_ptr[y+1]).
 *
 * Structuring element: a rectangle of se_w x se_h pixels (width x height) with
 * origin (origin_x, origin_y), 0 <= origin_x < se_w, 0 <= origin_y < se_h; the
 * centre of an odd rectangle is (se_w/2, se_h/2).  Definitions (clipped
 * window: pixels outside the image are left out of the min / max, so erosion
 * sees the outside as 1 and dilation as 0):
 *   erode : E(x,y) = min { I(x+i-ox, y+j-oy) : 0<=i<se_w, 0<=j<se_h, in image }
 *   dilate: D(x,y) = max { I(x-i+ox, y-j+oy) : 0<=i<se_w, 0<=j<se_h, in image }
 *   open  = dilate(erode(I)), close = erode(dilate(I)), same SE and origin
 * (sections "Within-Line Morphological Operations" — 1D erosion and dilation,
 * opening and closing built from them — and "2D Morphological Operators for
 * Rectangular Masks" — separable composition of within-line and between-line
 * operations).
 */
#ifndef MORPH_H
#define MORPH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MORPH_ABI_VERSION 1

#if defined(__GNUC__)
#define MORPH_API __attribute__((visibility("default")))
#else
#define MORPH_API
#endif

typedef enum morph_status {
    MORPH_OK = 0,
    MORPH_EINVAL = 1,     /* bad argument (sizes, formats, SE, aliasing, NULL) */
    MORPH_ECAPACITY = 2,  /* an RLE output needed more runs than capacity_runs */
    MORPH_ENOMEM = 3,     /* workspace smaller than morph_workspace_size() */
    MORPH_ECUDA = 4,      /* a CUDA launch or copy failed (see morph_last_error) */
    MORPH_ETIMEOUT = 5    /* a bounded device-side wait gave up */
} morph_status;

typedef enum morph_format {
    MORPH_PACKED32 = 0,   /* rows of uint32 words */
    MORPH_PACKED64 = 1,   /* rows of uint64 words */
    MORPH_RLE = 2         /* CSR of uint16 (start, end) runs */
} morph_format;

typedef enum morph_op {
    MORPH_ERODE = 0,
    MORPH_DILATE = 1,
    MORPH_OPEN = 2,
    MORPH_CLOSE = 3,
    MORPH_TO_RLE = 4      /* batch jobs only: convert the packed src into the RLE dst */
} morph_op;

/* Descriptor of one image.  Only the fields of its format are read.
 *   packed: words (device, aligned to the word size), stride_words >=
 *           ceil(width / B) words of B bits between consecutive rows.
 *   RLE   : row_ptr (device int32[height+1], row_ptr[0] = 0), runs (device
 *           uint16[2*capacity_runs], aligned to 4 bytes: one (start, end)
 *           pair), n_runs (device int64, may be NULL for
 *           inputs).  As an OUTPUT, the producer writes row_ptr, the runs and
 *           *n_runs = total runs needed; if that exceeds capacity_runs the runs
 *           are not written and MORPH_ECAPACITY is latched (row_ptr and *n_runs
 *           still tell the caller how much room to provide).
 * The descriptor itself lives in host memory and is only read during the
 * call; the buffers it points to must stay valid until the stream work ends. */
typedef struct morph_image {
    int32_t fmt;            /* morph_format */
    int32_t width;          /* W >= 1 (<= 65535 for RLE) */
    int32_t height;         /* H >= 1 */
    int32_t reserved;       /* must be 0 */
    void *words;            /* packed: row 0 */
    int64_t stride_words;   /* packed: words per row, in the format's words */
    int32_t *row_ptr;       /* RLE: int32[H+1] */
    uint16_t *runs;         /* RLE: uint16[2*capacity_runs] */
    int64_t capacity_runs;  /* RLE: room in runs, in runs */
    int64_t *n_runs;        /* RLE output: int64 written on the device */
} morph_image;

/* ------------------------------------------------------------------ ops --
 * Rectangular morphology.  dst and src have the same width and height and
 * the same family of format: both packed (PACKED32 / PACKED64, may differ) or
 * both RLE.  dst may not overlap src (use a second buffer; the paper's
 * in-place convention is not kept because tiles of one launch read rows that
 * other tiles write).
 *
 * Packed path: one launch of the fused tile kernel (within-line pass on
 * packed words, between-line pass as bit-sliced run counters down word
 * columns; opening / closing fuse both operations in the same launch).
 * Workspace: none (workspace may be NULL, workspace_bytes 0), except for a
 * rectangle reaching more than 128 pixels left or right of its origin
 * (after clipping to the image), which runs as a chain of launches through
 * scratch images in the workspace.
 * RLE path: the row pass shrinks or grows every run and merges the grown
 * ones (section "Within-Line Morphological Operations"); the between-line
 * pass intersects (erode) or unites (dilate) se_h neighbouring rows, then a
 * count / prefix-sum / write sequence produces the CSR output.  Workspace:
 * morph_workspace_size() bytes, 256-byte aligned.
 *
 * Errors: MORPH_EINVAL for a bad SE, size, format, alias or NULL pointer;
 * MORPH_ENOMEM if workspace_bytes is too small; MORPH_ECUDA if a launch
 * failed.  MORPH_ECAPACITY for an RLE dst is latched on the device.
 */
MORPH_API morph_status morph_erode_rect(const morph_image *dst, const morph_image *src, int se_w,
                              int se_h, int origin_x, int origin_y, void *workspace,
                              size_t workspace_bytes, void *stream);
MORPH_API morph_status morph_dilate_rect(const morph_image *dst, const morph_image *src, int se_w,
                               int se_h, int origin_x, int origin_y, void *workspace,
                               size_t workspace_bytes, void *stream);
MORPH_API morph_status morph_open_rect(const morph_image *dst, const morph_image *src, int se_w,
                             int se_h, int origin_x, int origin_y, void *workspace,
                             size_t workspace_bytes, void *stream);
MORPH_API morph_status morph_close_rect(const morph_image *dst, const morph_image *src, int se_w,
                              int se_h, int origin_x, int origin_y, void *workspace,
                              size_t workspace_bytes, void *stream);

/* Same four operations selected by `op` (morph_op). */
MORPH_API morph_status morph_rect(int op, const morph_image *dst, const morph_image *src, int se_w,
                        int se_h, int origin_x, int origin_y, void *workspace,
                        size_t workspace_bytes, void *stream);

/* Bytes of workspace that morph_rect(op, dst, src, se_w, se_h, origin_x,
 * origin_y, ...) needs: 0 for the packed path unless the rectangle is wider
 * than one launch reaches; for RLE it depends on the op and image size only.
 * Returns 0 for invalid arguments (the op call then reports them). */
MORPH_API size_t morph_workspace_size(int op, const morph_image *dst, const morph_image *src,
                                      int se_w, int se_h, int origin_x, int origin_y);

/* Erosion or dilation of an RLE image with no workspace and no allocation.
 * The paper has no counterpart: this exists for callers that may not
 * allocate device memory at all (a serving loop with a fixed budget, a host
 * whose allocator owns the rest of the device).  Same result as
 * morph_rect(MORPH_ERODE / MORPH_DILATE, ...) on RLE images; op must be one
 * of those two.  The per-row scratch lives in a fixed array inside the
 * library, so src->height must be <= 65536 (else MORPH_EINVAL); every device
 * that loads the library holds that array (256 KiB) until exit.  The first
 * call on a device looks up the array's device address (make that first
 * call before any stream capture).  All calls on a device share the array:
 * calls that overlap on the GPU race on it — serialise them.  Errors as for
 * morph_rect; MORPH_ECAPACITY is latched on the device. */
MORPH_API morph_status morph_rle_rect_noalloc(int op, const morph_image *dst,
                                              const morph_image *src, int se_w, int se_h,
                                              int origin_x, int origin_y, void *stream);

/* ------------------------------------------------------- arbitrary masks --
 * Section "Morphology with Arbitrary Masks": erosion / dilation / opening /
 * closing of a packed or RLE image by an arbitrary structuring element.
 *   mask: HOST memory, mask_h rows of mask_w bytes, row 0 first; a nonzero
 *         byte puts that pixel (i, j) in the element (read during the call
 *         only).  1 <= mask_w, mask_h <= 4096; at least one pixel; at most
 *         1024 horizontal runs (maximal row segments of set pixels).
 *   origin (origin_x, origin_y) inside the mask (it need not be set).
 * Semantics are the rectangle ones with the window replaced by the element:
 *   E(x,y) = AND of src(x+i-ox, y+j-oy) over set (i,j) inside the image,
 *   D(x,y) = OR of src(x-i+ox, y-j+oy) over set (i,j) inside the image,
 *   open = D(E), close = E(D); a full mask gives exactly morph_rect.
 * Packed images (either word size): run at a time with doubling
 * accumulation — doubling levels of the image up to the longest run are
 * built in the workspace, then every output word is the AND of two level
 * words per run.
 * RLE images (src and dst both RLE): run at a time on the runs — for each
 * run of the element, every run of the image line it reaches (for an
 * erosion, every gap between runs: the erosion is the complement of the
 * dilation of the complement by the reflected element) is grown by the
 * element run and painted into the output line, which is then encoded into
 * runs; open / close encode their first stage into an intermediate RLE in the
 * workspace (never full: it holds ceil(W/2) runs per line).  dst's capacity
 * too small latches MORPH_ECAPACITY (read by morph_sync_status) and leaves
 * its runs unwritten, as for the rectangles.
 * src and dst the same size, not overlapping.  Workspace (device, 256-byte
 * aligned): morph_mask_workspace_size() bytes (0 = none needed; that
 * function returns 0 also for invalid arguments, which morph_mask then
 * reports).  Errors: MORPH_EINVAL (arguments, one packed and one RLE image,
 * empty or too large element), MORPH_ENOMEM (workspace too small),
 * MORPH_ECUDA. */
MORPH_API size_t morph_mask_workspace_size(int op, const morph_image *dst, const morph_image *src,
                                           const uint8_t *mask, int mask_w, int mask_h,
                                           int origin_x, int origin_y);
MORPH_API morph_status morph_mask(int op, const morph_image *dst, const morph_image *src,
                                  const uint8_t *mask, int mask_w, int mask_h, int origin_x,
                                  int origin_y, void *workspace, size_t workspace_bytes,
                                  void *stream);

/* ------------------------------------------------------------ conversion --
 * Section "Conversion Between Image Formats".
 * rle_from_bitmap: packed src -> RLE dst (canonical runs of every row).  A
 * row's transitions are found with shifts and XOR, counted with popcount,
 * their output positions come from a prefix sum over rows.  Workspace:
 * morph_convert_workspace_size(height) bytes.
 * rle_to_bitmap: RLE src -> packed dst; padding bits written 0.  No workspace.
 * The src RLE must be canonical (as every producer here writes it); a
 * non-canonical list gives an unspecified bitmap but no out-of-bounds access.
 */
MORPH_API size_t morph_convert_workspace_size(int height);
MORPH_API morph_status rle_from_bitmap(const morph_image *dst_rle, const morph_image *src_packed,
                             void *workspace, size_t workspace_bytes, void *stream);
MORPH_API morph_status rle_to_bitmap(const morph_image *dst_packed, const morph_image *src_rle,
                           void *stream);

/* ------------------------------------------------------ sheared lines --
 * Section "Morphology with Lines at Arbitrary Orientations": a line element
 * at an angle is applied by skewing the image perpendicular to the line,
 * applying the axis-parallel line and skewing back.  Here the skew is given
 * as a table (for an angle a from the vertical, shift[y] = round(y tan a)):
 * line y is moved right by shift[y], the vertical line of `length` pixels
 * with origin `origin` is applied (clipped window: positions holding no
 * image pixel are left out), and the lines are moved back.  Pixel by pixel
 *   erode:  E(x,y) = AND over j in [-origin, length-1-origin] of
 *                    src(x + shift[y] - shift[y+j], y + j)
 *   dilate: D(x,y) = OR over j in [-(length-1-origin), origin] of the same,
 * terms only where the source pixel lies in the image; open = D(E), close =
 * E(D).  horizontal = 1 is the transposed case (shift[x] moves column x
 * down, the line runs along the rows; n_shift = width), else n_shift =
 * height.  shift: HOST int32[n_shift], read during the call.  src and dst
 * packed (either word size), same size, not overlapping.  Workspace
 * (device, 256-byte aligned): morph_sheared_line_workspace_size() bytes
 * (0 for invalid arguments).  Errors: MORPH_EINVAL, MORPH_ENOMEM,
 * MORPH_ECUDA. */
MORPH_API size_t morph_sheared_line_workspace_size(int op, const morph_image *src, const int32_t *shift,
                                                   int n_shift, int length, int horizontal);
MORPH_API morph_status morph_sheared_line(int op, const morph_image *dst, const morph_image *src,
                                          const int32_t *shift, int n_shift, int length, int origin,
                                          int horizontal, void *workspace, size_t workspace_bytes,
                                          void *stream);

/* Skew table and line of a line element at an angle, built as the paper
 * builds one (section "Morphology with Lines at Arbitrary Orientations":
 * skew perpendicular to the line by the tangent of the line's angle from its
 * nearer axis, then an axis-parallel line of about 2 r cos(angle) pixels).
 * The outputs are the arguments of morph_sheared_line.
 *   angle_deg: degrees counterclockwise from the x axis, image rows growing
 *     downwards; any finite value (reduced to a in [-90, 90)).
 *   Lines with |a| <= 45 run along the rows: *horizontal = 1,
 *     *n_shift = width, shift[x] = floor(x tan(a) + 1/2) moves column x down.
 *   Other lines run along the columns: *horizontal = 0, *n_shift = height,
 *     shift[y] = floor(y tan(90 - a) + 1/2) moves row y right.
 *   *length = 2 c + 1, *origin = c, c = half_length |cos| of the same angle
 *     rounded to the nearest integer (ties away from zero).
 * shift: HOST int32[capacity], written up to *n_shift entries.  Double
 * precision throughout.  Errors: MORPH_EINVAL (NULL output, half_length < 0,
 * width or height < 1, a non-finite angle, capacity below the table's
 * length); nothing is written then. */
MORPH_API morph_status morph_line_element(double angle_deg, int half_length, int width, int height,
                                          int32_t *shift, int capacity, int *n_shift, int *length,
                                          int *origin, int *horizontal);

/* ------------------------------------------------------------- transpose --
 * Section "Efficient Transpose": dst(x, y) = src(y, x).
 * morph_transpose: packed src (W x H) -> packed dst (H x W), either word
 * size; padding bits of dst written 0.  No workspace.  A bit-matrix
 * transpose of 32 x 32 blocks in registers, tiles staged in shared memory.
 * morph_rle_transpose: RLE src (W x H) -> RLE dst (H x W, so H <= 65535):
 * the columns of src become the rows of dst (vertical runs, e.g. for
 * vertical run-length statistics or between-line operations done as
 * within-line ones).  Runs painted into a bitmap, transposed, encoded again
 * (capacity rules of rle_from_bitmap).  Workspace (device, 256-byte
 * aligned): morph_rle_transpose_workspace_size() bytes.
 * Errors: MORPH_EINVAL (formats, sizes, overlap), MORPH_ENOMEM, MORPH_ECUDA. */
MORPH_API morph_status morph_transpose(const morph_image *dst, const morph_image *src, void *stream);
MORPH_API size_t morph_rle_transpose_workspace_size(const morph_image *src_rle);
MORPH_API morph_status morph_rle_transpose(const morph_image *dst_rle, const morph_image *src_rle,
                                           void *workspace, size_t workspace_bytes, void *stream);

/* ------------------------------------------------ connected components --
 * Section "Connected Component Extraction and Statistics".
 * morph_rle_components labels every run of an RLE image by its connected
 * component: each run starts as its own set of a union-find structure, every
 * run is merged with the runs of the line above that it touches, and each
 * run is then relabelled by its set.
 *   connectivity 4: runs in adjacent lines touch when they share a column
 *                   ([s, e) and [s', e'): s < e' and s' < e);
 *                8: also when they meet at a corner (s <= e' and s' <= e).
 *   labels (device int32[src->capacity_runs]): labels[k] for the image's
 *     runs k = 0 .. n_runs-1 in row order; components are numbered 0, 1, ...
 *     in the raster order of their first run, so the labelling is unique.
 *   n_components (device int64, required): the number of components.
 *   stats (device, may be NULL): for component c < max_components,
 *     stats[c] = {x0, y0, x1, y1 (half-open bounding box), area (pixels),
 *     sum_x, sum_y (sums over its pixels; centroid = sum / area)}.
 *     If there are more than max_components components MORPH_ECAPACITY is
 *     latched (see morph_sync_status), labels and n_components are still
 *     complete and stats holds the first max_components.
 * The src RLE must be canonical (every producer here writes it so).
 * Workspace (device, 256-byte aligned): morph_components_workspace_size()
 * bytes.  Errors: MORPH_EINVAL (arguments, non-RLE src, NULL labels or
 * n_components, connectivity not 4 or 8, overlapping buffers), MORPH_ENOMEM
 * (workspace too small), MORPH_ECUDA. */
typedef struct morph_component {
    int64_t x0, y0, x1, y1;  /* bounding box [x0, x1) x [y0, y1) */
    int64_t area;            /* pixels */
    int64_t sum_x, sum_y;    /* sums of the pixels' coordinates */
} morph_component;

MORPH_API size_t morph_components_workspace_size(const morph_image *src_rle);
MORPH_API morph_status morph_rle_components(int32_t *labels, morph_component *stats,
                                            int64_t max_components, int64_t *n_components,
                                            const morph_image *src_rle, int connectivity,
                                            void *workspace, size_t workspace_bytes,
                                            void *stream);

/* Layout analysis (section "Document Analysis Performance"): the spacing of
 * words and of lines is estimated from the white run lengths along the lines
 * and along the columns (via the transpose): the gap estimate is the
 * smallest length L such that white runs of length <= L make up at least
 * coverage_pct percent of the white runs no longer than 1/16 of the line
 * (0 without such runs).  The page is dilated by a (gap_h + 1) x (gap_v + 1)
 * rectangle (origin at its centre), merging characters and lines into
 * blocks, and the 8-connected components of the result are returned as
 * records in `boxes` (as morph_rle_components, max_boxes of them; the count
 * in *n_boxes on the device).  gaps (HOST int32[2], may be NULL) receives
 * gap_h and gap_v.  page: packed, both sides <= 65535.  Synchronises the
 * stream once (the two histograms are read back to choose the rectangle).
 * Workspace (device, 256-byte aligned): morph_layout_workspace_size() bytes.
 * Errors: MORPH_EINVAL, MORPH_ENOMEM, MORPH_ECUDA; MORPH_ECAPACITY latched
 * when there are more blocks than max_boxes. */
MORPH_API size_t morph_layout_workspace_size(const morph_image *page);
MORPH_API morph_status morph_layout_boxes(morph_component *boxes, int64_t max_boxes, int64_t *n_boxes,
                                          int32_t *gaps, const morph_image *page, int coverage_pct,
                                          void *workspace, size_t workspace_bytes, void *stream);

/* Run-length statistics (section "Other Operations"): histograms of the
 * lengths of the black runs (1-pixels) and of the white runs (maximal gaps
 * of 0-pixels in a row, the ones at either end of the row included; an empty
 * row is one white run of length width) of an RLE image.  black_hist and
 * white_hist: device int64[width + 1], overwritten; entry L counts the runs
 * of length L (entry 0 stays 0).  Either may be NULL.  No workspace.
 * Errors: MORPH_EINVAL, MORPH_ECUDA. */
MORPH_API morph_status morph_run_length_hist(int64_t *black_hist, int64_t *white_hist,
                                             const morph_image *src_rle, void *stream);

/* ----------------------------------------------------------------- batch --
 * Many uneven pages, each with its own op, rectangle and path, in ONE
 * morph_batch_launch() call.  A job reads a packed src page and writes a
 * packed dst page (same size, no overlap), or with MORPH_TO_RLE converts it
 * into an RLE dst.  A job may depend on one earlier job (depends_on), which
 * chains per-page pipelines (e.g. close -> open -> dilate -> to RLE) inside
 * one call.  path MORPH_PATH_PACKED runs the fused rectangle tile on the
 * page; MORPH_PATH_RLE converts the page to runs, runs the RLE operation on
 * them and writes the result back as a bitmap.  The choice per page is the
 * caller's (the Python autotuner picks it by ink density and rectangle).
 *
 * How a call runs (the operations are those of sections "2D Morphological
 * Operators for Rectangular Masks" and "Conversion Between Image Formats"; the
 * grouping is this library's):
 *  - packed-path jobs with no dependency, or whose dependency is itself such
 *    a job, run as grouped launches of the rectangle tile: one launch per
 *    tile variant and dependency level, over a device table of the level's
 *    jobs of that variant; the levels run in order, the launches of a level
 *    concurrently on the library's auxiliary streams of the device, forked
 *    from and joined back into the caller's stream (a plan with at most one
 *    group per level and at most one RLE group runs in stream order on the
 *    caller's stream);
 *  - then one persistent kernel runs every other job (RLE-path jobs with a
 *    dependency or depended on, MORPH_TO_RLE jobs, packed
 *    jobs the tile cannot plan) and the bitmap -> RLE encodes of the
 *    source pages of RLE-path jobs;
 *  - then RLE-path jobs that neither depend on a job nor are depended on run
 *    as grouped launches of the run-length source tile, which read the
 *    persistent kernel's encodes (both stages of an opening or closing in
 *    one pass).
 * morph_batch_kernels() returns the number of kernel launches of one call.
 *
 * Use: morph_batch_plan_bytes() -> a host buffer; morph_batch_plan_build()
 * fills it (all checks happen here); the caller copies the plan to device
 * memory and calls morph_batch_launch() with that copy, the host plan and a
 * workspace of morph_batch_workspace_size() bytes (counters, encodes and the
 * RLE buffers of RLE-path jobs).  The launch does no host work beyond
 * kernel launches, one memset of the counters and the event records and
 * waits of the fork and join, so it can be captured in a CUDA graph and
 * replayed while the plan, workspace and pages stay valid.  Launches of one
 * device from several host threads share its auxiliary streams (a mutex
 * orders their use).
 * In the persistent kernel, work items are claimed from a device queue in
 * plan order; an item waits (bounded spin, acquire loads) only for items of
 * smaller index, which are already held by running CTAs, so the launch
 * cannot deadlock.  A wait longer than the plan's limit (4 s) latches
 * MORPH_ETIMEOUT and stops every CTA; an RLE buffer that is too small latches
 * MORPH_ECAPACITY and leaves that job's dst unwritten (and, when it is the
 * buffer of a shared source encode, the dst of every job sharing it).
 * RLE-path jobs without depends_on that read the same source page (same
 * words, stride, format and size) share one bitmap -> RLE encode of it.
 *
 * tile_rows: for jobs whose own tile_rows is 0, the row-band height of
 * packed tiles and the rows per work item of RLE-path and MORPH_TO_RLE jobs
 * (0 = library defaults; RLE items hold a multiple of 64 rows, at most 1024,
 * by default more the more RLE rows the plan holds).
 * rle_runs_per_row: room per row in each RLE buffer of RLE-path jobs
 * (0 = W/16 + 4, at most ceil(W/2)).
 * Limits: packed-path rectangles must reach <= 128 pixels left and right of
 * the origin after clipping; RLE-path pages must be <= 65535 pixels wide.
 */
typedef enum morph_path { MORPH_PATH_PACKED = 0, MORPH_PATH_RLE = 1 } morph_path;

typedef struct morph_job {
    int32_t op;          /* morph_op; MORPH_TO_RLE converts src to an RLE dst */
    int32_t path;        /* morph_path (ignored for MORPH_TO_RLE) */
    int32_t se_w, se_h, origin_x, origin_y;   /* ignored for MORPH_TO_RLE */
    int32_t depends_on;  /* index of an EARLIER job of the plan whose work must
                            finish before this one starts (e.g. the job that
                            writes this job's src), or -1 */
    int32_t tile_rows;   /* packed path: row-band height of its tiles; RLE path
                            and MORPH_TO_RLE: rows per work item (0 = the
                            plan's tile_rows, else the library default) */
    int32_t words_per_thread;  /* packed path: 32-bit words each thread of the
                            rectangle tile covers, 2 or 4 (0 = the planner's
                            choice; a tiling the tile cannot hold falls back
                            to the persistent kernel); ignored elsewhere */
    morph_image src;     /* packed */
    morph_image dst;     /* packed, same size; RLE for MORPH_TO_RLE */
} morph_job;

MORPH_API size_t morph_batch_plan_bytes(const morph_job *jobs, int n_jobs, int tile_rows,
                                        int rle_runs_per_row);
MORPH_API morph_status morph_batch_plan_build(void *host_plan, size_t plan_bytes,
                                              const morph_job *jobs, int n_jobs, int tile_rows,
                                              int rle_runs_per_row);
MORPH_API size_t morph_batch_workspace_size(const void *host_plan);
/* Number of work items in a plan (-1 for an invalid plan). */
MORPH_API int morph_batch_items(const void *host_plan);
/* Kernel launches that one morph_batch_launch() of the plan makes (-1 for an
 * invalid plan): the grouped tile launches plus the persistent kernel when
 * the plan has work items for it. */
MORPH_API int morph_batch_kernels(const void *host_plan);
/* Test and timing hooks on a host plan (what = 0 and 1 before the plan is
 * copied to the device; what = 2 at any time — the launch reads it there):
 * what = 0: set the wait limit to `value` ns (>= 1 ms; default 4 s);
 * what = 1: add `value` to the item count that the second phase of the first
 *           multi-phase (RLE-path) job waits for, so that its wait runs out —
 *           used to check that MORPH_ETIMEOUT is reported and the device stays
 *           usable;
 * what = 2: value != 0 launches the tile groups alone, without the
 *           persistent kernel — to time the groups once an earlier launch of
 *           the same plan has left its encodes in the workspace (the RLE
 *           groups read them); value 0 restores the full launch. */
MORPH_API morph_status morph_batch_plan_debug(void *host_plan, int what, long long value);
/* n_ctas <= 0: as many CTAs as fit on the device at once. */
MORPH_API morph_status morph_batch_launch(const void *dev_plan, const void *host_plan,
                                          void *workspace, size_t workspace_bytes, int n_ctas,
                                          void *stream);

/* The batch between host buffers: copies in_bytes from host memory h_in to
 * device memory d_in, runs morph_batch_launch() on the plan, and copies
 * out_bytes from device memory d_out to host memory h_out, in that order on
 * `stream` (one cudaMemcpyAsync per copy).  The caller lays the plan's
 * source pages out in d_in and its destination pages in d_out; h_in and
 * h_out should be page-locked (cudaHostAlloc) for the copies to be
 * asynchronous.  Returns once the work is queued; morph_sync_status(stream)
 * waits for it.  Two calls on two streams with two plans and buffer sets
 * overlap one step's copies with the other's kernels.  Errors: MORPH_EINVAL
 * (a NULL buffer with a nonzero size), those of morph_batch_launch(),
 * MORPH_ECUDA. */
MORPH_API morph_status morph_batch_launch_host(const void *dev_plan, const void *host_plan,
                                               void *workspace, size_t workspace_bytes,
                                               const void *h_in, void *d_in, size_t in_bytes,
                                               void *h_out, const void *d_out, size_t out_bytes,
                                               void *stream);

/* ---------------------------------------------------------------- status -- */
/* Wait for `stream`, then return (and clear) the first device-side condition
 * latched since the last call (MORPH_ECAPACITY, MORPH_ETIMEOUT), else the
 * stream's CUDA error as MORPH_ECUDA, else MORPH_OK. */
MORPH_API morph_status morph_sync_status(void *stream);
/* Message for the last non-OK status returned on this host thread. */
MORPH_API const char *morph_last_error(void);
MORPH_API const char *morph_status_string(int status);
MORPH_API int morph_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MORPH_H */
