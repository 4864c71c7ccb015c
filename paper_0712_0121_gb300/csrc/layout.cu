// Morphological layout analysis as in the paper's document-analysis
// experiment (section "Document Analysis Performance"): the spacing of
// words and of lines is estimated from the white run lengths along and
// across the lines, a rectangular dilation of that size merges characters
// and lines into blocks, and the bounding boxes of the connected components
// of the result are the blocks.  Host orchestration of the library's own
// entry points (conversion, histograms, transpose, packed dilation,
// components); the only host work on data is reading two histograms back
// to choose the rectangle.
#include <vector>

#include "morph_internal.cuh"

namespace morph {
namespace {

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

// smallest L in [1, lmax] such that the white runs of length <= L are at
// least pct percent of the white runs of length <= lmax (0: no such runs)
int gap_estimate(const std::vector<int64_t> &white, int lmax, int pct) {
    int64_t total = 0;
    for (int L = 1; L <= lmax; ++L) total += white[L];
    if (total == 0) return 0;
    int64_t c = 0;
    for (int L = 1; L <= lmax; ++L) {
        c += white[L];
        if (c * 100 >= (int64_t)pct * total) return L;
    }
    return lmax;
}

struct LayoutPlan {
    int W, H, lmax_h, lmax_v;
    int64_t cap_h, cap_v;  // runs of the page / of its transpose (worst case: every other pixel)
    int nw64;
    size_t off_rp, off_runs, off_n, off_conv, off_rpt, off_runst, off_nt, off_tws, off_wh, off_wv, off_bmp,
        off_rws, off_rpd, off_runsd, off_nd, off_lab, off_cws, total;
};

LayoutPlan layout_plan(int W, int H) {
    LayoutPlan p;
    p.W = W;
    p.H = H;
    p.lmax_h = W / 16 > 1 ? W / 16 : 1;
    p.lmax_v = H / 16 > 1 ? H / 16 : 1;
    p.cap_h = (int64_t)H * ((W + 1) / 2);
    p.cap_v = (int64_t)W * ((H + 1) / 2);
    p.nw64 = (W + 63) / 64;
    size_t o = 0;
    auto take = [&](size_t n) { const size_t at = o; o += a256(n); return at; };
    p.off_rp = take((size_t)(H + 1) * 4);
    p.off_runs = take((size_t)p.cap_h * 4);
    p.off_n = take(8);
    p.off_conv = take(morph_convert_workspace_size(H > W ? H : W));
    p.off_rpt = take((size_t)(W + 1) * 4);
    p.off_runst = take((size_t)p.cap_v * 4);
    p.off_nt = take(8);
    p.off_tws = take(rle_transpose_ws_bytes(W, H));
    p.off_wh = take((size_t)(W + 1) * 8);
    p.off_wv = take((size_t)(H + 1) * 8);
    p.off_bmp = take((size_t)H * p.nw64 * 8);
    // scratch of the dilation: the largest rectangle the estimates allow
    morph_image img{};
    img.fmt = MORPH_PACKED64;
    img.width = W;
    img.height = H;
    img.words = (void *)256;
    img.stride_words = p.nw64;
    p.off_rws = take(morph_workspace_size(MORPH_DILATE, &img, &img, p.lmax_h + 1, p.lmax_v + 1,
                                          (p.lmax_h + 1) / 2, (p.lmax_v + 1) / 2));
    p.off_rpd = take((size_t)(H + 1) * 4);
    p.off_runsd = take((size_t)p.cap_h * 4);
    p.off_nd = take(8);
    p.off_lab = take((size_t)p.cap_h * 4);
    morph_image r{};
    r.fmt = MORPH_RLE;
    r.width = W;
    r.height = H;
    r.capacity_runs = p.cap_h;
    p.off_cws = take(morph_components_workspace_size(&r));
    p.total = o;
    return p;
}

}  // namespace
}  // namespace morph

using namespace morph;

extern "C" {

size_t morph_layout_workspace_size(const morph_image *page) {
    if (!page || (page->fmt != MORPH_PACKED32 && page->fmt != MORPH_PACKED64) || page->width < 1 ||
        page->height < 1 || page->width > 65535 || page->height > 65535)
        return 0;
    return layout_plan(page->width, page->height).total;
}

morph_status morph_layout_boxes(morph_component *boxes, int64_t max_boxes, int64_t *n_boxes, int32_t *gaps,
                                const morph_image *page, int coverage_pct, void *workspace,
                                size_t workspace_bytes, void *stream) {
    if (!page || (page->fmt != MORPH_PACKED32 && page->fmt != MORPH_PACKED64)) {
        set_error("morph_layout_boxes needs a packed page");
        return MORPH_EINVAL;
    }
    if (page->width < 1 || page->height < 1 || page->width > 65535 || page->height > 65535) {
        set_error("page of %d x %d: both sides must be 1 .. 65535 (RLE of the page and of its transpose)",
                  page->width, page->height);
        return MORPH_EINVAL;
    }
    if (!boxes || !n_boxes || max_boxes < 0 || coverage_pct < 1 || coverage_pct > 100) {
        set_error("boxes / n_boxes NULL, max_boxes < 0 or coverage_pct outside 1..100");
        return MORPH_EINVAL;
    }
    const int W = page->width, H = page->height;
    const LayoutPlan p = layout_plan(W, H);
    if (!workspace || workspace_bytes < p.total) {
        set_error("the layout analysis needs %zu bytes of workspace, got %zu", p.total,
                  workspace ? workspace_bytes : (size_t)0);
        return MORPH_ENOMEM;
    }
    if ((uintptr_t)workspace % 256) {
        set_error("workspace is not 256-byte aligned");
        return MORPH_EINVAL;
    }
    char *ws = (char *)workspace;
    cudaStream_t s = (cudaStream_t)stream;
    morph_image R{};  // the page as runs
    R.fmt = MORPH_RLE;
    R.width = W;
    R.height = H;
    R.row_ptr = (int32_t *)(ws + p.off_rp);
    R.runs = (uint16_t *)(ws + p.off_runs);
    R.capacity_runs = p.cap_h;
    R.n_runs = (int64_t *)(ws + p.off_n);
    morph_image RT = R;  // its transpose: the columns as lines
    RT.width = H;
    RT.height = W;
    RT.row_ptr = (int32_t *)(ws + p.off_rpt);
    RT.runs = (uint16_t *)(ws + p.off_runst);
    RT.capacity_runs = p.cap_v;
    RT.n_runs = (int64_t *)(ws + p.off_nt);
    int64_t *wh = (int64_t *)(ws + p.off_wh), *wv = (int64_t *)(ws + p.off_wv);
    const size_t conv = morph_convert_workspace_size(H > W ? H : W);

    morph_status st = rle_from_bitmap(&R, page, ws + p.off_conv, conv, stream);
    if (!st) st = morph_run_length_hist(nullptr, wh, &R, stream);
    if (!st) st = morph_rle_transpose(&RT, &R, ws + p.off_tws, rle_transpose_ws_bytes(W, H), stream);
    if (!st) st = morph_run_length_hist(nullptr, wv, &RT, stream);
    if (st) return st;
    std::vector<int64_t> hh(W + 1), hv(H + 1);
    cudaError_t e = cudaMemcpyAsync(hh.data(), wh, (size_t)(W + 1) * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hv.data(), wv, (size_t)(H + 1) * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_error("layout analysis: histogram read: %s", cudaGetErrorString(e));
        return MORPH_ECUDA;
    }
    // word spacing along the lines, line spacing across them
    const int th = gap_estimate(hh, p.lmax_h, coverage_pct);
    const int tv = gap_estimate(hv, p.lmax_v, coverage_pct);
    if (gaps) {
        gaps[0] = th;
        gaps[1] = tv;
    }
    // dilation by (th + 1) x (tv + 1) closes gaps of up to th x tv pixels
    morph_image D{};
    D.fmt = MORPH_PACKED64;
    D.width = W;
    D.height = H;
    D.words = ws + p.off_bmp;
    D.stride_words = p.nw64;
    morph_image RD = R;
    RD.row_ptr = (int32_t *)(ws + p.off_rpd);
    RD.runs = (uint16_t *)(ws + p.off_runsd);
    RD.n_runs = (int64_t *)(ws + p.off_nd);
    const int sw = th + 1, sh = tv + 1;
    st = morph_dilate_rect(&D, page, sw, sh, sw / 2, sh / 2, ws + p.off_rws, p.off_rpd - p.off_rws, stream);
    if (!st) st = rle_from_bitmap(&RD, &D, ws + p.off_conv, conv, stream);
    if (!st)
        st = morph_rle_components((int32_t *)(ws + p.off_lab), boxes, max_boxes, n_boxes, &RD, 8,
                                  ws + p.off_cws, p.total - p.off_cws, stream);
    return st;
}

}  // extern "C"
