// morph_rle_rect_noalloc: RLE erosion / dilation for callers that cannot
// allocate device memory.
//
// Who needs it: code that must not call cudaMalloc or any allocating library
// routine on its hot path — a serving loop with a fixed memory budget that
// forbids allocation after start-up, a host application that hands the
// library only the images it owns (its allocator owns the rest of the
// device), or a caller running where allocating would synchronise the device
// or fail.  The regular RLE entry points need a caller-provided workspace
// for their per-row counts; this one keeps that scratch in a fixed array
// that lives in the library's own device image instead.
//
// The scratch is one int32 per image row, so images are limited to
// NOALLOC_MAX_ROWS rows (256 KiB, held by every device that loads the
// library until the process exits).  All calls on a device share the array:
// calls whose work overlaps on the GPU (different streams, no ordering)
// race on it and must be serialised by the caller.  Nothing in it needs to
// start at zero: the count pass writes the entry of every row before the
// prefix sum reads it, and entries beyond the image height are never read.
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "morph_internal.cuh"

namespace morph {
namespace {

constexpr int NOALLOC_MAX_ROWS = 65536;

// Per-row run counts written by the count pass and read by the prefix sum.
static __device__ __align__(256) int32_t g_noalloc_counts[NOALLOC_MAX_ROWS];

// Host: device address of the scratch array on the current device.  In host
// code the array's name is only a host-side stand-in, so the address is
// looked up once per device (with that device current) and cached.
int32_t *noalloc_scratch(cudaError_t *err) {
    static std::mutex mu;
    static int32_t *ptrs[128] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 128) {
        *err = e != cudaSuccess ? e : cudaErrorInvalidDevice;
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(mu);
    if (!ptrs[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_counts);
        if (e != cudaSuccess) {
            *err = e;
            return nullptr;
        }
        ptrs[dev] = (int32_t *)p;
    }
    *err = cudaSuccess;
    return ptrs[dev];
}

morph_status reject(morph_status st, const char *fmt, ...) {
    char buf[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    set_error("%s", buf);
    return st;
}

bool ranges_overlap(const void *a, size_t an, const void *b, size_t bn) {
    const uintptr_t a0 = (uintptr_t)a, b0 = (uintptr_t)b;
    return an && bn && a0 < b0 + bn && b0 < a0 + an;
}

}  // namespace
}  // namespace morph

using namespace morph;

extern "C" morph_status morph_rle_rect_noalloc(int op, const morph_image *dst,
                                               const morph_image *src, int se_w, int se_h,
                                               int origin_x, int origin_y, void *stream) {
    if (op != MORPH_ERODE && op != MORPH_DILATE)
        return reject(MORPH_EINVAL, "morph_rle_rect_noalloc supports MORPH_ERODE and MORPH_DILATE only");
    if (!dst || !src) return reject(MORPH_EINVAL, "dst or src is NULL");
    if (src->fmt != MORPH_RLE || dst->fmt != MORPH_RLE || src->reserved || dst->reserved)
        return reject(MORPH_EINVAL, "src and dst must be RLE images");
    if (src->width < 1 || src->height < 1 || src->width > 65535 || dst->width != src->width ||
        dst->height != src->height)
        return reject(MORPH_EINVAL, "bad or different image sizes (%d x %d, %d x %d)", src->width,
                      src->height, dst->width, dst->height);
    if (src->height > NOALLOC_MAX_ROWS)
        return reject(MORPH_EINVAL, "image height %d exceeds the %d rows of the fixed scratch of "
                      "morph_rle_rect_noalloc", src->height, NOALLOC_MAX_ROWS);
    if (!src->row_ptr || !dst->row_ptr || dst->capacity_runs < 0 || src->capacity_runs < 0 ||
        (dst->capacity_runs > 0 && !dst->runs))
        return reject(MORPH_EINVAL, "NULL row_ptr or runs, or negative capacity");
    if ((uintptr_t)src->runs % 4 || (uintptr_t)dst->runs % 4)
        return reject(MORPH_EINVAL, "runs must be aligned to 4 bytes (one (start, end) pair)");
    if (se_w < 1 || se_h < 1 || se_w > 65535 || se_h > 65535 || origin_x < 0 || origin_x >= se_w ||
        origin_y < 0 || origin_y >= se_h)
        return reject(MORPH_EINVAL, "bad structuring element %d x %d, origin (%d, %d)", se_w, se_h,
                      origin_x, origin_y);
    const size_t rp = (size_t)(src->height + 1) * sizeof(int32_t);
    if (ranges_overlap(dst->row_ptr, rp, src->row_ptr, rp) ||
        ranges_overlap(dst->runs, (size_t)dst->capacity_runs * 4, src->runs, (size_t)src->capacity_runs * 4) ||
        ranges_overlap(dst->row_ptr, rp, src->runs, (size_t)src->capacity_runs * 4) ||
        ranges_overlap(dst->runs, (size_t)dst->capacity_runs * 4, src->row_ptr, rp))
        return reject(MORPH_EINVAL, "dst overlaps src");

    cudaError_t e;
    int32_t *counts = noalloc_scratch(&e);
    if (!counts) return reject(MORPH_ECUDA, "scratch address: %s", cudaGetErrorString(e));

    // clip the rectangle to what can reach inside the image
    const int W = src->width, H = src->height;
    int l = origin_x, r = se_w - 1 - origin_x, u = origin_y, d = se_h - 1 - origin_y;
    if (l > W - 1) l = W - 1;
    if (r > W - 1) r = W - 1;
    if (u > H - 1) u = H - 1;
    if (d > H - 1) d = H - 1;

    const RleIn in{src->row_ptr, src->runs, W, H};
    const RleOut out{dst->row_ptr, dst->runs, dst->capacity_runs, dst->n_runs};
    e = launch_rle_rect(in, out, op == MORPH_DILATE, l + r + 1, u + d + 1, l, u, counts, nullptr,
                        device_status_ptr(), (cudaStream_t)stream);
    if (e != cudaSuccess) return reject(MORPH_ECUDA, "RLE morphology launch: %s", cudaGetErrorString(e));
    return MORPH_OK;
}
