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


}  // namespace
}  // namespace morph

using namespace morph;

extern "C" morph_status morph_rle_rect_noalloc(int op, const morph_image *dst,
                                               const morph_image *src, int se_w, int se_h,
                                               int origin_x, int origin_y, void *stream) {
    if (op != MORPH_ERODE && op != MORPH_DILATE)
        return reject(MORPH_EINVAL, "morph_rle_rect_noalloc supports MORPH_ERODE and MORPH_DILATE only");
    const morph_status st = check_op_args(op, dst, src, se_w, se_h, origin_x, origin_y);
    if (st != MORPH_OK) return st;
    if (src->fmt != MORPH_RLE)
        return reject(MORPH_EINVAL, "morph_rle_rect_noalloc takes RLE images");
    if (src->height > NOALLOC_MAX_ROWS)
        return reject(MORPH_EINVAL, "image height %d exceeds the %d rows of the fixed scratch of "
                      "morph_rle_rect_noalloc", src->height, NOALLOC_MAX_ROWS);

    cudaError_t e;
    int32_t *counts = noalloc_scratch(&e);
    if (!counts) return reject(MORPH_ECUDA, "scratch address: %s", cudaGetErrorString(e));

    const int W = src->width, H = src->height;
    const Se se = clip_se(W, H, se_w, se_h, origin_x, origin_y);
    const RleIn in{src->row_ptr, src->runs, W, H};
    const RleOut out{dst->row_ptr, dst->runs, dst->capacity_runs, dst->n_runs};
    e = launch_rle_rect(in, out, op == MORPH_DILATE, se.sw, se.sh, se.ox, se.oy, counts, nullptr,
                        device_status_ptr(), (cudaStream_t)stream);
    if (e != cudaSuccess) return reject(MORPH_ECUDA, "RLE morphology launch: %s", cudaGetErrorString(e));
    return MORPH_OK;
}
