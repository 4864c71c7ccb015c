// Kernel and launch dispatch of the packed rectangle tile (rect_tile.cuh);
// each rect_k*.cu instantiates one (stages, words per thread) family so that
// the variants compile in parallel.
#pragma once

#include <mutex>

#include "rect_tile.cuh"

namespace morph {

template <int NST, int NWT, int VM, int HM, int HALO>
__global__ void __launch_bounds__(256, 2) k_rect(const RectArgs a) {
    extern __shared__ __align__(16) uint32_t sm[];
    rect_tile<NST, NWT, VM, HM, HALO>(a, blockIdx.x, blockIdx.y, sm);
}

template <int NST, int NWT, int VM, int HM, int HALO>
cudaError_t rect_launch_t(const RectArgs &a0, cudaStream_t s) {
    RectArgs a = a0;
    // with the band chosen here the CTA may hold every group its tiling
    // allows: size the shared memory for that many (the fitted band can only
    // need as much or less)
    if (a.band_auto) a.groups = a.threads / a.tpr;
    const size_t smem = rect_smem_words(a) * sizeof(uint32_t);
    auto kern = k_rect<NST, NWT, VM, HM, HALO>;
    // resident CTAs per SM of this variant at this size (looked up once per
    // device, CTA size and shared memory)
    static std::mutex mu;
    static int c_dev = -1, c_threads = 0, c_occ = 0;
    static size_t c_smem = 0;
    int dev = 0, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (c_dev != dev || c_threads != a.threads || c_smem != smem) {
            if (smem > 48 * 1024) {
                e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e != cudaSuccess) return e;
            }
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c_occ, kern, a.threads, smem);
            if (e != cudaSuccess) return e;
            c_dev = dev;
            c_threads = a.threads;
            c_smem = smem;
        }
        occ = c_occ;
    }
    if (occ < 1) return cudaErrorInvalidConfiguration;
    if (a.band_auto) rect_fit_band(a, occ * rect_sm_count(dev));
    kern<<<rect_grid(a), a.threads, smem, s>>>(a);
    return cudaGetLastError();
}

template <int NST, int NWT, int VM>
cudaError_t rect_launch_h(const RectArgs &a, cudaStream_t s) {
    switch (a.hmode) {
    case RH_NONE: return rect_launch_t<NST, NWT, VM, RH_NONE, 1>(a, s);
    case RH_D1: return rect_launch_t<NST, NWT, VM, RH_D1, 1>(a, s);
    case RH_D2: return rect_launch_t<NST, NWT, VM, RH_D2, 1>(a, s);
    default:
        switch (a.halo) {
        case 1: return rect_launch_t<NST, NWT, VM, RH_LOG, 1>(a, s);
        case 2: return rect_launch_t<NST, NWT, VM, RH_LOG, 2>(a, s);
        case 4: return rect_launch_t<NST, NWT, VM, RH_LOG, 4>(a, s);
        default: return cudaErrorInvalidValue;
        }
    }
}

template <int NST, int NWT>
cudaError_t rect_launch_nw(const RectArgs &a, cudaStream_t s) {
    switch (a.vmode) {
    case RV_NONE: return rect_launch_h<NST, NWT, RV_NONE>(a, s);
    case RV_W3: return rect_launch_h<NST, NWT, RV_W3>(a, s);
    case RV_CNT: return rect_launch_h<NST, NWT, RV_CNT>(a, s);
    default: return rect_launch_h<NST, NWT, RV_VHGW>(a, s);
    }
}

}  // namespace morph
