// Kernel and launch dispatch of the packed rectangle tile (rect_tile.cuh);
// each rect_k*.cu instantiates one (stages, words per thread) family so that
// the variants compile in parallel.
#pragma once

#include <map>
#include <mutex>
#include <utility>

#include "rect_tile.cuh"

namespace morph {

// Raise a kernel's dynamic shared-memory limit to at least `bytes` (never
// lowers it: launches of other sizes share the attribute).  Recorded per
// kernel and device.
template <typename K>
cudaError_t raise_smem_limit(K kern, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, size_t> set_to;
    // (the default limit covers static shared memory too: raise early)
    if (bytes <= 32 * 1024) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    size_t &cur = set_to[std::make_pair((const void *)kern, dev)];
    if (bytes <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

// One image (jobs == nullptr: plan a, CTA (blockIdx.x, blockIdx.y)), or a
// table of images of the same variant: CTA b belongs to image j with
// starts[j] <= b < starts[j + 1]; its plan is copied into shared memory.
template <int NST, int NWT, int VM, int HM, int HALO>
__global__ void __launch_bounds__(256, 2) k_rect(const RectArgs a, const RectArgs *jobs, const int *starts,
                                                 int njobs) {
    extern __shared__ __align__(16) uint32_t sm[];
    if (jobs == nullptr) {
        rect_tile<NST, NWT, VM, HM, HALO>(a, blockIdx.x, blockIdx.y, sm);
        return;
    }
    __shared__ RectArgs sj;
    __shared__ int sbx, sby;
    if (threadIdx.x == 0) {
        const int j = rect_job_of(starts, njobs, blockIdx.x);
        sj = jobs[j];
        const int local = blockIdx.x - starts[j];
        const int gx = (int)rect_grid(sj).x;
        sbx = local % gx;
        sby = local / gx;
    }
    __syncthreads();
    // the job's plan in registers: read through shared memory, every field
    // would be loaded again after each of the tile's barriers
    const RectArgs la = sj;
    rect_tile<NST, NWT, VM, HM, HALO>(la, sbx, sby, sm);
}

template <int NST, int NWT, int VM, int HM, int HALO>
cudaError_t rect_launch_t(const RectArgs &a0, cudaStream_t s, const RectJobs *mj) {
    if (mj) {
        auto kern = k_rect<NST, NWT, VM, HM, HALO>;
        cudaError_t e = raise_smem_limit(kern, mj->smem);
        if (e != cudaSuccess) return e;
        kern<<<mj->ctas, a0.threads, mj->smem, s>>>(a0, mj->jobs, mj->starts, mj->njobs);
        return cudaGetLastError();
    }
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
        e = raise_smem_limit(kern, smem);
        if (e != cudaSuccess) return e;
        if (c_dev != dev || c_threads != a.threads || c_smem != smem) {
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
    kern<<<rect_grid(a), a.threads, smem, s>>>(a, nullptr, nullptr, 0);
    return cudaGetLastError();
}

template <int NST, int NWT, int VM>
cudaError_t rect_launch_h(const RectArgs &a, cudaStream_t s, const RectJobs *mj) {
    switch (a.hmode) {
    case RH_NONE: return rect_launch_t<NST, NWT, VM, RH_NONE, 1>(a, s, mj);
    case RH_D1: return rect_launch_t<NST, NWT, VM, RH_D1, 1>(a, s, mj);
    case RH_D2: return rect_launch_t<NST, NWT, VM, RH_D2, 1>(a, s, mj);
    default:
        switch (a.halo) {
        case 1: return rect_launch_t<NST, NWT, VM, RH_LOG, 1>(a, s, mj);
        case 2: return rect_launch_t<NST, NWT, VM, RH_LOG, 2>(a, s, mj);
        case 4: return rect_launch_t<NST, NWT, VM, RH_LOG, 4>(a, s, mj);
        default: return cudaErrorInvalidValue;
        }
    }
}

template <int NST, int NWT>
cudaError_t rect_launch_nw(const RectArgs &a, cudaStream_t s, const RectJobs *mj) {
    switch (a.vmode) {
    case RV_NONE: return rect_launch_h<NST, NWT, RV_NONE>(a, s, mj);
    case RV_W3: return rect_launch_h<NST, NWT, RV_W3>(a, s, mj);
    case RV_CNT: return rect_launch_h<NST, NWT, RV_CNT>(a, s, mj);
    case RV_CNT4:
        if constexpr (NST == 2 && NWT == 2) return rect_launch_h<NST, NWT, RV_CNT4>(a, s, mj);
        return cudaErrorInvalidValue;
    case RV_CNT5:
        if constexpr (NST == 2 && NWT == 2) return rect_launch_h<NST, NWT, RV_CNT5>(a, s, mj);
        return cudaErrorInvalidValue;
    default: return rect_launch_h<NST, NWT, RV_VHGW>(a, s, mj);
    }
}

}  // namespace morph
