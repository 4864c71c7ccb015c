// Kernel and launch dispatch of the run-length-source tile (rle_rect.cuh);
// rle_rect_w2.cu / rle_rect_w4.cu instantiate the 2- and 4-word families.
#pragma once

#include <mutex>

#include "rect_kernels.cuh"
#include "rle_rect.cuh"

namespace morph {

// One image (jobs == nullptr), or a table of images of the same variant
// (CTA b belongs to image j with starts[j] <= b < starts[j + 1]).
template <int NST, int NWT, int VM, int HM, int HALO>
__global__ void __launch_bounds__(256, 2) k_rle_rect(const RectArgs a, const RleSrc src, const RleJob *jobs,
                                                     const int *starts, int njobs, const uint8_t *base) {
    extern __shared__ __align__(16) uint32_t sm[];
    if (jobs == nullptr) {
        rle_rect_tile<NST, NWT, VM, HM, HALO>(a, src, blockIdx.x, sm);
        return;
    }
    __shared__ RectArgs sj;
    __shared__ RleSrc ss;
    __shared__ int sbx;
    if (threadIdx.x == 0) {
        const int j = rect_job_of(starts, njobs, blockIdx.x);
        sj = jobs[j].a;
        ss = RleSrc{reinterpret_cast<const int32_t *>(base + jobs[j].off_row_ptr),
                    reinterpret_cast<const uint32_t *>(base + jobs[j].off_runs), jobs[j].op1, jobs[j].cap};
        sbx = blockIdx.x - starts[j];
    }
    __syncthreads();
    // the job's plan in registers (see k_rect)
    const RectArgs la = sj;
    const RleSrc ls = ss;
    rle_rect_tile<NST, NWT, VM, HM, HALO>(la, ls, sbx, sm);
}

template <int NST, int NWT, int VM, int HM, int HALO>
cudaError_t rle_rect_launch_t(const RectArgs &a0, const RleSrc &src, cudaStream_t s, const RleJobs *mj) {
    if (mj) {
        auto kern = k_rle_rect<NST, NWT, VM, HM, HALO>;
        cudaError_t e = raise_smem_limit(kern, mj->smem);
        if (e != cudaSuccess) return e;
        kern<<<mj->ctas, a0.threads, mj->smem, s>>>(a0, src, mj->jobs, mj->starts, mj->njobs, mj->base);
        return cudaGetLastError();
    }
    RectArgs a = a0;
    if (a.band_auto) a.groups = a.threads / a.tpr;
    const size_t smem = rle_rect_smem_words(a) * sizeof(uint32_t);
    auto kern = k_rle_rect<NST, NWT, VM, HM, HALO>;
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
    kern<<<rect_grid(a).x, a.threads, smem, s>>>(a, src, nullptr, nullptr, 0, nullptr);
    return cudaGetLastError();
}

template <int NWT, int VM>
cudaError_t rle_rect_launch_h2(const RectArgs &a, const RleSrc &src, cudaStream_t s, const RleJobs *mj) {
    switch (a.hmode) {
    case RH_NONE: return rle_rect_launch_t<2, NWT, VM, RH_NONE, 1>(a, src, s, mj);
    case RH_D1: return rle_rect_launch_t<2, NWT, VM, RH_D1, 1>(a, src, s, mj);
    case RH_D2: return rle_rect_launch_t<2, NWT, VM, RH_D2, 1>(a, src, s, mj);
    default:
        switch (a.halo) {
        case 1: return rle_rect_launch_t<2, NWT, VM, RH_LOG, 1>(a, src, s, mj);
        case 2: return rle_rect_launch_t<2, NWT, VM, RH_LOG, 2>(a, src, s, mj);
        case 4: return rle_rect_launch_t<2, NWT, VM, RH_LOG, 4>(a, src, s, mj);
        default: return cudaErrorInvalidValue;
        }
    }
}

template <int NWT>
cudaError_t rle_rect_launch_nw(const RectArgs &a, const RleSrc &src, cudaStream_t s, const RleJobs *mj) {
    if (a.nst == 1) {
        if (a.hmode != RH_NONE) return cudaErrorInvalidValue;
        switch (a.vmode) {
        case RV_NONE: return rle_rect_launch_t<1, NWT, RV_NONE, RH_NONE, 1>(a, src, s, mj);
        case RV_W3: return rle_rect_launch_t<1, NWT, RV_W3, RH_NONE, 1>(a, src, s, mj);
        case RV_VHGW: return rle_rect_launch_t<1, NWT, RV_VHGW, RH_NONE, 1>(a, src, s, mj);
        default: return cudaErrorInvalidValue;
        }
    }
    switch (a.vmode) {
    case RV_NONE: return rle_rect_launch_h2<NWT, RV_NONE>(a, src, s, mj);  // sh == 1
    case RV_W3: return rle_rect_launch_h2<NWT, RV_W3>(a, src, s, mj);
    case RV_VHGW: return rle_rect_launch_h2<NWT, RV_VHGW>(a, src, s, mj);
    case RV_CNT:
        if constexpr (NWT == 2) return rle_rect_launch_h2<NWT, RV_CNT>(a, src, s, mj);
        return cudaErrorInvalidValue;
    case RV_CNT4:
        if constexpr (NWT == 2) return rle_rect_launch_h2<NWT, RV_CNT4>(a, src, s, mj);
        return cudaErrorInvalidValue;
    case RV_CNT5:
        if constexpr (NWT == 2) return rle_rect_launch_h2<NWT, RV_CNT5>(a, src, s, mj);
        return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace morph
