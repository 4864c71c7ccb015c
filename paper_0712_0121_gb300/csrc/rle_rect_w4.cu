// Run-length-source tile variants with 4 words per thread.
#include "rle_rect_kernels.cuh"

namespace morph {
cudaError_t launch_rle_rect_w4(const RectArgs &a, const RleSrc &src, cudaStream_t s, const RleJobs *mj) {
    return rle_rect_launch_nw<4>(a, src, s, mj);
}
}  // namespace morph
