// Packed rectangle tile variants with 1 stage(s) and 2 words per thread.
#include "rect_kernels.cuh"

namespace morph {
cudaError_t launch_rect_1_2(const RectArgs &a, cudaStream_t s, const RectJobs *mj) {
    return rect_launch_nw<1, 2>(a, s, mj);
}
}  // namespace morph
