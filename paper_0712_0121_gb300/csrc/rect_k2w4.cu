// Packed rectangle tile variants with 2 stage(s) and 4 words per thread.
#include "rect_kernels.cuh"

namespace morph {
cudaError_t launch_rect_2_4(const RectArgs &a, cudaStream_t s, const RectJobs *mj) {
    return rect_launch_nw<2, 4>(a, s, mj);
}
}  // namespace morph
