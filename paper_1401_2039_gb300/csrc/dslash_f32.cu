// Hopping-term kernels with float storage (instantiated in their own
// translation unit so the four precisions compile in parallel).
#include "dslash.cuh"

namespace wd {
cudaError_t launch_dslash_f32(const DslashLaunch &L, cudaStream_t s) {
    return launch_dslash_prec<float, float>(L, s);
}
}  // namespace wd
