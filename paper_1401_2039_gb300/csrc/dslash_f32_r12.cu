// Hopping-term kernels with float storage and 12-real links, in their own
// translation unit so the precision/link-format variants compile in parallel.
#include "dslash.cuh"

namespace wd {
cudaError_t launch_dslash_f32_r12(const DslashLaunch &L, cudaStream_t s) {
    return launch_dslash_t<float, float, 12>(L, s);
}
}  // namespace wd
