// Hopping-term kernels with __half storage and 12-real links, in their own
// translation unit so the precision/link-format variants compile in parallel.
#include "dslash.cuh"

namespace wd {
cudaError_t launch_dslash_f16_r12(const DslashLaunch &L, cudaStream_t s) {
    return launch_dslash_t<__half, float, 12>(L, s);
}
}  // namespace wd
