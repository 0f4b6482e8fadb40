// Hopping-term kernels with __half storage (instantiated in their own
// translation unit so the four precisions compile in parallel).
#include "dslash.cuh"

namespace wd {
cudaError_t launch_dslash_f16(const DslashLaunch &L, cudaStream_t s) {
    return launch_dslash_prec<__half, float>(L, s);
}
}  // namespace wd
