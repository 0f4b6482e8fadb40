// Hopping-term kernels with __nv_bfloat16 storage (instantiated in their own
// translation unit so the four precisions compile in parallel).
#include "dslash.cuh"

namespace wd {
cudaError_t launch_dslash_bf16(const DslashLaunch &L, cudaStream_t s) {
    return launch_dslash_prec<__nv_bfloat16, float>(L, s);
}
}  // namespace wd
