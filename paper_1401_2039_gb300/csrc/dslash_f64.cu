// Hopping-term kernels with double storage (instantiated in their own
// translation unit so the four precisions compile in parallel).
#include "dslash.cuh"

namespace wd {
cudaError_t launch_dslash_f64(const DslashLaunch &L, cudaStream_t s) {
    return launch_dslash_prec<double, double>(L, s);
}
}  // namespace wd
