// Hopping-term kernels with double storage and 18-real links, in their own
// translation unit so the precision/link-format variants compile in parallel.
#include "dslash.cuh"

namespace wd {
cudaError_t launch_dslash_f64_r18(const DslashLaunch &L, cudaStream_t s) {
    return launch_dslash_t<double, double, 18>(L, s);
}
}  // namespace wd
