// Hopping-term kernels in double-float arithmetic with double-float storage
// and 18-real links (the residuals of the reliable updates).
#include "dslash.cuh"

namespace wd {
cudaError_t launch_dslash_df64_r18(const DslashLaunch &L, cudaStream_t s) {
    return launch_dslash_t<df64, df64, 18>(L, s);
}
}  // namespace wd
