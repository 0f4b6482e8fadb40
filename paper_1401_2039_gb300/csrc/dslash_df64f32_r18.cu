// Hopping-term kernels that read double-float fields and 18-real links in
// FP32 arithmetic (each double-float rounded to one float on load, the
// output stored with a zero trailing part): the residual refreshes of a
// mixed-precision solve while the residual is still large, whose rounding
// the later double-float refreshes correct.
#include "dslash.cuh"

namespace wd {
cudaError_t launch_dslash_df64f32_r18(const DslashLaunch &L, cudaStream_t s) {
    return launch_dslash_t<df64, float, 18>(L, s);
}
}  // namespace wd
