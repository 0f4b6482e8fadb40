// Batched hopping term, FP32 storage, 12-real links: every launch configuration the
// batch autotuner chooses from (own translation unit for a parallel build).
#include "batch_internal.cuh"

namespace wd {
cudaError_t bt_launch_hop_f32_r12(int dagger, int variant, int cfg, const BtArgs &a, cudaStream_t s,
                   unsigned *grid_out) {
    return bt_launch_lo<float, float, 12>(dagger, variant, cfg, a, s, grid_out);
}
}  // namespace wd
