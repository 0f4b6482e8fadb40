// Batched hopping term in FP64 storage and in the double-float residual
// arithmetic (one configuration each; own translation unit for a parallel
// build).
#include "batch_internal.cuh"

namespace wd {
cudaError_t bt_launch_hop_f64_r18(int dagger, int variant, int, const BtArgs &a, cudaStream_t s,
                                  unsigned *grid_out) {
    return bt_launch_fixed<double, double, 18, 2>(dagger, variant, a, s, grid_out);
}
cudaError_t bt_launch_hop_f64_r12(int dagger, int variant, int, const BtArgs &a, cudaStream_t s,
                                  unsigned *grid_out) {
    return bt_launch_fixed<double, double, 12, 2>(dagger, variant, a, s, grid_out);
}
cudaError_t bt_launch_hop_df64_r18(int dagger, int variant, int, const BtArgs &a, cudaStream_t s,
                                   unsigned *grid_out) {
    return bt_launch_fixed<df64, df64, 18, 3>(dagger, variant, a, s, grid_out);
}
}  // namespace wd
