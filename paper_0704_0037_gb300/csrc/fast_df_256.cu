// Register-resident double-float product passes for M = 256 = 16 x 16.
#include "fast_impl.cuh"

namespace dda {
cudaError_t fast_pass_256_df(int pass, const FastArgs& a) {
  return fast::run_pass<df, 16, 16>(pass, a);
}
}  // namespace dda
