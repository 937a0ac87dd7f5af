// Register-resident double-float product passes for M = 270 = 15 x 18.
#include "fast_impl.cuh"

namespace dda {
cudaError_t fast_pass_270_df(int pass, const FastArgs& a) {
  return fast::run_pass<df, 15, 18>(pass, a);
}
}  // namespace dda
