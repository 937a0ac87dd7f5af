// Register-resident double-float product passes for M = 32, 64, 128.
#include "fast_impl.cuh"

namespace dda {
cudaError_t fast_pass_small_df(int M, int pass, const FastArgs& a) {
  switch (M) {
    case 32: return fast::run_pass<df, 4, 8>(pass, a);
    case 64: return fast::run_pass<df, 8, 8>(pass, a);
    case 128: return fast::run_pass<df, 8, 16>(pass, a);
  }
  return cudaErrorNotSupported;
}
}  // namespace dda
