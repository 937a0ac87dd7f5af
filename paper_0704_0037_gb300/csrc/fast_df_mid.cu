// Register-resident double-float product passes for M = 40, 48, 80, 96.
#include "fast_impl.cuh"

namespace dda {
cudaError_t fast_pass_mid_df(int M, int pass, const FastArgs& a) {
  switch (M) {
    case 40: return fast::run_pass<df, 5, 8>(pass, a);
    case 48: return fast::run_pass<df, 6, 8>(pass, a);
    case 80: return fast::run_pass<df, 8, 10>(pass, a);
    case 96: return fast::run_pass<df, 8, 12>(pass, a);
  }
  return cudaErrorNotSupported;
}
}  // namespace dda
