// Register-resident product passes for M = 256 = 16 x 16 (the 128^3 sphere).
#include "fast_impl.cuh"

namespace dda {
template <typename R> cudaError_t fast_pass_256(int pass, const FastArgs& a) {
  return fast::run_pass<R, 16, 16>(pass, a);
}
template cudaError_t fast_pass_256<float>(int, const FastArgs&);
template cudaError_t fast_pass_256<double>(int, const FastArgs&);
}  // namespace dda
