// Register-resident product passes for M = 270 = 15 x 18 (the 134^3 sphere).
#include "fast_impl.cuh"

namespace dda {
template <typename R> cudaError_t fast_pass_270(int pass, const FastArgs& a) {
  return fast::run_pass<R, 15, 18>(pass, a);
}
template cudaError_t fast_pass_270<float>(int, const FastArgs&);
template cudaError_t fast_pass_270<double>(int, const FastArgs&);
}  // namespace dda
