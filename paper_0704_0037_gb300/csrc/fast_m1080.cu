// Register-resident complex64 product passes for M = 1080 = 30 x 36 (the
// 536^3 sphere's padded grid).  Complex128 and double-float products on this
// length use the shared-memory Stockham passes.
#include "fast_impl.cuh"

namespace dda {
cudaError_t fast_pass_1080_c64(int pass, const FastArgs& a) {
  return fast::run_pass<float, 30, 36>(pass, a);
}
}  // namespace dda
