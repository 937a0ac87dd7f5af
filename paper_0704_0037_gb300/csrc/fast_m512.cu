// Register-resident complex64 product passes for M = 512 = 16 x 32 (the
// 256^3 sphere's padded grid).  Complex128 and double-float products on this
// length use the shared-memory Stockham passes.
#include "fast_impl.cuh"

namespace dda {
cudaError_t fast_pass_512_c64(int pass, const FastArgs& a) {
  return fast::run_pass<float, 16, 32>(pass, a);
}
}  // namespace dda
