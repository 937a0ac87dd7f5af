// Register-resident product passes for the padded lengths 40 = 5 x 8,
// 48 = 6 x 8, 80 = 8 x 10 and 96 = 8 x 12 (complex64 and complex128): with
// 32, 64 and 128 they give every lattice of up to 64 cells per axis a
// compiled length within 1.32 times its smallest 7-smooth padded length.
#include "fast_impl.cuh"

namespace dda {
template <typename R> cudaError_t fast_pass_mid(int M, int pass, const FastArgs& a) {
  switch (M) {
    case 40: return fast::run_pass<R, 5, 8>(pass, a);
    case 48: return fast::run_pass<R, 6, 8>(pass, a);
    case 80: return fast::run_pass<R, 8, 10>(pass, a);
    case 96: return fast::run_pass<R, 8, 12>(pass, a);
  }
  return cudaErrorNotSupported;
}
template cudaError_t fast_pass_mid<float>(int, int, const FastArgs&);
template cudaError_t fast_pass_mid<double>(int, int, const FastArgs&);
}  // namespace dda
