// Dispatch of one product pass to the Passes<R, M1, M2> launchers.
#pragma once

#include "fastfft.cuh"

namespace dda {
namespace fast {

template <typename R, int M1, int M2>
cudaError_t run_pass(int pass, const FastArgs& a) {
  using P = Passes<R, M1, M2>;
  const cpx<R>* tw = (const cpx<R>*)a.tw;
  switch (pass) {
    case FP_XFWD:
      return P::xfwd((const typename P::V*)a.in, (cpx<R>*)a.out, a.lat, (const cpx<R>*)a.beta, a.n_occ,
                     a.nrows, tw, a.adj, a.nrhs, a.bstride, a.skip, a.st, a.pdl);
    case FP_YFWD:
      return P::yfwd((const cpx<R>*)a.in, (cpx<R>*)a.out, a.ny, a.nz, a.Mx, tw, a.nrhs, a.skip, a.st,
                     a.var_yf, a.pdl, a.lat.yr);
    case FP_ZCONV:
      return P::zconv((cpx<R>*)a.out, (const cpx<R>*)a.D, a.nz, a.Mx, a.My, tw, a.nrhs, a.skip,
                      a.st, a.var_z, a.pdl);
    case FP_YINV:
      return P::yinv((const cpx<R>*)a.in, (cpx<R>*)a.out, a.ny, a.nz, a.Mx, tw, a.nrhs, a.skip, a.st,
                     a.var_yi, a.pdl);
    case FP_XINV:
      return P::xinv((const cpx<R>*)a.in, (const typename P::V*)a.x, (typename P::V*)a.out, a.lat,
                     (const cpx<R>*)a.beta, a.n_occ, a.nrows, tw, a.adj, a.dotp, a.nrhs, a.bstride,
                     a.skip, a.st, a.pdl);
    case FP_XFULL:
      return P::xfull((const cpx<R>*)a.in, (cpx<R>*)a.out, a.nrows, a.ny, a.My, tw, a.st);
    case FP_SFULL:
      return P::sfull((const cpx<R>*)a.in, (cpx<R>*)a.out, a.nrows, a.nz, a.Mx, a.msign, tw, a.st,
                      a.ostride);
  }
  return cudaErrorNotSupported;
}

}  // namespace fast
}  // namespace dda
