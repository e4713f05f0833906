// exchange.cu -- the state exchange of a coupling loop: the current state out to the caller's
// arrays and a new state in, in one pass over the element records, so that with page-locked host
// arrays both directions of the host link carry data at the same time.
#include "exchange.h"
#include "stage.cuh"

namespace dg {

// Thread c takes caller element c (coalesced in the caller's arrays): it reads the element's
// record, writes its modal coefficients out exactly as the unpacking kernel of dgswe_get_state
// does (mode 0 of each variable is sqrt(2) times the element mean), then sets the coefficients
// from the in arrays exactly as the packing kernel of dgswe_load_state does (bathymetry modes kept;
// depth and wet/dry flag are derived by the positive-depth pass that follows) and stores the
// record.  Each record is read and written by one thread only (inv is a permutation).
template <int P, class Pol>
__global__ void __launch_bounds__(256) exchange_kernel(uint4* rec, long long begin, long long n, const int32_t* inv,
                                                       const double* zi, const double* xi, const double* yi,
                                                       double* zo, double* xo, double* yo) {
  constexpr int RV = Pol::template RV<P>, NS = np_of(P) - 1;
  using T = typename Pol::T;
  const double s2 = 1.4142135623730951, is2 = 0.7071067811865476;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    const long long e = begin + inv[c];
    Raw<RV> r;
    load_raw<RV>(rec, e, r);
    Elem<P, Pol> E;
    unpack<P>(r, E);
    // the new state's coefficients, requested before the old ones are written out
    const double z0 = zi[c], x0 = xi[c], y0 = yi[c];
    double zn[NS > 0 ? NS : 1], xn[NS > 0 ? NS : 1], yn[NS > 0 ? NS : 1];
#pragma unroll
    for (int m = 0; m < NS; ++m) {
      zn[m] = zi[(m + 1) * n + c];
      xn[m] = xi[(m + 1) * n + c];
      yn[m] = yi[(m + 1) * n + c];
    }
    zo[c] = s2 * acc_d(E.zb);
    xo[c] = s2 * acc_d(E.xb);
    yo[c] = s2 * acc_d(E.yb);
#pragma unroll
    for (int m = 0; m < NS; ++m) {
      zo[(m + 1) * n + c] = (double)E.zs[m];
      xo[(m + 1) * n + c] = (double)E.xs[m];
      yo[(m + 1) * n + c] = (double)E.ys[m];
    }
    acc_set(E.zb, is2 * z0);
    acc_set(E.xb, is2 * x0);
    acc_set(E.yb, is2 * y0);
#pragma unroll
    for (int m = 0; m < NS; ++m) {
      E.zs[m] = (T)zn[m];
      E.xs[m] = (T)xn[m];
      E.ys[m] = (T)yn[m];
    }
    pack<P>(E, r);
    store_raw<RV>(rec, e, r);
  }
}

template <class Pol>
cudaError_t launch_exchange(int p, uint4* rec, long long begin, long long n, const int32_t* inv, const double* zi,
                            const double* xi, const double* yi, double* zo, double* xo, double* yo, cudaStream_t s) {
  const long long g0 = (n + 255) / 256;
  const int g = (int)(g0 < 1 ? 1 : (g0 > 65535 * 8 ? 65535 * 8 : g0));
  if (p == 1) exchange_kernel<1, Pol><<<g, 256, 0, s>>>(rec, begin, n, inv, zi, xi, yi, zo, xo, yo);
  else exchange_kernel<2, Pol><<<g, 256, 0, s>>>(rec, begin, n, inv, zi, xi, yi, zo, xo, yo);
  return cudaGetLastError();
}

template cudaError_t launch_exchange<Mixed>(int, uint4*, long long, long long, const int32_t*, const double*,
                                            const double*, const double*, double*, double*, double*, cudaStream_t);
template cudaError_t launch_exchange<Fp64>(int, uint4*, long long, long long, const int32_t*, const double*,
                                           const double*, const double*, double*, double*, double*, cudaStream_t);

}  // namespace dg
