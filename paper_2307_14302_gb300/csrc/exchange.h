// exchange.h -- launcher of the state exchange kernel (exchange.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace dg {

// One pass over the records of elements [begin, begin + n): the modal state [Np][n] in caller
// order goes out to (zo, xo, yo) and (zi, xi, yi), same layout, comes in; inv[c] is the position
// of caller element c relative to begin.  The arrays may be device memory or device-accessible
// page-locked host memory; in and out must not overlap.
template <class Pol>
cudaError_t launch_exchange(int p, uint4* rec, long long begin, long long n, const int32_t* inv, const double* zi,
                            const double* xi, const double* yi, double* zo, double* xo, double* yo, cudaStream_t s);

}  // namespace dg
