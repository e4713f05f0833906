// tile_spec.cu -- specialised instantiations of the mixed-precision tile kernel.
//
// Each instantiation compiles in only the features of its set (Feature bits): the code of
// absent boundary kinds, forcing kinds, friction laws and stage-weight kinds, and their run-time
// tests, are left out, which shortens the kernel's instruction stream and its code.  A run
// whose features a set covers is launched with the narrowest such instantiation; any other run
// uses the generic one (tile_mixed.cu).
#include <algorithm>

#include "tile_launch.cuh"

namespace dg {
namespace {

// tidal boundary, parametric storm rain, Manning friction, SSP(2,2)
constexpr int FT_TIDE_STORM = FT_OCEAN | FT_RAIN2 | FT_MANNING | FT_POW2;
// tidal boundary, gridded rain, Manning friction, SSP(2,2)
constexpr int FT_TIDE_GRID = FT_OCEAN | FT_RAIN3 | FT_MANNING | FT_POW2;
// walls only, constant nodal rain, Manning friction, SSP(2,2)
constexpr int FT_WALL_NODAL = FT_RAIN1 | FT_MANNING | FT_POW2;
// tidal boundary, parametric storm rain, pressure set-up, Manning friction, SSP(3,3) (p = 2)
constexpr int FT_TIDE_STORM_SETUP = FT_OCEAN | FT_RAIN2 | FT_PRESS | FT_MANNING | FT_POW2 | FT_GENSSP;

using Kernel = void (*)(const StageArgs<Mixed>);
struct Spec {
  int p, flux, ft;
  Kernel k;
};
const Spec kSpecs[] = {
    {1, 0, FT_WALL_NODAL, tile_kernel<1, 0, Mixed, FT_WALL_NODAL>},
    {1, 0, FT_TIDE_STORM, tile_kernel<1, 0, Mixed, FT_TIDE_STORM>},
    {1, 0, FT_TIDE_GRID, tile_kernel<1, 0, Mixed, FT_TIDE_GRID>},
    {2, 0, FT_TIDE_STORM_SETUP, tile_kernel<2, 0, Mixed, FT_TIDE_STORM_SETUP>},
};

int bits(int x) {
  int n = 0;
  for (; x; x &= x - 1) ++n;
  return n;
}
// the narrowest instantiation that covers feat, or null
const Spec* find_spec(int p, int flux, int feat) {
  const Spec* best = nullptr;
  for (const Spec& sp : kSpecs)
    if (sp.p == p && sp.flux == flux && ft_covers(sp.ft, feat) && (!best || bits(sp.ft) < bits(best->ft)))
      best = &sp;
  return best;
}
int smem_bytes(int p, int block) { return p == 1 ? tile_smem_bytes<1, Mixed>(block) : tile_smem_bytes<2, Mixed>(block); }

}  // namespace

cudaError_t launch_tile_spec(int p, int flux, int feat, const StageArgs<Mixed>& a, int grid, int block,
                             cudaStream_t s) {
  const Spec* sp = find_spec(p, flux, feat);
  if (!sp) return cudaErrorNotSupported;
  sp->k<<<grid, block, smem_bytes(p, block), s>>>(a);
  return cudaGetLastError();
}

int tile_spec_features(int p, int flux, int feat) {
  const Spec* sp = find_spec(p, flux, feat);
  return sp ? sp->ft : -1;
}

int tile_spec_blocks_per_sm(int p, int flux, int feat, int block) {
  const Spec* sp = find_spec(p, flux, feat);
  if (!sp) return -1;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sp->k, block, smem_bytes(p, block)) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

cudaError_t upload_tile_spec_tables(int p, const RefTab<float>& tf, const RefTab<double>& td) {
  cudaError_t e = cudaMemcpyToSymbol(c_tab_f, &tf, sizeof(RefTab<float>), p * sizeof(RefTab<float>));
  if (e != cudaSuccess) return e;
  e = cudaMemcpyToSymbol(c_tab_d, &td, sizeof(RefTab<double>), p * sizeof(RefTab<double>));
  if (e != cudaSuccess) return e;
  int dev = 0, optin = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
  for (const Spec& sp : kSpecs)
    if ((e = tile_smem_limit(sp.k, optin, smem_bytes(sp.p, 256))) != cudaSuccess) return e;
  return cudaSuccess;
}

}  // namespace dg
