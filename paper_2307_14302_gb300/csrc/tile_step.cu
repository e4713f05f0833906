// tile_step.cu -- instantiations of the fused step (every Runge-Kutta stage of one step in one
// launch of the tile form) for the mixed-precision path.
//
// The fused step serves runs without gridded rain (whose node kernel runs between stages) and
// without the slope limiter (a separate launch after each stage).  Like the stage kernel it has
// the generic instantiation and specialised ones for the feature sets of the benchmark families
// that qualify; a run takes the narrowest instantiation that covers its features.  It is
// launched cooperatively, so that every CTA of the grid is resident at once: the per-tile waits
// between stages rely on it.
#include <algorithm>

#include "tile_launch.cuh"

namespace dg {
namespace {

constexpr int FT_TIDE_STORM = FT_OCEAN | FT_RAIN2 | FT_MANNING | FT_POW2;
constexpr int FT_WALL_NODAL = FT_RAIN1 | FT_MANNING | FT_POW2;
constexpr int FT_TIDE_STORM_SETUP = FT_OCEAN | FT_RAIN2 | FT_PRESS | FT_MANNING | FT_POW2 | FT_GENSSP;

using Kernel = void (*)(const StepArgs<Mixed>);
struct Spec {
  int p, flux, ft;
  Kernel k;
};
const Spec kSpecs[] = {
    {1, 0, FT_WALL_NODAL, tile_step_kernel<1, 0, Mixed, FT_WALL_NODAL>},
    {1, 0, FT_TIDE_STORM, tile_step_kernel<1, 0, Mixed, FT_TIDE_STORM>},
    {2, 0, FT_TIDE_STORM_SETUP, tile_step_kernel<2, 0, Mixed, FT_TIDE_STORM_SETUP>},
    {1, 0, FT_ALL, tile_step_kernel<1, 0, Mixed>},
    {1, 1, FT_ALL, tile_step_kernel<1, 1, Mixed>},
    {2, 0, FT_ALL, tile_step_kernel<2, 0, Mixed>},
    {2, 1, FT_ALL, tile_step_kernel<2, 1, Mixed>},
};

int bits(int x) {
  int n = 0;
  for (; x; x &= x - 1) ++n;
  return n;
}
// the narrowest instantiation that covers feat (the generic ones cover every run)
const Spec* find_spec(int p, int flux, int feat) {
  const Spec* best = nullptr;
  for (const Spec& sp : kSpecs)
    if (sp.p == p && sp.flux == flux && ft_covers(sp.ft, feat) && (!best || bits(sp.ft) < bits(best->ft)))
      best = &sp;
  return best;
}
int smem_bytes(int p, int block) { return p == 1 ? tile_smem_bytes<1, Mixed>(block) : tile_smem_bytes<2, Mixed>(block); }

}  // namespace

cudaError_t launch_tile_step(int p, int flux, int feat, const StepArgs<Mixed>& a, int grid, int block, cudaStream_t s) {
  const Spec* sp = find_spec(p, flux, feat);
  if (!sp) return cudaErrorNotSupported;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = (size_t)smem_bytes(p, block);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, sp->k, a);
}

int tile_step_blocks_per_sm(int p, int flux, int feat, int block) {
  const Spec* sp = find_spec(p, flux, feat);
  if (!sp) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sp->k, block, smem_bytes(p, block)) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

cudaError_t upload_tile_step_tables(int p, const RefTab<float>& tf, const RefTab<double>& td) {
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
