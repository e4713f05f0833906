// tile_launch.cuh -- launchers of the tile-form stage kernel, instantiated per precision policy
// by tile_mixed.cu and tile_fp64.cu (their own translation units, compiled in parallel).
#pragma once
#include "tile.cuh"

namespace dg {
// dynamic shared memory a kernel may request: what its largest block needs, at most the
// per-block opt-in limit less the kernel's static shared memory
template <class K>
static cudaError_t tile_smem_limit(K kernel, int optin, int need) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  const int room = optin - (int)fa.sharedSizeBytes;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, need < room ? need : room);
}
// the specialised instantiations exist for the mixed path only
template <class Pol>
inline cudaError_t tile_try_spec(int, int, int, const StageArgs<Pol>&, int, int, cudaStream_t) {
  return cudaErrorNotSupported;
}
template <>
inline cudaError_t tile_try_spec<Mixed>(int p, int flux, int feat, const StageArgs<Mixed>& a, int grid, int block,
                                        cudaStream_t s) {
  return launch_tile_spec(p, flux, feat, a, grid, block, s);
}
template <class Pol>
inline int tile_try_spec_occ(int, int, int, int) { return -1; }
template <>
inline int tile_try_spec_occ<Mixed>(int p, int flux, int feat, int block) {
  return tile_spec_blocks_per_sm(p, flux, feat, block);
}
}  // namespace dg

#define DG_DEFINE_TILE_LAUNCHERS(POL)                                                                        \
  template <>                                                                                                \
  cudaError_t upload_tile_tables<POL>(int p, const RefTab<float>& tf, const RefTab<double>& td) {            \
    cudaError_t e = cudaMemcpyToSymbol(c_tab_f, &tf, sizeof(RefTab<float>), p * sizeof(RefTab<float>));     \
    if (e != cudaSuccess) return e;                                                                          \
    e = cudaMemcpyToSymbol(c_tab_d, &td, sizeof(RefTab<double>), p * sizeof(RefTab<double>));                \
    if (e != cudaSuccess) return e;                                                                          \
    int dev = 0, optin = 0;                                                                                  \
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;                                                  \
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)   \
      return e;                                                                                              \
    if ((e = tile_smem_limit(tile_kernel<1, 0, POL>, optin, tile_smem_bytes<1, POL>(256))) != cudaSuccess)   \
      return e;                                                                                              \
    if ((e = tile_smem_limit(tile_kernel<1, 1, POL>, optin, tile_smem_bytes<1, POL>(256))) != cudaSuccess)   \
      return e;                                                                                              \
    if ((e = tile_smem_limit(tile_kernel<2, 0, POL>, optin, tile_smem_bytes<2, POL>(256))) != cudaSuccess)   \
      return e;                                                                                              \
    return tile_smem_limit(tile_kernel<2, 1, POL>, optin, tile_smem_bytes<2, POL>(256));                     \
  }                                                                                                          \
  template <>                                                                                                \
  cudaError_t launch_tile<POL>(int p, int flux, int feat, const StageArgs<POL>& a, int grid, int block,      \
                               cudaStream_t s) {                                                            \
    const cudaError_t es = tile_try_spec<POL>(p, flux, feat, a, grid, block, s);                             \
    if (es != cudaErrorNotSupported) return es;                                                              \
    const int k = (p == 1 ? 0 : 2) + (flux ? 1 : 0);                                                         \
    switch (k) {                                                                                             \
      case 0: tile_kernel<1, 0, POL><<<grid, block, tile_smem_bytes<1, POL>(block), s>>>(a); break;          \
      case 1: tile_kernel<1, 1, POL><<<grid, block, tile_smem_bytes<1, POL>(block), s>>>(a); break;          \
      case 2: tile_kernel<2, 0, POL><<<grid, block, tile_smem_bytes<2, POL>(block), s>>>(a); break;          \
      default: tile_kernel<2, 1, POL><<<grid, block, tile_smem_bytes<2, POL>(block), s>>>(a); break;         \
    }                                                                                                        \
    return cudaGetLastError();                                                                               \
  }                                                                                                          \
  template <>                                                                                                \
  int tile_blocks_per_sm<POL>(int p, int flux, int feat, int block) {                                        \
    const int ns = tile_try_spec_occ<POL>(p, flux, feat, block);                                             \
    if (ns >= 0) return ns;                                                                                  \
    int n = 0;                                                                                               \
    cudaError_t e = cudaSuccess;                                                                             \
    const int k = (p == 1 ? 0 : 2) + (flux ? 1 : 0);                                                         \
    switch (k) {                                                                                             \
      case 0: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, tile_kernel<1, 0, POL>, block, tile_smem_bytes<1, POL>(block)); break; \
      case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, tile_kernel<1, 1, POL>, block, tile_smem_bytes<1, POL>(block)); break; \
      case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, tile_kernel<2, 0, POL>, block, tile_smem_bytes<2, POL>(block)); break; \
      default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, tile_kernel<2, 1, POL>, block, tile_smem_bytes<2, POL>(block)); break; \
    }                                                                                                        \
    if (e != cudaSuccess) {                                                                                  \
      cudaGetLastError();                                                                                    \
      return 0;                                                                                              \
    }                                                                                                        \
    return n;                                                                                                \
  }
