// tile_fp64.cu -- instantiation of the tile-form stage kernel for the FP64 path.
#include <algorithm>

#include "tile_launch.cuh"

namespace dg {
DG_DEFINE_TILE_LAUNCHERS(Fp64)
}  // namespace dg
