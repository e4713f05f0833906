// tile_mixed.cu -- instantiation of the tile-form stage kernel for the mixed-precision path.
#include <algorithm>

#include "tile_launch.cuh"

namespace dg {
DG_DEFINE_TILE_LAUNCHERS(Mixed)
}  // namespace dg
