// stage_fp64.cu -- instantiation of the stage and auxiliary kernels for the FP64 path (every
// operation in double precision).
#include "stage.cuh"

namespace dg {
DG_DEFINE_LAUNCHERS(Fp64)
}  // namespace dg
