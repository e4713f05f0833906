// stage_mixed.cu -- instantiation of the stage and auxiliary kernels for the mixed-precision
// path (FP32 bulk arithmetic, float-float element means, FP64 depth test near H0).
#include "stage.cuh"

namespace dg {
DG_DEFINE_LAUNCHERS(Mixed)
}  // namespace dg
