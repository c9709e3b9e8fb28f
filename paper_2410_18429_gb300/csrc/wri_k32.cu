// z-march kernels with complex64 stencils (FP32 arithmetic, FP64 reductions).
#include "wri_launch.h"
#include "wri_march_impl.cuh"

namespace wri {
#define WRI_R float
#define WRI_OR float
#define WRI_LAUNCH_NAME launch_march_f32
#define WRI_OCC_NAME occ_f32
#include "wri_dispatch.inc"
}  // namespace wri
