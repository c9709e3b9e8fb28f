// z-march kernels with complex128 stencils, and the FP64 -> FP32 normal-equation
// residual of the iterative refinement.
#include "wri_launch.h"
#include "wri_march_impl.cuh"

namespace wri {
#define WRI_R double
#define WRI_OR double
#define WRI_LAUNCH_NAME launch_march_f64
#define WRI_OCC_NAME occ_f64
#include "wri_dispatch.inc"
#undef WRI_R
#undef WRI_OR

template <int BY>
static int occ_df() {
  static int v = -1;
  if (v < 0) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_march<double, float, M_SH, true, BY>, WRI_TX * BY, 0) !=
        cudaSuccess)
      n = 1;
    v = n > 0 ? n : 1;
  }
  return v;
}

int occ_f64_to_f32(int by) {
  switch (by) {
    case 4: return occ_df<4>();
    case 8: return occ_df<8>();
    case 16: return occ_df<16>();
  }
  return 0;
}

cudaError_t launch_march_f64_to_f32(int mode, int by, const Batch& b, int grid, cudaStream_t st) {
  if (mode != M_SH) return cudaErrorInvalidValue;
  if (grid <= 0) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long g = (long long)sms * occ_f64_to_f32(by);
    grid = (int)(g < b.nitems ? g : b.nitems);
    if (grid < 1) grid = 1;
  }
  switch (by) {
    case 4: k_march<double, float, M_SH, true, 4><<<grid, dim3(WRI_TX, 4), 0, st>>>(b); break;
    case 8: k_march<double, float, M_SH, true, 8><<<grid, dim3(WRI_TX, 8), 0, st>>>(b); break;
    case 16: k_march<double, float, M_SH, true, 16><<<grid, dim3(WRI_TX, 16), 0, st>>>(b); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
}  // namespace wri
