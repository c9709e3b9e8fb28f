// TMA-pipelined CGLS phase kernels (complex64) and their launcher.
#include "wri_launch.h"
#include "wri_tma.cuh"

namespace wri {

template <int MODE, int BY, int S>
static cudaError_t launch_one(const Batch& b, const TmaSet& T, int grid, cudaStream_t st) {
  static int occ = -1;
  const size_t smem = TmaLayout<MODE, BY>::bytes(S);
  auto kern = k_phase_tma<MODE, BY, S, (BY <= 8 ? 3 : 1)>;
  if (occ < 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    int n = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, WRI_TX * BY, smem);
    if (e != cudaSuccess) return e;
    occ = n > 0 ? n : 1;
  }
  if (grid <= 0) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long g = (long long)sms * occ;
    grid = (int)(g < b.nitems ? g : b.nitems);
    if (grid < 1) grid = 1;
  }
  kern<<<grid, dim3(WRI_TX, BY), smem, st>>>(b, T);
  return cudaGetLastError();
}

template <int MODE, int BY, int S, int MINB>
static cudaError_t launch_two(const Batch& b, const TmaSet& T, int grid, cudaStream_t st) {
  static int occ = -1;
  const size_t smem = TmaLayout2<MODE, BY>::bytes(S);
  auto kern = k_phase_tma2<MODE, BY, S, MINB>;
  if (occ < 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    int n = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, 16 * BY, smem);
    if (e != cudaSuccess) return e;
    occ = n > 0 ? n : 1;
  }
  if (grid <= 0) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long g = (long long)sms * occ;
    grid = (int)(g < b.nitems ? g : b.nitems);
    if (grid < 1) grid = 1;
  }
  kern<<<grid, dim3(16, BY), smem, st>>>(b, T);
  return cudaGetLastError();
}

template <int MODE, int BY, int S, int MINB, bool PW = true, bool ER = false>
static cudaError_t launch_ws(const Batch& b, const TmaSet& T, int grid, cudaStream_t st) {
  static int occ[4] = {-1, -1, -1, -1};  // by the number of extra update boxes per stage
  const int xp = (MODE == M_P1) ? xsteps_of(b) - 1 : 0;
  const size_t smem = WsLayout<MODE, BY>::bytes(S, xp);
  auto kern = k_phase_ws<MODE, BY, S, MINB, PW, ER>;
  constexpr int threads = 16 * BY + (PW ? 32 : 0);
  if (occ[xp] < 0) {
    // the attribute covers the larger of the two sizes
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)WsLayout<MODE, BY>::bytes(S, 3));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    int n = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, threads, smem);
    if (e != cudaSuccess) return e;
    occ[xp] = n > 0 ? n : 1;
  }
  if (grid <= 0) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long g = (long long)sms * occ[xp];
    grid = (int)(g < b.nitems ? g : b.nitems);
    if (grid < 1) grid = 1;
  }
  kern<<<grid, threads, smem, st>>>(b, T);
  return cudaGetLastError();
}

int tma_config_count() { return 25; }

// config: 0 -> (BY 8, 4 stages), 1 -> (8, 6), 2 -> (16, 3), 3 -> (16, 4) with one node per thread;
// 4 -> (16, 4), 5 -> (16, 3), 6 -> (8, 6), 7 -> (8, 3; 5 CTAs/SM), 8 -> (8, 4; 4 CTAs/SM) with two
// x-adjacent nodes per thread; warp-specialised (copy warp + consumer warps, two nodes per
// thread): 9 -> (8, 4 stages; 4 CTAs/SM), 10 -> (8, 4; 5 CTAs/SM), 11 -> (8, 6; 3), 12 -> (16, 4; 2),
// 13 -> (8, 5; 4); without the copy warp (thread 0 issues the copies): 14 -> (8, 4; 5 CTAs/SM),
// 15 -> (8, 4; 4), 16 -> (16, 4; 3); copy warp and early stage release: 17 -> (8, 4; 4),
// 18 -> (8, 3; 4), 19 -> (8, 5; 4); early release with more stages in phase 2 than in phase 1
// (phase 2 copies two boxes per plane against phase 1's four): 20 -> phase 1 (8, 3; 4) and
// phase 2 (8, 4; 4), 21 -> phase 1 (8, 3; 4) and phase 2 (8, 5; 4); grouped iterate updates (x
// updated every m-th iteration): 22 -> as 18 with m = 2, 23 -> as 20 with m = 2, 24 -> as 18 with m = 4
int tma_config_by(int cfg) {
  return (cfg == 2 || cfg == 3 || cfg == 4 || cfg == 5 || cfg == 12 || cfg == 16) ? 16 : 8;
}

int tma_config_xsteps(int cfg) { return (cfg == 22 || cfg == 23) ? 2 : cfg == 24 ? 4 : 1; }

cudaError_t launch_phase_tma(int mode, int cfg, const Batch& b, const TmaSet& T, int grid, cudaStream_t st) {
  if (b.nitems <= 0) return cudaSuccess;
#define WRI_TMA_CASE(M, C_, BY_, S_) \
  if (mode == M && cfg == C_) return launch_one<M, BY_, S_>(b, T, grid, st);
  WRI_TMA_CASE(M_P1, 0, 8, 4)
  WRI_TMA_CASE(M_P2, 0, 8, 4)
  WRI_TMA_CASE(M_P1, 1, 8, 6)
  WRI_TMA_CASE(M_P2, 1, 8, 6)
  WRI_TMA_CASE(M_P1, 2, 16, 3)
  WRI_TMA_CASE(M_P2, 2, 16, 3)
  WRI_TMA_CASE(M_P1, 3, 16, 4)
  WRI_TMA_CASE(M_P2, 3, 16, 4)
#undef WRI_TMA_CASE
#define WRI_TMA2_CASE(M, C_, BY_, S_, MB_) \
  if (mode == M && cfg == C_) return launch_two<M, BY_, S_, MB_>(b, T, grid, st);
  WRI_TMA2_CASE(M_P1, 4, 16, 4, 2)
  WRI_TMA2_CASE(M_P2, 4, 16, 4, 2)
  WRI_TMA2_CASE(M_P1, 5, 16, 3, 2)
  WRI_TMA2_CASE(M_P2, 5, 16, 3, 2)
  WRI_TMA2_CASE(M_P1, 6, 8, 6, 3)
  WRI_TMA2_CASE(M_P2, 6, 8, 6, 3)
  WRI_TMA2_CASE(M_P1, 7, 8, 3, 5)
  WRI_TMA2_CASE(M_P2, 7, 8, 3, 5)
  WRI_TMA2_CASE(M_P1, 8, 8, 4, 4)
  WRI_TMA2_CASE(M_P2, 8, 8, 4, 4)
#undef WRI_TMA2_CASE
#define WRI_WS_CASE(M, C_, BY_, S_, MB_) \
  if (mode == M && cfg == C_) return launch_ws<M, BY_, S_, MB_>(b, T, grid, st);
  WRI_WS_CASE(M_P1, 9, 8, 4, 4)
  WRI_WS_CASE(M_P2, 9, 8, 4, 4)
  WRI_WS_CASE(M_P1, 10, 8, 4, 5)
  WRI_WS_CASE(M_P2, 10, 8, 4, 5)
  WRI_WS_CASE(M_P1, 11, 8, 6, 3)
  WRI_WS_CASE(M_P2, 11, 8, 6, 3)
  WRI_WS_CASE(M_P1, 12, 16, 4, 2)
  WRI_WS_CASE(M_P2, 12, 16, 4, 2)
  WRI_WS_CASE(M_P1, 13, 8, 5, 4)
  WRI_WS_CASE(M_P2, 13, 8, 5, 4)
#undef WRI_WS_CASE
#define WRI_WS1_CASE(M, C_, BY_, S_, MB_) \
  if (mode == M && cfg == C_) return launch_ws<M, BY_, S_, MB_, false>(b, T, grid, st);
  WRI_WS1_CASE(M_P1, 14, 8, 4, 5)
  WRI_WS1_CASE(M_P2, 14, 8, 4, 5)
  WRI_WS1_CASE(M_P1, 15, 8, 4, 4)
  WRI_WS1_CASE(M_P2, 15, 8, 4, 4)
  WRI_WS1_CASE(M_P1, 16, 16, 4, 3)
  WRI_WS1_CASE(M_P2, 16, 16, 4, 3)
#undef WRI_WS1_CASE
#define WRI_WSE_CASE(M, C_, BY_, S_, MB_) \
  if (mode == M && cfg == C_) return launch_ws<M, BY_, S_, MB_, true, true>(b, T, grid, st);
  WRI_WSE_CASE(M_P1, 17, 8, 4, 4)
  WRI_WSE_CASE(M_P2, 17, 8, 4, 4)
  WRI_WSE_CASE(M_P1, 18, 8, 3, 4)
  WRI_WSE_CASE(M_P2, 18, 8, 3, 4)
  WRI_WSE_CASE(M_P1, 19, 8, 5, 4)
  WRI_WSE_CASE(M_P2, 19, 8, 5, 4)
  WRI_WSE_CASE(M_P1, 20, 8, 3, 4)
  WRI_WSE_CASE(M_P2, 20, 8, 4, 4)
  WRI_WSE_CASE(M_P1, 21, 8, 3, 4)
  WRI_WSE_CASE(M_P2, 21, 8, 5, 4)
  // grouped updates: the same kernels as 18 and 20, with b.xsteps set by the caller
  WRI_WSE_CASE(M_P1, 22, 8, 3, 4)
  WRI_WSE_CASE(M_P2, 22, 8, 3, 4)
  WRI_WSE_CASE(M_P1, 23, 8, 3, 4)
  WRI_WSE_CASE(M_P2, 23, 8, 4, 4)
  WRI_WSE_CASE(M_P1, 24, 8, 3, 4)
  WRI_WSE_CASE(M_P2, 24, 8, 3, 4)
#undef WRI_WSE_CASE
  return cudaErrorInvalidValue;
}

}  // namespace wri
