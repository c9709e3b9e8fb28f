// Host-side launch entry points of the kernel translation units.
#pragma once

#include <cuda_runtime.h>

#include "wri_dev.cuh"

namespace wri {

// Kernel selection for the z-march: element type of the stencil (R), of its
// output (OR), mode and conjugation.  `grid` = 0 launches one persistent wave
// (SMs x resident CTAs, capped by the number of work items).
cudaError_t launch_march_f32(int mode, bool conj, int by, const Batch& b, int grid, cudaStream_t st);
cudaError_t launch_march_f64(int mode, bool conj, int by, const Batch& b, int grid, cudaStream_t st);
cudaError_t launch_march_f64_to_f32(int mode, int by, const Batch& b, int grid, cudaStream_t st);

// small kernels (wri_small.cu)
cudaError_t launch_setup_rhs(int dtype_bytes, int rl_bytes, const Batch& b, int nsys_total, cudaStream_t st);
cudaError_t launch_ztable(const Batch& b, cudaStream_t st);
// receiver bitmaps of every group (b: solver view with rmask / rcol set and zeroed)
cudaError_t launch_rmask(const Batch& b, int nsys_total, cudaStream_t st);
// control kernel of the device-side CG loop (one thread; sets the WHILE node's condition)
cudaError_t launch_loop_ctl(cudaGraphConditionalHandle h, int* counters, int cap, cudaStream_t st);
cudaError_t launch_export(const SysDev* sys, int nsys, int32_t* iters, double* relres, int32_t* status,
                          cudaStream_t st);
// FP64 refinement (b: inner complex64 view; u: the caller's wavefields, one per group)
cudaError_t launch_ir_init(const Batch& b, void* const* u, int warm, cudaStream_t st);
cudaError_t launch_ir_rmap(const Batch& b, int nsys_total, cudaStream_t st);  // b: outer view, map filled with -1
cudaError_t launch_ir_cold(const Batch& b, int nsys_total, cudaStream_t st);  // b: inner view
cudaError_t launch_ir_forcing(const Batch& b, const void* q2, cudaStream_t st);
cudaError_t launch_ir_update(const Batch& b, cudaStream_t st);
cudaError_t launch_ir_final(const Batch& b, void* const* u, cudaStream_t st);
cudaError_t launch_source_estimate(int rbytes, const Batch& b, int nsys_total, double* alpha_out, cudaStream_t st);
cudaError_t launch_data_term(int rbytes, int dbytes, const Batch& b, int nsys_total, cudaStream_t st);
// reduced FWI: weights, residuals, objective and adjoint right-hand sides; gradient of group gi
cudaError_t launch_fwi_adjoint_source(int rbytes, const Batch& b, int nsys_total, const double* alpha_in,
                                      double* alpha_out, void* const* q_adj, double* f, cudaStream_t st);
cudaError_t launch_fwi_gradient(int rbytes, const Batch& b, int gi, const double* alpha, const void* w, double* grad,
                                cudaStream_t st);
// gradient and objective from a refined solve's FP64 residual (b: outer view of that solve)
cudaError_t launch_grad_residual(const Batch& b, int gi, double* grad, double* f, cudaStream_t st);
cudaError_t launch_widen(const void* u, void* u64, long long count, cudaStream_t st);
cudaError_t launch_tv(const double* m, int nx, int ny, int nz, double beta, double gamma, double* tv, double* grad,
                      cudaStream_t st);

// unfused baseline kernels (wri_small.cu); pointers are complex of element size rbytes
cudaError_t plain_fill(int rbytes, void* r1, void* x, long long n, long long src, double ar, double ai,
                       cudaStream_t st);
cudaError_t plain_setr2(int rbytes, void* r2, const void* d, int nr, double lam, cudaStream_t st);
cudaError_t plain_scatter(int rbytes, void* s, const int* rec, const void* r2, int nr, double lam, cudaStream_t st);
cudaError_t plain_gather_mask(int rbytes, void* t2, const void* p, const int* rec, int nr, double lam, void* t1,
                              long long src, int masked, cudaStream_t st);
cudaError_t plain_dot(int rbytes, const void* a, long long n, double* partial, double* out, cudaStream_t st);
cudaError_t plain_axpy(int rbytes, void* y, const void* x, double a, long long n, cudaStream_t st);
cudaError_t plain_xpby(int rbytes, void* p, const void* s, double beta, long long n, cudaStream_t st);

}  // namespace wri

namespace wri {
struct TmaSet;
// TMA-pipelined phase 1 / phase 2 kernels (complex64); cfg selects tile height and stages.
int tma_config_count();
int tma_config_by(int cfg);
int tma_config_xsteps(int cfg);  // iterations per iterate update of phase 1 (1, 2 or 4)
cudaError_t launch_phase_tma(int mode, int cfg, const Batch& b, const TmaSet& T, int grid, cudaStream_t st);
}  // namespace wri
