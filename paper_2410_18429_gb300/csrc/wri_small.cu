// Launchers of the small kernels (setup, export, refinement, source estimate,
// data term) and of the unfused baseline path.
#include "wri_launch.h"
#include "wri_small.cuh"

namespace wri {

static int grid_for(long long n, int bs, int cap = 4096) {
  long long g = (n + bs - 1) / bs;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

cudaError_t launch_setup_rhs(int dtype_bytes, int rl_bytes, const Batch& b, int nsys_total, cudaStream_t st) {
  if (nsys_total <= 0) return cudaSuccess;
  if (dtype_bytes == 4 && rl_bytes == 4) k_setup_rhs<float, float><<<nsys_total, 128, 0, st>>>(b, nsys_total);
  else if (dtype_bytes == 4 && rl_bytes == 8) k_setup_rhs<float, double><<<nsys_total, 128, 0, st>>>(b, nsys_total);
  else if (dtype_bytes == 8 && rl_bytes == 8) k_setup_rhs<double, double><<<nsys_total, 128, 0, st>>>(b, nsys_total);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_rmask(const Batch& b, int nsys_total, cudaStream_t st) {
  if (nsys_total <= 0) return cudaSuccess;
  k_rmask<<<nsys_total, 128, 0, st>>>(b, nsys_total);
  return cudaGetLastError();
}

cudaError_t launch_loop_ctl(cudaGraphConditionalHandle h, int* counters, int cap, cudaStream_t st) {
  k_loop_ctl<<<1, 1, 0, st>>>(h, counters, cap);
  return cudaGetLastError();
}

cudaError_t launch_grad_residual(const Batch& b, int gi, double* grad, double* f, cudaStream_t st) {
  const long long n = b.g[gi].n;
  k_grad_residual<<<grid_for(n, 256, 8 * 152), 256, 0, st>>>(b, gi, grad, f);
  return cudaGetLastError();
}

cudaError_t launch_fwi_adjoint_source(int rbytes, const Batch& b, int nsys_total, const double* alpha_in,
                                      double* alpha_out, void* const* q_adj, double* f, cudaStream_t st) {
  if (nsys_total <= 0) return cudaSuccess;
  FwiPtrs Q;
  for (int g = 0; g < WRI_MAXG; ++g) Q.p[g] = g < b.ngroups ? q_adj[g] : nullptr;
  if (rbytes == 8) k_fwi_adjoint_source<double><<<nsys_total, 128, 0, st>>>(b, nsys_total, alpha_in, alpha_out, Q, f);
  else k_fwi_adjoint_source<float><<<nsys_total, 128, 0, st>>>(b, nsys_total, alpha_in, alpha_out, Q, f);
  return cudaGetLastError();
}

cudaError_t launch_fwi_gradient(int rbytes, const Batch& b, int gi, const double* alpha, const void* w, double* grad,
                                cudaStream_t st) {
  const int grid = grid_for(b.g[gi].n, 256, 8 * 152);
  if (rbytes == 8) k_fwi_gradient<double><<<grid, 256, 0, st>>>(b, gi, alpha, w, grad);
  else k_fwi_gradient<float><<<grid, 256, 0, st>>>(b, gi, alpha, w, grad);
  return cudaGetLastError();
}

cudaError_t launch_ztable(const Batch& b, cudaStream_t st) {
  k_ztable<<<dim3(4, b.ngroups), 128, 0, st>>>(b);
  return cudaGetLastError();
}

cudaError_t launch_export(const SysDev* sys, int nsys, int32_t* iters, double* relres, int32_t* status,
                          cudaStream_t st) {
  k_export<<<(nsys + 127) / 128, 128, 0, st>>>(sys, nsys, iters, relres, status);
  return cudaGetLastError();
}

static IrU ir_u(void* const* u, int ngroups) {
  IrU U;
  for (int g = 0; g < WRI_MAXG; ++g) U.u[g] = g < ngroups ? (float2*)u[g] : nullptr;
  return U;
}

cudaError_t launch_ir_init(const Batch& b, void* const* u, int warm, cudaStream_t st) {
  k_ir_init<<<1024, 256, 0, st>>>(b, ir_u(u, b.ngroups), warm);
  return cudaGetLastError();
}

cudaError_t launch_ir_rmap(const Batch& b, int nsys_total, cudaStream_t st) {
  if (nsys_total <= 0) return cudaSuccess;
  k_ir_rmap<<<nsys_total, 128, 0, st>>>(b);
  return cudaGetLastError();
}

cudaError_t launch_ir_cold(const Batch& b, int nsys_total, cudaStream_t st) {
  if (nsys_total <= 0) return cudaSuccess;
  k_ir_cold<<<nsys_total, 128, 0, st>>>(b, nsys_total);
  return cudaGetLastError();
}

cudaError_t launch_ir_forcing(const Batch& b, const void* q2, cudaStream_t st) {
  k_ir_forcing<<<1024, 256, 0, st>>>(b, (const double2*)q2);
  return cudaGetLastError();
}

cudaError_t launch_ir_update(const Batch& b, cudaStream_t st) {
  k_ir_update<<<1024, 256, 0, st>>>(b);
  return cudaGetLastError();
}

cudaError_t launch_ir_final(const Batch& b, void* const* u, cudaStream_t st) {
  k_ir_final<<<1024, 256, 0, st>>>(b, ir_u(u, b.ngroups));
  return cudaGetLastError();
}

cudaError_t launch_source_estimate(int rbytes, const Batch& b, int nsys_total, double* alpha_out, cudaStream_t st) {
  const int g = (nsys_total + 63) / 64;
  if (rbytes == 4) k_source_estimate<float><<<g, 64, 0, st>>>(b, nsys_total, alpha_out);
  else k_source_estimate<double><<<g, 64, 0, st>>>(b, nsys_total, alpha_out);
  return cudaGetLastError();
}

cudaError_t launch_data_term(int rbytes, int dbytes, const Batch& b, int nsys_total, cudaStream_t st) {
  if (rbytes == 4 && dbytes == 4) k_data_term<float, float><<<nsys_total, 256, 0, st>>>(b, nsys_total);
  else if (rbytes == 8 && dbytes == 4) k_data_term<double, float><<<nsys_total, 256, 0, st>>>(b, nsys_total);
  else if (rbytes == 8 && dbytes == 8) k_data_term<double, double><<<nsys_total, 256, 0, st>>>(b, nsys_total);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_tv(const double* m, int nx, int ny, int nz, double beta, double gamma, double* tv, double* grad,
                      cudaStream_t st) {
  const long long n = (long long)nx * ny * nz;
  k_tv<<<grid_for(n, 256, 4096), 256, 0, st>>>(m, nx, ny, nz, beta, gamma, tv, grad);
  return cudaGetLastError();
}

cudaError_t launch_widen(const void* u, void* u64, long long count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  k_widen<<<grid_for(count, 256), 256, 0, st>>>((const float2*)u, (double2*)u64, count);
  return cudaGetLastError();
}

#define WRI_BOTH(call_f, call_d) \
  if (rbytes == 4) {             \
    call_f;                      \
  } else {                       \
    call_d;                      \
  }                              \
  return cudaGetLastError();

cudaError_t plain_fill(int rbytes, void* r1, void* x, long long n, long long src, double ar, double ai,
                       cudaStream_t st) {
  const int g = grid_for(n, 256);
  WRI_BOTH((k_p_fill<float><<<g, 256, 0, st>>>((float2*)r1, (float2*)x, n, src, make_float2((float)ar, (float)ai))),
           (k_p_fill<double><<<g, 256, 0, st>>>((double2*)r1, (double2*)x, n, src, make_double2(ar, ai))))
}

cudaError_t plain_setr2(int rbytes, void* r2, const void* d, int nr, double lam, cudaStream_t st) {
  if (nr <= 0) return cudaSuccess;
  const int g = (nr + 127) / 128;
  WRI_BOTH((k_p_setr2<float><<<g, 128, 0, st>>>((float2*)r2, (const float2*)d, nr, (float)lam)),
           (k_p_setr2<double><<<g, 128, 0, st>>>((double2*)r2, (const double2*)d, nr, lam)))
}

cudaError_t plain_scatter(int rbytes, void* s, const int* rec, const void* r2, int nr, double lam, cudaStream_t st) {
  if (nr <= 0) return cudaSuccess;
  const int g = (nr + 127) / 128;
  WRI_BOTH((k_p_scatter<float><<<g, 128, 0, st>>>((float2*)s, rec, (const float2*)r2, nr, (float)lam)),
           (k_p_scatter<double><<<g, 128, 0, st>>>((double2*)s, rec, (const double2*)r2, nr, lam)))
}

cudaError_t plain_gather_mask(int rbytes, void* t2, const void* p, const int* rec, int nr, double lam, void* t1,
                              long long src, int masked, cudaStream_t st) {
  const int g = (nr > 0 ? nr + 127 : 128) / 128;
  WRI_BOTH((k_p_gather_mask<float><<<g, 128, 0, st>>>((float2*)t2, (const float2*)p, rec, nr, (float)lam,
                                                      (float2*)t1, src, masked)),
           (k_p_gather_mask<double><<<g, 128, 0, st>>>((double2*)t2, (const double2*)p, rec, nr, lam, (double2*)t1,
                                                       src, masked)))
}

cudaError_t plain_dot(int rbytes, const void* a, long long n, double* partial, double* out, cudaStream_t st) {
  const int g = grid_for(n, 256, 1024);
  if (rbytes == 4) k_p_dot<float><<<g, 256, 0, st>>>((const float2*)a, n, partial);
  else k_p_dot<double><<<g, 256, 0, st>>>((const double2*)a, n, partial);
  k_p_sum<<<1, 1024, 0, st>>>(partial, g, out);
  return cudaGetLastError();
}

cudaError_t plain_axpy(int rbytes, void* y, const void* x, double a, long long n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int g = grid_for(n, 256);
  WRI_BOTH((k_p_axpy<float><<<g, 256, 0, st>>>((float2*)y, (const float2*)x, (float)a, n)),
           (k_p_axpy<double><<<g, 256, 0, st>>>((double2*)y, (const double2*)x, a, n)))
}

cudaError_t plain_xpby(int rbytes, void* p, const void* s, double beta, long long n, cudaStream_t st) {
  const int g = grid_for(n, 256);
  WRI_BOTH((k_p_xpby<float><<<g, 256, 0, st>>>((float2*)p, (const float2*)s, (float)beta, n)),
           (k_p_xpby<double><<<g, 256, 0, st>>>((double2*)p, (const double2*)s, beta, n)))
}

}  // namespace wri
