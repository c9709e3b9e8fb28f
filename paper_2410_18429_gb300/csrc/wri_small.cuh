// Small kernels of libwri: right-hand-side setup, result export, refinement
// bookkeeping, the source-weight estimate, the data term of the objective, and the
// BLAS-1 kernels of the unfused baseline path.
#pragma once

#include "../../include/wri.h"
#include "wri_march.cuh"

namespace wri {

// lamd[k] = lambda_g d[k] and r2[k] = lamd[k] for every receiver entry (one block per system).
template <typename DT, typename RL>
__global__ void k_setup_rhs(const __grid_constant__ Batch b, int nsys_total) {
  const int s = blockIdx.x;
  if (s >= nsys_total) return;
  const SysDev& sd = b.sys[s];
  const GroupDev& G = b.g[sd.group];
  const cx<DT>* d = (const cx<DT>*)G.d;
  const int base = b.sys[G.sys0].rec_begin;  // the group's data starts at its first system
  cx<RL>* lamd = (cx<RL>*)b.lamd;
  cx<RL>* r2 = (cx<RL>*)b.r2;
  const RL lam = RL(G.lambda);
  for (int k = sd.rec_begin + threadIdx.x; k < sd.rec_end; k += blockDim.x) {
    const cx<RL> v = lam * to_c(d[k - base], RL(0));
    lamd[k] = v;
    r2[k] = v;
  }
}

// Receiver bitmaps of the normal-residual norms (rec_col_bits): one block per system; the
// caller zeroed both maps.  Receivers are distinct within a system, so every bit is set once.
__global__ void k_rmask(const __grid_constant__ Batch b, int nsys_total) {
  const int s = blockIdx.x;
  if (s >= nsys_total) return;
  const SysDev& sd = b.sys[s];
  const GroupDev& G = b.g[sd.group];
  if (!G.rmask) return;
  uint32_t* mask = const_cast<uint32_t*>(G.rmask);
  uint32_t* col = const_cast<uint32_t*>(G.rcol);
  const long long plane = (long long)G.nx * G.ny;
  for (int k = sd.rec_begin + threadIdx.x; k < sd.rec_end; k += blockDim.x) {
    const long long node = b.rec_idx[k];
    const int z = (int)(node / plane);
    const long long rem = node - (long long)z * plane;
    const int y = (int)(rem / G.nx);
    const int x = (int)(rem - (long long)y * G.nx);
    const uint32_t bit = 1u << (x & 31);
    atomicOr(mask + (((long long)sd.local * G.nz + z) * G.ny + y) * G.tiles_x + (x >> 5), bit);
    atomicOr(col + ((long long)sd.local * G.ny + y) * G.tiles_x + (x >> 5), bit);
  }
}

// Control kernel of the device-side CG loop (the WHILE node of the iteration graph): the body runs
// again while systems remain, no copy wait has timed out and fewer than `cap` bodies have run.
// counters: [0] systems not done, [1] copy-wait error flag, [2] bodies run (zeroed per solve).
__global__ void k_loop_ctl(cudaGraphConditionalHandle h, int* counters, int cap) {
  const int body = ++counters[2];
  const bool go = counters[0] > 0 && counters[1] == 0 && body < cap;
  cudaGraphSetConditional(h, go ? 1u : 0u);
}

// Gradient and objective of Eqs. VarG2 / VarObj2 from the FP64 residual q = b - S u that a refined
// solve leaves behind: node part q1 = b1 - Z A u, receiver part q2 = lambda (d - P u).  The PDE
// residual of the gradient is A u - a e = -q1: in source-free mode a = (A u)[src] zeroes the source
// row exactly as Z does, and with a known weight b1 = alpha e and Z = I.  So, with no stencil,
//   grad[node] += -omega^2 sum over the group's systems of Re(conj(w u) q1),
//   f          += 1/2 ||q1||^2 + 1/2 ||q2||^2.
// One thread per node of group gi (all its systems); b: the outer view (x64 = u, q64 = q1,
// r2 = q2 in FP64).
__global__ void k_grad_residual(const __grid_constant__ Batch b, int gi, double* grad, double* f) {
  __shared__ double red[8];
  const GroupDev& G = b.g[gi];
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long plane = (long long)G.nx * G.ny;
  const double2* u = (const double2*)G.x64;
  const double2* q = (const double2*)G.q64;
  const double om2 = G.omega * G.omega;
  double facc = 0.0;
  for (long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x; node < G.n; node += stride) {
    const int k = (int)(node / plane);
    const long long rem = node - (long long)k * plane;
    const int j = (int)(rem / G.nx);
    const int i = (int)(rem - (long long)j * G.nx);
    const double2 w = stretch_at<double, false>(G.ax, double(i)) * stretch_at<double, false>(G.ay, double(j)) *
                      stretch_at<double, false>(G.az, double(k));
    double acc = 0.0;
    for (int sl = 0; sl < G.nsys; ++sl) {
      const double2 wu = w * u[(long long)sl * G.n + node];
      const double2 r = q[(long long)sl * G.n + node];
      acc += wu.x * r.x + wu.y * r.y;
      facc += 0.5 * abs2(r);
    }
    grad[node] += -om2 * acc;
  }
  const double2* q2 = (const double2*)b.r2;
  const int r0 = b.sys[G.sys0].rec_begin, r1 = b.sys[G.sys0 + G.nsys - 1].rec_end;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < r1 - r0; e += stride)
    facc += 0.5 * abs2(q2[r0 + e]);
  const double fs = block_sum<256>(facc, red);
  if (threadIdx.x == 0 && fs != 0.0) atomicAdd(f, fs);
}

// ------------------------------------------------------------------ reduced FWI (Eqs. PDEsolve, FWI2)
struct FwiPtrs {
  void* p[WRI_MAXG];  // one device array per group, [nsys][n] complex
};

// Weights, data residuals, objective and adjoint right-hand sides of reduced FWI: one block of 128
// threads per system.  u = G = A^{-1} e (the forward solve with weight 1) in b.g[].x; the weight a
// is given or, source-free, the minimiser of ||a P G - d||: a = (P G)^H d / ||P G||^2; then
// r = a P G - d, f += 1/2 ||r||^2 and q_adj = conj(P^T r) (A complex symmetric: the solve of
// A w = q_adj gives the adjoint wavefield v = conj(w) of A^H v = P^T r).
template <typename R>
__global__ void k_fwi_adjoint_source(const __grid_constant__ Batch b, int nsys_total, const double* alpha_in,
                                     double* alpha_out, FwiPtrs Q, double* f) {
  __shared__ double red[4];
  const int s = blockIdx.x;
  if (s >= nsys_total) return;
  const SysDev& sd = b.sys[s];
  const GroupDev& G = b.g[sd.group];
  const cx<R>* u = (const cx<R>*)G.x + (long long)sd.local * G.n;
  const cx<R>* d = (const cx<R>*)G.d;
  const int base = b.sys[G.sys0].rec_begin;  // the group's data starts at its first system
  double a_re, a_im;
  if (alpha_in) {
    a_re = alpha_in[2 * s];
    a_im = alpha_in[2 * s + 1];
  } else {
    double nr = 0.0, ni = 0.0, den = 0.0;  // (P G)^H d and ||P G||^2
    for (int k = sd.rec_begin + threadIdx.x; k < sd.rec_end; k += blockDim.x) {
      const double2 g = to_c(u[b.rec_idx[k]], 0.0), dv = to_c(d[k - base], 0.0);
      nr += g.x * dv.x + g.y * dv.y;
      ni += g.x * dv.y - g.y * dv.x;
      den += g.x * g.x + g.y * g.y;
    }
    nr = block_sum<128>(nr, red);
    ni = block_sum<128>(ni, red);
    den = block_sum<128>(den, red);
    __shared__ double sa[2];
    if (threadIdx.x == 0) {
      sa[0] = den > 0.0 ? nr / den : 0.0;
      sa[1] = den > 0.0 ? ni / den : 0.0;
    }
    __syncthreads();
    a_re = sa[0];
    a_im = sa[1];
  }
  if (threadIdx.x == 0) {
    alpha_out[2 * s] = a_re;
    alpha_out[2 * s + 1] = a_im;
  }
  cx<R>* q = (cx<R>*)Q.p[sd.group] + (long long)sd.local * G.n;
  double fr = 0.0;
  for (int k = sd.rec_begin + threadIdx.x; k < sd.rec_end; k += blockDim.x) {
    const int node = b.rec_idx[k];
    const double2 g = to_c(u[node], 0.0), dv = to_c(d[k - base], 0.0);
    const double2 r = make_double2(a_re * g.x - a_im * g.y - dv.x, a_re * g.y + a_im * g.x - dv.y);
    fr += 0.5 * (r.x * r.x + r.y * r.y);
    q[node] = to_c(make_double2(r.x, -r.y), R(0));
  }
  fr = block_sum<128>(fr, red);
  if (threadIdx.x == 0 && fr != 0.0) atomicAdd(f, fr);
}

// Gradient of reduced FWI for group gi: one thread per node, the group's systems summed in order:
// grad += -omega^2 sum_i Re(w a_i G_i conj(v_i)) with conj(v_i) = w_i, the adjoint solve's wavefield.
template <typename R>
__global__ void k_fwi_gradient(const __grid_constant__ Batch b, int gi, const double* alpha, const void* wadj,
                               double* grad) {
  const GroupDev& G = b.g[gi];
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long plane = (long long)G.nx * G.ny;
  const cx<R>* u = (const cx<R>*)G.x;
  const cx<R>* wv = (const cx<R>*)wadj;
  const double om2 = G.omega * G.omega;
  for (long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x; node < G.n; node += stride) {
    const int k = (int)(node / plane);
    const long long rem = node - (long long)k * plane;
    const int j = (int)(rem / G.nx);
    const int i = (int)(rem - (long long)j * G.nx);
    const double2 w = stretch_at<double, false>(G.ax, double(i)) * stretch_at<double, false>(G.ay, double(j)) *
                      stretch_at<double, false>(G.az, double(k));
    double acc = 0.0;
    for (int sl = 0; sl < G.nsys; ++sl) {
      const double2 a = make_double2(alpha[2 * (G.sys0 + sl)], alpha[2 * (G.sys0 + sl) + 1]);
      const double2 t = (w * a) * to_c(u[(long long)sl * G.n + node], 0.0) * to_c(wv[(long long)sl * G.n + node], 0.0);
      acc += t.x;
    }
    grad[node] += -om2 * acc;
  }
}

// z-axis coefficient tables of every group (FP32 and FP64, where the batch has them): one thread
// per (group, plane).
template <typename R>
__device__ __forceinline__ void ztable_fill(const GroupDev& G, cx<R>* t, int k) {
  const ZCoef<R> a = z_coef<R, false>(G, k);
  const ZCoef<R> h = z_coef<R, true>(G, k);
  t[3 * k + 0] = a.sz;
  t[3 * k + 1] = a.izm;
  t[3 * k + 2] = a.izp;
  t[3 * (G.nz + k) + 0] = h.sz;
  t[3 * (G.nz + k) + 1] = h.izm;
  t[3 * (G.nz + k) + 2] = h.izp;
}

__global__ void k_ztable(const __grid_constant__ Batch b) {
  const int g = blockIdx.y;
  if (g >= b.ngroups) return;
  const GroupDev& G = b.g[g];
  float2* t = const_cast<float2*>(G.ztab);
  double2* t64 = const_cast<double2*>(G.ztab64);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < G.nz; k += gridDim.x * blockDim.x) {
    if (t) ztable_fill<float>(G, t, k);
    if (t64) ztable_fill<double>(G, t64, k);
  }
}

__global__ void k_export(const SysDev* sys, int nsys, int32_t* iters, double* relres, int32_t* status) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsys) return;
  iters[s] = sys[s].iter_total;
  relres[s] = sys[s].relres;
  status[s] = sys[s].status;
}

// ------------------------------------------------------------------ FP64 iterative refinement
// Augmented-system refinement of the least-squares problem min ||S x - b|| (Bjorck): the
// solution x64 and the residual r64 = (r64 on the nodes, r2_64 on the receivers) are kept
// in FP64; every outer step forms the FP64 residuals of the augmented system
//     f = b - r64 - S x64,   g = -S^H r64,
// and an FP32 CGLS inner solve of   min 1/2 ||S dx - f||^2 + Re<g, dx>   (same iterates as CGLS
// with s = S^H r + S^H r64 = S^H r - g) returns the corrections dx and dr = f - S dx.  The kernels below
// do the elementwise parts; b is the inner (complex64) view of the batch, with x64, r64, q64,
// r2_64 and r2_in set.  Systems whose refinement has finished (outer_done) are left alone.

struct IrU {
  float2* u[WRI_MAXG];  // the caller's complex64 wavefields, one pointer per group
};

__device__ __forceinline__ int nsys_of(const Batch& b) { return b.g[b.ngroups - 1].sys0 + b.g[b.ngroups - 1].nsys; }

// Receiver map of the refinement: rmap[system][node] = receiver entry (the map was filled with
// -1 before); one block per system.
__global__ void k_ir_rmap(const __grid_constant__ Batch b) {
  const int s = blockIdx.x;
  if (s >= nsys_of(b)) return;
  const SysDev& sd = b.sys[s];
  const GroupDev& G = b.g[sd.group];
  int* rmap = const_cast<int*>(G.rmap) + (long long)sd.local * G.n;
  for (int k = sd.rec_begin + threadIdx.x; k < sd.rec_end; k += blockDim.x) rmap[b.rec_idx[k]] = k;
}

// x64 = warm ? u : 0, r64 = 0, x32 = 0 on every node; r2_64 = 0 on every receiver entry.
__global__ void k_ir_init(const __grid_constant__ Batch b, IrU U, int warm) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (int g = 0; g < b.ngroups; ++g) {
    const GroupDev& G = b.g[g];
    const long long tot = (long long)G.nsys * G.n;
    const float2* u = U.u[g];
    double2* x64 = (double2*)G.x64;
    double2* r64 = (double2*)G.r64;
    float2* x32 = (float2*)G.x;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += stride) {
      x64[e] = warm ? make_double2(u[e].x, u[e].y) : make_double2(0.0, 0.0);
      r64[e] = make_double2(0.0, 0.0);
      x32[e] = make_float2(0.f, 0.f);
    }
  }
  const int ns = nsys_of(b);
  double2* r2 = (double2*)b.r2_64;
  for (int s = blockIdx.x; s < ns; s += gridDim.x)
    for (int k = b.sys[s].rec_begin + threadIdx.x; k < b.sys[s].rec_end; k += blockDim.x) r2[k] = make_double2(0.0, 0.0);
}

// Cold start of the refinement (x64 = 0, r64 = 0, so b - S x64 = b): the first inner solve's
// receiver residual is lambda d, rounded to complex64.  b: the inner view (r2 = r2_in, lamd FP64).
__global__ void k_ir_cold(const __grid_constant__ Batch b, int nsys_total) {
  const int s = blockIdx.x;
  if (s >= nsys_total) return;
  const double2* lamd = (const double2*)b.lamd;
  float2* r2 = (float2*)b.r2;
  for (int k = b.sys[s].rec_begin + threadIdx.x; k < b.sys[s].rec_end; k += blockDim.x)
    r2[k] = make_float2((float)lamd[k].x, (float)lamd[k].y);
}

// Forcing of an outer step: inner r1[0] = q64 - r64 (= f on the nodes) and inner receiver
// residual r2_in = q2 - r2_64, both rounded to complex64.  q = b - S x64 comes from the FP64
// residual kernel (q2: its receiver part).
__global__ void k_ir_forcing(const __grid_constant__ Batch b, const double2* q2) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (int g = 0; g < b.ngroups; ++g) {
    const GroupDev& G = b.g[g];
    const long long tot = (long long)G.nsys * G.n;
    const double2* q = (const double2*)G.q64;
    const double2* r64 = (const double2*)G.r64;
    float2* f = (float2*)G.r1[0];
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += stride) {
      if (b.sys[G.sys0 + (int)(e / G.n)].outer_done) continue;
      const double2 a = q[e], r = r64[e];
      f[e] = make_float2((float)(a.x - r.x), (float)(a.y - r.y));
    }
  }
  const int ns = nsys_of(b);
  const double2* r2 = (const double2*)b.r2_64;
  float2* f2 = (float2*)b.r2_in;
  for (int s = blockIdx.x; s < ns; s += gridDim.x) {
    if (b.sys[s].outer_done) continue;
    for (int k = b.sys[s].rec_begin + threadIdx.x; k < b.sys[s].rec_end; k += blockDim.x)
      f2[k] = make_float2((float)(q2[k].x - r2[k].x), (float)(q2[k].y - r2[k].y));
  }
}

// Update after an inner solve: x64 += dx (then dx = 0), r64 += dr on the nodes (the inner
// residual of the system's last iteration sits in r1[iter & 1]) and r2_64 += r2_in.
__global__ void k_ir_update(const __grid_constant__ Batch b) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (int g = 0; g < b.ngroups; ++g) {
    const GroupDev& G = b.g[g];
    const long long tot = (long long)G.nsys * G.n;
    double2* x64 = (double2*)G.x64;
    double2* r64 = (double2*)G.r64;
    float2* x32 = (float2*)G.x;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += stride) {
      const SysDev& sd = b.sys[G.sys0 + (int)(e / G.n)];
      if (sd.outer_done) continue;
      const float2 dx = x32[e];
      const float2 dr = ((const float2*)G.r1[sd.iter & 1])[e];
      double2 v = x64[e];
      v.x += dx.x;
      v.y += dx.y;
      x64[e] = v;
      x32[e] = make_float2(0.f, 0.f);
      double2 r = r64[e];
      r.x += dr.x;
      r.y += dr.y;
      r64[e] = r;
    }
  }
  const int ns = nsys_of(b);
  double2* r2 = (double2*)b.r2_64;
  const float2* d2 = (const float2*)b.r2_in;
  for (int s = blockIdx.x; s < ns; s += gridDim.x) {
    if (b.sys[s].outer_done) continue;
    for (int k = b.sys[s].rec_begin + threadIdx.x; k < b.sys[s].rec_end; k += blockDim.x) {
      double2 r = r2[k];
      r.x += d2[k].x;
      r.y += d2[k].y;
      r2[k] = r;
    }
  }
}

// u = x64 rounded to complex64.
__global__ void k_ir_final(const __grid_constant__ Batch b, IrU U) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (int g = 0; g < b.ngroups; ++g) {
    const GroupDev& G = b.g[g];
    const long long tot = (long long)G.nsys * G.n;
    const double2* x64 = (const double2*)G.x64;
    float2* u = U.u[g];
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += stride)
      u[e] = make_float2((float)x64[e].x, (float)x64[e].y);
  }
}

// alpha_out[s] = (A u_s)[src_s]; one thread per system.
template <typename R>
__global__ void k_source_estimate(const __grid_constant__ Batch b, int nsys_total, double* alpha_out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsys_total) return;
  const SysDev& sd = b.sys[s];
  const GroupDev& G = b.g[sd.group];
  const cx<R>* u = (const cx<R>*)G.x + (long long)sd.local * G.n;
  const cx<R> a = stencil_at<R, false>(G, u, sd.src);
  alpha_out[2 * s] = (double)a.x;
  alpha_out[2 * s + 1] = (double)a.y;
}

// f += 1/2 lambda^2 ||P u - d||^2 for every system (one block per system); u in R, d in DT.
template <typename R, typename DT>
__global__ void k_data_term(const __grid_constant__ Batch b, int nsys_total) {
  __shared__ double red[8];
  const int s = blockIdx.x;
  if (s >= nsys_total) return;
  const SysDev& sd = b.sys[s];
  const GroupDev& G = b.g[sd.group];
  const cx<R>* u = (const cx<R>*)G.x + (long long)sd.local * G.n;
  const cx<DT>* d = (const cx<DT>*)G.d;
  const int base = b.sys[G.sys0].rec_begin;
  double acc = 0.0;
  for (int k = sd.rec_begin + threadIdx.x; k < sd.rec_end; k += blockDim.x) {
    const cx<R> r = u[b.rec_idx[k]] - to_c(d[k - base], R(0));
    acc += (double)abs2(r);
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    t *= 0.5 * G.lambda * G.lambda;
    if (t != 0.0) atomicAdd(b.f, t);
  }
}

// u64 = u widened to complex128 (the FP64 wavefield output of a complex64 solve without refinement).
__global__ void k_widen(const float2* u, double2* u64, long long count) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count; e += (long long)gridDim.x * blockDim.x)
    u64[e] = make_double2(u[e].x, u[e].y);
}

// ------------------------------------------------------------------ total variation (Eq. TVAWRI)
// Smoothed isotropic TV of a model on its grid (our reading of ||m||_TV):
//   TV(m) = sum over nodes of sqrt(dx^2 + dy^2 + dz^2 + beta^2),
// forward differences in grid units (dx = m[i+1] - m[i]; zero on the last node of an axis).
// tv += gamma TV(m); grad (if not null) += gamma dTV/dm.  One thread per node, grid-stride.
__device__ __forceinline__ double tv_cell(const double* m, int nx, int ny, int nz, int i, int j, int k,
                                          double beta2, double& dx, double& dy, double& dz) {
  const long long plane = (long long)nx * ny;
  const long long c = (long long)k * plane + (long long)j * nx + i;
  const double v = m[c];
  dx = (i + 1 < nx) ? m[c + 1] - v : 0.0;
  dy = (j + 1 < ny) ? m[c + nx] - v : 0.0;
  dz = (k + 1 < nz) ? m[c + plane] - v : 0.0;
  return sqrt(dx * dx + dy * dy + dz * dz + beta2);
}

__global__ void k_tv(const double* m, int nx, int ny, int nz, double beta, double gamma, double* tv, double* grad) {
  __shared__ double red[8];
  const long long n = (long long)nx * ny * nz;
  const double beta2 = beta * beta;
  double acc = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(e / ((long long)nx * ny));
    const long long rem = e - (long long)k * nx * ny;
    const int j = (int)(rem / nx);
    const int i = (int)(rem - (long long)j * nx);
    double dx, dy, dz;
    const double q = tv_cell(m, nx, ny, nz, i, j, k, beta2, dx, dy, dz);
    acc += q;
    if (grad) {
      double gsum = -(dx + dy + dz) / q;  // this node's own cell
      double ax, ay, az;
      if (i > 0) {  // the cell of node i-1, whose x difference contains this node
        const double qq = tv_cell(m, nx, ny, nz, i - 1, j, k, beta2, ax, ay, az);
        gsum += ax / qq;
      }
      if (j > 0) {
        const double qq = tv_cell(m, nx, ny, nz, i, j - 1, k, beta2, ax, ay, az);
        gsum += ay / qq;
      }
      if (k > 0) {
        const double qq = tv_cell(m, nx, ny, nz, i, j, k - 1, beta2, ax, ay, az);
        gsum += az / qq;
      }
      grad[e] += gamma * gsum;
    }
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    if (t != 0.0) atomicAdd(tv, gamma * t);
  }
}

// ------------------------------------------------------------------ unfused baseline kernels
template <typename R>
__global__ void k_p_fill(cx<R>* r1, cx<R>* x, long long n, long long src, cx<R> a_src) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    r1[e] = (e == src) ? a_src : czero<R>();
    x[e] = czero<R>();
  }
}

template <typename R>
__global__ void k_p_setr2(cx<R>* r2, const cx<R>* d, int nr, R lam) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nr) r2[k] = lam * d[k];
}

template <typename R>
__global__ void k_p_scatter(cx<R>* s, const int* rec, const cx<R>* r2, int nr, R lam) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nr) s[rec[k]] = s[rec[k]] + lam * r2[k];
}

template <typename R>
__global__ void k_p_gather_mask(cx<R>* t2, const cx<R>* p, const int* rec, int nr, R lam, cx<R>* t1,
                                long long src, int masked) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nr) t2[k] = lam * p[rec[k]];
  if (k == 0 && masked) t1[src] = czero<R>();
}

// partial[block] = sum |a|^2 over a grid-stride slice (FP64), then k_p_sum adds the partials.
template <typename R>
__global__ void k_p_dot(const cx<R>* a, long long n, double* partial) {
  __shared__ double red[32];
  double acc = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    acc += (double)abs2(a[e]);
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) partial[blockIdx.x] = v;
  }
}

__global__ void k_p_sum(const double* partial, int nb, double* out) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int e = threadIdx.x; e < nb; e += blockDim.x) acc += partial[e];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) *out = v;
  }
}

template <typename R>
__global__ void k_p_axpy(cx<R>* y, const cx<R>* x, R a, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    y[e] = y[e] + a * x[e];
}

template <typename R>
__global__ void k_p_xpby(cx<R>* p, const cx<R>* s, R beta, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    p[e] = s[e] + beta * p[e];
}

}  // namespace wri
