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

// z-axis coefficient tables of every group (FP32): one thread per (group, plane).
__global__ void k_ztable(const __grid_constant__ Batch b) {
  const int g = blockIdx.y;
  if (g >= b.ngroups) return;
  const GroupDev& G = b.g[g];
  float2* t = const_cast<float2*>(G.ztab);
  if (!t) return;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < G.nz; k += gridDim.x * blockDim.x) {
    const ZCoef<float> a = z_coef<float, false>(G, k);
    const ZCoef<float> h = z_coef<float, true>(G, k);
    t[3 * k + 0] = a.sz;
    t[3 * k + 1] = a.izm;
    t[3 * k + 2] = a.izp;
    t[3 * (G.nz + k) + 0] = h.sz;
    t[3 * (G.nz + k) + 1] = h.izm;
    t[3 * (G.nz + k) + 2] = h.izp;
  }
}

__global__ void k_export(const SysDev* sys, int nsys, int32_t* iters, double* relres, int32_t* status) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsys) return;
  iters[s] = sys[s].iter_total;
  relres[s] = sys[s].relres;
  status[s] = sys[s].status;
}

// Refinement: x64 = warm ? u : 0 and x32 = 0 for every node of every system.
__global__ void k_ir_init(const __grid_constant__ Batch b, int warm) {
  for (int g = 0; g < b.ngroups; ++g) {
    const GroupDev& G = b.g[g];
    const long long tot = (long long)G.nsys * G.n;
    const float2* u = (const float2*)G.d;  // caller's u (C64), passed through the d slot
    double2* x64 = (double2*)G.x64;
    float2* x32 = (float2*)G.x;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
      x64[e] = warm ? make_double2(u[e].x, u[e].y) : make_double2(0.0, 0.0);
      x32[e] = make_float2(0.f, 0.f);
    }
  }
}

// Refinement: x64 += x32, x32 = 0 (systems still refining), or u = (complex64) x64 (final).
__global__ void k_ir_accum(const __grid_constant__ Batch b, int final_cast) {
  for (int g = 0; g < b.ngroups; ++g) {
    const GroupDev& G = b.g[g];
    const long long tot = (long long)G.nsys * G.n;
    double2* x64 = (double2*)G.x64;
    float2* x32 = (float2*)G.x;
    float2* u = (float2*)G.t1;  // caller's u, passed through the t1 slot
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
      if (final_cast) {
        const double2 v = x64[e];
        u[e] = make_float2((float)v.x, (float)v.y);
      } else {
        const float2 d = x32[e];
        if (d.x != 0.f || d.y != 0.f) {
          double2 v = x64[e];
          v.x += d.x;
          v.y += d.y;
          x64[e] = v;
          x32[e] = make_float2(0.f, 0.f);
        }
      }
    }
  }
}

// (A u)[node] for one node with the general coefficients (7 loads).
template <typename R>
__device__ cx<R> apply_at(const GroupDev& G, const cx<R>* u, long long node) {
  const long long plane = (long long)G.nx * G.ny;
  const int k = (int)(node / plane);
  const long long rem = node - (long long)k * plane;
  const int j = (int)(rem / G.nx);
  const int i = (int)(rem - (long long)j * G.nx);
  auto at = [&](int ii, int jj, int kk) -> cx<R> {
    if (ii < 0 || jj < 0 || kk < 0 || ii >= G.nx || jj >= G.ny || kk >= G.nz) return czero<R>();
    return u[(long long)kk * plane + (long long)jj * G.nx + ii];
  };
  const XYCoef<R> c = xy_coef<R, false>(G, i, j);
  const ZCoef<R> z = z_coef<R, false>(G, k);
  const R om2m = pick<R>(G.omega * G.omega, G.om2f) * model_at<R>(G.m, G.m_double, node);
  return stencil_general<R, false>(G, c, z, om2m, at(i, j, k), at(i - 1, j, k), at(i + 1, j, k),
                                   at(i, j - 1, k), at(i, j + 1, k), at(i, j, k - 1), at(i, j, k + 1));
}

// alpha_out[s] = (A u_s)[src_s]; one thread per system.
template <typename R>
__global__ void k_source_estimate(const __grid_constant__ Batch b, int nsys_total, double* alpha_out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsys_total) return;
  const SysDev& sd = b.sys[s];
  const GroupDev& G = b.g[sd.group];
  const cx<R>* u = (const cx<R>*)G.x + (long long)sd.local * G.n;
  const cx<R> a = apply_at<R>(G, u, sd.src);
  alpha_out[2 * s] = (double)a.x;
  alpha_out[2 * s + 1] = (double)a.y;
}

// f += 1/2 lambda^2 ||P u - d||^2 for every system (one block per system).
template <typename R>
__global__ void k_data_term(const __grid_constant__ Batch b, int nsys_total) {
  __shared__ double red[8];
  const int s = blockIdx.x;
  if (s >= nsys_total) return;
  const SysDev& sd = b.sys[s];
  const GroupDev& G = b.g[sd.group];
  const cx<R>* u = (const cx<R>*)G.x + (long long)sd.local * G.n;
  const cx<R>* d = (const cx<R>*)G.d;
  const int base = b.sys[G.sys0].rec_begin;
  double acc = 0.0;
  for (int k = sd.rec_begin + threadIdx.x; k < sd.rec_end; k += blockDim.x) {
    const cx<R> r = u[b.rec_idx[k]] - d[k - base];
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
