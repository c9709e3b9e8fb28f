// The z-marching stencil kernel and its fused CGLS phases.
//
// One CTA owns a tile of WRI_TX x BY nodes in the x-y plane and marches through a
// z-chunk [z0, z1).  For every plane it holds the input field F of the stencil in
// shared memory (own nodes plus a one-node halo ring, double buffered) and keeps the
// planes k-1, k, k+1 of its own column in registers, so each input value is read
// from memory once per tile (plus the halo ring).  The field F is formed on the fly
// from the stored vectors (e.g. p_new = s + beta p_old), so a CG vector update and
// the following operator application cost one pass over memory.
//
// Every work item is (group, tile, system); a persistent grid strides over items.
// Per-system reductions are FP64: each tile writes one partial sum, and the CTA that
// completes a system's last tile (atomic ticket) sums the partials in tile order,
// adds the receiver terms and updates the system's CG scalars on the device.
#pragma once

#include "wri_dev.cuh"

namespace wri {


template <typename T>
__device__ __forceinline__ T ldcg_c(const T* p);
template <>
__device__ __forceinline__ float2 ldcg_c(const float2* p) { return __ldcg(p); }
template <>
__device__ __forceinline__ double2 ldcg_c(const double2* p) { return __ldcg(p); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Barrier of the threads that take part in a reduction: the whole CTA ...
struct CtaSync {
  static __device__ __forceinline__ void sync() { __syncthreads(); }
};
// ... or only the first NC threads (named barrier 1), when other warps of the CTA run
// independently (the copy-issuing warp of the warp-specialised phases).
template <int NC>
struct FirstThreadsSync {
  static __device__ __forceinline__ void sync() { asm volatile("bar.sync 1, %0;" ::"n"(NC) : "memory"); }
};

// Deterministic block sum (fixed order) over the NT threads of SYNC; every one of them must
// call it.  Result valid in thread 0.
template <int NT, typename SYNC = CtaSync>
__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int ltid = threadIdx.y * blockDim.x + threadIdx.x;  // any block shape
  const int lane = ltid & 31;
  const int wid = ltid >> 5;
  SYNC::sync();
  if (lane == 0) red[wid] = v;
  SYNC::sync();
  double r = 0.0;
  if (wid == 0) {
    r = (lane < NT / 32) ? red[lane] : 0.0;
    r = warp_sum(r);
  }
  return r;
}

// Per-thread coefficients of the x and y axes for node (i, j).
template <typename R>
struct XYCoef {
  cx<R> sx, sy, sxy, ixm, ixp, iym, iyp;  // ixm = 1/(s_x(i-1/2) h^2), ...
};

template <typename R>
__device__ __forceinline__ R inv_h2(const GroupDev& G) {
  return pick<R>(1.0 / (G.h * G.h), G.ih2f);
}

template <typename R, bool CONJ>
__device__ __forceinline__ XYCoef<R> xy_coef(const GroupDev& G, int i, int j) {
  XYCoef<R> c;
  const R ih2 = inv_h2<R>(G);
  c.sx = stretch_at<R, CONJ>(G.ax, R(i));
  c.sy = stretch_at<R, CONJ>(G.ay, R(j));
  c.sxy = c.sx * c.sy;
  c.ixm = ih2 * inv(stretch_at<R, CONJ>(G.ax, R(i) - R(0.5)));
  c.ixp = ih2 * inv(stretch_at<R, CONJ>(G.ax, R(i) + R(0.5)));
  c.iym = ih2 * inv(stretch_at<R, CONJ>(G.ay, R(j) - R(0.5)));
  c.iyp = ih2 * inv(stretch_at<R, CONJ>(G.ay, R(j) + R(0.5)));
  return c;
}

template <typename R>
struct ZCoef {
  cx<R> sz, izm, izp;
};

template <typename R, bool CONJ>
__device__ __forceinline__ ZCoef<R> z_coef(const GroupDev& G, int k) {
  ZCoef<R> c;
  const R ih2 = inv_h2<R>(G);
  c.sz = stretch_at<R, CONJ>(G.az, R(k));
  c.izm = ih2 * inv(stretch_at<R, CONJ>(G.az, R(k) - R(0.5)));
  c.izp = ih2 * inv(stretch_at<R, CONJ>(G.az, R(k) + R(0.5)));
  return c;
}

// General right-hand side b1 = q of system sl at a node, in the precision of the kernel.
template <typename R>
__device__ __forceinline__ cx<R> q_at(const GroupDev& G, int sl, long long node) {
  const long long e = (long long)sl * G.n + node;
  if (G.q_double) return to_c(((const double2*)G.q)[e], R(0));
  return to_c(((const float2*)G.q)[e], R(0));
}

// z-axis coefficients of plane k from the per-call table (no FP64 division per node-plane on the
// narrow FP64 pipe), or computed when the call built no table.
__device__ __forceinline__ const float2* ztab_of(const GroupDev& G, float) { return G.ztab; }
__device__ __forceinline__ const double2* ztab_of(const GroupDev& G, double) { return G.ztab64; }

template <typename R, bool CONJ>
__device__ __forceinline__ ZCoef<R> z_lookup(const GroupDev& G, int k) {
  const cx<R>* t = ztab_of(G, R(0));
  if (!t) return z_coef<R, CONJ>(G, k);
  t += (CONJ ? 3 * G.nz : 0) + 3 * k;
  ZCoef<R> c;
  c.sz = __ldg(t);
  c.izm = __ldg(t + 1);
  c.izp = __ldg(t + 2);
  return c;
}

// Receiver nodes in the normal-residual norms ||S^H r||^2.  At a receiver node of system sl the
// finalizer adds lambda P^T r2 to the stencil value A^H r1 and accounts |s|^2 of the sum itself,
// so the stencil passes leave those nodes out of their partial sums.  (Summing |A^H r1|^2 over
// every node and correcting by |s|^2 - |A^H r1|^2 afterwards cancels catastrophically near
// convergence, where A^H r1 and -lambda P^T r2 are large and nearly equal at the receivers: the
// norm of a converged complex128 solve came out as exactly 0.)
// Bits of the thread's 32-node row segment (x0 .. x0+31, row j) that hold a receiver at any z ...
__device__ __forceinline__ uint32_t rec_col_bits(const GroupDev& G, int sl, int j, int x0) {
  if (!G.rmask) return 0u;
  return __ldg(G.rcol + ((long long)sl * G.ny + j) * G.tiles_x + (x0 >> 5));
}
// ... and at plane k
__device__ __forceinline__ uint32_t rec_plane_bits(const GroupDev& G, int sl, int k, int j, int x0) {
  return __ldg(G.rmask + (((long long)sl * G.nz + k) * G.ny + j) * G.tiles_x + (x0 >> 5));
}

// First/last node index of an axis whose own stretch and both half-point stretches are 1.
__device__ __forceinline__ void interior_range(const AxisPml& a, int& lo, int& hi) {
  if (a.npml > 0) {
    lo = a.npml + 1;
    hi = a.n - 2 - a.npml;
  } else {
    lo = 0;
    hi = a.n - 1;
  }
}

// (A u) at one node with the general (stretched) coefficients.
template <typename R, bool CONJ>
__device__ __forceinline__ cx<R> stencil_general(const GroupDev& G, const XYCoef<R>& c, const ZCoef<R>& z,
                                                 R om2m, cx<R> u, cx<R> uxm, cx<R> uxp, cx<R> uym,
                                                 cx<R> uyp, cx<R> uzm, cx<R> uzp) {
  const cx<R> syz = c.sy * z.sz;
  const cx<R> sxz = c.sx * z.sz;
  const cx<R> w = c.sxy * z.sz;
  const cx<R> lx = c.ixp * (uxp - u) - c.ixm * (u - uxm);
  const cx<R> ly = c.iyp * (uyp - u) - c.iym * (u - uym);
  const cx<R> lz = z.izp * (uzp - u) - z.izm * (u - uzm);
  return om2m * (w * u) + syz * lx + sxz * ly + c.sxy * lz;
}

// (A u) at one node when only the axes flagged XP, YP, ZP are stretched; the others have
// s = 1 and real coefficients 1/h^2.  Same value as stencil_general, written as
//   A u = s_z (s_y Lx + s_x Ly) + s_x s_y (Lz + omega^2 m s_z u),
//   L_a = c_a(+1/2) (u_next - u) - c_a(-1/2) (u - u_prev),  c_a = 1/(s_a(half) h^2).
template <bool XP, bool YP, bool ZP, typename R>
__device__ __forceinline__ cx<R> stencil_axes(R ih2, R om2m, cx<R> u, cx<R> uxm, cx<R> uxp, cx<R> uym, cx<R> uyp,
                                              cx<R> uzm, cx<R> uzp, cx<R> sx, cx<R> ixm, cx<R> ixp, cx<R> sy,
                                              cx<R> iym, cx<R> iyp, cx<R> sz, cx<R> izm, cx<R> izp) {
  cx<R> lx, ly, lz;
  if (XP) lx = ixp * (uxp - u) - ixm * (u - uxm);
  else lx = ih2 * ((uxp + uxm) - R(2) * u);
  if (YP) ly = iyp * (uyp - u) - iym * (u - uym);
  else ly = ih2 * ((uyp + uym) - R(2) * u);
  if (ZP) lz = izp * (uzp - u) - izm * (u - uzm);
  else lz = ih2 * ((uzp + uzm) - R(2) * u);
  const cx<R> a = (YP ? sy * lx : lx) + (XP ? sx * ly : ly);
  const cx<R> zu = ZP ? sz * u : u;
  const cx<R> b = lz + om2m * zu;
  const cx<R> za = ZP ? sz * a : a;
  cx<R> bb = b;
  if (XP && YP) bb = (sx * sy) * b;
  else if (XP) bb = sx * b;
  else if (YP) bb = sy * b;
  return za + bb;
}

// Dispatch of stencil_axes on the stretched axes var = 4 x + 2 y + z (var = 0: every factor is
// 1, the plain 7-point formula).
template <typename R>
__device__ __forceinline__ cx<R> stencil_var(int var, R ih2, R om2m, cx<R> u, cx<R> uxm, cx<R> uxp, cx<R> uym,
                                             cx<R> uyp, cx<R> uzm, cx<R> uzp, const XYCoef<R>& c, const ZCoef<R>& z) {
#define WRI_VAR(X_, Y_, Z_) \
  return stencil_axes<X_, Y_, Z_>(ih2, om2m, u, uxm, uxp, uym, uyp, uzm, uzp, c.sx, c.ixm, c.ixp, c.sy, c.iym, c.iyp, \
                                  z.sz, z.izm, z.izp);
  switch (var) {
    case 1: WRI_VAR(false, false, true)
    case 2: WRI_VAR(false, true, false)
    case 3: WRI_VAR(false, true, true)
    case 4: WRI_VAR(true, false, false)
    case 5: WRI_VAR(true, false, true)
    case 6: WRI_VAR(true, true, false)
    case 7: WRI_VAR(true, true, true)
    default: WRI_VAR(false, false, false)
  }
#undef WRI_VAR
}

// (A u) at one node in the interior (all stretch factors 1): omega^2 m u + Laplacian.
template <typename R>
__device__ __forceinline__ cx<R> stencil_interior(R ih2, R om2m, cx<R> u, cx<R> uxm, cx<R> uxp, cx<R> uym,
                                                  cx<R> uyp, cx<R> uzm, cx<R> uzp) {
  const cx<R> sum = (uxm + uxp) + (uym + uyp) + (uzm + uzp);
  return mkc(om2m * u.x + ih2 * (sum.x - R(6) * u.x), om2m * u.y + ih2 * (sum.y - R(6) * u.y));
}

// (A F)[node] (CONJ = false) or (A^H F)[node] (CONJ = true) at one node of a system's field F,
// with the general coefficients (7 loads, Dirichlet outside the grid).
template <typename R, bool CONJ>
__device__ cx<R> stencil_at(const GroupDev& G, const cx<R>* F, long long node) {
  const long long plane = (long long)G.nx * G.ny;
  const int k = (int)(node / plane);
  const long long rem = node - (long long)k * plane;
  const int j = (int)(rem / G.nx);
  const int i = (int)(rem - (long long)j * G.nx);
  auto at = [&](int ii, int jj, int kk) -> cx<R> {
    if (ii < 0 || jj < 0 || kk < 0 || ii >= G.nx || jj >= G.ny || kk >= G.nz) return czero<R>();
    return F[(long long)kk * plane + (long long)jj * G.nx + ii];
  };
  const XYCoef<R> c = xy_coef<R, CONJ>(G, i, j);
  const ZCoef<R> z = z_coef<R, CONJ>(G, k);
  const R om2m = pick<R>(G.omega * G.omega, G.om2f) * model_at<R>(G.m, G.m_double, node);
  return stencil_general<R, CONJ>(G, c, z, om2m, at(i, j, k), at(i - 1, j, k), at(i + 1, j, k), at(i, j - 1, k),
                                  at(i, j + 1, k), at(i, j, k - 1), at(i, j, k + 1));
}

}  // namespace wri
