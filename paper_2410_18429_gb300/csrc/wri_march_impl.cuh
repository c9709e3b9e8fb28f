// Kernel template of the z-march (see wri_march.cuh for the design) and the
// per-system finalizers that run in the CTA completing a system's last tile.
#pragma once

#include <math.h>

#include "../../include/wri.h"
#include "wri_march.cuh"

namespace wri {

template <typename R>
__device__ __forceinline__ cx<R> ldg_c(const cx<R>* p) {
  return __ldg(p);
}

// ------------------------------------------------------------------ finalizers
// Run by every thread of the CTA that completed the last tile of system `sd`.
// NT is the number of threads that run it (the whole CTA, any 2-D shape, or the first NT
// threads of a 1-D CTA with SYNC = FirstThreadsSync<NT>).
template <typename R, typename OR, int MODE, int NT, typename SYNC = CtaSync>
__device__ void finalize(const Batch& b, const GroupDev& G, SysDev* sd, int sl, bool xonly, double* red,
                         double* bcast) {
  typedef cx<R> C;
  typedef cx<OR> OC;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  __threadfence();
  const long long off = (long long)sl * G.n;
  const int cur = sd->iter & 1;

  if (MODE == M_P1 && xonly) {
    if (tid == 0) {
      sd->state = ST_DONE;
      sd->ticket = 0u;
      atomicSub(b.remaining, 1);
    }
    return;
  }

  // partial sums of the tiles, in tile order
  double part = 0.0;
  if (MODE != M_RES) {
    const double* pp = b.partial + sd->part_off;
    for (int t = tid; t < G.ntiles; t += NT) part += __ldcg(pp + t);
  }
  part = block_sum<NT, SYNC>(part, red);

  // receiver terms
  const int rb = sd->rec_begin, re = sd->rec_end;
  const R lam = R(G.lambda);
  C* r2 = (C*)b.r2;
  double rec = 0.0;
  for (int k = rb + tid; k < re; k += NT) {
    const long long node = off + b.rec_idx[k];
    if (MODE == M_P1) {
      const C pn = ldcg_c((const C*)G.p[pslot(b, sd->iter)] + node);
      rec += (double)lam * (double)lam * (double)abs2(pn);
    } else if (MODE == M_SH && G.rmap) {
      // the receiver terms were added in the stencil pass (refinement): nothing left to do
    } else if (MODE == M_SH || MODE == M_P2) {
      OC* S = (OC*)G.s;
      const OC sv = ldcg_c(S + node);
      const C add = lam * r2[k];
      const OC sn = to_c(to_c(sv, R(0)) + add, OR(0));
      S[node] = sn;
      // the stencil pass left receiver nodes out of its partial sums (rec_col_bits)
      rec += (double)abs2(sn);
    } else if (MODE == M_RES) {
      const C xv = ldcg_c((const C*)G.x + node);
      r2[k] = ((const C*)b.lamd)[k] - lam * xv;
    }
  }
  rec = block_sum<NT, SYNC>(rec, red);

  if (tid == 0) {
    const double tot = part + rec;
    if (MODE == M_P1) {
      const double delta = tot;
      double alpha = 0.0;
      sd->delta = delta;
      if (!(delta > 0.0) || !isfinite(delta)) {
        sd->status = isfinite(delta) ? WRI_SYS_BREAKDOWN : WRI_SYS_NONFINITE;
        if (sd->iter % xsteps_of(b) != 0) {
          // grouped updates: steps of earlier iterations are still pending (this pass added none);
          // the step history is left as it is, newest = the previous iteration's, and the x-only
          // pass adds them
          sd->state = ST_FINISHING;
        } else {
          sd->state = ST_DONE;
          sd->alpha = 0.0;
          atomicSub(b.remaining, 1);
        }
      } else {
        alpha = sd->gamma / delta;
        sd->alpha_hist[2] = sd->alpha_hist[1];
        sd->alpha_hist[1] = sd->alpha_hist[0];
        sd->alpha_hist[0] = sd->alpha;
        sd->alpha = alpha;
      }
      *bcast = alpha;  // step of the receiver residual (none on breakdown)
    } else if (MODE == M_P2) {
      const double g = tot;
      const int it = sd->iter + 1;
      sd->iter = it;
      sd->iter_total += 1;
      const double rn = sqrt(g);
      sd->relres = sd->snorm_ref > 0.0 ? rn / sd->snorm_ref : 0.0;
      if (!isfinite(g)) {
        sd->status = WRI_SYS_NONFINITE;
        sd->state = ST_FINISHING;
      } else if (rn <= sd->tol * sd->snorm_ref) {
        sd->status = WRI_SYS_OK;
        sd->state = ST_FINISHING;
      } else if (it >= b.max_iter) {
        sd->status = WRI_SYS_MAXITER;
        sd->state = ST_FINISHING;
      } else {
        sd->beta = g / sd->gamma;
      }
      sd->gamma = g;
    } else if (MODE == M_SH) {
      const double g = tot;
      const double rn = sqrt(g);
      if (b.flavor == SH_PLAIN) {
        // S^H r64 of the refinement: output vector only, no scalar changes
      } else if (b.flavor == SH_REF) {
        sd->snorm_b = rn;
      } else if (b.flavor == SH_INIT || b.flavor == SH_WARM) {
        if (b.flavor == SH_INIT) sd->snorm_b = rn;
        sd->snorm_ref = sd->snorm_b;
        sd->gamma = g;
        sd->beta = 0.0;
        sd->alpha = 0.0;
        sd->alpha_hist[0] = sd->alpha_hist[1] = sd->alpha_hist[2] = 0.0;
        sd->iter = 0;
        sd->iter_total = 0;
        sd->tol = b.tol;
        sd->relres = sd->snorm_b > 0.0 ? rn / sd->snorm_b : 0.0;
        if (!isfinite(g)) {
          sd->status = WRI_SYS_NONFINITE;
          sd->state = ST_DONE;
        } else if (g == 0.0 || rn <= b.tol * sd->snorm_b) {
          sd->status = WRI_SYS_OK;
          sd->state = ST_DONE;
        } else {
          sd->status = WRI_SYS_OK;
          sd->state = ST_ACTIVE;
          atomicAdd(b.remaining, 1);
        }
      } else {  // SH_REFINE: outer step of the FP64 refinement
        if (b.outer == 0 && !b.warm) {
          sd->snorm_b = rn;
          sd->iter_total = 0;
        }
        const double rr = sd->snorm_b > 0.0 ? rn / sd->snorm_b : 0.0;
        sd->relres = rr;
        const bool bad = !isfinite(g) || sd->status == WRI_SYS_NONFINITE;
        if (bad) {
          sd->status = WRI_SYS_NONFINITE;
          sd->outer_done = 1;
          sd->state = ST_DONE;
        } else if (g == 0.0 || rr <= b.refine_tol) {
          sd->status = WRI_SYS_OK;
          sd->outer_done = 1;
          sd->state = ST_DONE;
        } else if (b.outer >= b.max_refine) {
          sd->status = WRI_SYS_MAXITER;
          sd->outer_done = 1;
          sd->state = ST_DONE;
        } else {
          sd->status = WRI_SYS_OK;
          sd->gamma = g;
          sd->snorm_ref = rn;
          // the correction needs no more accuracy than the outer target asks for, with 5 % of
          // margin for the drift between the FP32 recurrence and the FP64 residual (measured about
          // 0.5 % at 1e-2): a tighter inner tolerance would only add iterations, and CGLS's normal
          // residual can stall for thousands of iterations just below a target
          sd->tol = fmax(b.inner_tol, 0.95 * b.refine_tol * sd->snorm_b / rn);
          sd->beta = 0.0;
          sd->alpha = 0.0;
          sd->alpha_hist[0] = sd->alpha_hist[1] = sd->alpha_hist[2] = 0.0;
          sd->iter = 0;
          sd->state = ST_ACTIVE;
          atomicAdd(b.remaining, 1);
        }
      }
    }
    sd->ticket = 0u;
  }
  if (MODE == M_P1) {
    SYNC::sync();
    const double a = *bcast;
    if (a != 0.0) {
      for (int k = rb + tid; k < re; k += NT) {
        const long long node = off + b.rec_idx[k];
        const C pn = ldcg_c((const C*)G.p[pslot(b, sd->iter)] + node);
        r2[k] = r2[k] - R(a * (double)lam) * pn;
      }
    }
  }
}

// ------------------------------------------------------------------ the kernel
template <typename R, typename OR, int MODE, bool CONJ, int BY>
__global__ void __launch_bounds__(WRI_TX * BY) k_march(const __grid_constant__ Batch b) {
  typedef cx<R> C;
  typedef cx<OR> OC;
  constexpr int NT = WRI_TX * BY;
  constexpr int RING = 2 * WRI_TX + 2 * BY;
  constexpr int GZ = grad_zc(BY);  // z-chunk of the gradient kernel
  __shared__ C buf[2][BY + 2][WRI_TX + 2];
  __shared__ double red[NT / 32];
  __shared__ double bcast;
  __shared__ int s_last;
  __shared__ double gacc[MODE == M_GRAD ? GZ : 1][BY][WRI_TX];

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * WRI_TX + tx;

  for (long long item = blockIdx.x; item < b.nitems; item += gridDim.x) {
    const int gi = find_group(b, item);
    const GroupDev& G = b.g[gi];
    const long long local = item - G.item0;
    int sl0, tile;
    if (MODE == M_GRAD) {
      sl0 = 0;
      tile = (int)local;
    } else {
      sl0 = (int)(local % G.nsys);
      tile = (int)(local / G.nsys);
    }
    SysDev* sd = (MODE == M_APPLY) ? nullptr : b.sys + (G.sys0 + sl0);

    // ---- what this item does (uniform across the CTA)
    int state = ST_ACTIVE;
    if (MODE == M_P1 || MODE == M_P2) state = sd->state;
    bool skip = false;
    if (MODE == M_P1) skip = (state == ST_DONE);
    if (MODE == M_P2) skip = (state != ST_ACTIVE);
    if ((MODE == M_SH || MODE == M_RES) && (b.flavor == SH_REFINE || b.flavor == SH_PLAIN))
      skip = sd->outer_done != 0;
    if (skip) continue;
    const bool xonly = (MODE == M_P1 && state == ST_FINISHING);

    // ---- tile geometry
    const int nx = G.nx, ny = G.ny, nz = G.nz;
    const int tzi = tile % G.zsplit;
    const int txy = tile / G.zsplit;
    const int x0 = (txy % G.tiles_x) * WRI_TX;
    const int y0 = (txy / G.tiles_x) * BY;
    const int z0 = tzi * G.zc;
    const int z1 = min(z0 + G.zc, nz);
    const int i = x0 + tx, j = y0 + ty;
    const bool own = (i < nx) && (j < ny);
    const long long plane = (long long)nx * ny;
    const long long col = (long long)j * nx + i;

    double accd = 0.0;   // FP64 accumulator of the tile's reduction
    double facc = 0.0;   // gradient: objective contribution

    if (xonly) {
      // the system converged in the last phase 2: apply the pending x += alpha p
      const long long off = (long long)sl0 * G.n;
      C* X = (C*)G.x + off;
      const C* Pc = (const C*)G.p[sd->iter & 1] + off;
      const R a = R(sd->alpha);
      if (own)
        for (int k = z0; k < z1; ++k) {
          const long long node = k * plane + col;
          X[node] = X[node] + a * ldg_c<R>(Pc + node);
        }
    } else {
      // ---- coefficients of this thread's column
      const XYCoef<R> cxy = xy_coef<R, CONJ>(G, min(i, nx - 1), min(j, ny - 1));
      int xlo, xhi, ylo, yhi, zlo, zhi;
      interior_range(G.ax, xlo, xhi);
      interior_range(G.ay, ylo, yhi);
      interior_range(G.az, zlo, zhi);
      // stretched axes of this tile (bit 2: x, bit 1: y); bit 0 (z) is set per plane
      const int xyvar = (((x0 >= xlo) && (min(x0 + WRI_TX, nx) - 1 <= xhi)) ? 0 : 4) |
                        (((y0 >= ylo) && (min(y0 + BY, ny) - 1 <= yhi)) ? 0 : 2);
      const R om2 = pick<R>(G.omega * G.omega, G.om2f);
      const R ih2 = inv_h2<R>(G);

      if (MODE == M_GRAD) {
        for (int e = tid; e < GZ * BY * WRI_TX; e += NT) (&gacc[0][0][0])[e] = 0.0;
      }
      const int nsl = (MODE == M_GRAD) ? G.nsys : 1;
      for (int sl = sl0; sl < sl0 + nsl; ++sl) {
        const long long off = (long long)sl * G.n;
        SysDev* sdl = (MODE == M_APPLY) ? nullptr : b.sys + (G.sys0 + sl);
        const long long src = (MODE == M_APPLY) ? -1 : sdl->src;
        const int cur = (MODE == M_P1 || MODE == M_P2) ? (sd->iter & 1) : 0;
        // receivers of this system in this thread's column (left out of the norm, rec_col_bits)
        const uint32_t rcb = ((MODE == M_P2 || (MODE == M_SH && !G.rmap)) && own)
                                 ? (rec_col_bits(G, sl, j, x0) >> tx) & 1u : 0u;

        // field F = Fa + coef * Fb, or the right-hand side b1 (cold start): the point field alpha e,
        // 0 (source-free) or the general right-hand side q
        const bool point = (MODE == M_SH) && (b.flavor == SH_INIT || b.flavor == SH_REF);
        C pval = czero<R>();
        if (point && G.alpha) pval = mkc(R(G.alpha[2 * sl]), R(G.alpha[2 * sl + 1]));
        auto b1_at = [&](long long node) -> C {
          if (G.q) return q_at<R>(G, sl, node);
          return (node == src) ? pval : czero<R>();
        };
        const C* Fa = nullptr;
        const C* Fb = nullptr;
        C* Fst = nullptr;
        C* X = nullptr;
        R coef = R(0), xal = R(0);
        if (MODE == M_APPLY || MODE == M_RES || MODE == M_GRAD) {
          Fa = (const C*)G.x + off;
        } else if (MODE == M_SH) {
          if (!point) Fa = (const C*)G.r1[0] + off;
          else Fst = (C*)G.r1[0] + off;
          if (b.flavor == SH_INIT) X = (C*)G.x + off;
        } else if (MODE == M_P1) {
          Fa = (const C*)G.s + off;
          if (sd->iter > 0) Fb = (const C*)G.p[cur] + off;
          coef = R(sd->beta);
          xal = R(sd->alpha);
          Fst = (C*)G.p[cur ^ 1] + off;
          X = (C*)G.x + off;
        } else if (MODE == M_P2) {
          Fa = (const C*)G.r1[cur] + off;
          Fb = (const C*)G.t1 + off;
          coef = -R(sd->alpha);
          Fst = (C*)G.r1[cur ^ 1] + off;
        }
        C a_src = czero<R>();
        if ((MODE == M_RES || MODE == M_GRAD) && G.alpha) a_src = mkc(R(G.alpha[2 * sl]), R(G.alpha[2 * sl + 1]));

        // F at any node (no side effects)
        auto fieldF = [&](long long node) -> C {
          if (point) return b1_at(node);
          C v = ldg_c<R>(Fa + node);
          if (Fb) v = v + coef * ldg_c<R>(Fb + node);
          return v;
        };
        // F at the thread's own node of plane kk, with the stores of the fused vector update
        auto ownF = [&](int kk) -> C {
          if (kk < 0 || kk >= nz || !own) return czero<R>();
          const long long node = kk * plane + col;
          const bool mine = (kk >= z0) && (kk < z1);
          if (point) {
            const C v = b1_at(node);
            if (mine) {
              Fst[node] = v;
              if (X) X[node] = czero<R>();
            }
            return v;
          }
          C v = ldg_c<R>(Fa + node);
          if (Fb) {
            const C o = ldg_c<R>(Fb + node);
            v = v + coef * o;
            if (MODE == M_P1 && mine) X[node] = X[node] + xal * o;
          }
          if (Fst && mine) Fst[node] = v;
          return v;
        };
        auto ring_node = [&](int e, int& rx, int& ry, int& si, int& sj) {
          if (e < WRI_TX) { rx = x0 + e; ry = y0 - 1; si = e + 1; sj = 0; }
          else if (e < 2 * WRI_TX) { rx = x0 + e - WRI_TX; ry = y0 + BY; si = e - WRI_TX + 1; sj = BY + 1; }
          else if (e < 2 * WRI_TX + BY) { rx = x0 - 1; ry = y0 + e - 2 * WRI_TX; si = 0; sj = ry - y0 + 1; }
          else { rx = x0 + WRI_TX; ry = y0 + e - 2 * WRI_TX - BY; si = WRI_TX + 1; sj = ry - y0 + 1; }
        };
        auto load_ring = [&](int kk, int slot) {
          for (int e = tid; e < RING; e += NT) {
            int rx, ry, si, sj;
            ring_node(e, rx, ry, si, sj);
            C v = czero<R>();
            if (kk >= 0 && kk < nz && rx >= 0 && rx < nx && ry >= 0 && ry < ny)
              v = fieldF(kk * plane + (long long)ry * nx + rx);
            buf[slot][sj][si] = v;
          }
        };

        // ---- prologue
        __syncthreads();  // previous item / system done with buf
        C Fm = ownF(z0 - 1);
        C Fc = ownF(z0);
        C Fp = (z0 + 1 <= z1) ? ownF(z0 + 1) : czero<R>();
        buf[0][ty + 1][tx + 1] = Fc;
        load_ring(z0, 0);
        float accf = 0.f;

        for (int k = z0; k < z1; ++k) {
          const int cb = (k - z0) & 1;
          __syncthreads();
          // issue the loads of the next planes early
          const C Fn = (k + 2 <= z1) ? ownF(k + 2) : czero<R>();
          // stencil at (i, j, k)
          const C u = Fc;
          const C uxm = buf[cb][ty + 1][tx];
          const C uxp = buf[cb][ty + 1][tx + 2];
          const C uym = buf[cb][ty][tx + 1];
          const C uyp = buf[cb][ty + 2][tx + 1];
          const long long node = k * plane + col;
          const R om2m = own ? om2 * model_at<R>(G.m, G.m_double, node) : R(0);
          C AF;
          ZCoef<R> zc;
          const int var = xyvar | ((k >= zlo && k <= zhi) ? 0 : 1);
          const bool fast = var == 0;
          if (fast) {
            AF = stencil_interior<R>(ih2, om2m, u, uxm, uxp, uym, uyp, Fm, Fp);
          } else {
            // only the stretched axes take complex coefficients (stencil_axes)
            zc = z_lookup<R, CONJ>(G, k);
            AF = stencil_var<R>(var, ih2, om2m, u, uxm, uxp, uym, uyp, Fm, Fp, cxy, zc);
          }
          if (own) {
            const long long gnode = off + node;
            if (MODE == M_APPLY) {
              ((OC*)G.s)[gnode] = to_c(AF, OR(0));
            } else if (MODE == M_SH) {
              if (G.rmap) {
                // FP64 normal residual of the refinement: near convergence A^H F and lambda P^T r2
                // nearly cancel at a receiver, so they are added here, before the one rounding and
                // before the norm
                const int rk = G.rmap[gnode];
                if (rk >= 0) AF = AF + R(G.lambda) * ((const C*)b.r2)[rk];
              }
              ((OC*)G.s)[gnode] = to_c(AF, OR(0));
              if (!(rcb && ((rec_plane_bits(G, sl, k, j, x0) >> tx) & 1u))) {
                if (sizeof(R) == 4) accf += (float)abs2(AF);
                else accd += (double)abs2(AF);
              }
            } else if (MODE == M_RES) {
              C r = czero<R>() - AF;
              if (G.q) r = q_at<R>(G, sl, node) - AF;
              else if (node == src) r = G.masked ? czero<R>() : a_src - AF;
              ((C*)G.r1[0])[gnode] = r;
            } else if (MODE == M_P1) {
              const C t = (G.masked && node == src) ? czero<R>() : AF;
              ((C*)G.t1)[gnode] = t;
              if (sizeof(R) == 4) accf += (float)abs2(t);
              else accd += (double)abs2(t);
            } else if (MODE == M_P2) {
              // refinement inner solve: s = S^H r + S^H r64, the normal residual of the correction
              // system S^H S dx = S^H f - g with g = -S^H r64
              if (G.gvec) AF = AF + to_c(((const float2*)G.gvec)[gnode], R(0));
              ((C*)G.s)[gnode] = AF;
              if (!(rcb && ((rec_plane_bits(G, sl, k, j, x0) >> tx) & 1u))) {
                if (sizeof(R) == 4) accf += (float)abs2(AF);
                else accd += (double)abs2(AF);
              }
            } else if (MODE == M_GRAD) {
              C r = AF;
              if (G.q) r = r - q_at<R>(G, sl, node);
              else if (node == src) r = r - a_src;
              if (fast) {
                gacc[k - z0][ty][tx] += (double)(om2 * (u.x * r.x + u.y * r.y));
              } else {
                const C w = cxy.sxy * zc.sz;
                const C wu = w * u;
                gacc[k - z0][ty][tx] += (double)(om2 * (wu.x * r.x + wu.y * r.y));
              }
              facc += 0.5 * (double)abs2(r);
            }
          }
          if (sizeof(R) == 4 && ((k - z0) & 7) == 7) {
            accd += (double)accf;
            accf = 0.f;
          }
          // next plane into the other buffer
          buf[cb ^ 1][ty + 1][tx + 1] = Fp;
          if (k + 1 < z1) load_ring(k + 1, cb ^ 1);
          Fm = Fc;
          Fc = Fp;
          Fp = Fn;
        }
        accd += (double)accf;
      }  // systems (gradient) / single system

      if (MODE == M_GRAD) {
        __syncthreads();
        if (own)
          for (int k = z0; k < z1; ++k) {
            const long long node = k * plane + col;
            G.grad[node] += gacc[k - z0][ty][tx];
          }
        const double fs = block_sum<NT>(facc, red);
        if (tid == 0 && fs != 0.0) atomicAdd(b.f, fs);
      }
    }

    if (MODE == M_APPLY || MODE == M_GRAD) continue;

    // ---- tile partial, ticket, and the system's finalizer
    const double tsum = block_sum<NT>(accd, red);
    if (tid == 0 && MODE != M_RES && !xonly) b.partial[sd->part_off + tile] = tsum;
    __threadfence();
    __syncthreads();
    if (tid == 0) {
      const unsigned t = atomicAdd(&sd->ticket, 1u);
      s_last = (t == (unsigned)(G.ntiles - 1));
    }
    __syncthreads();
    if (s_last) finalize<R, OR, MODE, WRI_TX * BY>(b, G, sd, sl0, xonly, red, &bcast);
  }
}

}  // namespace wri
