// TMA-pipelined CGLS phases (complex64 stencil, FP64 reductions) for sm_103a.
//
// Same work decomposition and finalizers as the z-march of wri_march_impl.cuh, but the
// planes of every input vector stream through a ring of S shared-memory stages filled
// by cp.async.bulk.tensor (TMA) copies:
//   * a halo'd field (the two vectors that form F) is copied as a 36 x (BY+2) box that
//     starts at x0-2 (16-byte aligned) and y0-1; out-of-grid elements arrive as zeros,
//     which is the Dirichlet boundary of the operator;
//   * the iterate x and the model m are copied as 32 x BY boxes;
//   * one thread arms an mbarrier per stage with the expected byte count and issues the
//     copies S planes ahead, so every CTA keeps S planes of all its inputs in flight
//     independently of its registers and warps.
// The consumers form F = a + c b on the halo'd tile into a ring of 4 F planes (own
// nodes stored as the updated CG vector), then apply the stencil one plane behind.
// Every mbarrier wait is bounded (2 s of the global timer): on time-out the CTA records an error
// flag, drains its own copies (again bounded) and stops.
#pragma once

#include <cuda.h>

#include "wri_march_impl.cuh"

namespace wri {

// halo boxes of s, t1, r1 and of the p slots; 32 x BY boxes of x and (grouped iterate updates) of
// the p slots; the model
enum TmaMap : int {
  TM_S = 0, TM_X, TM_T1, TM_R0, TM_R1, TM_M,
  TM_P0, TM_P1, TM_P2, TM_P3,
  TM_PC0, TM_PC1, TM_PC2, TM_PC3,
  TM_COUNT
};

struct TmaSet {
  CUtensorMap map[WRI_MAXG][TM_COUNT];
  int* err;                // set to 1 by a CTA whose copy wait timed out
  unsigned long long wait_ns;  // time limit of every copy-pipeline wait (global timer, ns)
  int withhold;            // test hook, -1 = off: the copy warp of CTA 0 never issues its fill of this
                           // index, so the consumers' wait for it runs out (the bounded-wait path)
  int pad_;
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Default time limit of every wait of the copy pipelines (TmaSet::wait_ns): only a copy that
// never completes (a broken descriptor or protocol, or the withheld fill of the test hook) can
// reach it.
constexpr uint64_t kWaitLimitNs = 2000000000ull;

// bounded wait: false after `limit` ns of polling (or 2^26 polls, whichever comes first)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit) {
  const uint64_t t0 = global_ns();
  for (int i = 0; i < (1 << 26); ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 255) == 255 && global_ns() - t0 > limit) return false;
  }
  return false;
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int x, int y, int z, int w,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5}], [%6];" ::"r"(smem_addr(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_addr(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
      : "memory");
}

// Shared-memory layout of one CTA.  Every TMA destination starts on a 128-byte boundary
// (the bulk tensor copy requires it): each box is padded to a multiple of 128 bytes and
// the dynamic region is re-aligned at run time (bytes() includes 128 bytes of slack).
template <int MODE, int BY>
struct TmaLayout {
  static constexpr int HW = WRI_TX + 4;  // halo box width: x0-2 .. x0+33
  static constexpr int HH = BY + 2;      // halo box height: y0-1 .. y0+BY
  static constexpr int FW = WRI_TX + 2;  // F tile width: x0-1 .. x0+32
  static constexpr int pad(int v) { return (v + 127) / 128 * 128; }
  static constexpr int HALO = HW * HH * 8;     // bytes copied per halo box
  static constexpr int CTR = WRI_TX * BY * 8;  // bytes copied per 32 x BY complex box
  static constexpr int MB = WRI_TX * BY * 4;   // bytes copied per 32 x BY float box
  static constexpr int OFF_B = pad(HALO);
  static constexpr int OFF_X = OFF_B + pad(HALO);
  static constexpr int OFF_M = OFF_X + (MODE == M_P1 ? pad(CTR) : 0);
  static constexpr int STAGE = OFF_M + pad(MB);
  static constexpr int FRING = 4 * HH * FW * 8;
  static size_t bytes(int S) { return 128 + (size_t)S * STAGE + FRING + 8 * S; }
};

// Neumaier-compensated FP32 accumulation of non-negative terms: the per-thread part of
// the FP64 reductions, kept in FP32 because GB300's FP64 pipe is narrow.
struct CompSum {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float t = s + v;
    c += (s >= v) ? ((s - t) + v) : ((v - t) + s);
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

template <int MODE, int BY, int S, int MINB>
__global__ void __launch_bounds__(WRI_TX* BY, MINB) k_phase_tma(const __grid_constant__ Batch b,
                                                                const __grid_constant__ TmaSet T) {
  static_assert(MODE == M_P1 || MODE == M_P2, "TMA path covers the two CGLS phases");
  typedef float2 C;
  typedef TmaLayout<MODE, BY> L;
  constexpr bool CONJ = (MODE == M_P2);
  constexpr int NT = WRI_TX * BY;
  constexpr int RING = 2 * WRI_TX + 2 * BY;
  static_assert(RING <= NT, "one halo-ring element per thread");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ double red[NT / 32];
  __shared__ double bcast;
  __shared__ int s_last;
  __shared__ int s_abort;
  unsigned char* smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
  C* Fbase = reinterpret_cast<C*>(smem + (size_t)S * L::STAGE);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + (size_t)S * L::STAGE + L::FRING);
  constexpr int FPL = L::HH * L::FW;  // elements of one F plane

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * WRI_TX + tx;
  // self-check of the copy destinations (uniform): never issue a misaligned bulk copy
  if ((smem_addr(smem) & 127u) != 0u || (L::OFF_B & 127) || (L::OFF_X & 127) || (L::OFF_M & 127) ||
      (L::STAGE & 127)) {
    if (tid == 0) atomicExch(T.err, 2);
    return;
  }
  // this thread's halo-ring element (fixed for the whole kernel); the RING elements are
  // dealt round-robin over the warps so every warp carries the same share
  constexpr int NW = NT / 32;
  static_assert((RING + NW - 1) / NW <= 32, "ring share fits a warp");
  const int r_e = (tid & 31) * NW + (tid >> 5);
  const bool has_ring = r_e < RING;
  int r_si = 0, r_sj = 0;
  if (r_e < WRI_TX) { r_si = r_e + 1; r_sj = 0; }
  else if (r_e < 2 * WRI_TX) { r_si = r_e - WRI_TX + 1; r_sj = BY + 1; }
  else if (r_e < 2 * WRI_TX + BY) { r_si = 0; r_sj = r_e - 2 * WRI_TX + 1; }
  else { r_si = WRI_TX + 1; r_sj = r_e - 2 * WRI_TX - BY + 1; }
  const int r_raw = r_sj * L::HW + r_si + 1;   // element in a halo box
  const int r_f = r_sj * L::FW + r_si;         // element in an F plane
  const int o_raw = (ty + 1) * L::HW + tx + 2;  // own node in a halo box
  const int o_f = (ty + 1) * L::FW + tx + 1;    // own node in an F plane
  const int o_ctr = ty * WRI_TX + tx;           // own node in a 32 x BY box

  if (tid == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&bar[s], 1);
    s_abort = 0;
  }
  __syncthreads();
  unsigned uses = 0;  // stage uses so far (uniform across the CTA)

  for (long long item = blockIdx.x; item < b.nitems; item += gridDim.x) {
    const int gi = find_group(b, item);
    const GroupDev& G = b.g[gi];
    const long long local = item - G.item0;
    int sl, tile;
    item_coords(b, G, local, sl, tile);
    SysDev* sd = b.sys + (G.sys0 + sl);
    const int state = sd->state;
    if (MODE == M_P1 ? (state == ST_DONE) : (state != ST_ACTIVE)) continue;
    const bool xonly = (MODE == M_P1 && state == ST_FINISHING);

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
    const long long off = (long long)sl * G.n;
    const int iter = sd->iter;
    const int cur = iter & 1;
    double accd = 0.0;

    if (xonly) {
      C* X = (C*)G.x + off + col;
      const C* Pc = (const C*)G.p[cur] + off + col;
      const float a = (float)sd->alpha;
      if (own)
        for (int k = z0; k < z1; ++k) {
          const long long o = k * plane;
          X[o] = X[o] + a * __ldg(Pc + o);
        }
    } else {
      const CUtensorMap* mapA = &T.map[gi][MODE == M_P1 ? TM_S : (cur ? TM_R1 : TM_R0)];
      const bool hasB = (MODE == M_P2) || iter > 0;
      const CUtensorMap* mapB = &T.map[gi][MODE == M_P1 ? (cur ? TM_P1 : TM_P0) : TM_T1];
      const bool hasX = (MODE == M_P1) && iter > 0;
      const CUtensorMap* mapX = &T.map[gi][TM_X];
      const CUtensorMap* mapM = &T.map[gi][TM_M];
      const uint32_t tx_bytes = L::HALO + (hasB ? L::HALO : 0) + (hasX ? L::CTR : 0) + L::MB;
      const float coef = (MODE == M_P1) ? (float)sd->beta : -(float)sd->alpha;
      const float xal = (float)sd->alpha;
      // own-node pointers (plane offsets are added in the loop)
      C* pF = ((MODE == M_P1) ? (C*)G.p[cur ^ 1] : (C*)G.r1[cur ^ 1]) + off + col;
      C* pX = (C*)G.x + off + col;
      C* pO = ((MODE == M_P1) ? (C*)G.t1 : (C*)G.s) + off + col;
      // the masked source node as (plane, column) of this system, or none
      int src_k = -1;
      long long src_col = -1;
      if (MODE == M_P1 && G.masked) {
        src_k = (int)(sd->src / plane);
        src_col = sd->src - (long long)src_k * plane;
      }
      const bool own_src_col = (src_col == col);
      // receivers of this system in the thread's column: left out of the phase-2 norm
      const uint32_t rcb = (MODE == M_P2 && own) ? (rec_col_bits(G, sl, j, x0) >> tx) & 1u : 0u;
      const int count = z1 - z0 + 2;  // planes z0-1 .. z1

      auto issue = [&](int q) {
        const int st = (int)((uses + q) % S);
        unsigned char* base = smem + (size_t)st * L::STAGE;
        const int kq = z0 - 1 + q;
        mbar_expect_tx(&bar[st], tx_bytes);
        tma_load_4d(base, mapA, x0 - 2, y0 - 1, kq, sl, &bar[st]);
        if (hasB) tma_load_4d(base + L::OFF_B, mapB, x0 - 2, y0 - 1, kq, sl, &bar[st]);
        if (hasX) tma_load_4d(base + L::OFF_X, mapX, x0, y0, kq, sl, &bar[st]);
        tma_load_3d(base + L::OFF_M, mapM, x0, y0, kq, &bar[st]);
      };

      const XYCoef<float> cxy = xy_coef<float, CONJ>(G, min(i, nx - 1), min(j, ny - 1));
      int xlo, xhi, ylo, yhi, zlo, zhi;
      interior_range(G.ax, xlo, xhi);
      interior_range(G.ay, ylo, yhi);
      interior_range(G.az, zlo, zhi);
      const bool xy_int =
          (x0 >= xlo) && (min(x0 + WRI_TX, nx) - 1 <= xhi) && (y0 >= ylo) && (min(y0 + BY, ny) - 1 <= yhi);
      const float om2 = G.om2f;
      const float ih2 = G.ih2f;
      const float2* ztab = G.ztab + (CONJ ? 3 * nz : 0);

      __syncthreads();  // the previous item no longer reads the stages, the F ring or zring
      if (tid == 0)
        for (int q = 0; q < S && q < count; ++q) issue(q);

      CompSum acc;
      float m_prev = 0.f;
      int issued = min(S, count);
      int q_fail = -1;
      long long po = (long long)(z0 - 1) * plane;  // offset of plane kq
      for (int q = 0; q < count; ++q, po += plane) {
        const int st = (int)((uses + q) % S);
        const uint32_t par = ((uses + q) / S) & 1u;
        // every thread waits for the stage itself; a time-out is made uniform at the
        // plane barrier below (the F values of a failed plane are never used)
        if (!mbar_wait(&bar[st], par, T.wait_ns)) s_abort = 1;
        const unsigned char* base = smem + (size_t)st * L::STAGE;
        const C* A = reinterpret_cast<const C*>(base);
        const C* B = reinterpret_cast<const C*>(base + L::OFF_B);
        const C* XT = reinterpret_cast<const C*>(base + L::OFF_X);
        const float* MT = reinterpret_cast<const float*>(base + L::OFF_M);
        const int kq = z0 - 1 + q;
        C* Fq = Fbase + (q & 3) * FPL;
        const bool mine = own && kq >= z0 && kq < z1;
        // F on the own node (stored as the updated CG vector on own planes)
        {
          const C a = A[o_raw];
          C v = a;
          if (hasB) {
            const C bb = B[o_raw];
            v = a + coef * bb;
            if (MODE == M_P1 && mine) pX[po] = XT[o_ctr] + xal * bb;
          }
          Fq[o_f] = v;
          if (mine) pF[po] = v;
        }
        const float m_new = MT[o_ctr];
        // F on this thread's halo-ring element (zeros outside the grid come from the copies)
        if (has_ring) Fq[r_f] = hasB ? A[r_raw] + coef * B[r_raw] : A[r_raw];
        __syncthreads();
        if (s_abort) {
          q_fail = q;
          break;
        }
        if (tid == 0 && issued < count) {
          issue(issued);
          ++issued;
        }
        if (q >= 2) {
          const int kp = kq - 1;  // plane of the stencil
          const C* Fm = Fbase + ((q - 2) & 3) * FPL;
          const C* Fc = Fbase + ((q - 1) & 3) * FPL;
          const C u = Fc[o_f];
          const C uxm = Fc[o_f - 1];
          const C uxp = Fc[o_f + 1];
          const C uym = Fc[o_f - L::FW];
          const C uyp = Fc[o_f + L::FW];
          const C uzm = Fm[o_f];
          const C uzp = Fq[o_f];
          const float om2m = om2 * m_prev;
          C AF;
          if (xy_int && kp >= zlo && kp <= zhi) {
            AF = stencil_interior<float>(ih2, om2m, u, uxm, uxp, uym, uyp, uzm, uzp);
          } else {
            ZCoef<float> zc;
            const C* zr = ztab + 3 * kp;
            zc.sz = __ldg(zr);
            zc.izm = __ldg(zr + 1);
            zc.izp = __ldg(zr + 2);
            AF = stencil_general<float, CONJ>(G, cxy, zc, om2m, u, uxm, uxp, uym, uyp, uzm, uzp);
          }
          if (own) {
            C o = AF;
            if (MODE == M_P1 && own_src_col && kp == src_k) o = czero<float>();
            pO[po - plane] = o;
            if (!(rcb && ((rec_plane_bits(G, sl, kp, j, x0) >> tx) & 1u))) acc.add(abs2(o));
          }
        }
        m_prev = m_new;
      }
      if (q_fail >= 0) {
        // a copy never completed: record it, drain the copies this CTA issued (bounded), stop
        if (tid == 0) {
          atomicExch(T.err, 1);
          for (int qq = q_fail; qq < issued; ++qq) mbar_wait(&bar[(uses + qq) % S], ((uses + qq) / S) & 1u, T.wait_ns);
        }
        __syncthreads();
        return;
      }
      uses += (unsigned)count;
      accd = acc.value();
    }

    // ---- tile partial, ticket, and the system's finalizer (shared with the generic kernel)
    const double tsum = block_sum<NT>(accd, red);
    if (tid == 0 && !xonly) b.partial[sd->part_off + tile] = tsum;
    __threadfence();
    __syncthreads();
    if (tid == 0) {
      const unsigned t = atomicAdd(&sd->ticket, 1u);
      s_last = (t == (unsigned)(G.ntiles - 1));
    }
    __syncthreads();
    if (s_last) finalize<float, float, MODE, NT>(b, G, sd, sl, xonly, red, &bcast);
  }
}

// ------------------------------------------------------------------ two nodes per thread
// Same pipeline as k_phase_tma, with every thread owning the two x-adjacent nodes
// (x0 + 2 tx, x0 + 2 tx + 1) of row y0 + ty: shared-memory and global accesses move 16
// bytes per instruction and the per-plane control, barrier and address work is paid once
// per pair.  F planes use the copy boxes' 36-column layout so pairs stay 16-byte aligned.
template <int MODE, int BY>
struct TmaLayout2 {
  static constexpr int HW = WRI_TX + 4;  // 36 columns: x0-2 .. x0+33 (boxes and F planes)
  static constexpr int HH = BY + 2;
  static constexpr int pad(int v) { return (v + 127) / 128 * 128; }
  static constexpr int HALO = HW * HH * 8;
  static constexpr int CTR = WRI_TX * BY * 8;
  static constexpr int MB = WRI_TX * BY * 4;
  static constexpr int OFF_B = pad(HALO);
  static constexpr int OFF_X = OFF_B + pad(HALO);
  static constexpr int OFF_M = OFF_X + (MODE == M_P1 ? pad(CTR) : 0);
  static constexpr int STAGE = OFF_M + pad(MB);
  static constexpr int FPL = HH * HW;  // complex elements of one F plane
  static constexpr int FRING = 4 * FPL * 8;
  static size_t bytes(int S) { return 128 + (size_t)S * STAGE + FRING + 8 * S; }
};

__device__ __forceinline__ float4 ld4(const float2* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float2* p, float2 a, float2 b) {
  *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }

template <int MODE, int BY, int S, int MINB>
__global__ void __launch_bounds__(16 * BY, MINB) k_phase_tma2(const __grid_constant__ Batch b,
                                                              const __grid_constant__ TmaSet T) {
  static_assert(MODE == M_P1 || MODE == M_P2, "TMA path covers the two CGLS phases");
  typedef float2 C;
  typedef TmaLayout2<MODE, BY> L;
  constexpr bool CONJ = (MODE == M_P2);
  constexpr int NT = 16 * BY;
  constexpr int NW = NT / 32;
  constexpr int RW = 32 + 2 * BY;  // ring work items: 2 x 16 pairs (y halo rows) + 2 x BY singles (x halo)
  static_assert(NT % 32 == 0 && (RW + NW - 1) / NW <= 32, "ring share fits a warp");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ double red[NT / 32];
  __shared__ double bcast;
  __shared__ int s_last;
  __shared__ int s_abort;
  // x/y stretch coefficients of the current tile (general stencil only), rebuilt per item:
  // node stretch s(i) and half-point 1/(s(i-1/2) h^2) for the 32 columns and BY rows
  __shared__ C xs_tab[WRI_TX], xh_tab[WRI_TX + 1], ys_tab[BY], yh_tab[BY + 1];
  unsigned char* smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
  C* Fbase = reinterpret_cast<C*>(smem + (size_t)S * L::STAGE);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + (size_t)S * L::STAGE + L::FRING);

  const int tx = threadIdx.x, ty = threadIdx.y;  // tx in [0, 16)
  const int tid = ty * 16 + tx;
  if ((smem_addr(smem) & 127u) != 0u || (L::OFF_B & 127) || (L::OFF_X & 127) || (L::OFF_M & 127) ||
      (L::STAGE & 127)) {
    if (tid == 0) atomicExch(T.err, 2);
    return;
  }
  // ring work item of this thread, dealt round-robin over warps
  const int r_e = (tid & 31) * NW + (tid >> 5);
  const bool has_ring = r_e < RW;
  const bool r_pair = r_e < 32;
  int r_idx;  // element index in a box / F plane (both 36 wide)
  if (r_e < 16) r_idx = 2 * r_e + 2;                                  // row 0, pair
  else if (r_e < 32) r_idx = (BY + 1) * L::HW + 2 * (r_e - 16) + 2;  // row BY+1, pair
  else if (r_e < 32 + BY) r_idx = (r_e - 32 + 1) * L::HW + 1;        // column x0-1
  else r_idx = (r_e - 32 - BY + 1) * L::HW + 34;                     // column x0+32
  const int o = (ty + 1) * L::HW + 2 * tx + 2;  // own pair in a box / F plane
  const int oc = ty * WRI_TX + 2 * tx;          // own pair in a 32 x BY box

  if (tid == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&bar[s], 1);
    s_abort = 0;
  }
  __syncthreads();
  unsigned uses = 0;

  for (long long item = blockIdx.x; item < b.nitems; item += gridDim.x) {
    const int gi = find_group(b, item);
    const GroupDev& G = b.g[gi];
    const long long local = item - G.item0;
    int sl, tile;
    item_coords(b, G, local, sl, tile);
    SysDev* sd = b.sys + (G.sys0 + sl);
    const int state = sd->state;
    if (MODE == M_P1 ? (state == ST_DONE) : (state != ST_ACTIVE)) continue;
    const bool xonly = (MODE == M_P1 && state == ST_FINISHING);

    const int nx = G.nx, ny = G.ny, nz = G.nz;
    const int tzi = tile % G.zsplit;
    const int txy = tile / G.zsplit;
    const int x0 = (txy % G.tiles_x) * WRI_TX;
    const int y0 = (txy / G.tiles_x) * BY;
    const int z0 = tzi * G.zc;
    const int z1 = min(z0 + G.zc, nz);
    const int i0 = x0 + 2 * tx, j = y0 + ty;
    const bool own = (i0 < nx) && (j < ny);  // nx is even: the pair is in or out as a whole
    const long long plane = (long long)nx * ny;
    const long long col = (long long)j * nx + i0;
    const long long off = (long long)sl * G.n;
    const int iter = sd->iter;
    const int cur = iter & 1;
    double accd = 0.0;

    if (xonly) {
      C* X = (C*)G.x + off + col;
      const C* Pc = (const C*)G.p[cur] + off + col;
      const float a = (float)sd->alpha;
      if (own)
        for (int k = z0; k < z1; ++k) {
          const long long q = k * plane;
          const float4 xv = ld4(X + q), pv = __ldg(reinterpret_cast<const float4*>(Pc + q));
          st4(X + q, lo2(xv) + a * lo2(pv), hi2(xv) + a * hi2(pv));
        }
    } else {
      const CUtensorMap* mapA = &T.map[gi][MODE == M_P1 ? TM_S : (cur ? TM_R1 : TM_R0)];
      const bool hasB = (MODE == M_P2) || iter > 0;
      const CUtensorMap* mapB = &T.map[gi][MODE == M_P1 ? (cur ? TM_P1 : TM_P0) : TM_T1];
      const bool hasX = (MODE == M_P1) && iter > 0;
      const CUtensorMap* mapX = &T.map[gi][TM_X];
      const CUtensorMap* mapM = &T.map[gi][TM_M];
      const uint32_t tx_bytes = L::HALO + (hasB ? L::HALO : 0) + (hasX ? L::CTR : 0) + L::MB;
      const float coef = (MODE == M_P1) ? (float)sd->beta : -(float)sd->alpha;
      const float xal = (float)sd->alpha;
      C* pF = ((MODE == M_P1) ? (C*)G.p[cur ^ 1] : (C*)G.r1[cur ^ 1]) + off + col;
      C* pX = (C*)G.x + off + col;
      C* pO = ((MODE == M_P1) ? (C*)G.t1 : (C*)G.s) + off + col;
      int src_k = -1;
      long long src_col = -1;
      if (MODE == M_P1 && G.masked) {
        src_k = (int)(sd->src / plane);
        src_col = sd->src - (long long)src_k * plane;
      }
      const int src_lane = (src_col == col) ? 0 : (src_col == col + 1) ? 1 : -1;
      // receivers of this system in the thread's two columns: left out of the phase-2 norm
      const uint32_t rcb = (MODE == M_P2 && own) ? (rec_col_bits(G, sl, j, x0) >> (2 * tx)) & 3u : 0u;
      const int count = z1 - z0 + 2;

      auto issue = [&](int q) {
        const int st = (int)((uses + q) % S);
        unsigned char* base = smem + (size_t)st * L::STAGE;
        const int kq = z0 - 1 + q;
        mbar_expect_tx(&bar[st], tx_bytes);
        tma_load_4d(base, mapA, x0 - 2, y0 - 1, kq, sl, &bar[st]);
        if (hasB) tma_load_4d(base + L::OFF_B, mapB, x0 - 2, y0 - 1, kq, sl, &bar[st]);
        if (hasX) tma_load_4d(base + L::OFF_X, mapX, x0, y0, kq, sl, &bar[st]);
        tma_load_3d(base + L::OFF_M, mapM, x0, y0, kq, &bar[st]);
      };

      int xlo, xhi, ylo, yhi, zlo, zhi;
      interior_range(G.ax, xlo, xhi);
      interior_range(G.ay, ylo, yhi);
      interior_range(G.az, zlo, zhi);
      // which axes are stretched anywhere in this tile (uniform): selects the stencil variant
      const int xpf = ((x0 >= xlo) && (min(x0 + WRI_TX, nx) - 1 <= xhi)) ? 0 : 4;
      const int ypf = ((y0 >= ylo) && (min(y0 + BY, ny) - 1 <= yhi)) ? 0 : 2;
      {
        // coefficient tables of this tile (read only in the absorbing layer)
        const float ih2t = G.ih2f;
        for (int e = tid; e < 2 * WRI_TX + 2 * BY + 2; e += NT) {
          if (e < WRI_TX) {
            xs_tab[e] = stretch_at<float, CONJ>(G.ax, float(x0 + e));
          } else if (e < 2 * WRI_TX + 1) {
            const int c = e - WRI_TX;
            xh_tab[c] = ih2t * inv(stretch_at<float, CONJ>(G.ax, float(x0 + c) - 0.5f));
          } else if (e < 2 * WRI_TX + 1 + BY) {
            const int r = e - 2 * WRI_TX - 1;
            ys_tab[r] = stretch_at<float, CONJ>(G.ay, float(y0 + r));
          } else {
            const int r = e - 2 * WRI_TX - 1 - BY;
            yh_tab[r] = ih2t * inv(stretch_at<float, CONJ>(G.ay, float(y0 + r) - 0.5f));
          }
        }
      }
      const float om2 = G.om2f;
      const float ih2 = G.ih2f;
      const float2* ztab = G.ztab + (CONJ ? 3 * nz : 0);

      __syncthreads();
      if (tid == 0)
        for (int q = 0; q < S && q < count; ++q) issue(q);

      CompSum acc;
      float2 m_prev = make_float2(0.f, 0.f);
      int issued = min(S, count);
      int q_fail = -1;
      long long po = (long long)(z0 - 1) * plane;
      for (int q = 0; q < count; ++q, po += plane) {
        const int st = (int)((uses + q) % S);
        const uint32_t par = ((uses + q) / S) & 1u;
        if (!mbar_wait(&bar[st], par, T.wait_ns)) s_abort = 1;
        const unsigned char* base = smem + (size_t)st * L::STAGE;
        const C* A = reinterpret_cast<const C*>(base);
        const C* B = reinterpret_cast<const C*>(base + L::OFF_B);
        const C* XT = reinterpret_cast<const C*>(base + L::OFF_X);
        const float* MT = reinterpret_cast<const float*>(base + L::OFF_M);
        const int kq = z0 - 1 + q;
        C* Fq = Fbase + (q & 3) * L::FPL;
        const bool mine = own && kq >= z0 && kq < z1;
        {
          const float4 a = ld4(A + o);
          C v0 = lo2(a), v1 = hi2(a);
          if (hasB) {
            const float4 bb = ld4(B + o);
            v0 = v0 + coef * lo2(bb);
            v1 = v1 + coef * hi2(bb);
            if (MODE == M_P1 && mine) {
              const float4 xv = ld4(XT + oc);
              st4(pX + po, lo2(xv) + xal * lo2(bb), hi2(xv) + xal * hi2(bb));
            }
          }
          st4(Fq + o, v0, v1);
          if (mine) st4(pF + po, v0, v1);
        }
        const float2 m_new = *reinterpret_cast<const float2*>(MT + oc);
        if (has_ring) {
          if (r_pair) {
            const float4 a = ld4(A + r_idx);
            if (hasB) {
              const float4 bb = ld4(B + r_idx);
              st4(Fq + r_idx, lo2(a) + coef * lo2(bb), hi2(a) + coef * hi2(bb));
            } else {
              st4(Fq + r_idx, lo2(a), hi2(a));
            }
          } else {
            Fq[r_idx] = hasB ? A[r_idx] + coef * B[r_idx] : A[r_idx];
          }
        }
        __syncthreads();
        if (s_abort) {
          q_fail = q;
          break;
        }
        if (tid == 0 && issued < count) {
          issue(issued);
          ++issued;
        }
        if (q >= 2) {
          const int kp = kq - 1;
          const C* Fm = Fbase + ((q - 2) & 3) * L::FPL;
          const C* Fc = Fbase + ((q - 1) & 3) * L::FPL;
          const float4 U = ld4(Fc + o);
          const C u0 = lo2(U), u1 = hi2(U);
          const C l = Fc[o - 1], r = Fc[o + 2];
          const float4 YM = ld4(Fc + o - L::HW), YP = ld4(Fc + o + L::HW);
          const float4 ZM = ld4(Fm + o), ZP = ld4(Fq + o);
          C a0, a1;
          const int var = xpf | ypf | ((kp >= zlo && kp <= zhi) ? 0 : 1);
          if (var == 0) {
            a0 = stencil_interior<float>(ih2, om2 * m_prev.x, u0, l, u1, lo2(YM), lo2(YP), lo2(ZM), lo2(ZP));
            a1 = stencil_interior<float>(ih2, om2 * m_prev.y, u1, u0, r, hi2(YM), hi2(YP), hi2(ZM), hi2(ZP));
          } else {
            // coefficients of the stretched axes only (tables of this tile / plane)
            C sx0 = mkc(1.f, 0.f), sx1 = sx0, ixa = mkc(ih2, 0.f), ixb = ixa, ixc = ixa;
            C sy = mkc(1.f, 0.f), iym = mkc(ih2, 0.f), iyp = iym;
            C sz = mkc(1.f, 0.f), izm = mkc(ih2, 0.f), izp = izm;
            if (var & 4) {
              sx0 = xs_tab[2 * tx];
              sx1 = xs_tab[2 * tx + 1];
              ixa = xh_tab[2 * tx];
              ixb = xh_tab[2 * tx + 1];
              ixc = xh_tab[2 * tx + 2];
            }
            if (var & 2) {
              sy = ys_tab[ty];
              iym = yh_tab[ty];
              iyp = yh_tab[ty + 1];
            }
            if (var & 1) {
              const C* zr = ztab + 3 * kp;
              sz = __ldg(zr);
              izm = __ldg(zr + 1);
              izp = __ldg(zr + 2);
            }
            const float om0 = om2 * m_prev.x, om1 = om2 * m_prev.y;
#define WRI_AX(AX_, AY_, AZ_)                                                                                 \
  a0 = stencil_axes<AX_, AY_, AZ_>(ih2, om0, u0, l, u1, lo2(YM), lo2(YP), lo2(ZM), lo2(ZP), sx0, ixa, ixb, sy, iym, \
                                iyp, sz, izm, izp);                                                           \
  a1 = stencil_axes<AX_, AY_, AZ_>(ih2, om1, u1, u0, r, hi2(YM), hi2(YP), hi2(ZM), hi2(ZP), sx1, ixb, ixc, sy, iym, \
                                iyp, sz, izm, izp);
            switch (var) {
              case 1: WRI_AX(false, false, true) break;
              case 2: WRI_AX(false, true, false) break;
              case 3: WRI_AX(false, true, true) break;
              case 4: WRI_AX(true, false, false) break;
              case 5: WRI_AX(true, false, true) break;
              case 6: WRI_AX(true, true, false) break;
              default: WRI_AX(true, true, true) break;
            }
#undef WRI_AX
          }
          if (own) {
            if (MODE == M_P1 && kp == src_k) {
              if (src_lane == 0) a0 = czero<float>();
              if (src_lane == 1) a1 = czero<float>();
            }
            st4(pO + po - plane, a0, a1);
            float e0 = abs2(a0), e1 = abs2(a1);
            if (rcb) {
              const uint32_t w = rec_plane_bits(G, sl, kp, j, x0) >> (2 * tx);
              if (w & 1u) e0 = 0.f;
              if (w & 2u) e1 = 0.f;
            }
            acc.add(e0);
            acc.add(e1);
          }
        }
        m_prev = m_new;
      }
      if (q_fail >= 0) {
        if (tid == 0) {
          atomicExch(T.err, 1);
          for (int qq = q_fail; qq < issued; ++qq) mbar_wait(&bar[(uses + qq) % S], ((uses + qq) / S) & 1u, T.wait_ns);
        }
        __syncthreads();
        return;
      }
      uses += (unsigned)count;
      accd = acc.value();
    }

    const double tsum = block_sum<NT>(accd, red);
    if (tid == 0 && !xonly) b.partial[sd->part_off + tile] = tsum;
    __threadfence();
    __syncthreads();
    if (tid == 0) {
      const unsigned t = atomicAdd(&sd->ticket, 1u);
      s_last = (t == (unsigned)(G.ntiles - 1));
    }
    __syncthreads();
    if (s_last) finalize<float, float, MODE, NT>(b, G, sd, sl, xonly, red, &bcast);
  }
}

// ------------------------------------------------------------------ warp-specialised phases
// Same work, decomposition, boxes and finalizers as k_phase_tma2, with the plane pipeline
// decoupled from the CTA barrier:
//   * the last warp only issues the TMA copies: before refilling a stage it waits on that
//     stage's "empty" mbarrier, which every consumer warp arrives on once it is done with the
//     stage; consumers wait on the stage's "full" mbarrier (armed with the byte count);
//   * consumer warps never synchronise with each other inside a tile column: a thread forms
//     the stencil input F = a + c b of its own nodes and keeps it in registers for the three
//     planes the z-stencil needs, and forms the in-plane neighbours' F straight from the
//     stage's copy boxes (each F value is the same rounded a + c b wherever it is formed);
//   * a stage is released once the stencil of its plane is done, so a CTA holds two planes
//     and keeps S - 2 planes of copies in flight.
// All waits are bounded: a time-out raises a CTA-wide abort flag and the error flag of the
// launch; the other roles see the flag in their waits, every consumer warp still reaches the
// same named barriers, and the copy warp waits (bounded) for its copies before it exits.
template <int MODE, int BY>
struct WsLayout {
  static constexpr int HW = WRI_TX + 4;  // 36 columns: x0-2 .. x0+33
  static constexpr int HH = BY + 2;
  static constexpr int pad(int v) { return (v + 127) / 128 * 128; }
  static constexpr int HALO = HW * HH * 8;
  static constexpr int CTR = WRI_TX * BY * 8;
  static constexpr int MB = WRI_TX * BY * 4;
  static constexpr int OFF_B = pad(HALO);
  static constexpr int OFF_X = OFF_B + pad(HALO);
  static constexpr int OFF_M = OFF_X + (MODE == M_P1 ? pad(CTR) : 0);
  static constexpr int STAGE = OFF_M + pad(MB);
  // grouped iterate updates (phase 1): the older directions of the group, in boxes appended to
  // each stage (box i at OFF_X2 + i X2)
  static constexpr int OFF_X2 = STAGE;
  static constexpr int X2 = (MODE == M_P1) ? pad(CTR) : 0;
  static size_t bytes(int S, int extra) { return 128 + (size_t)S * (STAGE + extra * X2) + 16 * S; }
};

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// bounded wait that also gives up as soon as another role raised the abort flag
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t* bar, uint32_t parity, const volatile int* abort_flag,
                                                   uint64_t limit) {
  const uint64_t t0 = global_ns();
  for (int i = 0; i < (1 << 26); ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63) == 63 && (*abort_flag || global_ns() - t0 > limit)) return false;
  }
  return false;
}

// OR of a predicate over the first NC threads (named barrier 1): the same answer in every one
// of them, so a decision taken on it keeps them on the same barriers.
template <int NC>
__device__ __forceinline__ bool first_threads_any(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(NC)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ float2 fma_c(float c, float2 b, float2 a) {
  return make_float2(__fmaf_rn(c, b.x, a.x), __fmaf_rn(c, b.y, a.y));
}

// PW = true: a dedicated copy warp (16 BY + 32 threads).  PW = false: no copy warp (16 BY threads,
// so more CTAs fit the register file); thread 0 issues the copies of its CTA's planes itself,
// S - 2 planes ahead of the plane it consumes, each after that stage's "empty" barrier (the
// stage of two planes back, which every warp has released by then); copies never run ahead
// across a work item.
//
// ER = true ("early release"): a stage is used in one pass only.  When plane k arrives a thread
// forms its own F(k), completes the pending stencil of plane k-1 with it as the z+1 neighbour,
// and computes everything of plane k's stencil except the z+1 term (A u is linear in it: the
// partial value and the z+1 coefficient stay in registers), then releases the stage at once:
// S - 1 planes of copies stay in flight instead of S - 2.
//
// b.xsteps = m > 1 ("grouped iterate updates", phase 1 only): x is needed only at the end of a
// solve, so phase 1 updates it every m-th iteration, x += alpha_{k-m} p_{k-m} + ... +
// alpha_{k-1} p_{k-1} in iteration k = m, 2m, ...  The directions live in a ring of R slots (R = 2
// for m = 2, 4 for m = 4, p_j in slot (j + 1) mod R): p_{k-1} is the stencil input anyway, the older
// m - 1 arrive in 32 x BY boxes, and p_{k-m} lies in the slot iteration k overwrites with p_k (each
// thread reads its own nodes there before it writes them).  Phase 1 moves 32 bytes per
// node-system in the other iterations and 32 + 16 + 8 (m - 1) in the updating one: 44 (m = 2) or
// 42 (m = 4) instead of 48 on average.  The steps are added oldest first, so x rounds exactly as
// with one update per iteration.  The x-only pass of a finishing system adds whatever is pending.
// A run-time switch of the same kernel (the stencil and reduction code is the same machine code
// with and without it); each stage then holds m - 1 more boxes (the launch sizes the shared memory).
template <int MODE, int BY, int S, int MINB, bool PW = true, bool ER = false>
__global__ void __launch_bounds__(16 * BY + (PW ? 32 : 0), MINB) k_phase_ws(const __grid_constant__ Batch b,
                                                                             const __grid_constant__ TmaSet T) {
  static_assert(MODE == M_P1 || MODE == M_P2, "the warp-specialised path covers the two CGLS phases");
  static_assert(S >= 3, "two stages are held by the consumers");
  static_assert(PW || !ER, "early release is built with the copy warp");
  typedef float2 C;
  typedef WsLayout<MODE, BY> L;
  const int XS = (MODE == M_P1) ? xsteps_of(b) : 1;  // iterations per iterate update
  const int SB = L::STAGE + (XS - 1) * L::X2;          // bytes of one stage
  typedef FirstThreadsSync<16 * BY> CSync;
  constexpr bool CONJ = (MODE == M_P2);
  constexpr int NC = 16 * BY;   // consumer threads: two x-adjacent nodes each
  constexpr int NCW = NC / 32;  // consumer warps
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ double red[NCW];
  __shared__ double bcast;
  __shared__ int s_last;
  __shared__ volatile int s_abort;
  __shared__ C xs_tab[WRI_TX], xh_tab[WRI_TX + 1], ys_tab[BY], yh_tab[BY + 1];
  unsigned char* smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)S * SB);
  uint64_t* empty = full + S;

  const int tid = threadIdx.x;
  if ((smem_addr(smem) & 127u) != 0u || (L::OFF_B & 127) || (L::OFF_X & 127) || (L::OFF_X2 & 127) ||
      (L::OFF_M & 127) || (L::STAGE & 127) || (SB & 127)) {
    if (tid == 0) atomicExch(T.err, 2);
    return;
  }
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NCW);
    }
    // a copy wait of an earlier launch of this solve timed out: the solve is being stopped, and
    // this launch does nothing (read once here so that the whole CTA takes the same decision)
    s_abort = (*(volatile const int*)T.err != 0) ? 1 : 0;
  }
  __syncthreads();  // the only CTA-wide barrier: the copy warp leaves the consumers' barriers after it
  if (s_abort) return;

  // ================================================================ copy warp
  if (PW && tid >= NC) {
    if (tid != NC) return;
    unsigned fills = 0;
    bool stop = false;
    for (long long item = blockIdx.x; item < b.nitems && !stop; item += gridDim.x) {
      const int gi = find_group(b, item);
      const GroupDev& G = b.g[gi];
      int sl, tile;
      item_coords(b, G, item - G.item0, sl, tile);
      const SysDev* sd = b.sys + (G.sys0 + sl);
      const int state = sd->state;
      if (MODE == M_P1 ? (state == ST_DONE) : (state != ST_ACTIVE)) continue;
      if (MODE == M_P1 && state == ST_FINISHING) continue;  // x-only pass: no copies
      const int tzi = tile % G.zsplit;
      const int txy = tile / G.zsplit;
      const int x0 = (txy % G.tiles_x) * WRI_TX;
      const int y0 = (txy / G.tiles_x) * BY;
      const int z0 = tzi * G.zc;
      const int z1 = min(z0 + G.zc, G.nz);
      const int iter = sd->iter;
      const int cur = iter & 1;
      const CUtensorMap* mapA = &T.map[gi][MODE == M_P1 ? TM_S : (cur ? TM_R1 : TM_R0)];
      const bool hasB = (MODE == M_P2) || iter > 0;
      const CUtensorMap* mapB = &T.map[gi][MODE == M_P1 ? TM_P0 + pslot(b, iter - 1) : TM_T1];
      const bool hasX = (MODE == M_P1) && iter >= XS && iter % XS == 0;
      const int nX2 = hasX ? XS - 1 : 0;  // older directions of the group: p_{iter-XS} .. p_{iter-2}
      const uint32_t tx_bytes = L::HALO + (hasB ? L::HALO : 0) + (hasX ? L::CTR : 0) + nX2 * L::CTR + L::MB;
      const int count = z1 - z0 + 2;
      for (int q = 0; q < count; ++q, ++fills) {
        const int st = (int)(fills % S);
        if (fills >= (unsigned)S && !mbar_wait_or_abort(&empty[st], ((fills / S) - 1) & 1u, &s_abort, T.wait_ns)) {
          s_abort = 1;
          atomicExch(T.err, 1);
          stop = true;
          break;
        }
        if (s_abort) {
          stop = true;
          break;
        }
        // test hook (off unless the caller asks): this fill is never issued, so its "full" barrier
        // never completes and the consumers' bounded wait for it runs out
        if (blockIdx.x == 0 && (int)fills == T.withhold) continue;
        unsigned char* base = smem + (size_t)st * SB;
        const int kq = z0 - 1 + q;
        mbar_expect_tx(&full[st], tx_bytes);
        tma_load_4d(base, mapA, x0 - 2, y0 - 1, kq, sl, &full[st]);
        if (hasB) tma_load_4d(base + L::OFF_B, mapB, x0 - 2, y0 - 1, kq, sl, &full[st]);
        if (hasX) tma_load_4d(base + L::OFF_X, &T.map[gi][TM_X], x0, y0, kq, sl, &full[st]);
        for (int i = 0; i < nX2; ++i)
          tma_load_4d(base + L::OFF_X2 + i * L::X2, &T.map[gi][TM_PC0 + pslot(b, iter - XS + i)], x0, y0, kq, sl,
                      &full[st]);
        tma_load_3d(base + L::OFF_M, &T.map[gi][TM_M], x0, y0, kq, &full[st]);
      }
    }
    if (stop) {
      // wait (bounded) until every copy issued into the ring has landed
      const unsigned first = fills > (unsigned)S ? fills - S : 0u;
      for (unsigned u = first; u < fills; ++u) mbar_wait(&full[u % S], (u / S) & 1u, T.wait_ns);
    }
    return;
  }

  // ================================================================ consumer warps
  const int lane = tid & 31;
  const int tx = tid & 15, ty = tid >> 4;
  const int o = (ty + 1) * L::HW + 2 * tx + 2;  // own pair in a halo box
  const int oc = ty * WRI_TX + 2 * tx;          // own pair in a 32 x BY box
  unsigned fills = 0;
  unsigned issued = 0;  // PW = false: copies issued by thread 0

  for (long long item = blockIdx.x; item < b.nitems; item += gridDim.x) {
    const int gi = find_group(b, item);
    const GroupDev& G = b.g[gi];
    int sl, tile;
    item_coords(b, G, item - G.item0, sl, tile);
    SysDev* sd = b.sys + (G.sys0 + sl);
    const int state = sd->state;
    if (MODE == M_P1 ? (state == ST_DONE) : (state != ST_ACTIVE)) continue;
    const bool xonly = (MODE == M_P1 && state == ST_FINISHING);

    const int nx = G.nx, ny = G.ny, nz = G.nz;
    const int tzi = tile % G.zsplit;
    const int txy = tile / G.zsplit;
    const int x0 = (txy % G.tiles_x) * WRI_TX;
    const int y0 = (txy / G.tiles_x) * BY;
    const int z0 = tzi * G.zc;
    const int z1 = min(z0 + G.zc, nz);
    const int i0 = x0 + 2 * tx, j = y0 + ty;
    const bool own = (i0 < nx) && (j < ny);  // nx is even: the pair is in or out as a whole
    const long long plane = (long long)nx * ny;
    const long long col = (long long)j * nx + i0;
    const long long off = (long long)sl * G.n;
    const int iter = sd->iter;
    const int cur = iter & 1;
    double accd = 0.0;

    if (xonly) {
      // the steps not yet in x: those of iterations iter - c .. iter - 1, oldest first (c = 1 with
      // one update per iteration; grouped updates: the rest of the last group, or on a breakdown
      // the steps before it)
      C* X = (C*)G.x + off + col;
      const int c = (iter - 1) % XS + 1;
      if (own)
        for (int k = z0; k < z1; ++k) {
          const long long q = k * plane;
          float4 xv = ld4(X + q);
          for (int jj = c - 1; jj >= 0; --jj) {
            const float a = (float)(jj == 0 ? sd->alpha : sd->alpha_hist[jj - 1]);
            const C* Pj = (const C*)G.p[pslot(b, iter - 1 - jj)] + off + col;
            const float4 pv = __ldg(reinterpret_cast<const float4*>(Pj + q));
            // explicit fma (as in the iteration's own update): the rounding must not depend on how
            // the compiler contracts this instantiation
            xv = make_float4(__fmaf_rn(a, pv.x, xv.x), __fmaf_rn(a, pv.y, xv.y), __fmaf_rn(a, pv.z, xv.z),
                             __fmaf_rn(a, pv.w, xv.w));
          }
          st4(X + q, lo2(xv), hi2(xv));
        }
    } else {
      const bool hasB = (MODE == M_P2) || iter > 0;
      const bool hasX = (MODE == M_P1) && iter >= XS && iter % XS == 0;
      const int nX2 = hasX ? XS - 1 : 0;
      const float coef = (MODE == M_P1) ? (float)sd->beta : -(float)sd->alpha;
      const float xal = (float)sd->alpha;
      // steps of the older directions in the update boxes: box i holds p_{iter-XS+i}
      float xh[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int i = 0; i < 3; ++i)
        if (i < nX2) xh[i] = (float)sd->alpha_hist[XS - 2 - i];
      C* pF = ((MODE == M_P1) ? (C*)G.p[pslot(b, iter)] : (C*)G.r1[cur ^ 1]) + off + col;
      C* pX = (C*)G.x + off + col;
      C* pO = ((MODE == M_P1) ? (C*)G.t1 : (C*)G.s) + off + col;
      const C* pG = (MODE == M_P2 && G.gvec) ? (const C*)G.gvec + off + col : nullptr;
      int src_k = -1;
      long long src_col = -1;
      if (MODE == M_P1 && G.masked) {
        src_k = (int)(sd->src / plane);
        src_col = sd->src - (long long)src_k * plane;
      }
      const int src_lane = (src_col == col) ? 0 : (src_col == col + 1) ? 1 : -1;
      // receivers of this system in the thread's two columns: left out of the phase-2 norm
      const uint32_t rcb = (MODE == M_P2 && own) ? (rec_col_bits(G, sl, j, x0) >> (2 * tx)) & 3u : 0u;
      const int count = z1 - z0 + 2;
      // PW = false: thread 0 issues fill q of this item (plane z0 - 1 + q) into stage (fills + q) % S
      auto fill = [&](int q) {
        const unsigned u = fills + (unsigned)q;
        const int st = (int)(u % S);
        if (u >= (unsigned)S && !mbar_wait_or_abort(&empty[st], ((u / S) - 1) & 1u, &s_abort, T.wait_ns)) {
          s_abort = 1;
          atomicExch(T.err, 1);
          return;
        }
        if (s_abort) return;
        const CUtensorMap* mapA = &T.map[gi][MODE == M_P1 ? TM_S : (cur ? TM_R1 : TM_R0)];
        const CUtensorMap* mapB = &T.map[gi][MODE == M_P1 ? TM_P0 + pslot(b, iter - 1) : TM_T1];
        const uint32_t tx_bytes = L::HALO + (hasB ? L::HALO : 0) + (hasX ? L::CTR : 0) + nX2 * L::CTR + L::MB;
        unsigned char* base = smem + (size_t)st * SB;
        const int kq = z0 - 1 + q;
        mbar_expect_tx(&full[st], tx_bytes);
        tma_load_4d(base, mapA, x0 - 2, y0 - 1, kq, sl, &full[st]);
        if (hasB) tma_load_4d(base + L::OFF_B, mapB, x0 - 2, y0 - 1, kq, sl, &full[st]);
        if (hasX) tma_load_4d(base + L::OFF_X, &T.map[gi][TM_X], x0, y0, kq, sl, &full[st]);
        for (int i = 0; i < nX2; ++i)
          tma_load_4d(base + L::OFF_X2 + i * L::X2, &T.map[gi][TM_PC0 + pslot(b, iter - XS + i)], x0, y0, kq, sl,
                      &full[st]);
        tma_load_3d(base + L::OFF_M, &T.map[gi][TM_M], x0, y0, kq, &full[st]);
        issued = u + 1;
      };
      if (!PW && tid == 0)
        for (int q = 0; q < S - 2 && q < count; ++q) fill(q);

      int xlo, xhi, ylo, yhi, zlo, zhi;
      interior_range(G.ax, xlo, xhi);
      interior_range(G.ay, ylo, yhi);
      interior_range(G.az, zlo, zhi);
      const int xpf = ((x0 >= xlo) && (min(x0 + WRI_TX, nx) - 1 <= xhi)) ? 0 : 4;
      const int ypf = ((y0 >= ylo) && (min(y0 + BY, ny) - 1 <= yhi)) ? 0 : 2;
      if (xpf | ypf) {
        const float ih2t = G.ih2f;
        for (int e = tid; e < 2 * WRI_TX + 2 * BY + 2; e += NC) {
          if (e < WRI_TX) {
            xs_tab[e] = stretch_at<float, CONJ>(G.ax, float(x0 + e));
          } else if (e < 2 * WRI_TX + 1) {
            const int c = e - WRI_TX;
            xh_tab[c] = ih2t * inv(stretch_at<float, CONJ>(G.ax, float(x0 + c) - 0.5f));
          } else if (e < 2 * WRI_TX + 1 + BY) {
            const int r = e - 2 * WRI_TX - 1;
            ys_tab[r] = stretch_at<float, CONJ>(G.ay, float(y0 + r));
          } else {
            const int r = e - 2 * WRI_TX - 1 - BY;
            yh_tab[r] = ih2t * inv(stretch_at<float, CONJ>(G.ay, float(y0 + r) - 0.5f));
          }
        }
        CSync::sync();  // tables complete (the previous item's readers passed its final barrier)
      }
      const float om2 = G.om2f;
      const float ih2 = G.ih2f;
      const float2* ztab = G.ztab + (CONJ ? 3 * nz : 0);

      // per-thread partial sum: FP32 over 4 planes (8 terms), then FP64
      float accf = 0.f;
      if constexpr (ER) {
        C fc0 = czero<float>(), fc1 = fc0;                       // own F of plane kq-1
        C p0 = fc0, p1 = fc0, c0 = fc0, c1 = fc0;               // pending stencil of kq-1 without z+1
        long long po = (long long)(z0 - 1) * plane;
        for (int q = 0; q < count; ++q, po += plane) {
          const unsigned u = fills + q;
          const int st = (int)(u % S);
          bool ok = true;
          if (!s_abort) {
            ok = mbar_wait_or_abort(&full[st], (u / S) & 1u, &s_abort, T.wait_ns);
            if (!ok) {
              s_abort = 1;
              atomicExch(T.err, 1);
            }
          } else {
            ok = false;
          }
          C v0 = czero<float>(), v1 = v0;
          if (ok) {
            const unsigned char* base = smem + (size_t)st * SB;
            const C* A = reinterpret_cast<const C*>(base);
            const C* B = reinterpret_cast<const C*>(base + L::OFF_B);
            const int kq = z0 - 1 + q;
            const bool mine = own && kq >= z0 && kq < z1;
            const float4 a = ld4(A + o);
            v0 = lo2(a);
            v1 = hi2(a);
            if (hasB) {
              const float4 bb = ld4(B + o);
              v0 = fma_c(coef, lo2(bb), v0);
              v1 = fma_c(coef, hi2(bb), v1);
              if (MODE == M_P1 && hasX && mine) {
                float4 xv = ld4(reinterpret_cast<const C*>(base + L::OFF_X) + oc);
                // the older steps first: the same order as single updates
                #pragma unroll
                for (int e = 0; e < 3; ++e) {
                  if (e >= nX2) break;
                  const float4 ov = ld4(reinterpret_cast<const C*>(base + L::OFF_X2 + e * L::X2) + oc);
                  const float h = xh[e];
                  xv = make_float4(__fmaf_rn(h, ov.x, xv.x), __fmaf_rn(h, ov.y, xv.y), __fmaf_rn(h, ov.z, xv.z),
                                   __fmaf_rn(h, ov.w, xv.w));
                }
                st4(pX + po, fma_c(xal, lo2(bb), lo2(xv)), fma_c(xal, hi2(bb), hi2(xv)));
              }
            }
            if (mine) st4(pF + po, v0, v1);
            if (q >= 2 && own) {
              // plane kq-1: add the z+1 term (this plane's own F) to the pending partial stencil
              C a0 = p0 + c0 * v0, a1 = p1 + c1 * v1;
              if (MODE == M_P1 && kq - 1 == src_k) {
                if (src_lane == 0) a0 = czero<float>();
                if (src_lane == 1) a1 = czero<float>();
              }
              if (MODE == M_P2 && pG) {
                // refinement inner solve: s = S^H r + S^H r64
                const float4 gv = __ldg(reinterpret_cast<const float4*>(pG + po - plane));
                a0 = a0 + lo2(gv);
                a1 = a1 + hi2(gv);
              }
              st4(pO + po - plane, a0, a1);
              float e0 = abs2(a0), e1 = abs2(a1);
              if (rcb) {
                const uint32_t w = rec_plane_bits(G, sl, kq - 1, j, x0) >> (2 * tx);
                if (w & 1u) e0 = 0.f;
                if (w & 2u) e1 = 0.f;
              }
              accf += e0 + e1;
            }
            if (q >= 1 && q <= count - 2) {
              // plane kq: every stencil term but the z+1 one, from this stage and registers
              const float2 mk = *reinterpret_cast<const float2*>(reinterpret_cast<const float*>(base + L::OFF_M) + oc);
              C l = A[o - 1], r = A[o + 2];
              float4 ym = ld4(A + o - L::HW), yp = ld4(A + o + L::HW);
              C ym0 = lo2(ym), ym1 = hi2(ym), yp0 = lo2(yp), yp1 = hi2(yp);
              if (hasB) {
                l = fma_c(coef, B[o - 1], l);
                r = fma_c(coef, B[o + 2], r);
                const float4 bym = ld4(B + o - L::HW), byp = ld4(B + o + L::HW);
                ym0 = fma_c(coef, lo2(bym), ym0);
                ym1 = fma_c(coef, hi2(bym), ym1);
                yp0 = fma_c(coef, lo2(byp), yp0);
                yp1 = fma_c(coef, hi2(byp), yp1);
              }
              const C zero = czero<float>();
              const int var = xpf | ypf | ((kq >= zlo && kq <= zhi) ? 0 : 1);
              if (var == 0) {
                p0 = stencil_interior<float>(ih2, om2 * mk.x, v0, l, v1, ym0, yp0, fc0, zero);
                p1 = stencil_interior<float>(ih2, om2 * mk.y, v1, v0, r, ym1, yp1, fc1, zero);
                c0 = c1 = mkc(ih2, 0.f);
              } else {
                C sx0 = mkc(1.f, 0.f), sx1 = sx0, ixa = mkc(ih2, 0.f), ixb = ixa, ixc = ixa;
                C sy = mkc(1.f, 0.f), iym = mkc(ih2, 0.f), iyp = iym;
                C sz = mkc(1.f, 0.f), izm = mkc(ih2, 0.f), izp = izm;
                if (var & 4) {
                  sx0 = xs_tab[2 * tx];
                  sx1 = xs_tab[2 * tx + 1];
                  ixa = xh_tab[2 * tx];
                  ixb = xh_tab[2 * tx + 1];
                  ixc = xh_tab[2 * tx + 2];
                }
                if (var & 2) {
                  sy = ys_tab[ty];
                  iym = yh_tab[ty];
                  iyp = yh_tab[ty + 1];
                }
                if (var & 1) {
                  const C* zr = ztab + 3 * kq;
                  sz = __ldg(zr);
                  izm = __ldg(zr + 1);
                  izp = __ldg(zr + 2);
                }
                const float om0 = om2 * mk.x, om1 = om2 * mk.y;
#define WRI_AX(AX_, AY_, AZ_)                                                                                       \
  p0 = stencil_axes<AX_, AY_, AZ_>(ih2, om0, v0, l, v1, ym0, yp0, fc0, zero, sx0, ixa, ixb, sy, iym, iyp, sz, izm,    \
                                   izp);                                                                            \
  p1 = stencil_axes<AX_, AY_, AZ_>(ih2, om1, v1, v0, r, ym1, yp1, fc1, zero, sx1, ixb, ixc, sy, iym, iyp, sz, izm,    \
                                   izp);
                switch (var) {
                  case 1: WRI_AX(false, false, true) break;
                  case 2: WRI_AX(false, true, false) break;
                  case 3: WRI_AX(false, true, true) break;
                  case 4: WRI_AX(true, false, false) break;
                  case 5: WRI_AX(true, false, true) break;
                  case 6: WRI_AX(true, true, false) break;
                  default: WRI_AX(true, true, true) break;
                }
#undef WRI_AX
                // coefficient of the z+1 neighbour: (s_x s_y of the stretched axes) x (1/(s_z h^2) or 1/h^2)
                const C zc = (var & 1) ? izp : mkc(ih2, 0.f);
                const C syz = (var & 2) ? sy * zc : zc;
                c0 = (var & 4) ? sx0 * syz : syz;
                c1 = (var & 4) ? sx1 * syz : syz;
              }
            }
          }
          if ((q & 3) == 3) {
            accd += (double)accf;
            accf = 0.f;
          }
          // this plane's stage is no longer needed: hand it back to the copy warp
          __syncwarp();
          if (lane == 0) mbar_arrive(&empty[st]);
          fc0 = v0;
          fc1 = v1;
        }
        fills += (unsigned)count;
        accd += (double)accf;
      } else {
      C fm0 = czero<float>(), fm1 = fm0, fc0 = fm0, fc1 = fm0;  // own F of planes kq-2, kq-1
      float2 m_c = make_float2(0.f, 0.f);                        // m of plane kq-1
      long long po = (long long)(z0 - 1) * plane;
      for (int q = 0; q < count; ++q, po += plane) {
        const unsigned u = fills + q;
        const int st = (int)(u % S);
        bool ok = true;
        if (!s_abort) {
          ok = mbar_wait_or_abort(&full[st], (u / S) & 1u, &s_abort, T.wait_ns);
          if (!ok) {
            s_abort = 1;
            atomicExch(T.err, 1);
          }
        } else {
          ok = false;
        }
        C v0 = czero<float>(), v1 = v0;
        float2 m_new = make_float2(0.f, 0.f);
        if (ok) {
          const unsigned char* base = smem + (size_t)st * SB;
          const C* A = reinterpret_cast<const C*>(base);
          const C* B = reinterpret_cast<const C*>(base + L::OFF_B);
          const int kq = z0 - 1 + q;
          const bool mine = own && kq >= z0 && kq < z1;
          const float4 a = ld4(A + o);
          v0 = lo2(a);
          v1 = hi2(a);
          if (hasB) {
            const float4 bb = ld4(B + o);
            v0 = fma_c(coef, lo2(bb), v0);
            v1 = fma_c(coef, hi2(bb), v1);
            if (MODE == M_P1 && hasX && mine) {
              float4 xv = ld4(reinterpret_cast<const C*>(base + L::OFF_X) + oc);
              // the older steps first: the same order as single updates
              #pragma unroll
              for (int e = 0; e < 3; ++e) {
                if (e >= nX2) break;
                const float4 ov = ld4(reinterpret_cast<const C*>(base + L::OFF_X2 + e * L::X2) + oc);
                const float h = xh[e];
                xv = make_float4(__fmaf_rn(h, ov.x, xv.x), __fmaf_rn(h, ov.y, xv.y), __fmaf_rn(h, ov.z, xv.z),
                                 __fmaf_rn(h, ov.w, xv.w));
              }
              st4(pX + po, fma_c(xal, lo2(bb), lo2(xv)), fma_c(xal, hi2(bb), hi2(xv)));
            }
          }
          if (mine) st4(pF + po, v0, v1);
          m_new = *reinterpret_cast<const float2*>(reinterpret_cast<const float*>(base + L::OFF_M) + oc);
          if (q >= 2) {
            // stencil of plane kp = kq - 1: z neighbours from registers, in-plane neighbours
            // formed from the copy boxes of plane kp
            const int kp = kq - 1;
            const unsigned char* bp = smem + (size_t)((u - 1) % S) * SB;
            const C* Ap = reinterpret_cast<const C*>(bp);
            const C* Bp = reinterpret_cast<const C*>(bp + L::OFF_B);
            C l = Ap[o - 1], r = Ap[o + 2];
            float4 ym = ld4(Ap + o - L::HW), yp = ld4(Ap + o + L::HW);
            C ym0 = lo2(ym), ym1 = hi2(ym), yp0 = lo2(yp), yp1 = hi2(yp);
            if (hasB) {
              l = fma_c(coef, Bp[o - 1], l);
              r = fma_c(coef, Bp[o + 2], r);
              const float4 bym = ld4(Bp + o - L::HW), byp = ld4(Bp + o + L::HW);
              ym0 = fma_c(coef, lo2(bym), ym0);
              ym1 = fma_c(coef, hi2(bym), ym1);
              yp0 = fma_c(coef, lo2(byp), yp0);
              yp1 = fma_c(coef, hi2(byp), yp1);
            }
            C a0, a1;
            const int var = xpf | ypf | ((kp >= zlo && kp <= zhi) ? 0 : 1);
            if (var == 0) {
              a0 = stencil_interior<float>(ih2, om2 * m_c.x, fc0, l, fc1, ym0, yp0, fm0, v0);
              a1 = stencil_interior<float>(ih2, om2 * m_c.y, fc1, fc0, r, ym1, yp1, fm1, v1);
            } else {
              C sx0 = mkc(1.f, 0.f), sx1 = sx0, ixa = mkc(ih2, 0.f), ixb = ixa, ixc = ixa;
              C sy = mkc(1.f, 0.f), iym = mkc(ih2, 0.f), iyp = iym;
              C sz = mkc(1.f, 0.f), izm = mkc(ih2, 0.f), izp = izm;
              if (var & 4) {
                sx0 = xs_tab[2 * tx];
                sx1 = xs_tab[2 * tx + 1];
                ixa = xh_tab[2 * tx];
                ixb = xh_tab[2 * tx + 1];
                ixc = xh_tab[2 * tx + 2];
              }
              if (var & 2) {
                sy = ys_tab[ty];
                iym = yh_tab[ty];
                iyp = yh_tab[ty + 1];
              }
              if (var & 1) {
                const C* zr = ztab + 3 * kp;
                sz = __ldg(zr);
                izm = __ldg(zr + 1);
                izp = __ldg(zr + 2);
              }
              const float om0 = om2 * m_c.x, om1 = om2 * m_c.y;
#define WRI_AX(AX_, AY_, AZ_)                                                                                  \
  a0 = stencil_axes<AX_, AY_, AZ_>(ih2, om0, fc0, l, fc1, ym0, yp0, fm0, v0, sx0, ixa, ixb, sy, iym, iyp, sz, izm, \
                                   izp);                                                                       \
  a1 = stencil_axes<AX_, AY_, AZ_>(ih2, om1, fc1, fc0, r, ym1, yp1, fm1, v1, sx1, ixb, ixc, sy, iym, iyp, sz, izm, \
                                   izp);
              switch (var) {
                case 1: WRI_AX(false, false, true) break;
                case 2: WRI_AX(false, true, false) break;
                case 3: WRI_AX(false, true, true) break;
                case 4: WRI_AX(true, false, false) break;
                case 5: WRI_AX(true, false, true) break;
                case 6: WRI_AX(true, true, false) break;
                default: WRI_AX(true, true, true) break;
              }
#undef WRI_AX
            }
            if (own) {
              if (MODE == M_P1 && kp == src_k) {
                if (src_lane == 0) a0 = czero<float>();
                if (src_lane == 1) a1 = czero<float>();
              }
              if (MODE == M_P2 && pG) {
                // refinement inner solve: s = S^H r + S^H r64
                const float4 gv = __ldg(reinterpret_cast<const float4*>(pG + po - plane));
                a0 = a0 + lo2(gv);
                a1 = a1 + hi2(gv);
              }
              st4(pO + po - plane, a0, a1);
              float e0 = abs2(a0), e1 = abs2(a1);
              if (rcb) {
                const uint32_t w = rec_plane_bits(G, sl, kp, j, x0) >> (2 * tx);
                if (w & 1u) e0 = 0.f;
                if (w & 2u) e1 = 0.f;
              }
              accf += e0 + e1;
            }
          }
        }
        if ((q & 3) == 3) {
          accd += (double)accf;
          accf = 0.f;
        }
        if (q >= 1) {
          // plane kq-1 is done: hand its stage back to the copy warp
          __syncwarp();
          if (lane == 0) mbar_arrive(&empty[(u - 1) % S]);
        }
        if (!PW && tid == 0 && q + S - 2 < count) fill(q + S - 2);
        fm0 = fc0;
        fm1 = fc1;
        fc0 = v0;
        fc1 = v1;
        m_c = m_new;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[(fills + count - 1) % S]);
      fills += (unsigned)count;
      accd += (double)accf;
      }  // ER
    }

    // ---- tile partial, ticket and the system's finalizer (consumer threads only)
    const double tsum = block_sum<NC, CSync>(accd, red);
    // the copy warp may raise the flag at any time: decide on one reduced value
    if (first_threads_any<NC>(s_abort != 0)) break;
    if (tid == 0 && !xonly) b.partial[sd->part_off + tile] = tsum;
    __threadfence();
    CSync::sync();
    if (tid == 0) {
      const unsigned t = atomicAdd(&sd->ticket, 1u);
      s_last = (t == (unsigned)(G.ntiles - 1));
    }
    CSync::sync();
    if (s_last) finalize<float, float, MODE, NC, CSync>(b, G, sd, sl, xonly, red, &bcast);
  }
  if (!PW && tid == 0 && s_abort) {
    // stopped early: wait (bounded) until every copy thread 0 issued has landed
    const unsigned first = issued > (unsigned)S ? issued - S : 0u;
    for (unsigned u = first; u < issued; ++u) mbar_wait(&full[u % S], (u / S) & 1u, T.wait_ns);
  }
}

}  // namespace wri
