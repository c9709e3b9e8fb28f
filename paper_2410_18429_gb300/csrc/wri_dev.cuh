// Device-side definitions shared by the libwri translation units: complex helpers,
// the stretched-coordinate factors of the absorbing layer, and the batch
// descriptors passed to every kernel by value.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define WRI_MAXG 8   // frequency groups per batched launch
#define WRI_TX 32    // tile width in x: one warp spans one x-row of a tile

namespace wri {

// z-chunk of the gradient kernel (its FP64 accumulator tile lives in shared memory)
__host__ __device__ constexpr int grad_zc(int by) { return by >= 16 ? 8 : 16; }

// squared slowness at a node, in the precision of the caller's model array
template <typename R>
__device__ __forceinline__ R model_at(const void* m, int m_double, long long node) {
  return m_double ? R(((const double*)m)[node]) : R(((const float*)m)[node]);
}

// ------------------------------------------------------------------ complex helpers
template <typename R> struct CT;
template <> struct CT<float> { typedef float2 T; };
template <> struct CT<double> { typedef double2 T; };
template <typename R> using cx = typename CT<R>::T;

__host__ __device__ __forceinline__ float2 mkc(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ double2 mkc(double a, double b) { return make_double2(a, b); }
template <typename R> __host__ __device__ __forceinline__ cx<R> czero() { return mkc(R(0), R(0)); }

#define WRI_COPS(T, R)                                                                              \
  __device__ __forceinline__ T operator+(T a, T b) { return mkc(a.x + b.x, a.y + b.y); }         \
  __device__ __forceinline__ T operator-(T a, T b) { return mkc(a.x - b.x, a.y - b.y); }         \
  __device__ __forceinline__ T operator*(T a, T b) {                                               \
    return mkc(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);                                     \
  }                                                                                                \
  __device__ __forceinline__ T operator*(R s, T a) { return mkc(s * a.x, s * a.y); }             \
  __device__ __forceinline__ T conjc(T a) { return mkc(a.x, -a.y); }                              \
  __device__ __forceinline__ R abs2(T a) { return a.x * a.x + a.y * a.y; }                        \
  __device__ __forceinline__ T inv(T a) {                                                          \
    R d = R(1) / (a.x * a.x + a.y * a.y);                                                          \
    return mkc(a.x * d, -a.y * d);                                                                 \
  }
WRI_COPS(float2, float)
WRI_COPS(double2, double)
#undef WRI_COPS

__device__ __forceinline__ float2 to_c(float2 a, float) { return a; }
__device__ __forceinline__ float2 to_c(double2 a, float) { return make_float2((float)a.x, (float)a.y); }
__device__ __forceinline__ double2 to_c(float2 a, double) { return make_double2(a.x, a.y); }
__device__ __forceinline__ double2 to_c(double2 a, double) { return a; }

// ------------------------------------------------------------------ absorbing layer (step a1)
// s(xi) = 1 + i sigma(xi)/omega, sigma = sigma_max (xi/L)^2, xi = distance into the
// padding from the last physical node, measured at position `pos` (node units,
// half-integers for the half points).  CONJ returns conj(s), used by A^H.
// Parameters are kept in both precisions so FP32 kernels never convert from FP64
// (conversions run on the FP64 pipe, which is narrow on GB300).
struct AxisPml {
  int n, npml;
  double h, inv_omega, smax, invL;
  float hf, inv_omegaf, smaxf, invLf;
};

template <typename R> __device__ __forceinline__ R pick(double d, float f);
template <> __device__ __forceinline__ float pick<float>(double, float f) { return f; }
template <> __device__ __forceinline__ double pick<double>(double d, float) { return d; }

template <typename R, bool CONJ>
__device__ __forceinline__ cx<R> stretch_at(const AxisPml& a, R pos) {
  R xi = R(0);
  const R lo = R(a.npml), hi = R(a.n - 1 - a.npml);
  if (a.npml > 0) {
    if (pos < lo) xi = (lo - pos) * pick<R>(a.h, a.hf);
    else if (pos > hi) xi = (pos - hi) * pick<R>(a.h, a.hf);
  }
  const R q = xi * pick<R>(a.invL, a.invLf);
  const R im = pick<R>(a.smax, a.smaxf) * q * q * pick<R>(a.inv_omega, a.inv_omegaf);
  return mkc(R(1), CONJ ? -im : im);
}

// ------------------------------------------------------------------ kernel modes
enum Mode : int {
  M_APPLY = 0,  // y = A x (or A^H x); no reduction
  M_SH = 1,     // s = A^H r1 (+ lambda P^T r2 in the finalizer); init of a solve
  M_RES = 2,    // r1 = b1 - Z A x, r2 = lambda (d - P x)
  M_P1 = 3,     // p = s + beta p_old, t1 = Z A p, x += (step of the previous iteration) p_old
  M_P2 = 4,     // r1 = r1_old - alpha t1, s = A^H r1 (CGLS)
  M_GRAD = 6,   // g += omega^2 Re(conj(w u)(A u - a e)), f += 1/2 |A u - a e|^2
};

// flavors of M_SH finalization
enum ShFlavor : int {
  SH_INIT = 0,      // cold start: F = b1 (point), writes r1 = b1, x = 0; sets snorm_b
  SH_REF = 1,       // F = b1 (point), computes ||S^H b|| only (warm start); writes r1 = b1
  SH_WARM = 2,      // F = r1 (from M_RES), starts the solve from the stored x
  SH_REFINE = 3,    // F = q64 = b - S x64 (FP64), output c = S^H q cast to the inner s; outer test
  SH_PLAIN = 4,     // F = r64 (FP64 residual iterate), output S^H r64 cast to gvec; no scalars
};

// ------------------------------------------------------------------ batch descriptors
enum SysState : int { ST_ACTIVE = 0, ST_FINISHING = 1, ST_DONE = 2 };

// Per-system scalars, FP64, living in the workspace.
struct SysDev {
  double gamma;      // ||s||^2 of the current normal-equation residual
  double delta;      // ||S p||^2
  double alpha;      // step length of the current iteration
  double alpha_hist[3];  // step lengths of the three iterations before it, newest first (iterate
                         // updated every m-th iteration: the steps not yet added to x)
  double beta;       // p = s + beta p
  double snorm_b;    // ||S^H b|| (reference of the relative residual)
  double snorm_ref;  // reference norm of the current (inner) solve
  double relres;     // last relative residual
  double tol;        // tolerance of the current (inner) solve, relative to snorm_ref
  int iter;          // iterations of the current (inner) solve
  int iter_total;    // iterations summed over refinements
  int state;         // SysState
  int status;        // WRI_SYS_*
  int outer_done;    // refinement finished for this system
  unsigned ticket;   // tile-completion counter of the running launch
  int group;         // group index
  int local;         // index inside the group
  int rec_begin, rec_end;  // receiver range in the batch-wide receiver arrays
  int part_off;      // first slot of this system in the partial-sum array
  long long src;     // source node
};

struct GroupDev {
  int nx, ny, nz, npml;
  double h, omega, lambda;
  float ih2f, om2f, lambdaf;  // 1/h^2, omega^2, lambda in FP32
  AxisPml ax, ay, az;
  int nsys, sys0;          // systems of the group and global index of the first
  int tiles_x, tiles_y, zsplit, zc, ntiles;
  long long item0, nitems;  // work items (tile x system) of the group in the batched launch
  int masked;               // 1 = source-free (Z applied), 0 = known weight or general right-hand side
  long long n;              // nodes
  const void* m;            // [n] real, float or double (m_double)
  int m_double;             // 1 if m is double (complex128 problems), 0 if float
  const void* d;            // [nnz] complex observed data
  const double* alpha;      // [2*nsys] known weights or null
  const void* q;            // [nsys][n] general PDE right-hand side b1 (complex, q_double), or null
  int q_double;             // 1 if q is double2 (complex128 problems), 0 if float2
  void* x;                  // [nsys][n] iterate (dtype of the stencil)
  void* r1[2];              // [nsys][n] data-space residual, ping-pong
  void* p[4];               // [nsys][n] search direction: p_j in slot (j + 1) mod R, R = 2 (ping-pong) or
                            // 4 (iterate updated every fourth iteration; slots 2, 3 null otherwise)
  void* s;                  // [nsys][n] normal-equation residual S^H r
  void* t1;                 // [nsys][n] Z A p
  void* x64;                // [nsys][n] double2 refinement master of the solution (or null)
  void* r64;                // [nsys][n] double2 refinement master of the residual b1 - Z A x (or null)
  void* q64;                // [nsys][n] double2 true residual b1 - Z A x64 of the outer step (or null)
  const void* gvec;         // [nsys][n] complex64 S^H r64, added to s in phase 2 (or null)
  const int* rmap;          // [nsys][n] receiver entry of a node (-1: none): the FP64 S^H kernels of
                            // the refinement add lambda P^T r2 in the stencil pass (or null)
  const uint32_t* rmask;    // [nsys][nz][ny][tiles_x] receiver bits of the normal-residual norms
                            // (bit b of word (k, j, t): node (32 t + b, j, k) is a receiver), or null
  const uint32_t* rcol;     // [nsys][ny][tiles_x] OR of rmask over k (columns holding a receiver)
  double* grad;             // [n] gradient accumulator (gradient kernel only)
  const float2* ztab;       // [2][nz][3] z-axis coefficients (s_z, 1/(s_z(k-1/2) h^2), 1/(s_z(k+1/2) h^2)),
                            // [0] for A, [1] conjugated for A^H; FP32, built once per call (or null)
  const double2* ztab64;    // the same table in FP64 (the z-march FP64 kernels), or null
};

struct Batch {
  int ngroups;
  int bx, by;           // thread block shape (bx = WRI_TX)
  long long nitems;     // total work items
  SysDev* sys;
  double* partial;      // per (system, tile) FP64 partial sums
  const int* rec_idx;   // batch-wide receiver nodes
  void* r2;             // batch-wide receiver residual (type of the kernel's stencil)
  void* r2_64;          // refinement: FP64 receiver part of the residual master (or null)
  void* r2_in;          // refinement: complex64 receiver residual of the inner solve (or null)
  const void* lamd;     // batch-wide lambda*d (same type as r2)
  int* remaining;       // systems not yet DONE
  double* f;            // objective accumulator (gradient kernel only)
  int max_iter;
  int flavor;           // kernel-specific sub-mode
  int order;            // TMA phases: work-item order, 0 = systems fastest, 1 = tiles of a system
                        // consecutive, 2 = z-chunk slowest (the resident wave shares z-slabs),
                        // 3 = blocks of sblock systems, tiles in order, systems fastest in a block
  int sblock;           // systems per block of order 3
  int xsteps;           // m: phase 1 adds the steps of m iterations to x every m-th iteration (m = 2, 4:
                        // the warp-specialised grouped-update configurations; 0 or 1: every iteration)
  double tol;           // tolerance of a cold-start solve
  double refine_tol, inner_tol;
  int outer, max_refine, warm;
  GroupDev g[WRI_MAXG];
};

// steps per iterate update (1, 2 or 4) and the p ring of a batch
__host__ __device__ __forceinline__ int xsteps_of(const Batch& b) { return b.xsteps > 1 ? b.xsteps : 1; }
__host__ __device__ __forceinline__ int pring_of(const Batch& b) { return b.xsteps == 4 ? 4 : 2; }
// slot of p_j
__host__ __device__ __forceinline__ int pslot(const Batch& b, int j) { return (j + 1) & (pring_of(b) - 1); }

// (system, tile) of a work item of group G under the batch's work order
__device__ __forceinline__ void item_coords(const Batch& b, const GroupDev& G, long long local, int& sl, int& tile) {
  if (b.order == 1) {
    sl = (int)(local / G.ntiles);
    tile = (int)(local % G.ntiles);
  } else if (b.order == 2) {
    const int nxy = G.tiles_x * G.tiles_y;
    const long long per_z = (long long)G.nsys * nxy;
    const int tz = (int)(local / per_z);
    const long long rem = local - (long long)tz * per_z;
    sl = (int)(rem / nxy);
    tile = (int)(rem % nxy) * G.zsplit + tz;
  } else if (b.order == 3) {
    const int sb = min(b.sblock, G.nsys);
    const int nb = (G.nsys + sb - 1) / sb;
    const long long per_block = (long long)sb * G.ntiles;
    const int blk = (int)min(local / per_block, (long long)(nb - 1));
    const long long rem = local - (long long)blk * per_block;
    const int cnt = min(sb, G.nsys - blk * sb);
    tile = (int)(rem / cnt);
    sl = blk * sb + (int)(rem % cnt);
  } else {
    sl = (int)(local % G.nsys);
    tile = (int)(local / G.nsys);
  }
}

__device__ __forceinline__ int find_group(const Batch& b, long long item) {
  int g = 0;
#pragma unroll 1
  for (; g < b.ngroups - 1; ++g)
    if (item < b.g[g + 1].item0) break;
  return g;
}

}  // namespace wri
