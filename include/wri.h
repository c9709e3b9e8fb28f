/*
 * wri.h -- C ABI of libwri: the per-source, per-frequency hot path of source-free
 * Wavefield Reconstruction Inversion (arXiv 2410.18429) on one NVIDIA GB300 (sm_103a).
 *
 * The library solves, for every (source i, frequency j) system of a batch, the
 * augmented least-squares problem of Eqs. ObjPen / CmpctWRIobj / Sandb,
 *
 *     min_u  1/2 || Z A_j u - b1 ||^2 + 1/2 lambda^2 || P_i u - d_ij ||^2 ,
 *
 * with the matrix-free Helmholtz operator A_j = omega_j^2 diag(w m) + L_pml
 * (Sec. "3D Source free WRI": A = omega^2 diag(m) + Laplacian, plus a stretched-
 * coordinate absorbing layer), estimates the source weight a = (A u)[src]
 * (Eq. SimpObj, second block row) and accumulates the model gradient of Eq. VarG2.
 *
 *   source-free mode (alpha == NULL):  Z = I - e e^H,  b1 = 0           (Eq. SimpObj)
 *   known-weight mode (alpha != NULL): Z = I,          b1 = alpha e     (Eq. ObjPen)
 *
 * Conventions shared by every entry point
 *   - lambda weights the DATA term (the paper's lambda_p on the PDE term is 1/lambda);
 *     the minimiser is the same as the paper's.
 *   - Grids are C-ordered [nz][ny][nx], x fastest; node index (k*ny + j)*nx + i.
 *     nx, ny, nz count the computational nodes INCLUDING npml padding cells per face.
 *   - Complex arrays are interleaved (re, im): float2 for WRI_C64, double2 for WRI_C128.
 *     Real arrays (m) are float for WRI_C64 and double for WRI_C128.
 *   - "device" pointers are CUDA device memory owned by the caller; "host" pointers
 *     are ordinary host memory read before the call returns.  The library never
 *     allocates device memory: scratch comes from the caller's workspace.
 *   - Every call enqueues its work on `stream` (a cudaStream_t; 0 is the legacy
 *     default stream).  wri_solve_batch additionally waits on the host for the end of
 *     the solve: the CG iterations loop on the device (a CUDA-graph WHILE node that a
 *     small control kernel keeps going while systems remain), and the host reads the
 *     device counters once per inner solve to return an error code.
 *   - Calls from different host threads may run at the same time on different streams
 *     with different workspaces (per-thread host read-back buffers, a mutex around the
 *     shared graph cache); wri_gradient_noalloc is the exception (see there).
 *   - Return value: WRI_OK or an error code (wri_strerror).  Argument errors are
 *     detected before any work is enqueued.  Per-system outcomes go to device arrays.
 */
#ifndef WRI_H
#define WRI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* wri_stream_t; /* identical to cudaStream_t */

#if defined(__GNUC__)
#define WRI_API __attribute__((visibility("default")))
#else
#define WRI_API
#endif

/* return codes */
#define WRI_OK 0
#define WRI_EINVAL 1      /* invalid argument (null pointer, size, index out of range, ...) */
#define WRI_ECUDA 2       /* a CUDA launch or runtime call failed */
#define WRI_EWORKSPACE 3  /* workspace pointer null, misaligned (256 B) or too small */
#define WRI_ENOTSUP 4     /* valid but unsupported combination of options */
#define WRI_ESCRATCH 5    /* problem larger than the static scratch of wri_gradient_noalloc */

/* per-system status written by wri_solve_batch */
#define WRI_SYS_OK 0         /* relative normal-equation residual <= tol */
#define WRI_SYS_MAXITER 1    /* max_iter reached before tol */
#define WRI_SYS_BREAKDOWN 2  /* ||S p|| = 0 with a non-zero residual (cannot progress) */
#define WRI_SYS_NONFINITE 3  /* a NaN/Inf appeared in a step length or norm */

/* arithmetic of the iterative solve */
#define WRI_C64 0   /* complex64 vectors and stencil, FP64 inner products and scalars */
#define WRI_C128 1  /* complex128 throughout */

/* Grid of one frequency group.  Stretch factor of the absorbing layer on each axis
 * (our reading; the paper states no boundary condition):
 *   s(xi) = 1 + i sigma(xi)/omega,  sigma = sigma_max (xi/L)^2,  L = npml*h,
 *   sigma_max = 3 v_max ln(1/pml_R) / (2 L),  xi = distance into the layer. */
typedef struct {
  int32_t nx, ny, nz; /* computational nodes per axis, >= 3 each, including padding */
  int32_t npml;       /* padding cells per face (0 = no absorbing layer, Dirichlet box) */
  double h;           /* grid spacing (m), > 0 */
  double omega;       /* angular frequency omega_j (rad/s), > 0 */
  double pml_R;       /* target reflection of the layer, in (0, 1) */
  double v_max;       /* velocity (m/s) that sets sigma_max, > 0 */
} wri_grid;

/* One group of systems sharing a grid, a frequency and a model (a "grouped
 * inversion" block of Eq. Mmatrix2, read as block diagonal). */
typedef struct {
  wri_grid grid;
  const void* m;            /* device [n] squared slowness (float | double per dtype) */
  int32_t nsys;             /* systems in the group, >= 1 */
  const int64_t* src_idx;   /* host [nsys] source node of each system */
  const int32_t* rec_off;   /* host [nsys+1] CSR offsets into rec_idx / d, rec_off[0] = 0 */
  const int32_t* rec_idx;   /* host [rec_off[nsys]] receiver nodes; distinct within a system */
  const void* d;            /* device [rec_off[nsys]] observed data (complex, dtype) */
  const double* alpha;      /* device [2*nsys] known weights (complex128) or NULL = source-free */
  double lambda;            /* data weight, > 0; 0 allowed with a known right-hand side (alpha or q):
                               then the solve is the PDE least-squares problem min ||A u - b1||
                               (the forward and adjoint solves of reduced FWI, Eqs. PDEsolve / FWI2) */
  void* u;                  /* device [nsys][n] complex (dtype): in = x0 if warm_start, out = u */
  void* u64;                /* WRI_C64 only, optional: device [nsys][n] complex128 (16-byte aligned)
                               or NULL.  wri_solve_batch also writes the solution here, in FP64
                               (the refinement's FP64 master; without refinement, u widened), and
                               wri_source_estimate / wri_gradient then read it instead of u and use
                               FP64 stencils: the gradient needs the PDE residual A u - a e, which
                               rounding u to complex64 would swamp.  In one call either every
                               group sets it or none does.  Ignored for WRI_C128. */
  const void* q;            /* device [nsys][n] complex (dtype) or NULL: a general PDE right-hand side,
                               b1 = q in place of alpha e (Z = I); alpha must then be NULL.  The
                               adjoint solve of reduced FWI uses it (see wri_fwi_adjoint_source). */
} wri_group;

typedef struct {
  double tol;          /* stop when ||S^H (b - S u)|| <= tol ||S^H b||  (tol >= 0) */
  int32_t max_iter;    /* iteration cap per system (per inner solve when refining), >= 1 */
  int32_t dtype;       /* WRI_C64 or WRI_C128 */
  int32_t warm_start;  /* 1: start from the values in u; 0: start from u = 0 */
  int32_t max_refine;  /* WRI_C64 only: > 0 enables FP64 iterative refinement, at most this
                          many outer corrections; each inner FP32 solve runs to inner_tol, or to
                          the looser tolerance that already meets refine_tol with 5 % of margin
                          (a cold start's first inner solve: max(inner_tol, 0.95 refine_tol)) */
  double refine_tol;   /* refinement stops when the FP64 relative residual <= refine_tol */
  double inner_tol;    /* relative tolerance of each inner FP32 solve (e.g. 1e-3) */
  int32_t plain;       /* 1: unbatched, unfused baseline (one system at a time, separate
                          BLAS-1 kernels, scalars read back by the host every iteration) */
  int32_t poll_every;  /* CG iterations per body of the device-side loop, between two runs of
                          its control kernel (0 = library default, about 300 us of work) */
  int32_t tile;        /* tile configuration (0 = autotuned / default, see wri_tile_count) */
  int32_t zsplit;      /* z-chunks per tile column (0 = chosen from the batch size) */
  int32_t kernel;      /* 0 = automatic (TMA-pipelined phases when the batch allows them),
                          1 = z-march kernels only, 2 + c = TMA configuration c (0..24; 9..24
                          are the warp-specialised kernels; 22 and 23 update the
                          iterate every second iteration, 24 every fourth); see wri_autotune */
  int32_t order;       /* TMA phases: 0 = automatic (6), 1 = tiles of a system consecutive,
                          2 = systems of a tile consecutive, 3 = z-chunk slowest,
                          4 / 5 / 6 = blocks of 4 / 8 / 16 systems, tiles in order */
  int32_t l2_promotion; /* TMA copies: L2 fill size on a miss, 0 = automatic, 1 = none,
                           2 = 64 B, 3 = 128 B, 4 = 256 B */
  int32_t wait_limit_us; /* TMA phases: time limit of every wait of the copy pipelines, in
                            microseconds (0 = 2 s).  A wait that runs out stops the solve:
                            wri_solve_batch returns WRI_ECUDA and the context stays usable. */
  int32_t host_loop;     /* 1: the host replays a graph of poll_every iterations and reads the
                            counters after each replay, instead of the device-side loop (a graph
                            WHILE node).  Kernel profilers cannot see kernels inside conditional
                            graph nodes; this keeps the phase kernels visible to them.  The
                            environment variable WRI_HOST_LOOP=1 sets it for every solve. */
  int32_t test_withhold; /* test hook of the bounded waits, 0 = off.  k > 0: in the warp-specialised
                            TMA phases the copy warp of block 0 never issues its (k-1)-th plane
                            fill, so the wait for it runs out after wait_limit_us.  Nothing
                            faults or hangs; the call returns WRI_ECUDA. */
} wri_solve_opts;

/* y = A x (wri_apply_A) or y = A^H x (wri_apply_AH) for `nsys` vectors that share the
 * grid and model: x, y device [nsys][n] complex (dtype), m device [n] real (dtype).
 * x and y must not overlap.  Operator: Sec. "3D Source free WRI", first paragraph.
 * A is complex symmetric, so A^H x = conj(A conj(x)). */
WRI_API int wri_apply_A(const wri_grid* grid, int dtype, const void* m, int nsys, const void* x, void* y,
                wri_stream_t stream);
WRI_API int wri_apply_AH(const wri_grid* grid, int dtype, const void* m, int nsys, const void* x, void* y,
                 wri_stream_t stream);

/* Bytes of device workspace wri_solve_batch needs for these groups and options
 * (0 on invalid arguments).  The workspace must be 256-byte aligned.  With opts->kernel = 0
 * (automatic) it also covers the four search-direction vectors per system of TMA configuration
 * 24, so that a workspace sized before wri_autotune fits every configuration it may choose. */
WRI_API size_t wri_workspace_size(const wri_group* groups, int ngroups, const wri_solve_opts* opts);

/* Solve every system of every group (the LSQR/CG solve of Eq. SimpObj, Algorithm 1
 * read as CGLS, grouped as in Eq. Mmatrix2 with per-system scalars).
 *   iters  device [sum nsys] int32   iterations per system (summed over refinements)
 *   relres device [sum nsys] double  final ||S^H (b - S u)|| / ||S^H b||
 *   status device [sum nsys] int32   WRI_SYS_*
 * Systems are numbered group by group.  On return the stopping decision has been
 * taken; the results are ordered on `stream`. */
WRI_API int wri_solve_batch(const wri_group* groups, int ngroups, const wri_solve_opts* opts, int32_t* iters,
                    double* relres, int32_t* status, void* workspace, size_t ws_bytes,
                    wri_stream_t stream);

/* Bytes of device workspace wri_source_estimate and wri_gradient need (the device
 * copy of the geometry); wri_workspace_size is always at least this much. */
WRI_API size_t wri_aux_workspace_size(const wri_group* groups, int ngroups);

/* Source-weight estimate a_i = e_i^H A u_i = (A u_i)[src_i] (Eq. SimpObj, second
 * block row), for every system of every group, from the wavefields in groups[g].u.
 * alpha_out: device [2 * sum nsys] complex128.  workspace: >= wri_aux_workspace_size. */
WRI_API int wri_source_estimate(const wri_group* groups, int ngroups, int dtype, double* alpha_out,
                        void* workspace, size_t ws_bytes, wri_stream_t stream);

/* Gradient and objective of Eqs. VarG2 / VarObj2 accumulated over every system:
 *   grad[g][k] += sum_i omega^2 Re( conj(w_k u_ik) (A u_i - a_i e_i)_k )
 *   f[0]       += sum_i 1/2 ||A u_i - a_i e_i||^2 + 1/2 lambda^2 ||P_i u_i - d_i||^2
 * a_i = alpha_in (device [2 * sum nsys] complex128), normally wri_source_estimate's output
 * in source-free mode or the known weights otherwise.  grad: host array of ngroups
 * device pointers, each [n_g] double; f: device [1] double.  The caller zeroes them.
 * Systems of a group are summed in a fixed order per node; f is summed with FP64
 * atomics (last-bit order dependence).  workspace: >= wri_aux_workspace_size. */
WRI_API int wri_gradient(const wri_group* groups, int ngroups, int dtype, const double* alpha_in,
                 double* const* grad, double* f, void* workspace, size_t ws_bytes,
                 wri_stream_t stream);

/* Gradient and objective of Eqs. VarG2 / VarObj2 (the same results as wri_gradient) after a refined
 * solve, without a stencil pass: wri_solve_batch with max_refine > 0 and u64 on every group ends
 * with an FP64 residual step, and leaves q = b - S u64 of every system in its workspace.  Its node
 * part is b1 - Z A u64, and A u - a e = -(b1 - Z A u) (source-free: a = (A u)[src] zeroes the
 * source row as Z does; known weight: b1 = alpha e), so
 *   grad[g][k] += -omega^2 sum_i Re( conj(w_k u_ik) q1_ik ),   f[0] += 1/2 ||q1||^2 + 1/2 ||q2||^2
 * with q2 = lambda (d - P u).  It reads u64 and q once (32 bytes per node and system).
 *   - Call it after that wri_solve_batch, with the same groups (unchanged arrays) and options and
 *     the same workspace, on the same stream or after synchronising with it.  The library records
 *     which problem's residual a workspace holds (a later wri_solve_batch or wri_autotune on the
 *     workspace drops the record; wri_source_estimate and wri_gradient do not touch that part of
 *     it) and returns WRI_EINVAL when the record does not match these arguments.
 *   - grad: host array of ngroups device pointers, each [n_g] double; f: device [1] double; the
 *     caller zeroes them.  f is summed with FP64 atomics (last-bit order dependence).
 *   - The source weights, when wanted, come from wri_source_estimate (one stencil per system). */
WRI_API int wri_gradient_refined(const wri_group* groups, int ngroups, const wri_solve_opts* opts,
                                 double* const* grad, double* f, const void* workspace, size_t ws_bytes,
                                 wri_stream_t stream);

/* Reduced FWI, the paper's comparison method (Eqs. FWI, PDEsolve and FWI2), on libwri's solves:
 *   1. forward solves A G_i = e_i: wri_solve_batch with alpha = 1 and lambda = 0 (u = G);
 *   2. wri_fwi_adjoint_source: the weights a_i (given, or source-free the minimiser of
 *      ||a P G_i - d_i||: a_i = (P G_i)^H d_i / ||P G_i||^2), the data residuals
 *      r_i = a_i P G_i - d_i, f += 1/2 sum ||r_i||^2 (Eq. FWI2), and the adjoint right-hand sides
 *      conj(P^T r_i);
 *   3. adjoint solves A w_i = conj(P^T r_i): wri_solve_batch with q set and lambda = 0.  A is
 *      complex symmetric, so v_i = conj(w_i) solves A^H v_i = P^T r_i;
 *   4. wri_fwi_gradient: grad[k] += -omega^2 sum_i Re(w_k a_i G_ik conj(v_ik))
 *      = -omega^2 sum_i Re(w_k a_i G_ik w_ik)  (the adjoint-state gradient; the weight's own
 *      derivative vanishes at its optimum).
 * groups: the forward solves' groups (grid, m, geometry, d; u = G).
 *   alpha_in:  device [2 * sum nsys] complex128 known weights, or NULL (source-free)
 *   alpha_out: device [2 * sum nsys] complex128, the weights used
 *   q_adj:     host array of ngroups device pointers, each [nsys][n] complex (dtype); written only
 *              at the receiver nodes, so the caller zeroes them first
 *   f:         device [1] double, accumulated (FP64 atomics)
 *   workspace: >= wri_aux_workspace_size(groups, ngroups) */
WRI_API int wri_fwi_adjoint_source(const wri_group* groups, int ngroups, int dtype, const double* alpha_in,
                                   double* alpha_out, void* const* q_adj, double* f, void* workspace,
                                   size_t ws_bytes, wri_stream_t stream);
/*   w: host array of ngroups device pointers, each [nsys][n] complex (dtype), the adjoint solves'
 *      wavefields; alpha: the weights of wri_fwi_adjoint_source; grad: host array of ngroups device
 *      pointers, each [n] double, accumulated (the caller zeroes them).  Systems of a group are
 *      summed in a fixed order per node. */
WRI_API int wri_fwi_gradient(const wri_group* groups, int ngroups, int dtype, const double* alpha,
                             void* const* w, double* const* grad, wri_stream_t stream);

/* Allocation-free variant of wri_gradient (the paper has no counterpart: this is an
 * interface for callers that cannot call cudaMalloc, e.g. code whose device memory is
 * owned by another allocator such as a framework's caching pool that has reserved the
 * GPU, or a latency-critical loop that must not pay cudaMalloc's implicit device
 * synchronisation).  Same arguments and results as wri_gradient, without the
 * workspace: the device copy of the geometry goes to a static device array of
 * WRI_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until exit.
 *   - Problems whose geometry needs more than that (wri_aux_workspace_size) are
 *     rejected with WRI_ESCRATCH before any work is enqueued.
 *   - The first call on a device looks up the array's device address (with that device
 *     current); make that first call before any stream capture.
 *   - Every call reuses the same array and overwrites what it needs; two calls whose
 *     work overlaps on the GPU (different streams, or different host threads) race on
 *     it and must be serialised by the caller.
 *   - The call itself allocates no device memory (no cudaMalloc / cudaFree, no
 *     allocating library routine); grad and f are the caller's. */
#define WRI_NOALLOC_SCRATCH_BYTES (4u << 20)
WRI_API int wri_gradient_noalloc(const wri_group* groups, int ngroups, int dtype, const double* alpha_in,
                                 double* const* grad, double* f, wri_stream_t stream);

/* Autotuner of the batched solve (an interface outside the paper, which prescribes no
 * kernel configuration).  For a complex64 batch it times `trial_iters` CGLS iterations (>= 2)
 * of every candidate pair (TMA configuration 8, 9, 12, 13, 17, 18, 22 or 24 x work-item order 2, 5
 * or 6)
 * on the caller's own batch, on `stream`, and writes the fastest into opts->kernel and
 * opts->order (other fields unchanged).  With refinement (max_refine > 0) the candidates are
 * the warp-specialised configurations (9, 12, 13, 17, 18, 22, 24), which run its inner solves, and the
 * trials are plain CGLS solves.  Candidates whose workspace exceeds ws_bytes are skipped.
 *   - groups[g].u is used as the iterate of the trial solves: its contents are overwritten.
 *   - The choice is cached for the process, keyed by the device, the grids, the system counts
 *     and the receiver counts: a repeated call for the same batch shape returns the cached
 *     choice without timing anything (and without touching u).
 *   - Batches the TMA phases cannot take (complex128, the unfused baseline, an x extent that is
 *     not a multiple of 4) keep opts unchanged and return WRI_OK.
 *   - Synchronises `stream` (it reads event timings on the host). */
WRI_API int wri_autotune(const wri_group* groups, int ngroups, wri_solve_opts* opts, int trial_iters,
                         void* workspace, size_t ws_bytes, wri_stream_t stream);

/* Total-variation term of Eq. TVAWRI, for the outer loop (Algorithm 2), not the solve.  Our
 * reading of the paper's ||m||_TV: the smoothed isotropic TV
 *     TV(m) = sum over nodes of sqrt(dx^2 + dy^2 + dz^2 + beta^2),
 * forward differences in grid units (dx = m[i+1] - m[i], zero on the last node of an axis).
 *   m    device [n] double on the grid of `grid` (only nx, ny, nz are used; the grid must be
 *        valid as for the other calls)
 *   tv   device [1] double: tv += gamma TV(m) (FP64 atomics: last-bit order dependence)
 *   grad device [n] double: grad += gamma dTV/dm, or NULL
 * beta > 0 and gamma >= 0 (WRI_EINVAL otherwise).  Enqueued on `stream`. */
WRI_API int wri_tv(const wri_grid* grid, const double* m, double beta, double gamma, double* tv, double* grad,
                   wri_stream_t stream);

/* Number of built tile configurations of the z-march kernels and the thread-block shape of one
 * of them (tile = 1..count; WRI_EINVAL otherwise).  Outside the paper: an implementation
 * choice exposed for tuning. */
WRI_API int wri_tile_count(void);
WRI_API int wri_tile_shape(int tile, int* bx, int* by);

/* Static description of an error code (never NULL; "unknown error code" for other values). */
WRI_API const char* wri_strerror(int code);

/* Library version string, with the hash of the kernel sources it was built from (profiles
 * record it, so measurements taken on another build can be told apart). */
WRI_API const char* wri_version(void);

#ifdef __cplusplus
}
#endif
#endif /* WRI_H */
