// C ABI of libwri (include/wri.h): argument validation, workspace layout, launch
// sequencing, the CUDA-graph-captured CG iteration loop, FP64 iterative refinement
// and the unfused baseline path.  All arithmetic runs in the kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "../../include/wri.h"
#include "wri_launch.h"
#include "wri_tma.cuh"

using namespace wri;

namespace {

constexpr int kRefSMs = 152;  // SMs of a GB300; sets the z-split of small batches
// Measured defaults of the TMA phases on GB300 (128 sources x 3 frequency grids): the
// warp-specialised kernel (a copy warp and 4 consumer warps, two nodes per thread, 32 x 8
// tiles, 4 stages, 4 CTAs/SM); work items in blocks of 16 systems (neighbouring tiles of a
// system run together, so their halos meet in L2); L2 fills of 64 bytes on a copy miss
// (128-byte fills over-fetch the halo columns).  wri_autotune refines the choice per batch.
constexpr int kDefaultTmaCfg = 9;
constexpr int kFirstWsCfg = 9;  // configurations from here on are the warp-specialised kernels
constexpr int kDefaultOrder = 6;
constexpr int kDefaultPromotion = 2;
constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

int by_of_tile(int tile) {
  switch (tile) {
    case 1: return 4;
    case 3: return 16;
    default: return 8;
  }
}

#define WRI_CK(call)                          \
  do {                                        \
    cudaError_t e_ = (call);                  \
    if (e_ != cudaSuccess) return WRI_ECUDA;  \
  } while (0)

bool grid_valid(const wri_grid* g) {
  if (!g) return false;
  if (g->nx < 3 || g->ny < 3 || g->nz < 3) return false;
  if (g->npml < 0 || 2 * g->npml >= g->nx || 2 * g->npml >= g->ny || 2 * g->npml >= g->nz) return false;
  if (!(g->h > 0) || !std::isfinite(g->h) || !(g->omega > 0) || !std::isfinite(g->omega)) return false;
  if (g->npml > 0) {
    if (!(g->pml_R > 0 && g->pml_R < 1)) return false;
    if (!(g->v_max > 0) || !std::isfinite(g->v_max)) return false;
  }
  const long long n = (long long)g->nx * g->ny * g->nz;
  return n > 0 && n < (1LL << 40);
}

long long grid_n(const wri_grid& g) { return (long long)g.nx * g.ny * g.nz; }

AxisPml axis(int n, const wri_grid& g) {
  AxisPml a;
  a.n = n;
  a.npml = g.npml;
  a.h = g.h;
  a.inv_omega = 1.0 / g.omega;
  if (g.npml > 0) {
    const double L = g.npml * g.h;
    a.smax = 3.0 * g.v_max * std::log(1.0 / g.pml_R) / (2.0 * L);
    a.invL = 1.0 / L;
  } else {
    a.smax = 0.0;
    a.invL = 0.0;
  }
  a.hf = (float)a.h;
  a.inv_omegaf = (float)a.inv_omega;
  a.smaxf = (float)a.smax;
  a.invLf = (float)a.invL;
  return a;
}

void fill_geom(GroupDev& G, const wri_grid& g) {
  G.nx = g.nx;
  G.ny = g.ny;
  G.nz = g.nz;
  G.npml = g.npml;
  G.h = g.h;
  G.omega = g.omega;
  G.ih2f = (float)(1.0 / (g.h * g.h));
  G.om2f = (float)(g.omega * g.omega);
  G.ax = axis(g.nx, g);
  G.ay = axis(g.ny, g);
  G.az = axis(g.nz, g);
  G.n = grid_n(g);
}

// tiles_x, tiles_y, zsplit, zc of a grid for a given batch size
void decompose(const wri_grid& g, int by, int zs_req, GroupDev& G) {
  G.tiles_x = (g.nx + WRI_TX - 1) / WRI_TX;
  G.tiles_y = (g.ny + by - 1) / by;
  int zs = std::max(1, std::min(zs_req, std::max(1, g.nz / 4)));
  G.zc = (g.nz + zs - 1) / zs;
  G.zsplit = (g.nz + G.zc - 1) / G.zc;
  G.ntiles = G.tiles_x * G.tiles_y * G.zsplit;
}

// z-chunks per tile column when the caller leaves it open: the count that minimises the modelled
// time of one launch, the waves of resident CTAs (items / (152 SMs x 4 CTAs), rounded up) times the
// planes each item streams (its chunk plus the two halo planes), over 1..16 chunks of >= 4 planes.
// Large batches keep whole columns (one chunk); a single system of a 148^3 grid gets 6 chunks of 25
// planes, one wave of 570 items.
int auto_zsplit(long long xy_items, int nz) {
  const long long wave = (long long)kRefSMs * 4;
  int best = 1;
  double best_cost = 0.0;
  for (int zs = 1; zs <= 16 && zs <= std::max(1, nz / 4); ++zs) {
    const int zc = (nz + zs - 1) / zs;
    const long long items = xy_items * ((nz + zc - 1) / zc);
    const double cost = (double)((items + wave - 1) / wave) * (zc + 2);
    if (zs == 1 || cost < best_cost) {
      best_cost = cost;
      best = zs;
    }
  }
  return best;
}

int validate_groups(const wri_group* groups, int ngroups, bool need_data) {
  if (!groups || ngroups < 1 || ngroups > WRI_MAXG) return WRI_EINVAL;
  long long nsys_total = 0;
  for (int gi = 0; gi < ngroups; ++gi) {
    const wri_group& G = groups[gi];
    if (!grid_valid(&G.grid)) return WRI_EINVAL;
    if (!G.m || !G.u || G.nsys < 1 || !G.src_idx || !G.rec_off || !G.rec_idx) return WRI_EINVAL;
    if (!(G.lambda >= 0) || !std::isfinite(G.lambda)) return WRI_EINVAL;
    if (G.alpha && G.q) return WRI_EINVAL;                   // one right-hand side
    if (G.lambda == 0 && !G.alpha && !G.q) return WRI_EINVAL;  // source-free needs the data term
    const long long n = grid_n(G.grid);
    if (G.rec_off[0] != 0) return WRI_EINVAL;
    for (int s = 0; s < G.nsys; ++s) {
      if (G.src_idx[s] < 0 || G.src_idx[s] >= n) return WRI_EINVAL;
      const int a = G.rec_off[s], b = G.rec_off[s + 1];
      if (b < a) return WRI_EINVAL;
      std::vector<int> r(G.rec_idx + a, G.rec_idx + b);
      for (int v : r)
        if (v < 0 || v >= n) return WRI_EINVAL;
      std::sort(r.begin(), r.end());
      if (std::adjacent_find(r.begin(), r.end()) != r.end()) return WRI_EINVAL;
    }
    if (need_data && G.rec_off[G.nsys] > 0 && !G.d) return WRI_EINVAL;
    nsys_total += G.nsys;
  }
  if (nsys_total > (1 << 24)) return WRI_EINVAL;
  return WRI_OK;
}

struct Plan {
  int ngroups = 0, nsys_total = 0, nnz_total = 0, dtype = 0, ir = 0, by = 8;
  int tma_cfg = -1;  // TMA configuration of the CG phases, -1 = z-march kernels
  bool host_loop = false;  // the host replays the iteration graph (no conditional node)
  int vbytes = 8;   // bytes of one complex of the iteration vectors
  int rlbytes = 8;  // bytes of one complex of lamd / r2
  long long nitems = 0;
  long long nparts = 0;
  size_t off_sys = 0, off_rec = 0, off_part = 0, off_rem = 0, off_lamd = 0, off_r2 = 0;
  size_t off_r2_64 = 0, off_r2_in = 0;  // refinement: FP64 receiver residual master, complex64 inner r2
  size_t aux_total = 0, total = 0;
  GroupDev g[WRI_MAXG];
  size_t v_r1[WRI_MAXG][2], v_p[WRI_MAXG][4], v_s[WRI_MAXG], v_t1[WRI_MAXG];
  int pslots = 2;  // search-direction slots: 4 when the phases may update x every fourth iteration
  size_t v_x32[WRI_MAXG], v_x64[WRI_MAXG], v_r64[WRI_MAXG], v_q64[WRI_MAXG], v_g32[WRI_MAXG], v_rmap[WRI_MAXG];
  size_t off_ztab[WRI_MAXG], off_ztab64[WRI_MAXG];  // z-coefficient tables (FP32, FP64) per group
  size_t off_rmask[WRI_MAXG], off_rcol[WRI_MAXG], rmask_bytes[WRI_MAXG], rcol_bytes[WRI_MAXG];
  std::vector<int> rec_base;  // first receiver entry of every group
};

void plan_aux(const wri_group* groups, int ngroups, Plan& P) {
  P.ngroups = ngroups;
  P.nsys_total = 0;
  P.nnz_total = 0;
  P.rec_base.assign(ngroups, 0);
  for (int gi = 0; gi < ngroups; ++gi) {
    P.rec_base[gi] = P.nnz_total;
    P.nsys_total += groups[gi].nsys;
    P.nnz_total += groups[gi].rec_off[groups[gi].nsys];
  }
  size_t off = 0;
  P.off_sys = off;
  off += align_up(sizeof(SysDev) * (size_t)P.nsys_total);
  P.off_rec = off;
  off += align_up(sizeof(int) * (size_t)std::max(P.nnz_total, 1));
  for (int gi = 0; gi < ngroups; ++gi) {  // [2][nz][3] complex coefficients in FP32 and FP64
    P.off_ztab[gi] = off;
    off += align_up(sizeof(float) * 2 * 2 * 3 * (size_t)groups[gi].grid.nz);
    P.off_ztab64[gi] = off;
    off += align_up(sizeof(double) * 2 * 2 * 3 * (size_t)groups[gi].grid.nz);
  }
  P.aux_total = off;
  P.total = off;
}

bool host_loop_forced() {
  static const bool forced = [] {
    const char* v = std::getenv("WRI_HOST_LOOP");
    return v && v[0] == '1';
  }();
  return forced;
}

void plan_solve(const wri_group* groups, int ngroups, const wri_solve_opts* o, Plan& P) {
  plan_aux(groups, ngroups, P);
  P.dtype = o->dtype;
  P.host_loop = o->host_loop != 0 || host_loop_forced();
  P.ir = (o->dtype == WRI_C64 && o->max_refine > 0) ? 1 : 0;
  P.by = by_of_tile(o->tile);
  P.tma_cfg = -1;
  if (!o->plain && o->kernel != 1 && o->dtype == WRI_C64) {
    bool ok = true;
    // the refinement's inner iterate lives in the workspace; otherwise the TMA phases update u
    for (int gi = 0; gi < ngroups; ++gi)
      ok = ok && (groups[gi].grid.nx % 4 == 0) && (P.ir || (uintptr_t)groups[gi].u % 16 == 0);
    if (ok) {
      P.tma_cfg = o->kernel >= 2 ? o->kernel - 2 : kDefaultTmaCfg;
      // the refinement's inner phase 2 adds S^H r64, which only the warp-specialised kernels do
      if (P.ir && P.tma_cfg < kFirstWsCfg) P.tma_cfg = kDefaultTmaCfg;
      P.by = tma_config_by(P.tma_cfg);
      // a ring of four directions for the configurations that update x every fourth iteration; the
      // automatic choice reserves it too, so that wri_autotune may pick them in the same workspace
      P.pslots = (o->kernel == 0 || tma_config_xsteps(P.tma_cfg) == 4) ? 4 : 2;
    }
  }
  P.vbytes = (o->dtype == WRI_C128) ? 16 : 8;
  P.rlbytes = (o->dtype == WRI_C128 || P.ir) ? 16 : 8;
  long long xy_items = 0;
  for (int gi = 0; gi < ngroups; ++gi) {
    const wri_grid& g = groups[gi].grid;
    xy_items += (long long)groups[gi].nsys * ((g.nx + WRI_TX - 1) / WRI_TX) * ((g.ny + P.by - 1) / P.by);
  }
  int nz_max = 0;
  for (int gi = 0; gi < ngroups; ++gi) nz_max = std::max(nz_max, groups[gi].grid.nz);
  const int zs = o->zsplit > 0 ? o->zsplit
                               : auto_zsplit(o->plain ? xy_items / std::max(1, P.nsys_total) : xy_items, nz_max);
  long long item = 0, parts = 0;
  int sys0 = 0;
  for (int gi = 0; gi < ngroups; ++gi) {
    GroupDev& G = P.g[gi];
    std::memset(&G, 0, sizeof(G));
    fill_geom(G, groups[gi].grid);
    decompose(groups[gi].grid, P.by, zs, G);
    G.nsys = groups[gi].nsys;
    G.sys0 = sys0;
    G.item0 = item;
    G.nitems = (long long)G.ntiles * G.nsys;
    item += G.nitems;
    parts += G.nitems;
    sys0 += G.nsys;
  }
  P.nitems = item;
  P.nparts = parts;
  size_t off = P.total;
  P.off_part = off;
  off += align_up(sizeof(double) * (size_t)std::max<long long>(parts, 4096));
  P.off_rem = off;
  off += kAlign;
  P.off_lamd = off;
  off += align_up((size_t)P.rlbytes * std::max(P.nnz_total, 1));
  P.off_r2 = off;
  off += align_up((size_t)P.rlbytes * std::max(P.nnz_total, 1));
  P.off_r2_64 = P.off_r2_in = 0;
  if (P.ir) {
    P.off_r2_64 = off;
    off += align_up(16 * (size_t)std::max(P.nnz_total, 1));
    P.off_r2_in = off;
    off += align_up(8 * (size_t)std::max(P.nnz_total, 1));
  }
  for (int gi = 0; gi < ngroups; ++gi) {  // receiver bitmaps (one bit per node and system)
    const GroupDev& G = P.g[gi];
    P.rcol_bytes[gi] = 4 * (size_t)G.nsys * G.ny * G.tiles_x;
    P.rmask_bytes[gi] = P.rcol_bytes[gi] * (size_t)G.nz;
    P.off_rcol[gi] = off;
    off += align_up(P.rcol_bytes[gi]);
    P.off_rmask[gi] = off;
    off += align_up(P.rmask_bytes[gi]);
  }
  for (int gi = 0; gi < ngroups; ++gi) {
    const size_t vb = align_up((size_t)P.vbytes * (size_t)P.g[gi].nsys * (size_t)P.g[gi].n);
    P.v_r1[gi][0] = off; off += vb;
    P.v_r1[gi][1] = off; off += vb;
    P.v_p[gi][0] = off; off += vb;
    P.v_p[gi][1] = off; off += vb;
    P.v_p[gi][2] = P.v_p[gi][3] = 0;
    if (P.pslots == 4) {
      P.v_p[gi][2] = off; off += vb;
      P.v_p[gi][3] = off; off += vb;
    }
    P.v_s[gi] = off; off += vb;
    P.v_t1[gi] = off; off += vb;
    P.v_x32[gi] = P.v_x64[gi] = P.v_r64[gi] = P.v_q64[gi] = P.v_g32[gi] = P.v_rmap[gi] = 0;
    if (P.ir) {
      const size_t nn = (size_t)P.g[gi].nsys * (size_t)P.g[gi].n;
      P.v_x32[gi] = off; off += align_up(8 * nn);
      P.v_x64[gi] = off; off += align_up(16 * nn);
      P.v_r64[gi] = off; off += align_up(16 * nn);
      P.v_q64[gi] = off; off += align_up(16 * nn);
      P.v_g32[gi] = off; off += align_up(8 * nn);
      P.v_rmap[gi] = off; off += align_up(4 * nn);
    }
  }
  P.total = off;
}

int validate_opts(const wri_solve_opts* o) {
  if (!o) return WRI_EINVAL;
  if (o->dtype != WRI_C64 && o->dtype != WRI_C128) return WRI_EINVAL;
  if (!(o->tol >= 0) || !std::isfinite(o->tol) || o->max_iter < 1) return WRI_EINVAL;
  if (o->max_refine < 0 || o->poll_every < 0 || o->tile < 0 || o->tile > 3 || o->zsplit < 0) return WRI_EINVAL;
  if (o->kernel < 0 || o->kernel > 1 + tma_config_count()) return WRI_EINVAL;
  if (o->order < 0 || o->order > 6) return WRI_EINVAL;
  if (o->l2_promotion < 0 || o->l2_promotion > 4) return WRI_EINVAL;
  if (o->wait_limit_us < 0 || o->test_withhold < 0 || o->host_loop < 0 || o->host_loop > 1) return WRI_EINVAL;
  if (o->max_refine > 0) {
    if (o->dtype != WRI_C64) return WRI_ENOTSUP;
    if (!(o->refine_tol >= 0) || !(o->inner_tol > 0 && o->inner_tol < 1)) return WRI_EINVAL;
    if (o->plain) return WRI_ENOTSUP;
  }
  return WRI_OK;
}

// Host copies of the per-system descriptors and the batch-wide receiver list.
void build_sys(const wri_group* groups, int ngroups, const Plan& P, std::vector<SysDev>& sys,
               std::vector<int>& rec) {
  sys.assign(P.nsys_total, SysDev());
  rec.clear();
  rec.reserve(std::max(P.nnz_total, 1));
  int s = 0;
  long long part = 0;
  for (int gi = 0; gi < ngroups; ++gi) {
    const wri_group& G = groups[gi];
    for (int l = 0; l < G.nsys; ++l, ++s) {
      SysDev& d = sys[s];
      std::memset(&d, 0, sizeof(d));
      d.group = gi;
      d.local = l;
      d.src = G.src_idx[l];
      d.rec_begin = (int)rec.size();
      for (int k = G.rec_off[l]; k < G.rec_off[l + 1]; ++k) rec.push_back(G.rec_idx[k]);
      d.rec_end = (int)rec.size();
      d.part_off = (int)part;
      part += P.g[gi].ntiles;
      d.state = ST_DONE;
      d.status = WRI_SYS_OK;
    }
  }
  if (rec.empty()) rec.push_back(0);
}

// Per-device state shared by every call on that device: the stream graphs are captured on and
// the cache of instantiated CG-iteration graphs.  Both are guarded by g_mu; a cached graph is
// reference-counted, so evicting it while another thread still launches it is safe.
struct DevCtx {
  cudaStream_t cap = nullptr;
  struct Entry {
    std::vector<unsigned char> key;
    std::shared_ptr<CUgraphExec_st> exec;
    bool device_loop = false;  // the graph loops on the device (conditional WHILE node)
  };
  std::vector<Entry> graphs;
};
std::mutex g_mu;
DevCtx g_ctx[64];

// Pinned host words through which a call reads its own device counters (systems remaining, the
// copy-wait error flag, loop bodies run) and the unfused path its scalars: one block per host
// thread and device, so concurrent calls from different threads never share it.  A call runs
// on one host thread from start to end.
struct PollSlots {
  int* p[64] = {};
  ~PollSlots() {
    for (int* q : p)
      if (q) cudaFreeHost(q);
  }
};
thread_local PollSlots tl_poll;

int* poll_slot() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  if (!tl_poll.p[dev] && cudaHostAlloc((void**)&tl_poll.p[dev], 64, cudaHostAllocDefault) != cudaSuccess) {
    tl_poll.p[dev] = nullptr;
    return nullptr;
  }
  return tl_poll.p[dev];
}
struct Tuned {
  std::vector<long long> key;  // device, groups, then per group nx, ny, nz, nsys, receivers
  int kernel, order;
};
std::vector<Tuned> g_tuned;  // choices of wri_autotune, guarded by g_mu

// Workspaces that hold the FP64 residual b - S u64 of a finished refined solve, with the signature
// of that solve's problem (wri_gradient_refined reads the residual); guarded by g_mu.
struct ResidualStamp {
  const void* ws;
  std::vector<unsigned long long> sig;
};
std::vector<ResidualStamp> g_stamps;

unsigned long long fnv(const void* p, size_t bytes, unsigned long long h = 1469598103934665603ull) {
  const unsigned char* c = (const unsigned char*)p;
  for (size_t i = 0; i < bytes; ++i) h = (h ^ c[i]) * 1099511628211ull;
  return h;
}

// What the residual left in a workspace depends on: the workspace layout, every group's grid,
// arrays and geometry, and the precision options.
std::vector<unsigned long long> residual_signature(const wri_group* groups, int ngroups, const wri_solve_opts* o,
                                                   size_t total) {
  std::vector<unsigned long long> sig = {total, (unsigned long long)ngroups, (unsigned long long)o->dtype};
  for (int gi = 0; gi < ngroups; ++gi) {
    const wri_group& G = groups[gi];
    sig.push_back(fnv(&G.grid, sizeof(wri_grid)));
    const void* ptrs[6] = {G.m, G.d, (const void*)G.alpha, (const void*)G.u, G.u64, G.q};
    for (const void* p : ptrs) sig.push_back((uintptr_t)p);
    sig.push_back(fnv(&G.lambda, sizeof(double)));
    sig.push_back((unsigned long long)G.nsys);
    sig.push_back(fnv(G.src_idx, sizeof(int64_t) * G.nsys));
    sig.push_back(fnv(G.rec_off, sizeof(int32_t) * (G.nsys + 1)));
    sig.push_back(fnv(G.rec_idx, sizeof(int32_t) * G.rec_off[G.nsys]));
  }
  return sig;
}

void forget_residual(const void* ws) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_stamps.erase(std::remove_if(g_stamps.begin(), g_stamps.end(),
                                [&](const ResidualStamp& r) { return r.ws == ws; }),
                 g_stamps.end());
}

DevCtx* ctx() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  DevCtx* c = &g_ctx[dev];
  std::lock_guard<std::mutex> lk(g_mu);
  if (!c->cap && cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess) {
    c->cap = nullptr;
    return nullptr;
  }
  return c;
}

cudaError_t march(int rbytes, int obytes, int mode, bool conj, int by, const Batch& b, cudaStream_t st) {
  if (b.nitems <= 0) return cudaSuccess;
  if (rbytes == 4) return launch_march_f32(mode, conj, by, b, 0, st);
  if (obytes == 8) return launch_march_f64(mode, conj, by, b, 0, st);
  return launch_march_f64_to_f32(mode, by, b, 0, st);
}

// Base batch for the solver: geometry, workspace pointers, per-group vector views.
Batch solver_batch(const wri_group* groups, const Plan& P, char* ws, bool inner_view) {
  Batch b;
  std::memset(&b, 0, sizeof(b));
  b.ngroups = P.ngroups;
  b.bx = WRI_TX;
  b.by = P.by;
  b.nitems = P.nitems;
  b.sys = (SysDev*)(ws + P.off_sys);
  b.partial = (double*)(ws + P.off_part);
  b.rec_idx = (const int*)(ws + P.off_rec);
  b.r2 = ws + P.off_r2;
  b.lamd = ws + P.off_lamd;
  b.remaining = (int*)(ws + P.off_rem);
  if (P.ir) {
    b.r2_64 = ws + P.off_r2_64;
    b.r2_in = ws + P.off_r2_in;
    if (inner_view) b.r2 = b.r2_in;  // the FP32 inner solve keeps its receiver residual in complex64
  }
  for (int gi = 0; gi < P.ngroups; ++gi) {
    GroupDev G = P.g[gi];
    const wri_group& U = groups[gi];
    G.lambda = U.lambda;
    G.masked = (U.alpha || U.q) ? 0 : 1;
    G.m = U.m;
    G.m_double = P.dtype == WRI_C128 ? 1 : 0;
    G.d = U.d;
    G.alpha = U.alpha;
    G.q = U.q;
    G.q_double = P.dtype == WRI_C128 ? 1 : 0;
    G.r1[0] = ws + P.v_r1[gi][0];
    G.r1[1] = ws + P.v_r1[gi][1];
    G.p[0] = ws + P.v_p[gi][0];
    G.p[1] = ws + P.v_p[gi][1];
    G.p[2] = P.pslots == 4 ? ws + P.v_p[gi][2] : nullptr;
    G.p[3] = P.pslots == 4 ? ws + P.v_p[gi][3] : nullptr;
    G.s = ws + P.v_s[gi];
    G.t1 = ws + P.v_t1[gi];
    G.x = (P.ir && inner_view) ? (void*)(ws + P.v_x32[gi]) : U.u;
    G.x64 = P.ir ? ws + P.v_x64[gi] : nullptr;
    G.r64 = P.ir ? ws + P.v_r64[gi] : nullptr;
    G.q64 = P.ir ? ws + P.v_q64[gi] : nullptr;
    G.gvec = (P.ir && inner_view) ? ws + P.v_g32[gi] : nullptr;
    G.ztab = (const float2*)(ws + P.off_ztab[gi]);
    G.ztab64 = (const double2*)(ws + P.off_ztab64[gi]);
    G.rmask = (const uint32_t*)(ws + P.off_rmask[gi]);
    G.rcol = (const uint32_t*)(ws + P.off_rcol[gi]);
    b.g[gi] = G;
  }
  return b;
}

// Receiver bitmaps of every group (the normal-residual norms leave receiver nodes to the finalizer)
int setup_rmask(const Plan& P, const Batch& b, char* ws, cudaStream_t st) {
  for (int gi = 0; gi < P.ngroups; ++gi) {
    WRI_CK(cudaMemsetAsync(ws + P.off_rcol[gi], 0, P.rcol_bytes[gi], st));
    WRI_CK(cudaMemsetAsync(ws + P.off_rmask[gi], 0, P.rmask_bytes[gi], st));
  }
  WRI_CK(launch_rmask(b, P.nsys_total, st));
  return WRI_OK;
}

int poll_default(const Plan& P) {
  double bytes = 0;
  for (int gi = 0; gi < P.ngroups; ++gi) bytes += 80.0 * P.g[gi].nsys * (double)P.g[gi].n;
  const double t_iter = bytes / 6.0e12 + 6e-6;  // seconds per CG iteration of the batch (estimate)
  int k = (int)std::ceil(300e-6 / t_iter);
  return std::max(2, std::min(k, 256));
}

// ---------------------------------------------------------------- TMA descriptors
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

// 4-D map over [nsys][nz][ny][nx] complex64 vectors (8-byte elements); box bx x by x 1 x 1
CUtensorMapL2promotion promo_of(int p) {
  switch (p) {
    case 1: return CU_TENSOR_MAP_L2_PROMOTION_NONE;
    case 2: return CU_TENSOR_MAP_L2_PROMOTION_L2_64B;
    case 3: return CU_TENSOR_MAP_L2_PROMOTION_L2_128B;
    case 4: return CU_TENSOR_MAP_L2_PROMOTION_L2_256B;
  }
  return CU_TENSOR_MAP_L2_PROMOTION_NONE;
}

bool encode_vec(CUtensorMap* m, const void* base, const GroupDev& G, int bx, int by, int promo) {
  const cuuint64_t dims[4] = {(cuuint64_t)G.nx, (cuuint64_t)G.ny, (cuuint64_t)G.nz, (cuuint64_t)G.nsys};
  const cuuint64_t strides[3] = {(cuuint64_t)G.nx * 8, (cuuint64_t)G.nx * G.ny * 8, (cuuint64_t)G.n * 8};
  const cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)by, 1, 1};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  return encode_fn()(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, const_cast<void*>(base), dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, promo_of(promo),
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 3-D map over the float model [nz][ny][nx]; box 32 x by x 1
bool encode_model(CUtensorMap* m, const void* base, const GroupDev& G, int by, int promo) {
  const cuuint64_t dims[3] = {(cuuint64_t)G.nx, (cuuint64_t)G.ny, (cuuint64_t)G.nz};
  const cuuint64_t strides[2] = {(cuuint64_t)G.nx * 4, (cuuint64_t)G.nx * G.ny * 4};
  const cuuint32_t box[3] = {WRI_TX, (cuuint32_t)by, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  return encode_fn()(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, promo_of(promo),
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool build_tma(const Batch& b, const Plan& P, int* err, int promo, const wri_solve_opts* o, TmaSet& T) {
  if (!encode_fn()) return false;
  std::memset(&T, 0, sizeof(T));
  T.err = err;
  T.wait_ns = o->wait_limit_us > 0 ? 1000ull * (unsigned long long)o->wait_limit_us : kWaitLimitNs;
  T.withhold = o->test_withhold > 0 ? o->test_withhold - 1 : -1;
  const int hw = WRI_TX + 4, hh = P.by + 2, pr = promo;
  for (int gi = 0; gi < b.ngroups; ++gi) {
    const GroupDev& G = b.g[gi];
    bool ok = encode_vec(&T.map[gi][TM_S], G.s, G, hw, hh, pr) && encode_vec(&T.map[gi][TM_P0], G.p[0], G, hw, hh, pr) &&
              encode_vec(&T.map[gi][TM_P1], G.p[1], G, hw, hh, pr) &&
              encode_vec(&T.map[gi][TM_X], G.x, G, WRI_TX, P.by, pr) && encode_vec(&T.map[gi][TM_T1], G.t1, G, hw, hh, pr) &&
              encode_vec(&T.map[gi][TM_R0], G.r1[0], G, hw, hh, pr) && encode_vec(&T.map[gi][TM_R1], G.r1[1], G, hw, hh, pr) &&
              encode_model(&T.map[gi][TM_M], G.m, G, P.by, pr) &&
              encode_vec(&T.map[gi][TM_PC0], G.p[0], G, WRI_TX, P.by, pr) &&
              encode_vec(&T.map[gi][TM_PC1], G.p[1], G, WRI_TX, P.by, pr);
    for (int slot = 2; slot < 4 && ok; ++slot)
      if (G.p[slot])
        ok = encode_vec(&T.map[gi][TM_P0 + slot], G.p[slot], G, hw, hh, pr) &&
             encode_vec(&T.map[gi][TM_PC0 + slot], G.p[slot], G, WRI_TX, P.by, pr);
    if (!ok) return false;
  }
  return true;
}

// Conditional graph nodes (a WHILE node whose condition a device kernel sets) available?
bool device_loop_supported() {
  static int ok = -1;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaGraph_t g = nullptr;
    cudaGraphConditionalHandle h;
    ok = (cudaGraphCreate(&g, 0) == cudaSuccess &&
          cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) == cudaSuccess)
             ? 1
             : 0;
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
  });
  return ok == 1;
}

// Captures K CG iterations (phase 1 + phase 2 launches) on c->cap into whatever capture is open.
cudaError_t capture_iterations(const Plan& P, const Batch& b1, const Batch& b2, int mode2, int K, int rb,
                               bool use_tma, const TmaSet* tma, cudaStream_t cap) {
  cudaError_t err = cudaSuccess;
  for (int k = 0; k < K && err == cudaSuccess; ++k) {
    if (use_tma) {
      err = launch_phase_tma(M_P1, P.tma_cfg, b1, *tma, 0, cap);
      if (err == cudaSuccess) err = launch_phase_tma(M_P2, P.tma_cfg, b2, *tma, 0, cap);
    } else {
      err = march(rb, rb, M_P1, false, P.by, b1, cap);
      if (err == cudaSuccess) err = march(rb, rb, mode2, true, P.by, b2, cap);
    }
  }
  return err;
}

// Runs CG iterations (phase 1 + phase 2) until no system remains.  The iterations are captured
// once per batch shape in a CUDA graph whose WHILE node repeats a body of K iterations and a tiny
// control kernel on the device, with no host round trip; the host reads the counters once at the
// end.  (Without conditional nodes the graph holds K iterations and the host replays it, reading
// the counters after every replay.)  The workspace counters are: [0] systems not yet done, [1] the
// copy-wait error flag, [2] loop bodies run.
int run_loop(const Plan& P, const Batch& b1_in, const Batch& b2_in, int mode2, int K, int max_iter, cudaStream_t st,
             const TmaSet* tma = nullptr) {
  DevCtx* c = ctx();
  int* slot = poll_slot();
  if (!c || !slot) return WRI_ECUDA;
  const int rb = P.ir ? 4 : P.vbytes / 2;
  const bool use_tma = tma && P.tma_cfg >= 0 && mode2 == M_P2;
  // iterate updates every m-th iteration: only the grouped-update configurations' phase-1 kernel
  // does them (m = 4 needs the four direction slots)
  Batch b1 = b1_in, b2 = b2_in;
  int xs = use_tma ? tma_config_xsteps(P.tma_cfg) : 1;
  if (xs == 4 && !b1.g[0].p[2]) return WRI_EINVAL;
  b1.xsteps = b2.xsteps = xs;
  const bool dev_loop = !P.host_loop && device_loop_supported();
  // loop bodies after which the device loop gives up: every system stops by max_iter + 1 iterations
  const int cap_bodies = (max_iter + 2 + K - 1) / K + 2;
  // graph lookup / capture
  std::vector<unsigned char> key(sizeof(Batch) * 2 + 7 * sizeof(int) + (use_tma ? sizeof(TmaSet) : 0));
  std::memcpy(key.data(), &b1, sizeof(Batch));
  std::memcpy(key.data() + sizeof(Batch), &b2, sizeof(Batch));
  const int extra[7] = {mode2, K, P.by, rb, use_tma ? P.tma_cfg : -1, dev_loop ? 1 : 0, cap_bodies};
  std::memcpy(key.data() + 2 * sizeof(Batch), extra, sizeof(extra));
  if (use_tma) std::memcpy(key.data() + 2 * sizeof(Batch) + sizeof(extra), tma, sizeof(TmaSet));
  std::shared_ptr<CUgraphExec_st> exec;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto& e : c->graphs)
      if (e.key == key) exec = e.exec;
    if (!exec) {
      cudaGraph_t graph = nullptr;
      cudaGraphExec_t raw = nullptr;
      cudaError_t err = cudaSuccess;
      if (dev_loop) {
        WRI_CK(cudaGraphCreate(&graph, 0));
        cudaGraphConditionalHandle h;
        err = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
        cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        if (err == cudaSuccess) err = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np);
        if (err == cudaSuccess) {
          cudaGraph_t body = np.conditional.phGraph_out[0];
          err = cudaStreamBeginCaptureToGraph(c->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
          if (err == cudaSuccess) {
            err = capture_iterations(P, b1, b2, mode2, K, rb, use_tma, tma, c->cap);
            if (err == cudaSuccess) err = launch_loop_ctl(h, b1.remaining, cap_bodies, c->cap);
            const cudaError_t e2 = cudaStreamEndCapture(c->cap, &body);
            if (err == cudaSuccess) err = e2;
          }
        }
      } else {
        WRI_CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeRelaxed));
        err = capture_iterations(P, b1, b2, mode2, K, rb, use_tma, tma, c->cap);
        const cudaError_t e2 = cudaStreamEndCapture(c->cap, &graph);
        if (err == cudaSuccess) err = e2;
      }
      if (err == cudaSuccess) err = cudaGraphInstantiate(&raw, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (err != cudaSuccess) return WRI_ECUDA;
      exec = std::shared_ptr<CUgraphExec_st>(raw, [](cudaGraphExec_t x) { cudaGraphExecDestroy(x); });
      if (c->graphs.size() >= 8) c->graphs.erase(c->graphs.begin());  // freed once no launch holds it
      DevCtx::Entry e;
      e.key = key;
      e.exec = exec;
      e.device_loop = dev_loop;
      c->graphs.push_back(e);
    }
  }
  if (dev_loop) {
    WRI_CK(cudaMemsetAsync(b1.remaining + 2, 0, sizeof(int), st));
    WRI_CK(cudaGraphLaunch(exec.get(), st));
    WRI_CK(cudaMemcpyAsync(slot, b1.remaining, 3 * sizeof(int), cudaMemcpyDeviceToHost, st));
    WRI_CK(cudaStreamSynchronize(st));
    if (slot[1] != 0) return WRI_ECUDA;  // a bounded copy wait timed out
    if (slot[0] > 0) return WRI_ECUDA;   // a system failed to stop by max_iter (cannot happen)
    return WRI_OK;
  }
  long long launched = 0;
  for (;;) {
    WRI_CK(cudaGraphLaunch(exec.get(), st));
    launched += K;
    WRI_CK(cudaMemcpyAsync(slot, b1.remaining, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    WRI_CK(cudaStreamSynchronize(st));
    if (slot[1] != 0) return WRI_ECUDA;  // a bounded copy wait timed out
    if (slot[0] <= 0) break;
    if (launched > (long long)max_iter + 2 * K + 2) return WRI_ECUDA;  // a system failed to stop
  }
  return WRI_OK;
}

int upload(const wri_group* groups, int ngroups, const Plan& P, char* ws, cudaStream_t st) {
  std::vector<SysDev> sys;
  std::vector<int> rec;
  build_sys(groups, ngroups, P, sys, rec);
  WRI_CK(cudaMemcpyAsync(ws + P.off_sys, sys.data(), sizeof(SysDev) * sys.size(), cudaMemcpyHostToDevice, st));
  WRI_CK(cudaMemcpyAsync(ws + P.off_rec, rec.data(), sizeof(int) * rec.size(), cudaMemcpyHostToDevice, st));
  return WRI_OK;
}

int check_ws(const Plan& P, const void* ws, size_t bytes) {
  if (!ws || ((uintptr_t)ws % kAlign) != 0 || bytes < P.total) return WRI_EWORKSPACE;
  return WRI_OK;
}

// ---------------------------------------------------------------- fused, batched solve
int solve_fused(const wri_group* groups, int ngroups, const wri_solve_opts* o, const Plan& P, char* ws,
                cudaStream_t st) {
  Batch b = solver_batch(groups, P, ws, false);
  b.max_iter = o->max_iter;
  b.tol = o->tol;
  const int vb = P.vbytes / 2;
  if (setup_rmask(P, b, ws, st) != WRI_OK) return WRI_ECUDA;
  WRI_CK(launch_ztable(b, st));
  WRI_CK(launch_setup_rhs(o->dtype == WRI_C128 ? 8 : 4, vb, b, P.nsys_total, st));
  WRI_CK(cudaMemsetAsync(b.remaining, 0, 3 * sizeof(int), st));
  if (o->warm_start) {
    Batch r = b;
    r.flavor = SH_REF;
    WRI_CK(march(vb, vb, M_SH, true, P.by, r, st));
    r.flavor = 0;
    WRI_CK(march(vb, vb, M_RES, false, P.by, r, st));
    r.flavor = SH_WARM;
    WRI_CK(march(vb, vb, M_SH, true, P.by, r, st));
  } else {
    Batch r = b;
    r.flavor = SH_INIT;
    WRI_CK(march(vb, vb, M_SH, true, P.by, r, st));
  }
  Batch b1 = b, b2 = b;
  b1.flavor = b2.flavor = 0;
  const int ord = o->order ? o->order : kDefaultOrder;
  b1.order = b2.order = (ord == 1) ? 1 : (ord == 3) ? 2 : (ord >= 4) ? 3 : 0;
  b1.sblock = b2.sblock = (ord >= 4) ? (1 << (ord - 2)) : 1;  // 4 -> 4 systems, 5 -> 8, 6 -> 16
  const int K = o->poll_every > 0 ? o->poll_every : poll_default(P);
  if (P.tma_cfg >= 0) {
    static thread_local TmaSet T;  // ~8 KB: kept off the stack
    if (build_tma(b, P, b.remaining + 1, o->l2_promotion ? o->l2_promotion : kDefaultPromotion, o, T))
      return run_loop(P, b1, b2, M_P2, std::min(K, o->max_iter + 1), o->max_iter, st, &T);
    // descriptors rejected (e.g. an unaligned model array): same decomposition, z-march kernels
  }
  return run_loop(P, b1, b2, M_P2, std::min(K, o->max_iter + 1), o->max_iter, st);
}

// ---------------------------------------------------------------- FP64 iterative refinement
// Augmented-system refinement (Bjorck) of min ||S x - b|| with complex64 inner solves: the
// solution x64 and the residual r64 live in FP64.  Each outer step computes, with FP64
// stencils, q = b - S x64, the outer test c = S^H q (||c|| / ||S^H b|| <= refine_tol), the
// forcing f = q - r64 and g' = S^H r64; the complex64 CGLS inner solve (phase 2 adds g')
// then returns dx and dr = f - S dx, and x64 += dx, r64 += dr.  The inner accuracy needed
// scales with u32 kappa(S), not with u32 kappa(S)^2 as for refinement on the normal equations.
int solve_refined(const wri_group* groups, int ngroups, const wri_solve_opts* o, const Plan& P, char* ws,
                  cudaStream_t st) {
  int* slot = poll_slot();
  if (!slot) return WRI_ECUDA;
  // FP64 views: the residual kernel reads x64 and writes q64 (nodes) and b.r2 = q2 (receivers)
  Batch outer = solver_batch(groups, P, ws, false);
  for (int gi = 0; gi < P.ngroups; ++gi) {
    outer.g[gi].x = outer.g[gi].x64;
    outer.g[gi].r1[0] = outer.g[gi].q64;
    outer.g[gi].rmap = (const int*)(ws + P.v_rmap[gi]);
    WRI_CK(cudaMemsetAsync(ws + P.v_rmap[gi], 0xff, 4 * (size_t)P.g[gi].nsys * (size_t)P.g[gi].n, st));
  }
  WRI_CK(launch_ir_rmap(outer, P.nsys_total, st));
  outer.max_iter = o->max_iter;
  outer.tol = o->tol;
  outer.refine_tol = o->refine_tol;
  outer.inner_tol = o->inner_tol;
  outer.max_refine = o->max_refine;
  outer.warm = o->warm_start ? 1 : 0;
  // complex64 views: x = dx, r2 = r2_in, gvec = g'
  Batch inner = solver_batch(groups, P, ws, true);
  inner.max_iter = o->max_iter;
  if (setup_rmask(P, inner, ws, st) != WRI_OK) return WRI_ECUDA;
  WRI_CK(launch_ztable(inner, st));  // the outer view shares the tables
  void* u[WRI_MAXG] = {};
  for (int gi = 0; gi < P.ngroups; ++gi) u[gi] = groups[gi].u;
  // lambda d in FP64 (lamd and q2), x64 = warm ? u : 0, r64 = 0, dx = 0
  WRI_CK(launch_setup_rhs(4, 8, outer, P.nsys_total, st));
  WRI_CK(launch_ir_init(inner, u, o->warm_start ? 1 : 0, st));
  if (o->warm_start) {  // ||S^H b|| with the FP64 stencil (q2 still holds lambda d)
    Batch r = outer;
    r.flavor = SH_REF;
    WRI_CK(launch_march_f64_to_f32(M_SH, P.by, r, 0, st));
  }
  // g' = S^H r64 (FP64 stencil on r64 and r2_64, rounded into the inner gvec)
  Batch gb = outer;
  gb.flavor = SH_PLAIN;
  gb.r2 = gb.r2_64;
  for (int gi = 0; gi < P.ngroups; ++gi) {
    gb.g[gi].r1[0] = gb.g[gi].r64;
    gb.g[gi].s = const_cast<void*>(inner.g[gi].gvec);
  }
  const int K = o->poll_every > 0 ? o->poll_every : poll_default(P);
  // inner solves on the warp-specialised TMA phases when the batch allows them
  const TmaSet* tma = nullptr;
  static thread_local TmaSet T;
  if (P.tma_cfg >= 0) {
    const int ord = o->order ? o->order : kDefaultOrder;
    inner.order = (ord == 1) ? 1 : (ord == 3) ? 2 : (ord >= 4) ? 3 : 0;
    inner.sblock = (ord >= 4) ? (1 << (ord - 2)) : 1;
    if (build_tma(inner, P, inner.remaining + 1, o->l2_promotion ? o->l2_promotion : kDefaultPromotion, o, T))
      tma = &T;
  }
  int first_outer = 0;
  if (!o->warm_start) {
    // Cold start: x64 = 0 and r64 = 0, so the first outer step's residual is b itself and needs no
    // FP64 pass.  The first inner solve starts like an unrefined solve, from r = b (the point field
    // b1 and lambda d) and s = S^H b formed in FP32; ||S^H b|| is the reference of every outer test.
    WRI_CK(launch_ir_cold(inner, P.nsys_total, st));               // r2_in = lambda d (complex64)
    WRI_CK(cudaMemsetAsync(inner.remaining, 0, 3 * sizeof(int), st));
    Batch r = inner;
    r.flavor = SH_INIT;
    r.tol = std::max(o->inner_tol, 0.95 * o->refine_tol);
    WRI_CK(march(4, 4, M_SH, true, P.by, r, st));                  // s = S^H b, r1 = b1, dx = 0
    WRI_CK(cudaMemcpyAsync(slot, inner.remaining, sizeof(int), cudaMemcpyDeviceToHost, st));
    WRI_CK(cudaStreamSynchronize(st));
    if (*slot > 0) {
      Batch in = inner;
      for (int gi = 0; gi < P.ngroups; ++gi) in.g[gi].gvec = nullptr;  // r64 = 0: no g'
      const int rc = run_loop(P, in, in, M_P2, std::min(K, o->max_iter + 1), o->max_iter, st, tma);
      if (rc != WRI_OK) return rc;
      WRI_CK(launch_ir_update(inner, st));                         // x64 = dx, r64 = dr
    }
    first_outer = 1;
  }
  for (int outer_k = first_outer;; ++outer_k) {
    WRI_CK(cudaMemsetAsync(outer.remaining, 0, 3 * sizeof(int), st));
    Batch r = outer;
    r.outer = outer_k;
    r.flavor = SH_REFINE;
    WRI_CK(march(8, 8, M_RES, false, P.by, r, st));                // q = b - S x64
    WRI_CK(launch_ir_forcing(inner, outer.r2, st));                // f = q - r64 (complex64)
    WRI_CK(launch_march_f64_to_f32(M_SH, P.by, r, 0, st));         // c = S^H q, outer test
    WRI_CK(cudaMemcpyAsync(slot, outer.remaining, sizeof(int), cudaMemcpyDeviceToHost, st));
    WRI_CK(cudaStreamSynchronize(st));
    if (*slot <= 0) break;
    Batch in = inner;
    if (outer_k == 0) {
      // r64 = 0 (k_ir_init), so g' = S^H r64 = 0: the first inner solve is plain CGLS, and its
      // phase 2 reads no g'
      for (int gi = 0; gi < P.ngroups; ++gi) in.g[gi].gvec = nullptr;
    } else {
      WRI_CK(launch_march_f64_to_f32(M_SH, P.by, gb, 0, st));      // g' = S^H r64
    }
    const int rc = run_loop(P, in, in, M_P2, std::min(K, o->max_iter + 1), o->max_iter, st, tma);
    if (rc != WRI_OK) return rc;
    WRI_CK(launch_ir_update(inner, st));                           // x64 += dx, r64 += dr
    if (outer_k > o->max_refine + 1) return WRI_ECUDA;
  }
  WRI_CK(launch_ir_final(inner, u, st));
  return WRI_OK;
}

// ---------------------------------------------------------------- unfused baseline
// One system at a time: separate stencil, BLAS-1 and dot kernels, every scalar read
// back by the host.  Iterates and stopping rule are those of the fused path.
int solve_plain(const wri_group* groups, int ngroups, const wri_solve_opts* o, const Plan& P, char* ws,
                int32_t* iters, double* relres, int32_t* status, cudaStream_t st) {
  int* slot = poll_slot();
  if (!slot) return WRI_ECUDA;
  double* pinned_d = (double*)(slot + 4);
  const int rb = P.vbytes / 2;
  const size_t cb = P.vbytes;
  double* part = (double*)(ws + P.off_part);
  double* dres = part + 2048;  // two device scalars after the dot partials
  std::vector<SysDev> sys;
  std::vector<int> rec;
  build_sys(groups, ngroups, P, sys, rec);
  const int* rec_dev = (const int*)(ws + P.off_rec);
  int sidx = 0;
  for (int gi = 0; gi < ngroups; ++gi) {
    const wri_group& U = groups[gi];
    GroupDev G1 = P.g[gi];
    G1.lambda = U.lambda;
    G1.masked = (U.alpha || U.q) ? 0 : 1;
    G1.m = U.m;
    G1.m_double = P.dtype == WRI_C128 ? 1 : 0;
    decompose(U.grid, P.by, o->zsplit > 0 ? o->zsplit : auto_zsplit((long long)G1.tiles_x * G1.tiles_y, U.grid.nz),
              G1);
    G1.nsys = 1;
    G1.sys0 = 0;
    G1.item0 = 0;
    G1.nitems = G1.ntiles;
    const long long n = G1.n;
    for (int l = 0; l < U.nsys; ++l, ++sidx) {
      const SysDev& sd = sys[sidx];
      const int nr = sd.rec_end - sd.rec_begin;
      char* r1 = ws + P.v_r1[gi][0] + (size_t)l * n * cb;
      char* p = ws + P.v_p[gi][0] + (size_t)l * n * cb;
      char* s = ws + P.v_s[gi] + (size_t)l * n * cb;
      char* t1 = ws + P.v_t1[gi] + (size_t)l * n * cb;
      char* x = (char*)U.u + (size_t)l * n * cb;
      char* r2 = ws + P.off_r2 + (size_t)sd.rec_begin * cb;
      char* t2 = ws + P.off_lamd + (size_t)sd.rec_begin * cb;
      const char* dd = (const char*)U.d + (size_t)(sd.rec_begin - P.rec_base[gi]) * cb;
      const int* rc = rec_dev + sd.rec_begin;
      Batch a;
      std::memset(&a, 0, sizeof(a));
      a.ngroups = 1;
      a.bx = WRI_TX;
      a.by = P.by;
      a.nitems = G1.nitems;
      a.g[0] = G1;
      auto apply = [&](const void* in, void* out, bool conj) -> cudaError_t {
        Batch q = a;
        q.g[0].x = const_cast<void*>(in);
        q.g[0].s = out;
        return march(rb, rb, M_APPLY, conj, P.by, q, st);
      };
      auto dot2 = [&](const void* v1, long long n1, const void* v2, long long n2, double& out) -> int {
        WRI_CK(plain_dot(rb, v1, n1, part, dres, st));
        if (v2 && n2 > 0) WRI_CK(plain_dot(rb, v2, n2, part, dres + 1, st));
        WRI_CK(cudaMemcpyAsync(pinned_d, dres, sizeof(double) * ((v2 && n2 > 0) ? 2 : 1),
                               cudaMemcpyDeviceToHost, st));
        WRI_CK(cudaStreamSynchronize(st));
        out = pinned_d[0] + ((v2 && n2 > 0) ? pinned_d[1] : 0.0);
        return WRI_OK;
      };
      // b1 = alpha e (known weight) or 0; the weight lives on the device
      double ar = 0.0, ai = 0.0;
      if (U.alpha) {
        WRI_CK(cudaMemcpyAsync(pinned_d, U.alpha + 2 * l, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
        WRI_CK(cudaStreamSynchronize(st));
        ar = pinned_d[0];
        ai = pinned_d[1];
      }
      WRI_CK(plain_fill(rb, r1, x, n, U.alpha ? sd.src : -1, ar, ai, st));
      if (U.q)  // general right-hand side: r1 = b1 = q
        WRI_CK(cudaMemcpyAsync(r1, (const char*)U.q + (size_t)l * n * cb, (size_t)n * cb, cudaMemcpyDeviceToDevice, st));
      WRI_CK(plain_setr2(rb, r2, dd, nr, U.lambda, st));
      WRI_CK(apply(r1, s, true));
      WRI_CK(plain_scatter(rb, s, rc, r2, nr, U.lambda, st));
      double gamma = 0.0;
      if (dot2(s, n, nullptr, 0, gamma) != WRI_OK) return WRI_ECUDA;
      const double ref = std::sqrt(gamma);
      int it = 0, stat = WRI_SYS_OK;
      double rr = gamma > 0 ? 1.0 : 0.0;
      if (gamma > 0 && std::isfinite(gamma) && !(ref <= o->tol * ref)) {
        WRI_CK(cudaMemcpyAsync(p, s, (size_t)n * cb, cudaMemcpyDeviceToDevice, st));
        for (;;) {
          WRI_CK(apply(p, t1, false));
          WRI_CK(plain_gather_mask(rb, t2, p, rc, nr, U.lambda, t1, sd.src, (U.alpha || U.q) ? 0 : 1, st));
          double delta = 0.0;
          if (dot2(t1, n, t2, nr, delta) != WRI_OK) return WRI_ECUDA;
          if (!(delta > 0) || !std::isfinite(delta)) {
            stat = std::isfinite(delta) ? WRI_SYS_BREAKDOWN : WRI_SYS_NONFINITE;
            break;
          }
          const double al = gamma / delta;
          WRI_CK(plain_axpy(rb, x, p, al, n, st));
          WRI_CK(plain_axpy(rb, r1, t1, -al, n, st));
          WRI_CK(plain_axpy(rb, r2, t2, -al, nr, st));
          WRI_CK(apply(r1, s, true));
          WRI_CK(plain_scatter(rb, s, rc, r2, nr, U.lambda, st));
          double gn = 0.0;
          if (dot2(s, n, nullptr, 0, gn) != WRI_OK) return WRI_ECUDA;
          ++it;
          rr = std::sqrt(gn) / ref;
          if (!std::isfinite(gn)) {
            stat = WRI_SYS_NONFINITE;
            break;
          }
          if (std::sqrt(gn) <= o->tol * ref) break;
          if (it >= o->max_iter) {
            stat = WRI_SYS_MAXITER;
            break;
          }
          const double beta = gn / gamma;
          gamma = gn;
          WRI_CK(plain_xpby(rb, p, s, beta, n, st));
        }
      } else if (!std::isfinite(gamma)) {
        stat = WRI_SYS_NONFINITE;
      }
      if (gamma == 0.0) rr = 0.0;
      WRI_CK(cudaMemcpyAsync(iters + sidx, &it, sizeof(int), cudaMemcpyHostToDevice, st));
      WRI_CK(cudaMemcpyAsync(relres + sidx, &rr, sizeof(double), cudaMemcpyHostToDevice, st));
      WRI_CK(cudaMemcpyAsync(status + sidx, &stat, sizeof(int), cudaMemcpyHostToDevice, st));
      WRI_CK(cudaStreamSynchronize(st));
    }
  }
  return WRI_OK;
}

int apply_common(const wri_grid* grid, int dtype, const void* m, int nsys, const void* x, void* y,
                 cudaStream_t st, bool conj) {
  if (!grid_valid(grid) || !m || !x || !y || nsys < 1) return WRI_EINVAL;
  if (dtype != WRI_C64 && dtype != WRI_C128) return WRI_EINVAL;
  const long long n = grid_n(*grid);
  const size_t vb = (dtype == WRI_C128 ? 16 : 8);
  const char* xs = (const char*)x;
  const char* ys = (const char*)y;
  const size_t bytes = (size_t)n * nsys * vb;
  if (xs < ys + bytes && ys < xs + bytes) return WRI_EINVAL;  // overlap
  Batch b;
  std::memset(&b, 0, sizeof(b));
  b.ngroups = 1;
  b.bx = WRI_TX;
  b.by = 8;
  GroupDev& G = b.g[0];
  fill_geom(G, *grid);
  decompose(*grid, 8, auto_zsplit((long long)nsys * ((grid->nx + WRI_TX - 1) / WRI_TX) * ((grid->ny + 7) / 8), grid->nz),
            G);
  G.nsys = nsys;
  G.item0 = 0;
  G.nitems = (long long)G.ntiles * nsys;
  G.m = m;
  G.m_double = dtype == WRI_C128 ? 1 : 0;
  G.x = const_cast<void*>(x);
  G.s = y;
  b.nitems = G.nitems;
  const int rb = dtype == WRI_C128 ? 8 : 4;
  WRI_CK(march(rb, rb, M_APPLY, conj, 8, b, st));
  return WRI_OK;
}

// Precision of the source estimate / gradient: complex128 problems and complex64 problems whose
// groups all carry an FP64 wavefield (u64) run FP64 kernels (*wide); u64 on some groups only is an error.
int aux_precision(const wri_group* groups, int ngroups, int dtype, bool* wide) {
  int with = 0;
  for (int gi = 0; gi < ngroups; ++gi) {
    if (groups[gi].u64 && ((uintptr_t)groups[gi].u64 % 16) != 0) return WRI_EINVAL;
    with += groups[gi].u64 ? 1 : 0;
  }
  if (dtype == WRI_C128) {
    *wide = false;
    return WRI_OK;
  }
  if (with != 0 && with != ngroups) return WRI_EINVAL;
  *wide = with == ngroups;
  return WRI_OK;
}

// geometry-only batch for the source estimate / gradient
Batch aux_batch(const wri_group* groups, int ngroups, const Plan& P, char* ws, int dtype, bool wide = false) {
  Batch b;
  std::memset(&b, 0, sizeof(b));
  b.ngroups = ngroups;
  b.bx = WRI_TX;
  b.by = 8;
  // ws == nullptr: a geometry-only batch (no device copy of the systems, no tables)
  b.sys = ws ? (SysDev*)(ws + P.off_sys) : nullptr;
  b.rec_idx = ws ? (const int*)(ws + P.off_rec) : nullptr;
  int sys0 = 0;
  long long item = 0;
  for (int gi = 0; gi < ngroups; ++gi) {
    GroupDev& G = b.g[gi];
    fill_geom(G, groups[gi].grid);
    G.lambda = groups[gi].lambda;
    G.nsys = groups[gi].nsys;
    G.sys0 = sys0;
    G.masked = (groups[gi].alpha || groups[gi].q) ? 0 : 1;
    G.q = groups[gi].q;
    G.q_double = dtype == WRI_C128 ? 1 : 0;
    G.m = groups[gi].m;
    G.m_double = dtype == WRI_C128 ? 1 : 0;
    G.d = groups[gi].d;
    G.x = wide ? groups[gi].u64 : groups[gi].u;
    G.ztab = ws ? (const float2*)(ws + P.off_ztab[gi]) : nullptr;
    G.ztab64 = ws ? (const double2*)(ws + P.off_ztab64[gi]) : nullptr;
    // gradient decomposition: one work item per tile, systems looped inside
    G.tiles_x = (G.nx + WRI_TX - 1) / WRI_TX;
    G.tiles_y = (G.ny + 7) / 8;
    G.zc = grad_zc(8);
    G.zsplit = (G.nz + G.zc - 1) / G.zc;
    G.ntiles = G.tiles_x * G.tiles_y * G.zsplit;
    G.item0 = item;
    G.nitems = G.ntiles;
    item += G.nitems;
    sys0 += G.nsys;
  }
  b.nitems = item;
  return b;
}

// ---------------------------------------------------------------- allocation-free gradient
// Scratch of wri_gradient_noalloc: the device copy of the geometry (per-system
// descriptors and receiver list).  Host code must not hand the symbol itself to a
// kernel; it looks up the device address once per device (noalloc_scratch).
static __device__ __align__(256) unsigned char g_noalloc_scratch[WRI_NOALLOC_SCRATCH_BYTES];
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[64];

int noalloc_scratch(char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return WRI_ECUDA;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return WRI_ECUDA;
    g_noalloc_ptr[dev] = p;
  }
  *out = (char*)g_noalloc_ptr[dev];
  return WRI_OK;
}

}  // namespace

extern "C" {

int wri_gradient_noalloc(const wri_group* groups, int ngroups, int dtype, const double* alpha_in,
                         double* const* grad, double* f, wri_stream_t stream) {
  if (dtype != WRI_C64 && dtype != WRI_C128) return WRI_EINVAL;
  int rc = validate_groups(groups, ngroups, true);
  if (rc != WRI_OK) return rc;
  if (!alpha_in || !grad || !f) return WRI_EINVAL;
  for (int gi = 0; gi < ngroups; ++gi)
    if (!grad[gi]) return WRI_EINVAL;
  bool wide = false;
  rc = aux_precision(groups, ngroups, dtype, &wide);
  if (rc != WRI_OK) return rc;
  Plan P;
  plan_aux(groups, ngroups, P);
  if (P.aux_total > (size_t)WRI_NOALLOC_SCRATCH_BYTES) return WRI_ESCRATCH;
  char* ws = nullptr;
  rc = noalloc_scratch(&ws);
  if (rc != WRI_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  rc = upload(groups, ngroups, P, ws, st);  // overwrites every byte the kernels read
  if (rc != WRI_OK) return rc;
  Batch b = aux_batch(groups, ngroups, P, ws, dtype, wide);
  b.f = f;
  for (int gi = 0; gi < ngroups; ++gi) {
    b.g[gi].alpha = alpha_in + 2 * b.g[gi].sys0;
    b.g[gi].grad = grad[gi];
  }
  const int rb = (dtype == WRI_C128 || wide) ? 8 : 4;
  WRI_CK(launch_ztable(b, st));
  WRI_CK(march(rb, rb, M_GRAD, false, 8, b, st));
  WRI_CK(launch_data_term(rb, dtype == WRI_C128 ? 8 : 4, b, P.nsys_total, st));
  return WRI_OK;
}


int wri_apply_A(const wri_grid* grid, int dtype, const void* m, int nsys, const void* x, void* y,
                wri_stream_t stream) {
  return apply_common(grid, dtype, m, nsys, x, y, (cudaStream_t)stream, false);
}

int wri_apply_AH(const wri_grid* grid, int dtype, const void* m, int nsys, const void* x, void* y,
                 wri_stream_t stream) {
  return apply_common(grid, dtype, m, nsys, x, y, (cudaStream_t)stream, true);
}

size_t wri_workspace_size(const wri_group* groups, int ngroups, const wri_solve_opts* opts) {
  if (validate_opts(opts) != WRI_OK || validate_groups(groups, ngroups, false) != WRI_OK) return 0;
  Plan P;
  plan_solve(groups, ngroups, opts, P);
  return P.total;
}

size_t wri_aux_workspace_size(const wri_group* groups, int ngroups) {
  if (validate_groups(groups, ngroups, false) != WRI_OK) return 0;
  Plan P;
  plan_aux(groups, ngroups, P);
  return P.aux_total;
}

int wri_solve_batch(const wri_group* groups, int ngroups, const wri_solve_opts* opts, int32_t* iters,
                    double* relres, int32_t* status, void* workspace, size_t ws_bytes, wri_stream_t stream) {
  int rc = validate_opts(opts);
  if (rc != WRI_OK) return rc;
  rc = validate_groups(groups, ngroups, true);
  if (rc != WRI_OK) return rc;
  if (!iters || !relres || !status) return WRI_EINVAL;
  for (int gi = 0; gi < ngroups; ++gi)
    if (groups[gi].u64 && ((uintptr_t)groups[gi].u64 % 16) != 0) return WRI_EINVAL;
  Plan P;
  plan_solve(groups, ngroups, opts, P);
  rc = check_ws(P, workspace, ws_bytes);
  if (rc != WRI_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  forget_residual(workspace);
  rc = upload(groups, ngroups, P, ws, st);
  if (rc != WRI_OK) return rc;
  if (opts->plain) {
    rc = solve_plain(groups, ngroups, opts, P, ws, iters, relres, status, st);
  } else {
    rc = P.ir ? solve_refined(groups, ngroups, opts, P, ws, st) : solve_fused(groups, ngroups, opts, P, ws, st);
    if (rc == WRI_OK)
      WRI_CK(launch_export((const SysDev*)(ws + P.off_sys), P.nsys_total, iters, relres, status, st));
  }
  if (rc != WRI_OK) return rc;
  if (opts->dtype == WRI_C64)  // the FP64 wavefield output
    for (int gi = 0; gi < ngroups; ++gi) {
      if (!groups[gi].u64) continue;
      const long long cnt = (long long)groups[gi].nsys * grid_n(groups[gi].grid);
      if (P.ir)
        WRI_CK(cudaMemcpyAsync(groups[gi].u64, ws + P.v_x64[gi], 16 * (size_t)cnt, cudaMemcpyDeviceToDevice, st));
      else
        WRI_CK(launch_widen(groups[gi].u, groups[gi].u64, cnt, st));
    }
  if (P.ir) {  // the workspace now holds b - S u64 in FP64 (the last residual step of every system)
    std::lock_guard<std::mutex> lk(g_mu);
    g_stamps.push_back({workspace, residual_signature(groups, ngroups, opts, P.total)});
  }
  return WRI_OK;
}

int wri_source_estimate(const wri_group* groups, int ngroups, int dtype, double* alpha_out, void* workspace,
                        size_t ws_bytes, wri_stream_t stream) {
  if (dtype != WRI_C64 && dtype != WRI_C128) return WRI_EINVAL;
  int rc = validate_groups(groups, ngroups, false);
  if (rc != WRI_OK) return rc;
  if (!alpha_out) return WRI_EINVAL;
  bool wide = false;
  rc = aux_precision(groups, ngroups, dtype, &wide);
  if (rc != WRI_OK) return rc;
  Plan P;
  plan_aux(groups, ngroups, P);
  rc = check_ws(P, workspace, ws_bytes);
  if (rc != WRI_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  rc = upload(groups, ngroups, P, ws, st);
  if (rc != WRI_OK) return rc;
  Batch b = aux_batch(groups, ngroups, P, ws, dtype, wide);
  WRI_CK(launch_source_estimate((dtype == WRI_C128 || wide) ? 8 : 4, b, P.nsys_total, alpha_out, st));
  return WRI_OK;
}

int wri_gradient(const wri_group* groups, int ngroups, int dtype, const double* alpha_in, double* const* grad,
                 double* f, void* workspace, size_t ws_bytes, wri_stream_t stream) {
  if (dtype != WRI_C64 && dtype != WRI_C128) return WRI_EINVAL;
  int rc = validate_groups(groups, ngroups, true);
  if (rc != WRI_OK) return rc;
  if (!alpha_in || !grad || !f) return WRI_EINVAL;
  for (int gi = 0; gi < ngroups; ++gi)
    if (!grad[gi]) return WRI_EINVAL;
  bool wide = false;
  rc = aux_precision(groups, ngroups, dtype, &wide);
  if (rc != WRI_OK) return rc;
  Plan P;
  plan_aux(groups, ngroups, P);
  rc = check_ws(P, workspace, ws_bytes);
  if (rc != WRI_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  rc = upload(groups, ngroups, P, ws, st);
  if (rc != WRI_OK) return rc;
  Batch b = aux_batch(groups, ngroups, P, ws, dtype, wide);
  b.f = f;
  for (int gi = 0; gi < ngroups; ++gi) {
    b.g[gi].alpha = alpha_in + 2 * b.g[gi].sys0;
    b.g[gi].grad = grad[gi];
  }
  const int rb = (dtype == WRI_C128 || wide) ? 8 : 4;
  WRI_CK(launch_ztable(b, st));
  WRI_CK(march(rb, rb, M_GRAD, false, 8, b, st));
  WRI_CK(launch_data_term(rb, dtype == WRI_C128 ? 8 : 4, b, P.nsys_total, st));
  return WRI_OK;
}

int wri_gradient_refined(const wri_group* groups, int ngroups, const wri_solve_opts* opts, double* const* grad,
                         double* f, const void* workspace, size_t ws_bytes, wri_stream_t stream) {
  int rc = validate_opts(opts);
  if (rc != WRI_OK) return rc;
  rc = validate_groups(groups, ngroups, true);
  if (rc != WRI_OK) return rc;
  if (!grad || !f || opts->max_refine < 1 || opts->dtype != WRI_C64) return WRI_EINVAL;
  for (int gi = 0; gi < ngroups; ++gi)
    if (!grad[gi] || !groups[gi].u64) return WRI_EINVAL;
  Plan P;
  plan_solve(groups, ngroups, opts, P);
  rc = check_ws(P, workspace, ws_bytes);
  if (rc != WRI_OK) return rc;
  {
    const std::vector<unsigned long long> sig = residual_signature(groups, ngroups, opts, P.total);
    std::lock_guard<std::mutex> lk(g_mu);
    bool found = false;
    for (const auto& r : g_stamps) found = found || (r.ws == workspace && r.sig == sig);
    if (!found) return WRI_EINVAL;  // the workspace does not hold this problem's residual
  }
  char* ws = const_cast<char*>((const char*)workspace);
  Batch outer = solver_batch(groups, P, ws, false);
  cudaStream_t st = (cudaStream_t)stream;
  for (int gi = 0; gi < ngroups; ++gi) {
    outer.g[gi].x64 = groups[gi].u64;  // the solve copied its FP64 master there
    WRI_CK(launch_grad_residual(outer, gi, grad[gi], f, st));
  }
  return WRI_OK;
}

int wri_fwi_adjoint_source(const wri_group* groups, int ngroups, int dtype, const double* alpha_in, double* alpha_out,
                           void* const* q_adj, double* f, void* workspace, size_t ws_bytes, wri_stream_t stream) {
  if (dtype != WRI_C64 && dtype != WRI_C128) return WRI_EINVAL;
  int rc = validate_groups(groups, ngroups, true);
  if (rc != WRI_OK) return rc;
  if (!alpha_out || !q_adj || !f) return WRI_EINVAL;
  for (int gi = 0; gi < ngroups; ++gi)
    if (!q_adj[gi]) return WRI_EINVAL;
  Plan P;
  plan_aux(groups, ngroups, P);
  rc = check_ws(P, workspace, ws_bytes);
  if (rc != WRI_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  rc = upload(groups, ngroups, P, ws, st);
  if (rc != WRI_OK) return rc;
  const Batch b = aux_batch(groups, ngroups, P, ws, dtype);
  WRI_CK(launch_fwi_adjoint_source(dtype == WRI_C128 ? 8 : 4, b, P.nsys_total, alpha_in, alpha_out, q_adj, f, st));
  return WRI_OK;
}

int wri_fwi_gradient(const wri_group* groups, int ngroups, int dtype, const double* alpha, void* const* w,
                     double* const* grad, wri_stream_t stream) {
  if (dtype != WRI_C64 && dtype != WRI_C128) return WRI_EINVAL;
  int rc = validate_groups(groups, ngroups, false);
  if (rc != WRI_OK) return rc;
  if (!alpha || !w || !grad) return WRI_EINVAL;
  for (int gi = 0; gi < ngroups; ++gi)
    if (!w[gi] || !grad[gi]) return WRI_EINVAL;
  Plan P;
  plan_aux(groups, ngroups, P);
  // geometry only: no workspace is read (the batch's workspace views stay unset)
  const Batch b = aux_batch(groups, ngroups, P, nullptr, dtype);
  cudaStream_t st = (cudaStream_t)stream;
  for (int gi = 0; gi < ngroups; ++gi)
    WRI_CK(launch_fwi_gradient(dtype == WRI_C128 ? 8 : 4, b, gi, alpha, w[gi], grad[gi], st));
  return WRI_OK;
}

int wri_autotune(const wri_group* groups, int ngroups, wri_solve_opts* opts, int trial_iters, void* workspace,
                 size_t ws_bytes, wri_stream_t stream) {
  int rc = validate_opts(opts);
  if (rc != WRI_OK) return rc;
  rc = validate_groups(groups, ngroups, true);
  if (rc != WRI_OK) return rc;
  if (trial_iters < 2) return WRI_EINVAL;
  if (opts->dtype != WRI_C64 || opts->plain || opts->kernel == 1) return WRI_OK;
  for (int gi = 0; gi < ngroups; ++gi)
    if (groups[gi].grid.nx % 4 != 0 || (uintptr_t)groups[gi].u % 16 != 0) return WRI_OK;
  // with refinement the inner solves run on the warp-specialised kernels only (their phase 2 adds
  // S^H r64); the trials are plain CGLS solves on those kernels
  const bool refine = opts->max_refine > 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return WRI_ECUDA;
  std::vector<long long> key = {dev, ngroups, refine ? 1 : 0};
  for (int gi = 0; gi < ngroups; ++gi) {
    const wri_group& G = groups[gi];
    key.insert(key.end(), {G.grid.nx, G.grid.ny, G.grid.nz, G.nsys, G.rec_off[G.nsys]});
  }
  {
    std::lock_guard<std::mutex> lk(g_mu);
    for (const auto& e : g_tuned)
      if (e.key == key) {
        opts->kernel = e.kernel;
        opts->order = e.order;
        return WRI_OK;
      }
  }
  cudaStream_t st = (cudaStream_t)stream;
  forget_residual(workspace);  // the trial solves overwrite the workspace
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  WRI_CK(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return WRI_ECUDA;
  }
  static const int kCfgs[] = {8, 9, 12, 13, 17, 18, 22, 24};
  static const int kOrders[] = {2, 5, 6};  // systems of a tile consecutive, blocks of 8, blocks of 16
  float best = 0.f;
  int best_kernel = 0, best_order = 0;
  rc = WRI_OK;
  for (int cfg : kCfgs) {
    if (refine && cfg < kFirstWsCfg) continue;
    for (int ord : kOrders) {
      wri_solve_opts o = *opts;
      o.kernel = 2 + cfg;
      o.order = ord;
      o.tol = 0.0;
      o.warm_start = 0;
      o.max_iter = trial_iters;
      o.max_refine = 0;
      o.test_withhold = 0;
      Plan P;
      plan_solve(groups, ngroups, &o, P);
      if (P.tma_cfg != cfg || check_ws(P, workspace, ws_bytes) != WRI_OK) continue;
      char* ws = (char*)workspace;
      float ms = 0.f;
      for (int rep = 0; rep < 2 && rc == WRI_OK; ++rep) {  // the first run captures the graph
        if (cudaEventRecord(e0, st) != cudaSuccess) rc = WRI_ECUDA;
        if (rc == WRI_OK) rc = upload(groups, ngroups, P, ws, st);
        if (rc == WRI_OK) rc = solve_fused(groups, ngroups, &o, P, ws, st);
        if (rc == WRI_OK && cudaEventRecord(e1, st) != cudaSuccess) rc = WRI_ECUDA;
        if (rc == WRI_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = WRI_ECUDA;
        if (rc == WRI_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = WRI_ECUDA;
      }
      if (rc != WRI_OK) break;
      if (best_kernel == 0 || ms < best) {
        best = ms;
        best_kernel = o.kernel;
        best_order = ord;
      }
    }
    if (rc != WRI_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != WRI_OK) return rc;
  if (best_kernel == 0) return WRI_EWORKSPACE;  // no candidate fits the workspace
  opts->kernel = best_kernel;
  opts->order = best_order;
  std::lock_guard<std::mutex> lk(g_mu);
  g_tuned.push_back({key, best_kernel, best_order});
  return WRI_OK;
}

int wri_tv(const wri_grid* grid, const double* m, double beta, double gamma, double* tv, double* grad,
           wri_stream_t stream) {
  if (!grid_valid(grid) || !m || !tv) return WRI_EINVAL;
  if (!(beta > 0) || !std::isfinite(beta) || !(gamma >= 0) || !std::isfinite(gamma)) return WRI_EINVAL;
  WRI_CK(launch_tv(m, grid->nx, grid->ny, grid->nz, beta, gamma, tv, grad, (cudaStream_t)stream));
  return WRI_OK;
}

int wri_tile_count(void) { return 3; }

int wri_tile_shape(int tile, int* bx, int* by) {
  if (tile < 1 || tile > 3 || !bx || !by) return WRI_EINVAL;
  *bx = WRI_TX;
  *by = by_of_tile(tile);
  return WRI_OK;
}

const char* wri_strerror(int code) {
  switch (code) {
    case WRI_OK: return "success";
    case WRI_EINVAL: return "invalid argument";
    case WRI_ECUDA: return "CUDA launch or runtime error";
    case WRI_EWORKSPACE: return "workspace missing, misaligned or too small";
    case WRI_ENOTSUP: return "unsupported option combination";
    case WRI_ESCRATCH: return "problem exceeds the static scratch of the allocation-free entry point";
  }
  return "unknown error code";
}

#ifndef WRI_SRC_HASH
#define WRI_SRC_HASH "unknown"
#endif
const char* wri_version(void) { return "libwri 0.2 (sm_103a) src " WRI_SRC_HASH; }

}  // extern "C"
