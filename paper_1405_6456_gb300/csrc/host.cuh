// Host-side infrastructure shared by the translation units of the library:
// the context (device workspaces, reduction scratch, trace counters), error
// handling, stencil weights of Sec. 4, and kernel launch configuration.
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/ofdft.h"
#include "kernels.cuh"


// ----------------------------------------------------------------- context --
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

using ofd::CgScalars;

struct ofdft_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  int sms = 152;
  // reduction scratch
  DevBuf partials;
  unsigned int* counter = nullptr;
  // small device scalars: CG scalars (2 sets), functional outputs, dot outputs
  CgScalars* sc = nullptr;
  CgScalars* sc32 = nullptr;
  double* scal = nullptr;  // 64 doubles
  double* host_scal = nullptr;  // pinned mirror
  // named vector workspaces
  DevBuf v[32];
  // launch counters and optional CUDA-event timing of every launch
  long long launches = 0;
  long long kind_launches[OFDFT_K_COUNT] = {0};
  long long timed_launches[OFDFT_K_COUNT] = {0};
  double timed_ms[OFDFT_K_COUNT] = {0};
  int prof = 0;
  struct Pending {
    cudaEvent_t a, b;
    int kind;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> free_events;
  // pinned double buffer for polling CG flags without draining the stream
  CgScalars* ring = nullptr;
  cudaEvent_t ring_ev[2] = {nullptr, nullptr};
  // CUDA graphs of a chunk of CG iterations, keyed by everything they bake in
  struct GraphEntry {
    std::vector<long long> key;
    cudaGraphExec_t exec = nullptr;
  };
  std::vector<GraphEntry> graphs;
  int use_graphs = 1;
  cudaStream_t gstream = nullptr;  // private stream used only to capture graphs
  cudaEvent_t gev[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // sampling events recorded by CG graphs
  // autotuned z-splits of the z-streaming passes: key -> number of z chunks
  std::vector<std::pair<std::vector<long long>, int>> ztune;
  std::vector<std::vector<long long>> ztuned;  // (type, radius, grid, 16-byte staging) already tuned
  std::vector<long long> last_zkey;            // key of the last z-streaming launch
  int force_nz = -1;                           // >= 0: z-split of the next launches (autotuner)
  int pw_per_sm = 4;                           // blocks per SM of the pointwise passes
  int coop = 0;                                // persistent cooperative CG iterations (opt-in)
  unsigned int* coop_bar = nullptr;            // arrival counter of its grid barriers
  long long coop_iters = 0;                    // CG iterations run by it (trace counter)
  long long tma_launches = 0;                  // z-streaming passes staged by TMA (trace counter)
  int coop_nz = 0;                             // z-chunks of its grid (0: the default rule)
  int precond = 1;                             // Poisson CG preconditioner (OFDFT_PRECOND_*)
  int trace = 0;                               // OFDFT_TRACE=1: diagnostic lines on stderr
  double mg_omega = 0.9;                       // multigrid Jacobi weight (0 < omega < 1)
  int mg_sweeps = 20;                          // Jacobi sweeps on the multigrid bottom level
  DevBuf mgbuf;                                // multigrid levels below the finest
  int autotune = 1;
  double cg_fold_bytes = 96.0 * (1 << 20);     // fold the CG iterate update above this CG working set
  long long mg_fuse_nodes = -1;                // multigrid levels of at least this many nodes: two fused launches (-1: none)
  int ff_residual = 1;                         // mixed residual pass in float-float (else FP64)
  int cond_graphs = 1;                         // CG loops as one graph with a device-side WHILE node
  int mixed_ff = 0;                            // the last mixed Poisson solve ran the float-float residual pass
  int tma = 0;                                 // FP32 z-streaming passes stage planes by TMA where they can
  int pdl = 0;                                 // programmatic dependent launch for the CG-loop kernels
  int mg_finest_smooth = 1;                    // damped-Jacobi smoothing on the finest multigrid level
  long long mg_fuse_below = -1;                // coarser multigrid levels of at most this many nodes: fused
  int mg_cluster = 0;                          // coarse levels on one thread-block cluster (mg_cluster_kernel)
  int func_split_dots = 0;                     // G.d and G.s_old by a pass after the functional
  int mg_zstream = 0;                          // level smoothing passes as z-streaming radius-1 stencils
  long long mg_zstream_nodes = -1;             // ... on the levels of at least this many nodes (-1: none)
  // the b_J tables in V_BTAB belong to this geometry (atoms, charges, grid,
  // sigma, r_c, stencil radius); empty: none kept
  std::vector<double> btab_key;
};

namespace ofd {

enum Vec {
  V_R = 0, V_P0, V_P1, V_AP,           // CG vectors (prec type)
  V_R64, V_PHI64, V_B64, V_E32,        // mixed refinement (FP64 r, phi, b; FP32 correction)
  V_U, V_UT, V_PHI, V_B,               // solve state
  V_G, V_GT, V_S, V_ST, V_SN, V_D,     // NLCG vectors
  V_ATOM0, V_ATOM1, V_ATOM2,           // atom scratch
  V_W,                                 // u / Jacobi diagonal (rank-one preconditioner)
  V_PHI0,                              // FP64 potential at the origin of the current line search
  V_Z, V_T,                            // PCG: z = M r and the multigrid's finest-level scratch
  V_PHI2,                              // mixed: the FP64 potential as float-float pairs (residual pass)
  V_BACC,                              // FP64 running sums of the pseudocharge over atom ranges
  V_B2,                                // mixed: the FP64 pseudocharge as float-float pairs (residual pass)
  V_BTAB,                              // b_J tables of every atom, kept from the pseudocharge for the forces
  V_OC,                                // overlap correction: b, b~, V, V~ (FP64)
  V_COUNT
};

inline int fail(ofdft_ctx* c, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return code;
}

#define CU(call)                                                                   \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess)                                                         \
      return fail(c, e_ == cudaErrorMemoryAllocation ? OFDFT_ENOMEM : OFDFT_ECUDA, \
                  "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

#define TRY(expr)            \
  do {                       \
    int rc_ = (expr);        \
    if (rc_ != OFDFT_OK) return rc_; \
  } while (0)

inline int ensure(ofdft_ctx* c, DevBuf& b, size_t bytes) {
  if (b.bytes >= bytes && b.p) return OFDFT_OK;
  if (b.p) {
    CU(cudaStreamSynchronize(c->stream));
    CU(cudaFree(b.p));
    b.p = nullptr;
    b.bytes = 0;
  }
  const size_t want = std::max<size_t>(bytes, 256);
  CU(cudaMalloc(&b.p, want));
  b.bytes = want;
  return OFDFT_OK;
}

template <typename T>
T* vec(ofdft_ctx* c, int which) {
  return static_cast<T*>(c->v[which].p);
}

inline cudaEvent_t take_event(ofdft_ctx* c) {
  if (!c->free_events.empty()) {
    cudaEvent_t e = c->free_events.back();
    c->free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Folds the durations of completed timed launches into the totals (call after
// the stream has been synchronised) and recycles their events.
inline void harvest(ofdft_ctx* c) {
  for (auto& p : c->pending) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      c->timed_ms[p.kind] += ms;
      c->timed_launches[p.kind] += 1;
    }
    c->free_events.push_back(p.a);
    c->free_events.push_back(p.b);
  }
  c->pending.clear();
}

// Counts a kernel launch of `kind`; with profiling on, brackets it with events.
struct ProfScope {
  ofdft_ctx* c;
  int kind;
  cudaEvent_t a = nullptr, b = nullptr;
  ProfScope(ofdft_ctx* c_, int k) : c(c_), kind(k) {
    c->launches++;
    c->kind_launches[k]++;
    if (c->prof & (1 << k)) {
      a = take_event(c);
      b = take_event(c);
      if (a && b) cudaEventRecord(a, c->stream);
    }
  }
  ~ProfScope() {
    if (a && b) {
      cudaEventRecord(b, c->stream);
      c->pending.push_back({a, b, kind});
      if (c->pending.size() > 4096) {
        cudaEventSynchronize(b);
        harvest(c);
      }
    }
  }
};

inline RedBuf red(ofdft_ctx* c) { return RedBuf{static_cast<double*>(c->partials.p), c->counter}; }

inline int ensure_partials(ofdft_ctx* c, long long nblocks, int K) {
  return ensure(c, c->partials, (size_t)nblocks * K * sizeof(double) + 64);
}

inline GridDev gdev(const ofdft_grid* g) {
  GridDev d;
  d.n1 = g->n[0];
  d.n2 = g->n[1];
  d.n3 = g->n[2];
  d.G = (long long)d.n1 * d.n2 * d.n3;
  return d;
}

inline int check_grid(ofdft_ctx* c, const ofdft_grid* g) {
  if (!g) return fail(c, OFDFT_EINVAL, "grid is NULL");
  for (int d = 0; d < 3; ++d)
    if (g->n[d] < 1 || g->n[d] > (1 << 16)) return fail(c, OFDFT_EINVAL, "grid dimension %d is %d", d, g->n[d]);
  if (!(g->h > 0.0) || !isfinite(g->h)) return fail(c, OFDFT_EINVAL, "grid spacing must be positive");
  // the stencil kernels hold in-plane offsets in 32 bits
  if ((long long)g->n[0] * (g->n[1] + 2 * kMaxR) >= (1LL << 31))
    return fail(c, OFDFT_EINVAL, "grid plane of %d x %d nodes is too large", g->n[0], g->n[1]);
  return OFDFT_OK;
}

inline int check_order(ofdft_ctx* c, int fd_order) {
  if (fd_order < 2 || fd_order > 2 * kMaxR || (fd_order & 1))
    return fail(c, OFDFT_EINVAL, "fd_order must be even in [2, %d], got %d", 2 * kMaxR, fd_order);
  return OFDFT_OK;
}

inline int check_prec(ofdft_ctx* c, int prec) {
  if (prec != OFDFT_PREC_FP64 && prec != OFDFT_PREC_MIXED)
    return fail(c, OFDFT_EINVAL, "precision must be OFDFT_PREC_FP64 or OFDFT_PREC_MIXED");
  return OFDFT_OK;
}

// Laplacian weights of Sec. 4 (Eq. FD:Laplacian) in FP64, scaled by `scale`;
// c = 6 w_0 (the p = 0 term counts the centre six times).
inline Weights<double> lap_weights(int R, double h, double scale) {
  Weights<double> W;
  memset(&W, 0, sizeof(W));
  double s = 0.0;
  for (int q = 1; q <= R; ++q) s += 1.0 / ((double)q * q);
  W.c = scale * 6.0 * (-s / (h * h));
  // (R!)^2 / ((R-p)! (R+p)!) as a running product
  for (int p = 1; p <= R; ++p) {
    double ratio = 1.0;
    for (int i = 1; i <= p; ++i) ratio *= (double)(R - p + i) / (double)(R + i);
    const double sign = (p & 1) ? 1.0 : -1.0;
    W.w[p] = scale * 2.0 * sign * ratio / (h * h * (double)p * p);
  }
  return W;
}

// Gradient weights of Sec. 4: w~_p = (-1)^{p+1} (R!)^2 / (h p (R-p)! (R+p)!).
inline Weights<double> grad_weights(int R, double h) {
  Weights<double> W;
  memset(&W, 0, sizeof(W));
  for (int p = 1; p <= R; ++p) {
    double ratio = 1.0;
    for (int i = 1; i <= p; ++i) ratio *= (double)(R - p + i) / (double)(R + i);
    const double sign = (p & 1) ? 1.0 : -1.0;
    W.w[p] = sign * ratio / (h * (double)p);
  }
  return W;
}

template <typename T>
Weights<T> cast_weights(const Weights<double>& W) {
  Weights<T> o;
  o.c = (T)W.c;
  for (int p = 0; p <= kMaxR; ++p) o.w[p] = (T)W.w[p];
  return o;
}
// float-float weights: hi = nearest float, lo = nearest float of the remainder
inline float2 ff_of(double v) {
  const float hi = (float)v;
  return make_float2(hi, (float)(v - (double)hi));
}
template <>
inline Weights<float2> cast_weights<float2>(const Weights<double>& W) {
  Weights<float2> o;
  o.c = ff_of(W.c);
  for (int p = 0; p <= kMaxR; ++p) o.w[p] = ff_of(W.w[p]);
  return o;
}

inline int pointwise_blocks(ofdft_ctx* c, long long G) {
  long long b = (G + 1023) / 1024;
  return (int)std::max<long long>(1, std::min<long long>(b, (long long)c->sms * c->pw_per_sm));
}

// z-streaming launch shape: BX x BY columns; z split so that the grid fills
// the resident block slots (SMs x blocks per SM) in whole waves: a grid just
// above a wave would leave a nearly empty second wave.  z-chunks are at least
// 2R planes deep unless the grid is too small to fill the GPU at all.
// Poisson tolerance inside a solve's NLCG at a point with h^3 r.s = rs (see
// ofdft_params.poisson_adapt): the gradient's error from an inexact potential
// only has to stay small against the gradient itself.
inline double adaptive_poisson_tol(const ofdft_params* p, double rs, int M) {
  if (!(p->poisson_adapt > 0.0) || !(rs > 0.0) || !isfinite(rs)) return p->tol_poisson;
  const double t = p->poisson_adapt * p->tol_poisson * sqrt(rs / (p->tol_inner * M));
  return std::max(p->tol_poisson, std::min(1e-4, t));
}

// Poisson tolerance of a secant trial point (ofdft_params.trial_poisson_loosen).
inline double trial_poisson_tol(const ofdft_params* p, double tol) {
  if (!(p->trial_poisson_loosen > 1.0)) return tol;
  return std::max(tol, std::min(1e-4, tol * p->trial_poisson_loosen));
}

// Resolution of L in a MIXED evaluation: the FP32 energy densities (TF, vW
// with the FP32 stencil, XC) carry rounding noise that measured about 1e-9 of the
// summed magnitudes of the energy terms on the 666-atom cluster; a secant step
// whose L rises by less than that is not a rise the evaluation can resolve.
// FP64 evaluations resolve far below any step the NLCG takes: 0.
inline double l_resolution(const ofdft_energy& e, bool mixed) {
  if (!mixed) return 0.0;
  return 1e-9 * (fabs(e.E_tf) + fabs(e.E_vw) + fabs(e.E_xc) + fabs(e.E_es));
}

// Relative tolerance of one FP32 round of the mixed Poisson CG: cut the FP32
// residual by 1e-4 (the reduction FP32 recurrences track faithfully), but not
// below half of what the FP64 stopping test still asks for (||r|| <= tol ||b||),
// so that the last round does not over-solve.  rr = ||r64||^2, bb = ||b||^2.
inline double mixed_inner_tol(double rr, double bb, double tol) {
  const double want = (rr > 0.0) ? 0.5 * tol * sqrt(bb / rr) : 1e-4;
  return std::max(1e-4, std::min(want, 0.5));
}

struct ZShape {
  dim3 grid;
  int zchunk;
  long long nblocks;
};

template <typename T>
ZShape zshape(ofdft_ctx* c, const GridDev& g, int R, int blocks_per_sm = 4, int force_nz = 0) {
  ZShape s;
  const int gx = (g.n1 + BX - 1) / BX, gy = (g.n2 + ZCfg<T>::TY - 1) / ZCfg<T>::TY;
  const long long tiles = (long long)gx * gy;
  const long long slots = (long long)c->sms * std::max(blocks_per_sm, 1);
  int nz = (int)std::max<long long>(1, slots / tiles);  // one wave when tiles <= slots
  nz = std::min(nz, std::max(1, g.n3 / std::max(2 * R, 4)));
  if (force_nz > 0) nz = std::min(force_nz, g.n3);
  int zc = (g.n3 + nz - 1) / nz;
  nz = (g.n3 + zc - 1) / zc;
  s.grid = dim3(gx, gy, nz);
  s.zchunk = zc;
  s.nblocks = (long long)gx * gy * nz;
  return s;
}

// Key of an autotuned z-split: the kernel instantiation and the grid.
inline std::vector<long long> ztune_key(const void* fn, const GridDev& g) {
  return {(long long)(uintptr_t)fn, g.n1, g.n2, g.n3};
}

// True when a pass can stage 16-byte copies: rows of a whole number of copies
// (n1 % (16 / sizeof(T)) == 0) and 16-byte aligned stencil and epilogue inputs.
template <typename T, class L, class E>
bool zvec_ok(const GridDev& g, const L& ld, const E& ep) {
  if (g.n1 % (16 / (int)sizeof(T))) return false;
  auto aligned = [](const void* p) { return ((uintptr_t)p & 15u) == 0; };
  if (!aligned(ld.f)) return false;
  for (int j = 0; j < E::NIN; ++j)
    if (ep.input(j) && !aligned(ep.input(j))) return false;
  return true;
}

// Multigrid preconditioner of the Poisson CG (S3): the levels of a grid (kernels
// and the cycle's steps: mg_* in kernels.cuh).
constexpr int kMgCoarseNodes = 4096;  // levels from this size down run in one block
constexpr int kMgSweeps = 20;         // Jacobi sweeps from zero on the bottom level
constexpr double kMgOmega = 0.9;      // Jacobi weight (the cycle is SPD for 0 < omega < 1)

struct MgPlan {
  int nlev = 0;  // levels from the grid itself down to the bottom (smallest extent below 4)
  int lc = -1;   // first level handled by the one-block kernel
  MgLevel d[kMgMaxLevels];
  long long off[kMgMaxLevels] = {0};  // element offset of level l's r, z, t (l = 1 .. lc) in mgbuf
  long long elems = 0;                // mgbuf elements
  size_t smem = 0;                    // shared memory of the one-block kernel
  double s0 = 0.0;                    // omega h^2 / 6 of the finest level
  bool ok = false;
  // the cluster end (mg_cluster_kernel): levels lq .. lc-1 in the distributed
  // shared memory of one thread-block cluster (lq < 0: none fits)
  int lq = -1;
  MgSlab slab[kMgMaxLevels];
  size_t csmem = 0;       // dynamic shared memory per block of the cluster kernel
  unsigned tail_off = 0;  // byte offset of block 0's coarse-end arrays
};
constexpr size_t kMgClusterSmem = 220 * 1024;  // dynamic shared memory per cluster block (of 227 KB)

inline long long mg_nodes(const MgLevel& d) { return (long long)d.n1 * d.n2 * d.n3; }

inline MgPlan mg_plan(const GridDev& g, double h, size_t es, double omega = kMgOmega) {
  MgPlan P;
  MgLevel d{g.n1, g.n2, g.n3};
  P.d[0] = d;
  P.nlev = 1;
  while (std::min(d.n1, std::min(d.n2, d.n3)) >= 4 && P.nlev < kMgMaxLevels) {
    d = MgLevel{d.n1 / 2, d.n2 / 2, d.n3 / 2};
    P.d[P.nlev++] = d;
  }
  for (int l = 0; l < P.nlev; ++l)
    if (mg_nodes(P.d[l]) <= kMgCoarseNodes) {
      P.lc = l;
      break;
    }
  if (P.lc < 0) return P;  // the bottom level is too large for one block: plain CG
  if (mg_nodes(P.d[0]) >= (1LL << 31)) return P;  // the level kernels index with 32-bit integers
  long long e = 0;
  for (int l = 1; l <= P.lc; ++l) {
    P.off[l] = e;
    e += 3 * mg_nodes(P.d[l]);
  }
  P.elems = e;
  size_t sm = 0;
  for (int l = P.lc; l < P.nlev; ++l) sm += 3 * (size_t)mg_nodes(P.d[l]) * es;
  P.smem = sm;
  P.s0 = omega * h * h / 6.0;
  P.ok = sm <= 200 * 1024;
  if (!P.ok) return P;
  // the cluster end: the most levels above lc (level 0 excluded: its pass forms
  // r.z) whose z-plane slabs, with the coarse end's arrays in block 0, fit
  for (int lq = 1; lq < P.lc && P.lq < 0; ++lq) {
    size_t off = 0;  // bytes
    for (int l = lq; l < P.lc; ++l) {
      const MgLevel& d = P.d[l];
      const int pl = (d.n3 + kMgClusterCtas - 1) / kMgClusterCtas;
      P.slab[l] = MgSlab{d, pl, (unsigned)(off / es)};
      off += ((3 * (size_t)pl * d.n1 * d.n2 * es + 15) / 16) * 16;
    }
    P.slab[P.lc] = MgSlab{P.d[P.lc], 0, 0};
    if (off + sm <= kMgClusterSmem) {
      P.lq = lq;
      P.tail_off = (unsigned)off;
      P.csmem = off + sm;
    }
  }
  return P;
}

// Launches kern on the context's stream.  With c->pdl the launch allows
// programmatic dependent launch: the grid may be scheduled while the previous
// kernel of the stream is still finishing, and holds at pdl_wait() (the first
// statement of every kernel launched here) until that kernel has completed and
// its writes are visible; the previous kernel releases it early with
// pdl_launch_dependents().  Only the launch latency overlaps, never the work.
template <typename... KArgs, typename... Args>
cudaError_t launch_k(ofdft_ctx* c, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, Args... args) {
  if (c->pdl) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = c->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
  }
  kern<<<grid, block, smem, c->stream>>>(args...);
  return cudaGetLastError();
}

template <typename T, int R, int V, class L, class E>
int launch_zv(ofdft_ctx* c, const GridDev& g, const Weights<double>& W, L ld, E ep, int kind) {
  constexpr int smem = zsmem_bytes<T, R, V, E>();
  // resident blocks per SM of this kernel, per device (dynamic shared memory above
  // 48 KB needs an opt-in, a per-device setting)
  static int per_sm_dev[64] = {0};
  if (c->device < 0 || c->device >= 64) return fail(c, OFDFT_EINVAL, "device index out of range");
  int& per_sm = per_sm_dev[c->device];
  if (!per_sm) {
    CU(cudaFuncSetAttribute(zstream_kernel<T, R, V, L, E>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int nb = 0;
    CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, zstream_kernel<T, R, V, L, E>, NT, smem));
    per_sm = std::max(nb, 1);
  }
  const std::vector<long long> key = ztune_key((const void*)zstream_kernel<T, R, V, L, E>, g);
  int nz = 0;
  if (c->force_nz >= 0) {
    nz = c->force_nz;
  } else {
    for (auto& t : c->ztune)
      if (t.first == key) {
        nz = t.second;
        break;
      }
  }
  c->last_zkey = key;
  const ZShape s = zshape<T>(c, g, R, per_sm, nz);
  if (E::K > 0) TRY(ensure_partials(c, s.nblocks, E::K));
  {
    ProfScope ps_(c, kind);
    CU(launch_k(c, zstream_kernel<T, R, V, L, E>, s.grid, dim3(BX, BY), smem, g, cast_weights<T>(W), s.zchunk, ld,
                ep, red(c)));
  }
  return OFDFT_OK;
}

// cuTensorMapEncodeTiled of the driver, found through the runtime (no link
// against libcuda); nullptr when the driver does not offer it.
inline PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// Tensor map of an FP32 grid array (x-fastest, n1 x n2 x n3) read in boxes of
// bx x by x 1 elements; out-of-grid elements read as zero.
inline bool fp32_grid_map(CUtensorMap* m, const void* base, const GridDev& g, int bx, int by) {
  auto enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)g.n1, (cuuint64_t)g.n2, (cuuint64_t)g.n3};
  const cuuint64_t strides[2] = {(cuuint64_t)g.n1 * 4, (cuuint64_t)g.n1 * g.n2 * 4};
  const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The z-streaming pass with TMA staging (zstream_tma_kernel).  Returns false
// (nothing launched) when the pass cannot take it: another element type or
// staging width, a slot size off the 128-byte grid, an epilogue input that is
// NULL, or no tensor-map encoder.
template <typename T, int R, int V, class L, class E>
int launch_zv_tma(ofdft_ctx* c, const GridDev& g, const Weights<double>& W, L ld, E ep, int kind, bool* done) {
  *done = false;
  if constexpr (!ztma_fits<T, R, V>() || E::NIN > 3) {
    return OFDFT_OK;
  } else {
    if (!c->tma) return OFDFT_OK;
    constexpr int TY = ZCfg<T>::TY, RA = zhalo_x<T, R, V>();
    CUtensorMap mf, mi[3];
    if (!fp32_grid_map(&mf, ld.f, g, BX + 2 * RA, TY + 2 * R)) return OFDFT_OK;
    for (int j = 0; j < 3; ++j) mi[j] = mf;
    for (int j = 0; j < E::NIN; ++j) {
      const void* in = ep.input(j);
      if (!in || !fp32_grid_map(&mi[j], in, g, BX, TY)) return OFDFT_OK;
    }
    constexpr int smem = zsmem_bytes<T, R, V, E>() + 128;
    static int per_sm_dev[64] = {0};
    if (c->device < 0 || c->device >= 64) return fail(c, OFDFT_EINVAL, "device index out of range");
    int& per_sm = per_sm_dev[c->device];
    if (!per_sm) {
      CU(cudaFuncSetAttribute(zstream_tma_kernel<T, R, V, L, E>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
      int nb = 0;
      CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, zstream_tma_kernel<T, R, V, L, E>, NT, smem));
      per_sm = std::max(nb, 1);
    }
    const std::vector<long long> key = ztune_key((const void*)zstream_tma_kernel<T, R, V, L, E>, g);
    int nz = 0;
    if (c->force_nz >= 0) {
      nz = c->force_nz;
    } else {
      for (auto& t : c->ztune)
        if (t.first == key) {
          nz = t.second;
          break;
        }
    }
    c->last_zkey = key;
    const ZShape s = zshape<T>(c, g, R, per_sm, nz);
    if (E::K > 0) TRY(ensure_partials(c, s.nblocks, E::K));
    {
      ProfScope ps_(c, kind);
      CU(launch_k(c, zstream_tma_kernel<T, R, V, L, E>, s.grid, dim3(BX, BY), smem, mf, mi[0], mi[1], mi[2], g,
                  cast_weights<T>(W), s.zchunk, ld, ep, red(c)));
    }
    c->tma_launches++;
    *done = true;
    return OFDFT_OK;
  }
}

template <typename T, int R, class L, class E>
int launch_z(ofdft_ctx* c, const GridDev& g, const Weights<double>& W, L ld, E ep, int kind) {
  if (zvec_ok<T>(g, ld, ep)) {
    bool done = false;
    TRY((launch_zv_tma<T, R, 16 / (int)sizeof(T)>(c, g, W, ld, ep, kind, &done)));
    if (done) return OFDFT_OK;
    return launch_zv<T, R, 16 / (int)sizeof(T)>(c, g, W, ld, ep, kind);
  }
  return launch_zv<T, R, 1>(c, g, W, ld, ep, kind);
}

// Runtime radius -> template radius.
template <typename T, class L, class E>
int launch_z_r(ofdft_ctx* c, int R, const GridDev& g, const Weights<double>& W, L ld, E ep, int kind) {
  switch (R) {
    case 1: return launch_z<T, 1>(c, g, W, ld, ep, kind);
    case 2: return launch_z<T, 2>(c, g, W, ld, ep, kind);
    case 3: return launch_z<T, 3>(c, g, W, ld, ep, kind);
    case 4: return launch_z<T, 4>(c, g, W, ld, ep, kind);
    case 5: return launch_z<T, 5>(c, g, W, ld, ep, kind);
    case 6: return launch_z<T, 6>(c, g, W, ld, ep, kind);
  }
  return fail(c, OFDFT_EINVAL, "stencil radius %d not supported", R);
}


inline int sync_scalars(ofdft_ctx* c, const void* dev, size_t bytes, void* host) {
  CU(cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  if (!c->pending.empty()) harvest(c);
  return OFDFT_OK;
}

struct EvalOut {
  double sums[12];
};

inline void fill_energy(const EvalOut& o, double h, const ofdft_params* p, double E_self, double ezz, double eta,
                 double mu, ofdft_energy* e) {
  const double h3 = h * h * h;
  const bool es = p->terms & OFDFT_TERM_ES;
  e->E_tf = h3 * o.sums[0];
  e->E_vw = -0.5 * p->lambda * h3 * o.sums[1];
  e->E_xc = h3 * o.sums[2];
  e->E_self = es ? E_self : 0.0;
  e->E_es = es ? h3 * (0.5 * o.sums[3] + o.sums[4] / (8.0 * kPi)) - E_self : 0.0;
  e->E_zz_corr = ezz;
  e->E = e->E_tf + e->E_vw + e->E_xc + e->E_es + ezz;
  e->C = o.sums[9];
  e->L = e->E - eta * e->C + 0.5 * e->C * e->C / mu;
  e->gd = h3 * o.sums[5];
  e->gs_old = h3 * o.sums[6];
  e->rs = h3 * o.sums[7];
  e->rs_pc = e->rs;
  e->gnorm2 = h3 * o.sums[8];
}

// Routines of api.cu used by the batched engine (instantiated for double and float).
int check_atoms(ofdft_ctx* c, const double* R, const double* Z, int M);
int check_params(ofdft_ctx* c, const ofdft_params* p);
template <typename T>
int device_pseudocharge(ofdft_ctx* c, const ofdft_grid* gr, int R, const double* R_host, const double* Z_host,
                        int M, double sigma, double rc, T* b, double* E_self, bool keep_tables = false);
template <typename T>
int device_guess(ofdft_ctx* c, const ofdft_grid* gr, const double* R_host, const double* Z_host, int M,
                 double gsig, double gcut, double N, T* u);
template <typename T>
int device_forces(ofdft_ctx* c, const ofdft_grid* gr, int R, const double* R_host, const double* Z_host, int M,
                  double sigma, double rc, int variant, const T* phi, double* F);
int device_ezz(ofdft_ctx* c, const double* R_host, const double* Z_host, int M, double sigma, double* E,
               double* F);

}  // namespace ofd
