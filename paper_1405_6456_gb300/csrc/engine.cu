// Batched and continuously served ground states (S11, S12).
//
// Every solve ("slot") runs the same method as ofdft_solve: Algorithm 1 around
// the secant / Polak-Ribiere nonlinear CG with one CG Poisson solve per
// gradient evaluation.  Its control flow is written as a state machine that
// yields one request at a time (an evaluation of L and its gradient, or two dot
// products) after queueing the vector updates that precede it.  The engine
// advances all active slots in lockstep rounds and packs the work of a round
// into shared launches: one z-streaming launch per stencil stage over a work
// list of tiles drawn from every grid (uneven sizes), one pointwise launch per
// vector operation over segments of every grid, each grid reducing into its
// own scratch.  A converged CG drops out of the tile list at the next poll.
// New solves are admitted between rounds when their workspace fits in the
// HBM budget, so requests that arrive while others run join the mix.
#include "host.cuh"

#include <deque>
#include <functional>
#include <memory>
#include <type_traits>

namespace ofd {
namespace {

enum SlotState {
  S_AL_START,      // evaluation at u0 before the first inner solve
  S_NLCG_START,    // evaluation at u with the current (eta, mu)
  S_ITER,          // convergence test of the inner loop, then dots G.d, d.d
  S_DOTS,          // got G.d, d.d
  S_TRIAL,         // got the evaluation at the trial point
  S_SECANT,        // got the evaluation at a secant candidate
  S_AL_UPDATE,     // multiplier update of Algorithm 1
  S_FINAL,         // got the final evaluation at tol_poisson (after loose adaptive solves)
  S_DONE
};

enum ReqKind { REQ_NONE = 0, REQ_EVAL = 1, REQ_DOTS = 2 };
enum VopKind { VOP_AXPY_ABS = 0, VOP_DIRECTION = 1 };

template <typename T>
struct Vop {
  int kind;
  T* out;
  const T* a;
  const T* b;
  double scalar;
};

template <typename T>
struct Slot {
  int id = 0;
  ofdft_params p;
  std::vector<double> R, Z;
  int M = 0;
  double N = 0.0;
  ofdft_grid grid;
  GridDev g;
  int Rr = 6;
  int zdepth = 16;  // planes per CTA of this grid's tiles in the batched z-streaming passes
  int ztuned = 0;   // zdepth chosen (autotuner or the context's cache)
  double h = 0.5, h3 = 0.125;
  size_t bytes = 0;
  void* mem = nullptr;
  // fields
  T *u, *ut, *phi, *b, *G, *Gt, *s, *st, *sn, *d, *w, *r, *pv, *qv;
  double *phi64 = nullptr, *b64 = nullptr, *r64 = nullptr;
  double* phi0 = nullptr;  // FP64 potential at the origin of the current line search
  float* e32 = nullptr;
  double* partials = nullptr;
  unsigned int* counter = nullptr;
  int maxblk = 0;
  // multigrid preconditioner of the Poisson CG: z, finest scratch, coarser levels
  T *mz = nullptr, *mt = nullptr, *mgc = nullptr;
  MgPlan mg;
  int pc = 0;  // this solve's CG is preconditioned
  int index = 0;  // position in the engine's device scalar arrays
  // method state (host scalars)
  int state = S_AL_START;
  double eta = 0, mu = 1, E_prev = 0, delta_new = 0, alpha = 0, gprev = 0, gcur = 0, L0 = 0, sig = 0, dd = 0, g0 = 0;
  int k = 0, it = 0, q = 0, j = 0, bt = 0, inner_ok = 0, redo_dots = 0;
  T* s_old = nullptr;
  T* snew = nullptr;
  ofdft_energy e, et;
  ofdft_solve_stats stats;
  double E_self = 0.0, ezz = 0.0;
  std::vector<double> Fz, forces;
  int status = OFDFT_OK;
  std::string err;
  // pending request
  int req = REQ_NONE;
  const T* ev_at = nullptr;
  T* ev_G = nullptr;
  T* ev_s = nullptr;
  const T* ev_d = nullptr;
  const T* ev_sold = nullptr;
  double ev_eta = 0, ev_mu = 1;
  ofdft_energy* ev_out = nullptr;
  const T* dot_a[4] = {nullptr, nullptr, nullptr, nullptr};
  std::vector<Vop<T>> vops;
  std::vector<double> line_ops;  // OpLine parameters, applied before the next evaluation
  double line_l = 0.0, pos = 0.0;  // last solve's position along d; position of u along d
  double tol_p = 0.0;              // Poisson tolerance of the next evaluations (adaptive_poisson_tol)
  double ev_tol = 0.0;             // Poisson tolerance of the pending evaluation
  // Poisson phase (within a round)
  int pphase = 0, ptotal = 0;
  ofdft_cg_stats pstats;
};

struct DevArena {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace
}  // namespace ofd

using namespace ofd;

// The batch engine behind the ofdft_batch_* entry points.
struct ofdft_batch {
  ofdft_ctx* c = nullptr;
  int prec = OFDFT_PREC_MIXED;
  long long budget = 0, in_use = 0;
  int next_id = 1;
  int capacity = 0;           // slots the device scalar arrays hold
  CgScalars* sc = nullptr;    // per slot: FP64 residual / CG scalars
  CgScalars* sc32 = nullptr;  // per slot: FP32 correction CG (mixed)
  double* out = nullptr;      // per slot: 16 doubles
  std::vector<CgScalars> h_sc, h_sc32;
  std::vector<double> h_out;
  DevArena d_tiles, d_desc, d_segs, d_ops;
  std::vector<int> free_index;
  long long rounds = 0;
  // CUDA graphs of the batched CG loop: a device-side WHILE loop over one CG
  // iteration of every solve in the loop, keyed by the solves' buffers and the
  // launch shape; the work lists the captured launches read live in the graph's
  // own device arena
  struct LoopGraph {
    std::vector<long long> key;
    cudaGraphExec_t exec = nullptr;
    void* arena = nullptr;
  };
  std::vector<LoopGraph> graphs;
  long long graph_captures = 0, graph_replays = 0, graph_iters = 0, eager_iters = 0;
  int* one_pinned = nullptr;        // host-pinned 1: marks a slot's CG done without a host wait
  bool capturing = false;           // work-list uploads go to the capture arena
  std::vector<char> cap_host;       // staged contents of the capture arena
  char* cap_dev = nullptr;          // the capture arena (device)
  size_t cap_bytes = 0;
  // autotuned launch shape of the batched z-streaming passes: planes per CTA,
  // chosen per grid shape (the tiles of a grid fix the order of its partial
  // sums, so a request's result does not depend on the other grids in the mix)
  int zdepth = 16;                             // depth of the most recently tuned grid
  int ztuned = 0;
  std::vector<std::pair<int, float>> tune_log;  // (depth, us) of the last tuning
  // type-erased slot lists (only the engine of the batch precision is used)
  std::vector<std::unique_ptr<Slot<double>>> s64_active, s64_done;
  std::vector<std::unique_ptr<Slot<float>>> s32_active, s32_done;
  std::deque<std::unique_ptr<Slot<double>>> s64_queue;
  std::deque<std::unique_ptr<Slot<float>>> s32_queue;
};

namespace ofd {
namespace {

int grow_arena(ofdft_ctx* c, DevArena& a, size_t bytes) {
  if (a.bytes >= bytes && a.p) return OFDFT_OK;
  if (a.p) {
    CU(cudaStreamSynchronize(c->stream));
    CU(cudaFree(a.p));
    a.p = nullptr;
  }
  const size_t want = std::max<size_t>(bytes * 2, 4096);
  CU(cudaMalloc(&a.p, want));
  a.bytes = want;
  return OFDFT_OK;
}

template <typename V>
int upload(ofdft_ctx* c, DevArena& a, const std::vector<V>& v) {
  TRY(grow_arena(c, a, v.size() * sizeof(V) + 64));
  if (!v.empty())
    CU(cudaMemcpyAsync(a.p, v.data(), v.size() * sizeof(V), cudaMemcpyHostToDevice, c->stream));
  return OFDFT_OK;
}

// Workspace of one solve: every field it keeps resident between rounds.
long long slot_bytes(const ofdft_grid& g, int prec, int* maxblk) {
  const long long G = (long long)g.n[0] * g.n[1] * g.n[2];
  const long long es = (prec == OFDFT_PREC_MIXED) ? 4 : 8;
  auto chunk = [](long long n) { return (n + 255) & ~255LL; };  // carve() rounds every piece to 256 B
  long long bytes = 14 * chunk(G * es) + chunk(G * 8);
  if (prec == OFDFT_PREC_MIXED) bytes += 3 * chunk(G * 8) + chunk(G * 4);
  // multigrid preconditioner: z, the finest level's scratch, the coarser levels
  const MgPlan mg = mg_plan(gdev(&g), g.h, (size_t)es);
  if (mg.ok) bytes += 2 * chunk(G * es) + chunk(std::max<long long>(mg.elems, 1) * es);
  // reduction scratch: the larger of the tile count and the segment count
  const long long tiles = (long long)((g.n[0] + BX - 1) / BX) * ((g.n[1] + BY - 1) / BY) * ((g.n[2] + 15) / 16);
  const long long segs = (G + 16383) / 16384;
  const long long mb = std::max(tiles, segs) + 1;
  *maxblk = (int)mb;
  bytes += chunk(mb * 16 * 8) + chunk(256);
  return bytes;
}

template <typename T>
int carve(ofdft_ctx* c, Slot<T>* S, int prec) {
  const long long G = S->g.G;
  S->bytes = (size_t)slot_bytes(S->grid, prec, &S->maxblk);
  CU(cudaMalloc(&S->mem, S->bytes));
  char* p = (char*)S->mem;
  auto take = [&](size_t n) {
    char* q = p;
    p += (n + 255) & ~(size_t)255;
    return (void*)q;
  };
  T** vecs[] = {&S->u, &S->ut, &S->phi, &S->b, &S->G, &S->Gt, &S->s, &S->st, &S->sn, &S->d, &S->w, &S->r, &S->pv, &S->qv};
  for (T** v : vecs) *v = (T*)take(G * sizeof(T));
  S->phi0 = (double*)take(G * 8);
  if (prec == OFDFT_PREC_MIXED) {
    S->phi64 = (double*)take(G * 8);
    S->b64 = (double*)take(G * 8);
    S->r64 = (double*)take(G * 8);
    S->e32 = (float*)take(G * 4);
  }
  S->partials = (double*)take((size_t)S->maxblk * 16 * 8);
  S->counter = (unsigned int*)take(256);
  S->mg = mg_plan(S->g, S->h, sizeof(T), c->mg_omega);
  if (S->mg.ok) {
    S->mz = (T*)take(G * sizeof(T));
    S->mt = (T*)take(G * sizeof(T));
    S->mgc = (T*)take(std::max<long long>(S->mg.elems, 1) * sizeof(T));
  }
  S->pc = (S->mg.ok && c->precond == OFDFT_PRECOND_MG) ? 1 : 0;
  if ((size_t)(p - (char*)S->mem) > S->bytes) return fail(c, OFDFT_EINVAL, "slot workspace carve overflow");
  CU(cudaMemsetAsync(S->counter, 0, 256, c->stream));
  return OFDFT_OK;
}

// Tiles of one grid for the z-streaming batch launch (BX x rows columns, z chunks
// of zc planes).
void grid_tiles(const GridDev& g, int slot, int rows, int zc, std::vector<ZTile>& out, int* count) {
  const int gx = (g.n1 + BX - 1) / BX, gy = (g.n2 + rows - 1) / rows;
  int bid = 0;
  for (int z0 = 0; z0 < g.n3; z0 += zc)
    for (int by = 0; by < gy; ++by)
      for (int bx = 0; bx < gx; ++bx) out.push_back(ZTile{slot, bx, by, z0, std::min(z0 + zc, g.n3), bid++});
  *count = bid;
}

void grid_segs(const GridDev& g, int slot, std::vector<PSeg>& out, int* count) {
  const long long L = 16384;
  int bid = 0;
  for (long long b = 0; b < g.G; b += L) out.push_back(PSeg{slot, bid++, b, std::min(b + L, g.G)});
  *count = bid;
}

void count_segs(long long n, int slot, std::vector<PSeg>& out, int* count) {
  const long long L = 16384;
  int bid = 0;
  for (long long b = 0; b < n; b += L) out.push_back(PSeg{slot, bid++, b, std::min(b + L, n)});
  *count = bid;
}

template <typename T>
struct Engine {
  ofdft_batch* B;
  ofdft_ctx* c;
  std::vector<std::unique_ptr<Slot<T>>>* active;
  std::vector<std::unique_ptr<Slot<T>>>* done;
  std::deque<std::unique_ptr<Slot<T>>>* queue;
  bool mixed;

  RedBuf slot_red(Slot<T>* S) { return RedBuf{S->partials, S->counter}; }

  // A work list for the next launch: copied into arena `a` (ordinary launches),
  // or staged into the capture arena while a graph is being captured (the copy
  // to the device happens once, after the capture).  *dptr: its device address.
  template <typename V>
  int put(DevArena& a, const std::vector<V>& v, const void** dptr) {
    if (B->capturing) {
      const size_t off = (B->cap_host.size() + 255) & ~(size_t)255;
      const size_t bytes = v.size() * sizeof(V);
      if (off + bytes > B->cap_bytes) return fail(c, OFDFT_ENOMEM, "batched CG graph: work lists exceed the arena");
      B->cap_host.resize(off + bytes);
      if (bytes) memcpy(B->cap_host.data() + off, v.data(), bytes);
      *dptr = B->cap_dev + off;
      return OFDFT_OK;
    }
    TRY(upload(c, a, v));
    *dptr = a.p;
    return OFDFT_OK;
  }

  template <typename TT, int R, int V, class L, class E>
  int launch_zb(int kind, unsigned nb, const ZTile* dt, const ZSlot<TT, L, E>* ds) {
    constexpr int smem = zsmem_bytes<TT, R, V, E>();
    static bool attr_dev[64] = {false};  // a per-device setting
    if (c->device < 0 || c->device >= 64) return fail(c, OFDFT_EINVAL, "device index out of range");
    if (!attr_dev[c->device]) {
      CU(cudaFuncSetAttribute(zbatch_kernel<TT, R, V, L, E>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
      attr_dev[c->device] = true;
    }
    {
      ProfScope ps_(c, kind);
      zbatch_kernel<TT, R, V, L, E><<<nb, dim3(BX, BY), smem, c->stream>>>(dt, ds);
    }
    CU(cudaGetLastError());
    return OFDFT_OK;
  }

  // --- batched launches ---------------------------------------------------
  // z-streaming pass of kind `kind` over the given slots; make(S) returns the
  // loader/epilogue descriptor of that slot.  One launch per stencil radius.
  template <typename TT, class L, class E, class Make>
  int zpass(const std::vector<Slot<T>*>& slots, int kind, double wscale, Make make) {
    // one launch per stencil radius and staging width (16-byte copies where the
    // grid's rows allow them, element copies otherwise)
    for (int Rr = 1; Rr <= kMaxR; ++Rr)
      for (int wide = 1; wide >= 0; --wide) {
        std::vector<ZTile> tiles;
        std::vector<ZSlot<TT, L, E>> desc;
        for (Slot<T>* S : slots) {
          if (S->Rr != Rr) continue;
          auto le = make(S);
          if ((int)zvec_ok<TT>(S->g, le.first, le.second) != wide) continue;
          int cnt = 0;
          const int si = (int)desc.size();
          grid_tiles(S->g, si, ZCfg<TT>::TY, S->zdepth, tiles, &cnt);
          ZSlot<TT, L, E> z;
          z.g = S->g;
          z.W = cast_weights<TT>(lap_weights(Rr, S->h, wscale));
          z.ld = le.first;
          z.ep = le.second;
          z.red = slot_red(S);
          z.nblocks = cnt;
          desc.push_back(z);
        }
        if (tiles.empty()) continue;
        const void *pt = nullptr, *pd = nullptr;
        TRY(put(B->d_tiles, tiles, &pt));
        TRY(put(B->d_desc, desc, &pd));
        const ZTile* dt = (const ZTile*)pt;
        const ZSlot<TT, L, E>* ds = (const ZSlot<TT, L, E>*)pd;
        const unsigned nb = (unsigned)tiles.size();
        constexpr int VW = 16 / (int)sizeof(TT);
        switch (Rr * 2 + wide) {
#define ZB_CASE(RR)                                                             \
  case RR * 2 + 1: TRY((launch_zb<TT, RR, VW, L, E>(kind, nb, dt, ds))); break; \
  case RR * 2: TRY((launch_zb<TT, RR, 1, L, E>(kind, nb, dt, ds))); break;
          ZB_CASE(1)
          ZB_CASE(2)
          ZB_CASE(3)
          ZB_CASE(4)
          ZB_CASE(5)
          ZB_CASE(6)
#undef ZB_CASE
        }
      }
    return OFDFT_OK;
  }

  // pointwise pass over the given slots; make(S, nblocks) returns the op.
  template <class Op, class Make>
  int ppass(const std::vector<Slot<T>*>& slots, int kind, Make make) {
    std::vector<PSeg> segs;
    std::vector<Op> ops;
    for (Slot<T>* S : slots) {
      int cnt = 0;
      const int si = (int)ops.size();
      std::vector<PSeg> tmp;
      grid_segs(S->g, si, tmp, &cnt);
      segs.insert(segs.end(), tmp.begin(), tmp.end());
      ops.push_back(make(S, cnt));
    }
    if (segs.empty()) return OFDFT_OK;
    const void *ps = nullptr, *po = nullptr;
    TRY(put(B->d_segs, segs, &ps));
    TRY(put(B->d_ops, ops, &po));
    {
      ProfScope ps_(c, kind);
      pbatch_kernel<Op><<<(unsigned)segs.size(), 256, 0, c->stream>>>((const PSeg*)ps, (const Op*)po);
    }
    CU(cudaGetLastError());
    return OFDFT_OK;
  }

  // pointwise pass over n(S) elements of each slot (a multigrid level).
  template <class Op, class Count, class Make>
  int ppass_n(const std::vector<Slot<T>*>& slots, int kind, Count n, Make make) {
    std::vector<PSeg> segs;
    std::vector<Op> ops;
    for (Slot<T>* S : slots) {
      int cnt = 0;
      const int si = (int)ops.size();
      count_segs(n(S), si, segs, &cnt);
      ops.push_back(make(S, cnt));
    }
    if (segs.empty()) return OFDFT_OK;
    const void *ps = nullptr, *po = nullptr;
    TRY(put(B->d_segs, segs, &ps));
    TRY(put(B->d_ops, ops, &po));
    {
      ProfScope ps_(c, kind);
      pbatch_kernel<Op><<<(unsigned)segs.size(), 256, 0, c->stream>>>((const PSeg*)ps, (const Op*)po);
    }
    CU(cudaGetLastError());
    return OFDFT_OK;
  }

  // z = M r for every preconditioned slot: one V-cycle per grid, each pass of
  // the cycle shared by the grids that have that level (S3 + S11).
  template <class GetR, class GetSc>
  int mg_cycle(const std::vector<Slot<T>*>& slots, GetR getr, GetSc getsc) {
    std::vector<Slot<T>*> pcs;
    int maxlc = 0;
    for (Slot<T>* S : slots)
      if (S->pc) {
        pcs.push_back(S);
        maxlc = std::max(maxlc, S->mg.lc);
      }
    if (pcs.empty()) return OFDFT_OK;
    const T om = (T)c->mg_omega;
    auto nodes = [](Slot<T>* S, int l) { return mg_nodes(S->mg.d[l]); };
    auto rl = [&](Slot<T>* S, int l) -> T* { return l == 0 ? (T*)getr(S) : S->mgc + S->mg.off[l]; };
    auto zl = [&](Slot<T>* S, int l) -> T* { return l == 0 ? S->mz : S->mgc + S->mg.off[l] + nodes(S, l); };
    auto tl = [&](Slot<T>* S, int l) -> T* { return l == 0 ? S->mt : S->mgc + S->mg.off[l] + 2 * nodes(S, l); };
    auto sl = [&](Slot<T>* S, int l) { return (T)(S->mg.s0 * pow(4.0, l)); };
    auto having = [&](int l) {
      std::vector<Slot<T>*> v;
      for (Slot<T>* S : pcs)
        if (S->mg.lc > l) v.push_back(S);
      return v;
    };
    for (int l = 0; l < maxlc; ++l) {
      const std::vector<Slot<T>*> v = having(l);
      TRY((ppass_n<OpMgDown<T>>(v, OFDFT_K_MG, [&](Slot<T>* S) { return nodes(S, l); }, [&](Slot<T>* S, int nb) {
        return OpMgDown<T>{S->mg.d[l], rl(S, l), tl(S, l), om, getsc(S), slot_red(S), nb};
      })));
      TRY((ppass_n<OpMgRestrict<T>>(v, OFDFT_K_MG, [&](Slot<T>* S) { return nodes(S, l + 1); },
                                    [&](Slot<T>* S, int nb) {
                                      return OpMgRestrict<T>{S->mg.d[l], S->mg.d[l + 1], tl(S, l), rl(S, l + 1),
                                                             getsc(S), slot_red(S), nb};
                                    })));
    }
    for (int dot = 0; dot < 2; ++dot) {  // the coarse ends: whole grids (lc = 0) form r.z themselves
      std::vector<MgCoarseJob<T>> jobs;
      size_t smem = 0;
      for (Slot<T>* S : pcs)
        if ((S->mg.lc == 0) == (dot == 1)) {
          const int lc = S->mg.lc;
          jobs.push_back(MgCoarseJob<T>{S->mg.d[lc], S->mg.nlev - lc, rl(S, lc), zl(S, lc), sl(S, lc), getsc(S)});
          smem = std::max(smem, S->mg.smem);
        }
      if (jobs.empty()) continue;
      const void* pj = nullptr;
      TRY(put(B->d_ops, jobs, &pj));
      ProfScope ps_(c, OFDFT_K_MG);
      static bool attr_dev[64] = {false};  // per element type and device
      if (c->device < 0 || c->device >= 64) return fail(c, OFDFT_EINVAL, "device index out of range");
      if (!attr_dev[c->device]) {
        CU(cudaFuncSetAttribute(mg_coarse_batch_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                200 * 1024));
        CU(cudaFuncSetAttribute(mg_coarse_batch_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                200 * 1024));
        attr_dev[c->device] = true;
      }
      if (dot) {
        mg_coarse_batch_kernel<T, true><<<(unsigned)jobs.size(), 1024, smem, c->stream>>>(
            (const MgCoarseJob<T>*)pj, om, c->mg_sweeps);
      } else {
        mg_coarse_batch_kernel<T, false><<<(unsigned)jobs.size(), 1024, smem, c->stream>>>(
            (const MgCoarseJob<T>*)pj, om, c->mg_sweeps);
      }
      CU(cudaGetLastError());
    }
    for (int l = maxlc - 1; l >= 0; --l) {
      const std::vector<Slot<T>*> v = having(l);
      TRY((ppass_n<OpMgProlong<T>>(v, OFDFT_K_MG, [&](Slot<T>* S) { return nodes(S, l); }, [&](Slot<T>* S, int nb) {
        return OpMgProlong<T>{S->mg.d[l], S->mg.d[l + 1], rl(S, l), zl(S, l + 1), tl(S, l), sl(S, l), getsc(S),
                              slot_red(S), nb};
      })));
      if (l == 0)
        TRY((ppass_n<OpMgUp<T, true>>(v, OFDFT_K_MG, [&](Slot<T>* S) { return nodes(S, 0); }, [&](Slot<T>* S, int nb) {
          return OpMgUp<T, true>{S->mg.d[0], rl(S, 0), tl(S, 0), S->mz, om, sl(S, 0), getsc(S), slot_red(S), nb};
        })));
      else
        TRY((ppass_n<OpMgUp<T, false>>(v, OFDFT_K_MG, [&](Slot<T>* S) { return nodes(S, l); }, [&](Slot<T>* S, int nb) {
          return OpMgUp<T, false>{S->mg.d[l], rl(S, l), tl(S, l), zl(S, l), om, sl(S, l), getsc(S), slot_red(S), nb};
        })));
    }
    return OFDFT_OK;
  }

  int read_scalars() {
    CU(cudaMemcpyAsync(B->h_sc.data(), B->sc, B->capacity * sizeof(CgScalars), cudaMemcpyDeviceToHost, c->stream));
    if (mixed)
      CU(cudaMemcpyAsync(B->h_sc32.data(), B->sc32, B->capacity * sizeof(CgScalars), cudaMemcpyDeviceToHost,
                         c->stream));
    CU(cudaStreamSynchronize(c->stream));
    if (!c->pending.empty()) harvest(c);
    return OFDFT_OK;
  }

  // One CG iteration on the given slots (S3): the V-cycle of the preconditioned
  // slots, the stencil pass and the update; every kernel skips a slot whose CG
  // is done.
  template <class GetX, class GetR, class GetSc>
  int cg_iteration(const std::vector<Slot<T>*>& slots, bool fold, GetX getx, GetR getr, GetSc getsc) {
    // the stencil pass forms p and q from z = M r (preconditioned slots) or r
    TRY(mg_cycle(slots, getr, getsc));
    auto dir = [&](Slot<T>* S) -> const T* { return S->pc ? S->mz : getr(S); };
    if (fold) {
      TRY((zpass<T, LoadPlain<T>, EpiCgAX<T>>(slots, OFDFT_K_CG_DIR_STENCIL, -1.0, [&](Slot<T>* S) {
        return std::make_pair(LoadPlain<T>{dir(S)}, EpiCgAX<T>{S->pv, S->qv, (T*)getx(S), getsc(S)});
      })));
      TRY((ppass<OpCgUpdateR<T>>(slots, OFDFT_K_CG_UPDATE, [&](Slot<T>* S, int nb) {
        return OpCgUpdateR<T>{getr(S), S->qv, getsc(S), slot_red(S), nb};
      })));
    } else {
      TRY((zpass<T, LoadPlain<T>, EpiCgA<T>>(slots, OFDFT_K_CG_DIR_STENCIL, -1.0, [&](Slot<T>* S) {
        return std::make_pair(LoadPlain<T>{dir(S)}, EpiCgA<T>{S->pv, S->qv, getsc(S)});
      })));
      using X = std::remove_pointer_t<decltype(getx(slots[0]))>;
      TRY((ppass<OpCgUpdate<T, X>>(slots, OFDFT_K_CG_UPDATE, [&](Slot<T>* S, int nb) {
        return OpCgUpdate<T, X>{getx(S), getr(S), S->pv, S->qv, getsc(S), slot_red(S), nb};
      })));
    }
    return OFDFT_OK;
  }

  // Autotuner of the batched z-streaming passes (S11): the planes per CTA of
  // each grid's tiles in the CG stencil pass, timed on the grid itself (its r
  // or z as input) with scratch p and q and private CG scalars, so no solve's
  // state changes; chosen once per grid shape for the context's lifetime, so a
  // request's partial-sum order, and with it its result, is the same alone and
  // in any mix.
  template <class GetR>
  int tune_zdepth(const std::vector<Slot<T>*>& slots, GetR getr) {
    for (Slot<T>* S : slots) {
      if (S->ztuned) continue;
      // one choice per grid shape, stencil radius and element type for the
      // context's lifetime
      const std::vector<long long> key = {-1, (long long)sizeof(T), S->Rr, S->pc, S->g.n1, S->g.n2, S->g.n3};
      bool found = false;
      for (auto& t : c->ztune)
        if (t.first == key) {
          S->zdepth = t.second;
          B->zdepth = S->zdepth;
          B->ztuned = 1;  // chosen by the autotuner earlier in this context
          found = true;
          break;
        }
      if (!found) {
        TRY(tune_grid_zdepth(S, getr));
        c->ztune.push_back({key, S->zdepth});
      }
      S->ztuned = 1;
    }
    return OFDFT_OK;
  }

  // Times the batched CG stencil pass of one grid alone at 8, 16, 32 and 64
  // planes per CTA (scratch outputs, a private scalar block) and keeps the fastest.
  template <class GetR>
  int tune_grid_zdepth(Slot<T>* S, GetR getr) {
    const long long G = S->g.G;
    T* scratch = nullptr;
    CgScalars* psc = nullptr;
    CU(cudaMalloc(&scratch, 2 * G * sizeof(T)));
    if (cudaMalloc(&psc, sizeof(CgScalars)) != cudaSuccess) {
      cudaFree(scratch);
      return fail(c, OFDFT_ENOMEM, "autotune: no room for scratch scalars");
    }
    CgScalars init;
    memset(&init, 0, sizeof(init));
    init.first = 1;
    init.max_it = 1 << 30;
    const int prof = c->prof;
    c->prof = 0;
    const long long launches = c->launches;
    long long kinds[OFDFT_K_COUNT];
    memcpy(kinds, c->kind_launches, sizeof(kinds));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = OFDFT_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
      rc = fail(c, OFDFT_ECUDA, "autotune: event creation failed");
    const int saved = S->zdepth;
    int best = saved;
    float best_ms = 1e30f;
    B->tune_log.clear();
    const std::vector<Slot<T>*> one = {S};
    for (int zc : {8, 16, 32, 64}) {
      if (rc != OFDFT_OK) break;
      S->zdepth = zc;
      float ms = 0.0f;
      for (int rep = 0; rep < 4 && rc == OFDFT_OK; ++rep) {
        if (cudaMemcpyAsync(psc, &init, sizeof(CgScalars), cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
            cudaEventRecord(e0, c->stream) != cudaSuccess) {
          rc = fail(c, OFDFT_ECUDA, "autotune: enqueue failed");
          break;
        }
        rc = zpass<T, LoadPlain<T>, EpiCgA<T>>(one, OFDFT_K_CG_DIR_STENCIL, -1.0, [&](Slot<T>* X) {
          return std::make_pair(LoadPlain<T>{X->pc ? X->mz : getr(X)}, EpiCgA<T>{scratch, scratch + G, psc});
        });
        float t = 0.0f;
        if (rc == OFDFT_OK && (cudaEventRecord(e1, c->stream) != cudaSuccess ||
                               cudaEventSynchronize(e1) != cudaSuccess ||
                               cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
          rc = fail(c, OFDFT_ECUDA, "autotune: timing failed");
        if (rep > 0) ms += t;  // the first launch of each depth warms up
      }
      if (rc == OFDFT_OK) B->tune_log.push_back({zc, ms / 3.0f * 1000.0f});
      if (ms < best_ms) {
        best_ms = ms;
        best = zc;
      }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(c->stream);
    cudaFree(scratch);
    cudaFree(psc);
    c->prof = prof;
    c->launches = launches;  // tuning launches are not the caller's work
    memcpy(c->kind_launches, kinds, sizeof(kinds));
    S->zdepth = (rc == OFDFT_OK) ? best : saved;
    if (rc != OFDFT_OK) return rc;
    B->zdepth = S->zdepth;
    B->ztuned = 1;
    return OFDFT_OK;
  }

  // The CG loop of these slots as one CUDA graph (captured on first use): a
  // WHILE node over one iteration and batch_cond_kernel, which keeps the loop
  // going while any of the slots is not done.
  template <class GetX, class GetR, class GetSc>
  int loop_graph(const std::vector<Slot<T>*>& slots, bool fold, GetX getx, GetR getr, GetSc getsc,
                 cudaGraphExec_t* out) {
    std::vector<long long> key = {(long long)sizeof(T), fold ? 1 : 0, (long long)getsc(slots[0]),
                                  (long long)c->partials.p};
    std::vector<int> idx;
    for (Slot<T>* S : slots) {
      key.push_back((long long)S);
      key.push_back(S->zdepth);
      key.push_back((long long)getx(S));
      key.push_back((long long)getr(S));
      key.push_back((long long)getsc(S));
      key.push_back(S->pc);
      idx.push_back(S->index);
    }
    for (auto& e : B->graphs)
      if (e.key == key) {
        *out = e.exec;
        return OFDFT_OK;
      }
    // the graph's own arena for the work lists its launches read
    const size_t arena = (size_t)16 << 20;
    void* dev = nullptr;
    CU(cudaMalloc(&dev, arena));
    cudaGraph_t graph = nullptr;
    cudaGraphConditionalHandle handle;
    cudaGraphNode_t init = nullptr, loop = nullptr;
    cudaGraphNodeParams cp = {};
    const CgScalars* base = getsc(slots[0]) - slots[0]->index;
    int* idx_dev = (int*)dev;  // the slot indices first, then the work lists
    const int n = (int)idx.size();
    cudaError_t e = cudaGraphCreate(&graph, 0);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&handle, graph, 0, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) {
      cudaKernelNodeParams kp = {};
      const int* cidx = idx_dev;
      int nn = n;
      void* args[] = {&handle, &base, &cidx, &nn};
      kp.func = (void*)batch_cond_kernel;
      kp.gridDim = dim3(1);
      kp.blockDim = dim3(256);
      kp.kernelParams = args;
      e = cudaGraphAddKernelNode(&init, graph, nullptr, 0, &kp);
    }
    if (e == cudaSuccess) {
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = handle;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      e = cudaGraphAddNode(&loop, graph, &init, nullptr, 1, &cp);
    }
    if (e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaFree(dev);
      return fail(c, OFDFT_ECUDA, "batched CG graph: %s", cudaGetErrorString(e));
    }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    B->cap_host.assign(256, 0);
    memcpy(B->cap_host.data(), idx.data(), idx.size() * sizeof(int));
    if (idx.size() * sizeof(int) > 256) {
      B->cap_host.resize((idx.size() * sizeof(int) + 255) & ~(size_t)255);
      memcpy(B->cap_host.data(), idx.data(), idx.size() * sizeof(int));
    }
    B->cap_dev = (char*)dev;
    B->cap_bytes = arena;
    B->capturing = true;
    const int prof = c->prof;
    c->prof = 0;
    const long long launches = c->launches;
    long long kinds[OFDFT_K_COUNT];
    memcpy(kinds, c->kind_launches, sizeof(kinds));
    cudaStream_t user = c->stream;
    c->stream = c->gstream;
    int rc = OFDFT_OK;
    e = cudaStreamBeginCaptureToGraph(c->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      rc = cg_iteration(slots, fold, getx, getr, getsc);
      if (rc == OFDFT_OK) {
        batch_cond_kernel<<<1, 256, 0, c->stream>>>(handle, base, idx_dev, n);
        if (cudaGetLastError() != cudaSuccess) rc = fail(c, OFDFT_ECUDA, "batched CG graph: condition launch");
      }
      cudaGraph_t got = nullptr;
      const cudaError_t ee = cudaStreamEndCapture(c->stream, &got);
      if (rc == OFDFT_OK && ee != cudaSuccess) e = ee;
    }
    c->stream = user;
    c->prof = prof;
    c->launches = launches;
    memcpy(c->kind_launches, kinds, sizeof(kinds));
    B->capturing = false;
    cudaGraphExec_t exec = nullptr;
    if (rc == OFDFT_OK && e == cudaSuccess)
      e = cudaMemcpy(dev, B->cap_host.data(), B->cap_host.size(), cudaMemcpyHostToDevice);
    if (rc == OFDFT_OK && e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (rc != OFDFT_OK || e != cudaSuccess) {
      cudaFree(dev);
      if (rc != OFDFT_OK) return rc;
      return fail(c, OFDFT_ECUDA, "batched CG graph: %s", cudaGetErrorString(e));
    }
    // keep the most recent graphs (a batch's composition changes on admit and retire)
    if (B->graphs.size() >= 16) {
      CU(cudaStreamSynchronize(c->stream));
      cudaGraphExecDestroy(B->graphs.front().exec);
      cudaFree(B->graphs.front().arena);
      B->graphs.erase(B->graphs.begin());
    }
    B->graphs.push_back({key, exec, dev});
    B->graph_captures++;
    *out = exec;
    return OFDFT_OK;
  }

  // CG iterations on the given slots until each is done (S3), `x` the iterate,
  // `r` the residual, `scp` the slot's CG scalars.  With CUDA graphs: one eager
  // iteration, then the rest in the loop's WHILE graph; otherwise chunks of
  // eight iterations polled by the host.
  // `set` is the round's set of evaluating slots (a superset of `slots`): the
  // graph is captured for the whole set, so it is replayed round after round
  // while the set stays the same; its slots outside `slots` are marked done
  // first, and every kernel skips them.
  template <class GetX, class GetR, class GetSc, class HostSc>
  int cg_loop(std::vector<Slot<T>*> slots, const std::vector<Slot<T>*>& set, GetX getx, GetR getr, GetSc getsc,
              HostSc hostsc) {
    const int chunk = 8;
    if (slots.empty()) return OFDFT_OK;
    const bool graphs = c->use_graphs && c->cond_graphs && !(c->prof & (1 << OFDFT_K_CG_UPDATE));
    const std::vector<Slot<T>*> all = graphs ? set : slots;
    // as ofdft_solve: when the batch's CG vectors do not fit in L2 the iterate
    // update of an iteration is folded into the next stencil pass (EpiCgAX), the
    // update only moves r, and a last flush applies the final pending x += alpha p
    double bytes = 0.0;
    for (Slot<T>* S : all) bytes += 5.0 * (double)S->g.G * sizeof(T);
    const bool fold = bytes > c->cg_fold_bytes;
    if (graphs) {
      if (!B->one_pinned) {
        CU(cudaHostAlloc((void**)&B->one_pinned, sizeof(int), cudaHostAllocDefault));
        *B->one_pinned = 1;
      }
      std::vector<char> in(B->capacity + 1, 0);
      for (Slot<T>* S : slots) in[S->index] = 1;
      for (Slot<T>* S : set)
        if (!in[S->index])
          CU(cudaMemcpyAsync(&getsc(S)->done, B->one_pinned, sizeof(int), cudaMemcpyHostToDevice, c->stream));
      if (c->autotune) TRY(tune_zdepth(set, getr));
      TRY(cg_iteration(set, fold, getx, getr, getsc));  // also sets kernel attributes outside the capture
      B->eager_iters++;
      cudaGraphExec_t exec = nullptr;
      TRY(loop_graph(set, fold, getx, getr, getsc, &exec));
      CU(cudaGraphLaunch(exec, c->stream));
      B->graph_replays++;
      TRY(read_scalars());
      long long its = 0;
      for (Slot<T>* S : slots) its = std::max<long long>(its, hostsc(S).iters);
      B->graph_iters += its;
      std::vector<Slot<T>*> still;
      for (Slot<T>* S : slots)
        if (!hostsc(S).done) still.push_back(S);
      slots.swap(still);  // empty unless a graph failed to finish a loop
    }
    while (!slots.empty()) {
      for (int i = 0; i < chunk; ++i) TRY(cg_iteration(slots, fold, getx, getr, getsc));
      TRY(read_scalars());
      std::vector<Slot<T>*> still;
      for (Slot<T>* S : slots)
        if (!hostsc(S).done) still.push_back(S);
      slots.swap(still);
    }
    if (fold)
      TRY((ppass<OpXFlush<T>>(all, OFDFT_K_VECTOR, [&](Slot<T>* S, int nb) {
        return OpXFlush<T>{(T*)getx(S), S->pv, getsc(S), slot_red(S), nb};
      })));
    return OFDFT_OK;
  }

  // Batched Poisson solves at each slot's evaluation point.
  int poisson(const std::vector<Slot<T>*>& ev) {
    if (ev.empty()) return OFDFT_OK;
    if (!mixed) {
      TRY((zpass<T, LoadPlain<T>, EpiResidual<T>>(ev, OFDFT_K_RESIDUAL, 1.0, [&](Slot<T>* S) {
        return std::make_pair(LoadPlain<T>{S->phi}, EpiResidual<T>{nullptr, S->ev_at, S->b, S->r, B->sc + S->index,
                                                                  S->ev_tol, S->p.max_cg, 1, S->pc});
      })));
      TRY(read_scalars());
      std::vector<Slot<T>*> run;
      for (Slot<T>* S : ev)
        if (!B->h_sc[S->index].done) run.push_back(S);
      TRY(cg_loop(
          run, ev, [](Slot<T>* S) { return S->phi; }, [](Slot<T>* S) { return S->r; },
          [&](Slot<T>* S) { return B->sc + S->index; }, [&](Slot<T>* S) -> CgScalars& { return B->h_sc[S->index]; }));
      for (Slot<T>* S : ev) {
        const CgScalars& h = B->h_sc[S->index];
        S->pstats.iterations = h.iters;
        S->pstats.rel_residual = sqrt(h.rr / (h.bb > 0 ? h.bb : 1.0));
      }
      return OFDFT_OK;
    }
    // mixed: FP32 CG with residual replacement (per slot), as poisson_mixed
    for (Slot<T>* S : ev) {
      S->ptotal = 0;
      S->pphase = 1;  // 1: the next replacement restarts the FP32 CG
    }
    std::vector<Slot<T>*> resid = ev;
    for (Slot<T>* S : ev) CU(cudaMemsetAsync(S->e32, 0, S->g.G * sizeof(float), c->stream));
    for (int round = 0; round <= 60 && !resid.empty(); ++round) {
      if (round > 0)
        TRY((ppass<OpFold>(resid, OFDFT_K_VECTOR, [&](Slot<T>* S, int) { return OpFold{S->phi64, S->e32}; })));
      TRY((zpass<double, LoadPlain<double>, EpiResidual<double, float, double>>(
          resid, OFDFT_K_RESIDUAL, 1.0, [&](Slot<T>* S) {
            return std::make_pair(LoadPlain<double>{S->phi64},
                                  EpiResidual<double, float, double>{nullptr, (const float*)S->ev_at, S->b64, S->r64,
                                                                     B->sc + S->index, S->ev_tol, S->p.max_cg,
                                                                     1});
          })));
      TRY(read_scalars());
      std::vector<Slot<T>*> corr;
      for (Slot<T>* S : resid) {
        const CgScalars& h = B->h_sc[S->index];
        const double bb = h.bb > 0 ? h.bb : 1.0;
        S->pstats.iterations = S->ptotal;
        S->pstats.rel_residual = sqrt(h.rr / bb);
        if (h.rr <= S->ev_tol * S->ev_tol * bb || S->ptotal >= S->p.max_cg || !isfinite(h.rr)) continue;
        corr.push_back(S);
      }
      if (corr.empty()) break;
      TRY((ppass<OpRefineReplace>(corr, OFDFT_K_VECTOR, [&](Slot<T>* S, int nb) {
        const int budget = std::min(std::max(S->p.refine_every, 1), S->p.max_cg - S->ptotal);
        const CgScalars& h = B->h_sc[S->index];
        const double itol = mixed_inner_tol(h.rr, h.bb > 0 ? h.bb : 1.0, S->ev_tol);
        // preconditioned CG restarts every round (as poisson_mixed)
        return OpRefineReplace{(float*)S->r, S->r64, B->sc32 + S->index, itol, budget, S->pphase || S->pc ? 1 : 0,
                               slot_red(S), nb, S->pc};
      })));
      TRY(read_scalars());
      std::vector<int> before(B->capacity, 0);
      std::vector<Slot<T>*> run;
      for (Slot<T>* S : corr) {
        S->pphase = 0;
        before[S->index] = B->h_sc32[S->index].iters;
        if (!B->h_sc32[S->index].done) run.push_back(S);
      }
      TRY(cg_loop(
          run, ev, [](Slot<T>* S) { return (T*)S->e32; }, [](Slot<T>* S) { return S->r; },
          [&](Slot<T>* S) { return B->sc32 + S->index; },
          [&](Slot<T>* S) -> CgScalars& { return B->h_sc32[S->index]; }));
      for (Slot<T>* S : corr) S->ptotal += std::max(B->h_sc32[S->index].iters - before[S->index], 1);
      resid.swap(corr);
    }
    // FP32 potential (the gradient and the forces take it)
    TRY((ppass<OpConvert<double, float>>(ev, OFDFT_K_VECTOR, [&](Slot<T>* S, int) {
      return OpConvert<double, float>{(float*)S->phi, S->phi64};
    })));
    return OFDFT_OK;
  }

  int evaluate(const std::vector<Slot<T>*>& ev) {
    if (ev.empty()) return OFDFT_OK;
    TRY(poisson(ev));
    TRY((zpass<T, LoadPlain<T>, EpiFunctional<T>>(ev, OFDFT_K_FUNCTIONAL, 1.0, [&](Slot<T>* S) {
      const Weights<double> W = lap_weights(S->Rr, S->h, 1.0);
      FuncScalars f;
      f.h3 = S->h3;
      f.N = S->N;
      f.eta = S->ev_eta;
      f.inv_mu = 1.0 / S->ev_mu;
      f.lambda = S->p.lambda;
      f.CF = 0.3 * pow(3.0 * kPi * kPi, 2.0 / 3.0);
      f.kin_vw = -S->p.lambda * W.c;
      f.terms = S->p.terms;
      const bool es = S->p.terms & OFDFT_TERM_ES;
      EpiFunctional<T> ep{es ? S->phi : nullptr, S->b, (es && !mixed) ? S->r : nullptr, S->ev_d, S->ev_sold,
                          S->ev_G, S->ev_s, (S->p.precond_rank1 && S->ev_s) ? S->w : nullptr,
                          &B->sc[S->index].sum_uu, f, B->out + 16 * S->index};
      if (es && mixed) {  // FP64 potential, pseudocharge and residual (as the single-solve path)
        ep.phi64 = S->phi64;
        ep.b64 = S->b64;
        ep.r64 = S->r64;
      }
      return std::make_pair(LoadPlain<T>{S->ev_at}, ep);
    })));
    CU(cudaMemcpyAsync(B->h_out.data(), B->out, B->capacity * 16 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    std::vector<Slot<T>*> r1;
    std::vector<double> gam(B->capacity, 0.0);
    for (Slot<T>* S : ev) {
      EvalOut o;
      memcpy(o.sums, &B->h_out[16 * S->index], 12 * sizeof(double));
      fill_energy(o, S->h, &S->p, S->E_self, S->ezz, S->ev_eta, S->ev_mu, S->ev_out);
      S->ev_out->poisson = S->pstats;
      S->stats.stencil_apps += S->pstats.iterations + 3;
      S->stats.cg_iters += S->pstats.iterations;
      S->stats.grad_evals += 1;
      if (S->p.precond_rank1 && S->ev_s) {
        const double cpen = 4.0 * S->h3 / S->ev_mu;
        gam[S->index] = cpen * o.sums[10] / (1.0 + cpen * o.sums[11]);
        S->ev_out->rs_pc -= S->h3 * gam[S->index] * o.sums[10];
        r1.push_back(S);
      }
    }
    TRY((ppass<OpRank1<T>>(r1, OFDFT_K_VECTOR, [&](Slot<T>* S, int) {
      return OpRank1<T>{S->ev_s, S->w, gam[S->index]};
    })));
    return OFDFT_OK;
  }

  int dots(const std::vector<Slot<T>*>& dv) {
    if (dv.empty()) return OFDFT_OK;
    TRY((ppass<OpDot2<T>>(dv, OFDFT_K_VECTOR, [&](Slot<T>* S, int nb) {
      return OpDot2<T>{S->dot_a[0], S->dot_a[1], S->dot_a[2], S->dot_a[3], B->out + 16 * S->index + 12,
                       slot_red(S), nb};
    })));
    CU(cudaMemcpyAsync(B->h_out.data(), B->out, B->capacity * 16 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    return OFDFT_OK;
  }

  // Runs queued vector updates in lockstep (op i of every slot together).
  int flush_vops(const std::vector<Slot<T>*>& slots) {
    size_t depth = 0;
    for (Slot<T>* S : slots) depth = std::max(depth, S->vops.size());
    for (size_t i = 0; i < depth; ++i) {
      std::vector<Slot<T>*> ax, dr;
      for (Slot<T>* S : slots)
        if (i < S->vops.size()) (S->vops[i].kind == VOP_AXPY_ABS ? ax : dr).push_back(S);
      TRY((ppass<OpAxpyAbs<T>>(ax, OFDFT_K_VECTOR, [&](Slot<T>* S, int) {
        const Vop<T>& v = S->vops[i];
        return OpAxpyAbs<T>{v.out, v.a, v.b, v.scalar};
      })));
      TRY((ppass<OpDirection<T>>(dr, OFDFT_K_VECTOR, [&](Slot<T>* S, int) {
        const Vop<T>& v = S->vops[i];
        return OpDirection<T>{v.out, v.a, v.scalar};
      })));
    }
    for (Slot<T>* S : slots) S->vops.clear();
    size_t ldepth = 0;
    for (Slot<T>* S : slots) ldepth = std::max(ldepth, S->line_ops.size());
    for (size_t i = 0; i < ldepth; ++i) {
      std::vector<Slot<T>*> ls;
      for (Slot<T>* S : slots)
        if (i < S->line_ops.size()) ls.push_back(S);
      TRY((ppass<OpLine>(ls, OFDFT_K_VECTOR, [&](Slot<T>* S, int) {
        return OpLine{mixed ? S->phi64 : reinterpret_cast<double*>(S->phi), S->phi0, S->line_ops[i]};
      })));
    }
    for (Slot<T>* S : slots) S->line_ops.clear();
    return OFDFT_OK;
  }

  // --- the method as a state machine ---------------------------------------
  void request_eval(Slot<T>* S, const T* at, T* Gout, T* sout, const T* d, const T* sold, ofdft_energy* out) {
    S->req = REQ_EVAL;
    S->ev_at = at;
    S->ev_G = Gout;
    S->ev_s = sout;
    S->ev_d = d;
    S->ev_sold = sold;
    S->ev_eta = S->eta;
    S->ev_mu = S->mu;
    S->ev_out = out;
    S->ev_tol = S->tol_p;
  }
  void request_dots(Slot<T>* S) {
    S->req = REQ_DOTS;
    S->dot_a[0] = S->G;
    S->dot_a[1] = S->d;
    S->dot_a[2] = S->d;
    S->dot_a[3] = S->d;
  }
  void vop(Slot<T>* S, int kind, T* out, const T* a, const T* b, double x) { S->vops.push_back(Vop<T>{kind, out, a, b, x}); }
  // Warm start of the line search's Poisson solves (as Solver::line_start and
  // line_guess of the single-solve path): record phi0, then extrapolate
  // phi0 -> phi_l linearly to the next position a.
  void line_start(Slot<T>* S) {
    if (S->p.terms & OFDFT_TERM_ES) S->line_ops.push_back(0.0);
    S->line_l = 0.0;
    S->pos = 0.0;
  }
  void line_guess(Slot<T>* S, double a) {
    if (S->line_l != 0.0 && (S->p.terms & OFDFT_TERM_ES)) {
      const double t = a / S->line_l - 1.0;
      if (t != 0.0) S->line_ops.push_back(t);
    }
    S->line_l = a;
  }

  void finish(Slot<T>* S, int status, const char* msg) {
    S->status = status;
    if (msg) S->err = msg;
    S->state = S_DONE;
    S->req = REQ_NONE;
  }

  // Advances S until it issues a request or finishes (mirrors Solver::nlcg and
  // the Algorithm 1 loop of ofdft_solve step by step).
  void advance(Slot<T>* S) {
    const ofdft_params& p = S->p;
    const double h3 = S->h3;
    for (;;) {
      switch (S->state) {
        case S_AL_START:
          request_eval(S, S->u, S->G, S->s, nullptr, nullptr, &S->e);
          S->state = S_NLCG_START;
          S->inner_ok = -1;  // marks "E_prev not yet recorded"
          return;
        case S_NLCG_START:
          if (S->inner_ok == -1) {
            S->E_prev = S->e.E;
            S->inner_ok = 0;
          }
          // inner solve on L(., eta, mu) starts with an evaluation at u
          request_eval(S, S->u, S->G, S->s, nullptr, nullptr, &S->e);
          S->state = S_ITER;
          S->it = -1;
          return;
        case S_ITER: {
          if (S->it == -1) {  // first pass after the starting evaluation
            vop(S, VOP_DIRECTION, S->d, S->s, nullptr, 0.0);
            S->delta_new = S->e.rs_pc;
            S->k = 0;
            S->it = 0;
          }
          if (S->e.rs < p.tol_inner * S->M) {
            S->inner_ok = 1;
            S->state = S_AL_UPDATE;
            continue;
          }
          if (!isfinite(S->e.L) || !isfinite(S->e.rs)) {
            finish(S, OFDFT_ENONFINITE, "augmented Lagrangian is not finite");
            return;
          }
          if (S->it >= p.max_nlcg) {
            S->state = S_AL_UPDATE;
            continue;
          }
          S->tol_p = adaptive_poisson_tol(&p, S->e.rs, S->M);
          S->stats.nlcg_iters++;
          S->s_old = S->s;
          S->redo_dots = 0;
          request_dots(S);
          S->state = S_DOTS;
          return;
        }
        case S_DOTS: {
          const double* o = &B->h_out[16 * S->index + 12];
          S->g0 = h3 * o[0];
          S->dd = h3 * o[1];
          if (!(S->g0 < 0.0) && !S->redo_dots) {  // not a descent direction: restart along s
            vop(S, VOP_DIRECTION, S->d, S->s, nullptr, 0.0);
            S->k = 0;
            S->redo_dots = 1;
            request_dots(S);
            return;
          }
          S->sig = p.sigma0;
          if (p.trial_max_rel > 0.0 && S->dd > 0.0) S->sig = std::min(S->sig, p.trial_max_rel * sqrt(S->N / S->dd));
          line_start(S);
          line_guess(S, S->sig);
          vop(S, VOP_AXPY_ABS, S->ut, S->u, S->d, S->sig);
          request_eval(S, S->ut, S->Gt, S->st, S->d, S->s_old, &S->et);
          S->ev_tol = trial_poisson_tol(&p, S->tol_p);
          S->state = S_TRIAL;
          return;
        }
        case S_TRIAL: {
          S->alpha = -S->sig;
          S->gprev = S->et.gd;
          S->gcur = S->g0;
          if (!((S->gcur - S->gprev) / S->alpha > 0.0)) {
            std::swap(S->u, S->ut);
            std::swap(S->G, S->Gt);
            std::swap(S->s, S->st);
            S->e = S->et;
            goto direction;
          }
          S->snew = S->sn;
          S->L0 = S->e.L + l_resolution(S->e, mixed);
          S->j = 1;
          S->alpha = S->alpha * S->gcur / (S->gprev - S->gcur);
          S->bt = 0;
          line_guess(S, S->pos + S->alpha);
          vop(S, VOP_AXPY_ABS, S->ut, S->u, S->d, S->alpha);
          request_eval(S, S->ut, S->G, S->snew, S->d, S->s_old, &S->e);
          S->state = S_SECANT;
          return;
        }
        case S_SECANT: {
          if (S->bt < p.max_backtrack && !(S->e.L <= S->L0)) {
            S->bt++;
            S->alpha *= 0.5;
            line_guess(S, S->pos + S->alpha);
            vop(S, VOP_AXPY_ABS, S->ut, S->u, S->d, S->alpha);
            request_eval(S, S->ut, S->G, S->snew, S->d, S->s_old, &S->e);
            return;
          }
          std::swap(S->u, S->ut);
          S->pos += S->alpha;
          S->gprev = S->gcur;
          S->gcur = S->e.gd;
          const bool stop = (S->j == p.max_secant || S->alpha * S->alpha * S->dd <= p.eps_secant * p.eps_secant * S->N) ||
                            !((S->gcur - S->gprev) / S->alpha > 0.0);
          if (!stop) {
            S->j++;
            S->alpha = S->alpha * S->gcur / (S->gprev - S->gcur);
            S->bt = 0;
            line_guess(S, S->pos + S->alpha);
            vop(S, VOP_AXPY_ABS, S->ut, S->u, S->d, S->alpha);
            request_eval(S, S->ut, S->G, S->snew, S->d, S->s_old, &S->e);
            return;
          }
          S->sn = S->s;
          S->s = S->snew;
          goto direction;
        }
        case S_AL_UPDATE: {
          S->stats.outer_iters++;
          const double E = S->e.E, C = S->e.C;
          if (!isfinite(E) || !isfinite(C)) {
            finish(S, OFDFT_ENONFINITE, "energy or constraint is not finite");
            return;
          }
          const double eta_eff = S->eta - C / S->mu;
          S->stats.eta = eta_eff;
          if (p.method == OFDFT_METHOD_AL) S->eta = eta_eff;
          S->mu = p.kappa * S->mu;
          S->q++;
          const bool conv = fabs(E - S->E_prev) < p.tol_E * S->M;
          S->E_prev = E;
          if (conv || S->q >= p.max_outer) {
            S->stats.converged = conv ? 1 : 0;
            if (S->tol_p > p.tol_poisson) {
              // as ofdft_solve: the reported energy and the forces use a
              // potential solved to tol_poisson
              S->tol_p = p.tol_poisson;
              request_eval(S, S->u, nullptr, nullptr, nullptr, nullptr, &S->e);
              S->state = S_FINAL;
              return;
            }
            S->state = S_FINAL;
            continue;
          }
          S->state = S_NLCG_START;
          continue;
        }
        case S_FINAL:
          if (S->stats.converged)
            finish(S, OFDFT_OK, nullptr);
          else
            finish(S, OFDFT_ENOTCONV, "Algorithm 1 reached max_outer");
          return;
        default:
          return;
      }
    direction : {
      const double delta_old = S->delta_new;
      const double delta_mid = -S->e.gs_old;
      S->delta_new = S->e.rs_pc;
      const double beta = (S->delta_new - delta_mid) / delta_old;
      S->k++;
      if (S->k >= p.restart_every || !(beta > 0.0) || !std::isfinite(beta)) {
        vop(S, VOP_DIRECTION, S->d, S->s, nullptr, 0.0);
        S->k = 0;
      } else {
        vop(S, VOP_DIRECTION, S->d, S->s, nullptr, beta);
      }
      S->it++;
      S->state = S_ITER;
      continue;
    }
    }
  }

  // --- admission and completion --------------------------------------------
  int ensure_capacity(int need) {
    if (need <= B->capacity) return OFDFT_OK;
    const int cap = std::max(need, std::max(16, 2 * B->capacity));
    CU(cudaStreamSynchronize(c->stream));
    CgScalars *nsc = nullptr, *nsc32 = nullptr;
    double* nout = nullptr;
    CU(cudaMalloc(&nsc, cap * sizeof(CgScalars)));
    CU(cudaMalloc(&nsc32, cap * sizeof(CgScalars)));
    CU(cudaMalloc(&nout, cap * 16 * sizeof(double)));
    CU(cudaMemset(nsc, 0, cap * sizeof(CgScalars)));
    CU(cudaMemset(nsc32, 0, cap * sizeof(CgScalars)));
    CU(cudaMemset(nout, 0, cap * 16 * sizeof(double)));
    if (B->capacity > 0) {
      CU(cudaMemcpy(nsc, B->sc, B->capacity * sizeof(CgScalars), cudaMemcpyDeviceToDevice));
      CU(cudaMemcpy(nsc32, B->sc32, B->capacity * sizeof(CgScalars), cudaMemcpyDeviceToDevice));
      CU(cudaMemcpy(nout, B->out, B->capacity * 16 * sizeof(double), cudaMemcpyDeviceToDevice));
    }
    cudaFree(B->sc);
    cudaFree(B->sc32);
    cudaFree(B->out);
    B->sc = nsc;
    B->sc32 = nsc32;
    B->out = nout;
    for (int i = B->capacity; i < cap; ++i) B->free_index.push_back(i);
    B->capacity = cap;
    B->h_sc.resize(cap);
    B->h_sc32.resize(cap);
    B->h_out.resize((size_t)cap * 16);
    return OFDFT_OK;
  }

  int admit_one(Slot<T>* S) {
    TRY(carve(c, S, B->prec));
    if (B->free_index.empty()) TRY(ensure_capacity(B->capacity + 1));
    std::sort(B->free_index.begin(), B->free_index.end(), std::greater<int>());
    S->index = B->free_index.back();
    B->free_index.pop_back();
    B->in_use += (long long)S->bytes;
    const int rr = S->Rr;
    const ofdft_grid* gr = &S->grid;
    if (!mixed) {
      TRY(device_pseudocharge<double>(c, gr, rr, S->R.data(), S->Z.data(), S->M, S->p.sigma, S->p.rc, (double*)S->b,
                                      &S->E_self));
    } else {
      TRY(device_pseudocharge<double>(c, gr, rr, S->R.data(), S->Z.data(), S->M, S->p.sigma, S->p.rc, S->b64,
                                      &S->E_self));
      std::vector<Slot<T>*> one{S};
      TRY((ppass<OpConvert<double, float>>(one, OFDFT_K_VECTOR, [&](Slot<T>* X, int) {
        return OpConvert<double, float>{(float*)X->b, X->b64};
      })));
      CU(cudaMemsetAsync(S->phi64, 0, S->g.G * sizeof(double), c->stream));
    }
    TRY(device_guess<T>(c, gr, S->R.data(), S->Z.data(), S->M, S->p.guess_sigma, S->p.guess_cut, S->N, S->u));
    CU(cudaMemsetAsync(S->phi, 0, S->g.G * sizeof(T), c->stream));
    S->Fz.assign(3 * (size_t)S->M, 0.0);
    if (S->p.ezz_correction) TRY(device_ezz(c, S->R.data(), S->Z.data(), S->M, S->p.sigma, &S->ezz, S->Fz.data()));
    S->eta = (S->p.method == OFDFT_METHOD_PENALTY) ? 0.0 : S->p.eta0;
    S->mu = S->p.mu0;
    S->tol_p = (S->p.poisson_adapt > 0.0) ? std::max(S->p.tol_poisson, 1e-4) : S->p.tol_poisson;
    S->state = S_AL_START;
    S->stats.grid = S->grid;
    return OFDFT_OK;
  }

  int complete(Slot<T>* S) {
    S->stats.E = S->e.E;
    S->stats.C = S->e.C;
    S->stats.parts = S->e;
    if (S->status == OFDFT_OK || S->status == OFDFT_ENOTCONV) {
      S->forces.assign(3 * (size_t)S->M, 0.0);
      TRY(device_forces<T>(c, &S->grid, S->Rr, S->R.data(), S->Z.data(), S->M, S->p.sigma, S->p.rc,
                           S->p.force_variant, S->phi, S->forces.data()));
      if (S->p.ezz_correction)
        for (int i = 0; i < 3 * S->M; ++i) S->forces[i] += S->Fz[i];
    }
    CU(cudaStreamSynchronize(c->stream));
    CU(cudaFree(S->mem));
    S->mem = nullptr;
    B->in_use -= (long long)S->bytes;
    B->free_index.push_back(S->index);
    return OFDFT_OK;
  }

  // One round: admit what fits, advance every slot to its next request, run the
  // packed vector updates, evaluations and dot products, retire finished solves.
  int step() {
    while (!queue->empty()) {
      Slot<T>* S = queue->front().get();
      int mb = 0;
      const long long need = slot_bytes(S->grid, B->prec, &mb);
      if (B->in_use + need > B->budget && !active->empty()) break;
      TRY(admit_one(S));
      active->push_back(std::move(queue->front()));
      queue->pop_front();
    }
    std::vector<Slot<T>*> slots;
    for (auto& u : *active) slots.push_back(u.get());
    for (Slot<T>* S : slots) {
      S->req = REQ_NONE;
      advance(S);
    }
    TRY(flush_vops(slots));
    std::vector<Slot<T>*> ev, dv;
    for (Slot<T>* S : slots) {
      if (S->req == REQ_EVAL) ev.push_back(S);
      if (S->req == REQ_DOTS) dv.push_back(S);
    }
    TRY(evaluate(ev));
    TRY(dots(dv));
    for (size_t i = 0; i < active->size();) {
      Slot<T>* S = (*active)[i].get();
      if (S->state == S_DONE) {
        TRY(complete(S));
        done->push_back(std::move((*active)[i]));
        active->erase(active->begin() + i);
      } else {
        ++i;
      }
    }
    B->rounds++;
    return OFDFT_OK;
  }
};

template <typename T>
Engine<T> engine_of(ofdft_batch* b);

template <>
Engine<double> engine_of<double>(ofdft_batch* b) {
  return Engine<double>{b, b->c, &b->s64_active, &b->s64_done, &b->s64_queue, false};
}
template <>
Engine<float> engine_of<float>(ofdft_batch* b) {
  return Engine<float>{b, b->c, &b->s32_active, &b->s32_done, &b->s32_queue, true};
}

template <typename T>
int submit_impl(ofdft_batch* b, const double* R, const double* Z, int M, double h, const ofdft_params* p,
                const ofdft_grid* grid, int* id) {
  auto S = std::make_unique<Slot<T>>();
  S->p = *p;
  S->R.assign(R, R + 3 * (size_t)M);
  S->Z.assign(Z, Z + M);
  S->M = M;
  for (int i = 0; i < M; ++i) S->N += Z[i];
  if (grid) {
    S->grid = *grid;
  } else {
    const int rc = ofdft_grid_for_atoms(R, M, h, p->vacuum, p->round_to > 0 ? p->round_to : 1, &S->grid);
    if (rc != OFDFT_OK) return fail(b->c, rc, "box rule failed");
  }
  TRY(check_grid(b->c, &S->grid));
  S->g = gdev(&S->grid);
  S->h = S->grid.h;
  S->h3 = S->h * S->h * S->h;
  S->Rr = p->fd_order / 2;
  S->id = b->next_id++;
  *id = S->id;
  engine_of<T>(b).queue->push_back(std::move(S));
  return OFDFT_OK;
}

template <typename T>
int poll_impl(ofdft_batch* b, int id, int* done, double* energy, double* forces, ofdft_solve_stats* st) {
  Engine<T> E = engine_of<T>(b);
  for (size_t i = 0; i < E.done->size(); ++i) {
    Slot<T>* S = (*E.done)[i].get();
    if (S->id != id) continue;
    *done = 1;
    if (energy) *energy = S->stats.E;
    if (forces && !S->forces.empty()) memcpy(forces, S->forces.data(), S->forces.size() * sizeof(double));
    if (st) *st = S->stats;
    const int status = S->status;
    if (status != OFDFT_OK) fail(b->c, status, "%s", S->err.c_str());
    E.done->erase(E.done->begin() + i);
    return status;
  }
  *done = 0;
  for (auto& S : *E.active)
    if (S->id == id) return OFDFT_OK;
  for (auto& S : *E.queue)
    if (S->id == id) return OFDFT_OK;
  return fail(b->c, OFDFT_EINVAL, "unknown request id %d", id);
}

}  // namespace
}  // namespace ofd

// ===================================================================== C ABI
extern "C" {

int ofdft_batch_create(ofdft_ctx* c, int precision, long long hbm_budget_bytes, ofdft_batch** out) {
  if (!c || !out) return OFDFT_EINVAL;
  c->err.clear();
  *out = nullptr;
  if (precision != OFDFT_PREC_FP64 && precision != OFDFT_PREC_MIXED)
    return fail(c, OFDFT_EINVAL, "precision must be OFDFT_PREC_FP64 or OFDFT_PREC_MIXED");
  if (hbm_budget_bytes <= 0) return fail(c, OFDFT_EINVAL, "HBM budget must be positive");
  CU(cudaSetDevice(c->device));
  ofdft_batch* b = new ofdft_batch();
  b->c = c;
  b->prec = precision;
  b->budget = hbm_budget_bytes;
  *out = b;
  return OFDFT_OK;
}

int ofdft_batch_destroy(ofdft_batch* b) {
  if (!b) return OFDFT_OK;
  ofdft_ctx* c = b->c;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  auto drop = [](auto& v) {
    for (auto& S : v)
      if (S->mem) cudaFree(S->mem);
  };
  drop(b->s64_active);
  drop(b->s32_active);
  drop(b->s64_done);
  drop(b->s32_done);
  for (auto& gr : b->graphs) {
    cudaGraphExecDestroy(gr.exec);
    cudaFree(gr.arena);
  }
  if (b->one_pinned) cudaFreeHost(b->one_pinned);
  cudaFree(b->sc);
  cudaFree(b->sc32);
  cudaFree(b->out);
  for (DevArena* a : {&b->d_tiles, &b->d_desc, &b->d_segs, &b->d_ops}) cudaFree(a->p);
  delete b;
  return OFDFT_OK;
}

int ofdft_batch_submit(ofdft_batch* b, const double* R, const double* Z, int M, double h, const ofdft_params* p,
                       const ofdft_grid* grid, int* request_id) {
  if (!b || !request_id) return OFDFT_EINVAL;
  ofdft_ctx* c = b->c;
  c->err.clear();
  TRY(check_params(c, p));
  if (p->method == OFDFT_METHOD_LM)
    return fail(c, OFDFT_EINVAL, "the batch engine runs Algorithm 1 (AL or penalty); use ofdft_solve for LM");
  TRY(check_atoms(c, R, Z, M));
  if (p->precision != b->prec) return fail(c, OFDFT_EINVAL, "request precision differs from the batch precision");
  if (b->prec == OFDFT_PREC_FP64) return submit_impl<double>(b, R, Z, M, h, p, grid, request_id);
  return submit_impl<float>(b, R, Z, M, h, p, grid, request_id);
}

int ofdft_batch_step(ofdft_batch* b, int* n_active, int* n_queued) {
  if (!b) return OFDFT_EINVAL;
  ofdft_ctx* c = b->c;
  c->err.clear();
  CU(cudaSetDevice(c->device));
  int rc;
  if (b->prec == OFDFT_PREC_FP64) {
    Engine<double> E = engine_of<double>(b);
    rc = E.step();
    if (n_active) *n_active = (int)E.active->size();
    if (n_queued) *n_queued = (int)E.queue->size();
  } else {
    Engine<float> E = engine_of<float>(b);
    rc = E.step();
    if (n_active) *n_active = (int)E.active->size();
    if (n_queued) *n_queued = (int)E.queue->size();
  }
  return rc;
}

int ofdft_batch_poll(ofdft_batch* b, int request_id, int* done, double* energy, double* forces,
                     ofdft_solve_stats* st) {
  if (!b || !done) return OFDFT_EINVAL;
  b->c->err.clear();
  if (b->prec == OFDFT_PREC_FP64) return poll_impl<double>(b, request_id, done, energy, forces, st);
  return poll_impl<float>(b, request_id, done, energy, forces, st);
}

int ofdft_batch_run(ofdft_batch* b) {
  if (!b) return OFDFT_EINVAL;
  for (;;) {
    int na = 0, nq = 0;
    const int rc = ofdft_batch_step(b, &na, &nq);
    if (rc != OFDFT_OK) return rc;
    if (na == 0 && nq == 0) return OFDFT_OK;
  }
}

int ofdft_batch_info(const ofdft_batch* b, ofdft_batch_stats* out) {
  if (!b || !out) return OFDFT_EINVAL;
  memset(out, 0, sizeof(*out));
  out->rounds = b->rounds;
  out->graph_captures = b->graph_captures;
  out->graph_replays = b->graph_replays;
  out->graph_iterations = b->graph_iters;
  out->eager_iterations = b->eager_iters;
  out->z_depth = b->zdepth;
  out->z_tuned = b->ztuned;
  const int n = (int)std::min<size_t>(b->tune_log.size(), 8);
  out->tune_candidates = n;
  for (int i = 0; i < n; ++i) {
    out->tune_depth[i] = b->tune_log[i].first;
    out->tune_us[i] = b->tune_log[i].second;
  }
  return OFDFT_OK;
}

long long ofdft_batch_bytes(const ofdft_grid* g, int prec) {
  if (!g) return -1;
  int mb = 0;
  return slot_bytes(*g, prec, &mb);
}

}  // extern "C"
