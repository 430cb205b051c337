// C ABI of include/ofdft.h for single solves: Poisson CG control, the fused
// functional pass, the secant/Polak-Ribiere nonlinear CG and Algorithm 1 (host
// control of device work), atom kernels' launches, and the entry points.
// All arithmetic on fields runs in the kernels of kernels.cuh.
#include "host.cuh"

namespace ofd {

// Reads (and clears) the flag a z-streaming pass raises when a TMA copy it
// waited for never arrived (its waits are bounded); OFDFT_ETIMEOUT if raised.
int zstream_fault_check(ofdft_ctx* c) {
  if (!c->tma) return OFDFT_OK;
  int v = 0;
  CU(cudaMemcpyFromSymbolAsync(&v, zstream_fault, sizeof(int), 0, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  if (!v) return OFDFT_OK;
  const int zero = 0;
  CU(cudaMemcpyToSymbolAsync(zstream_fault, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return fail(c, OFDFT_ETIMEOUT, "a TMA copy of a z-streaming pass did not arrive (bounded wait ran out)");
}

// ------------------------------------------------------------ Poisson (S3) --
// The r update of one CG iteration with r.r (second kernel of cg_step); the
// iterate update x += alpha p is folded into the next stencil pass (EpiCgAX).
// Without folding (fold == false) the update also applies x += alpha p itself.
template <typename T>
int cg_update(ofdft_ctx* c, const GridDev& g, T* x, T* r, T* pv, T* qv, CgScalars* sc, int pb, bool fold) {
  {
    ProfScope ps_(c, OFDFT_K_CG_UPDATE);
    auto aligned = [](const void* q) { return ((uintptr_t)q & 15u) == 0; };
    const bool wide = g.G % (16 / (long long)sizeof(T)) == 0 && aligned(r) && aligned(qv) && aligned(x) &&
                      aligned(pv);
    const dim3 gr(pb), bl(256);
    const T* cqv = qv;
    if (fold) {
      if (wide)
        CU(launch_k(c, cg_update_r_kernel<T, true>, gr, bl, 0, g.G, r, cqv, sc, red(c)));
      else
        CU(launch_k(c, cg_update_r_kernel<T, false>, gr, bl, 0, g.G, r, cqv, sc, red(c)));
    } else {
      const T* cpv = pv;
      if (wide)
        CU(launch_k(c, cg_update_kernel<T, T, true>, gr, bl, 0, g.G, x, r, cpv, cqv, sc, red(c)));
      else
        CU(launch_k(c, cg_update_kernel<T, T, false>, gr, bl, 0, g.G, x, r, cpv, cqv, sc, red(c)));
    }
  }
  return OFDFT_OK;
}

// Whether a CG solve folds the iterate update into the stencil pass: it saves
// 8 bytes per node and iteration, which pays when the CG vectors stream from
// DRAM; when they stay in the 129 MB L2 the update kernel is bound by its fixed
// costs and the heavier stencil epilogue does not pay (measured at 128^3).  The
// threshold on the five CG vectors' bytes is 96 MiB unless OFDFT_CG_FOLD_BYTES
// set another at context creation.
template <typename T>
bool cg_fold(const ofdft_ctx* c, const GridDev& g) {
  return 5.0 * (double)g.G * sizeof(T) > c->cg_fold_bytes;
}

// The stencil pass of one CG iteration: q = A r + beta q, p = r + beta p, p.q,
// and the previous iteration's x += alpha p when it is pending.
template <typename T>
int cg_stencil(ofdft_ctx* c, int R, const GridDev& g, const Weights<double>& Wneg, T* x, const T* r, T* pv, T* qv,
               CgScalars* sc, bool fold) {
  if (fold)
    return launch_z_r<T>(c, R, g, Wneg, LoadPlain<T>{r}, EpiCgAX<T>{pv, qv, x, sc}, OFDFT_K_CG_DIR_STENCIL);
  return launch_z_r<T>(c, R, g, Wneg, LoadPlain<T>{r}, EpiCgA<T>{pv, qv, sc}, OFDFT_K_CG_DIR_STENCIL);
}

// Applies the last iteration's pending x += alpha p (after the CG loop of a call).
template <typename T>
int cg_flush(ofdft_ctx* c, const GridDev& g, T* x, const T* pv, CgScalars* sc) {
  {
    ProfScope ps_(c, OFDFT_K_VECTOR);
    cg_xflush_kernel<T><<<pointwise_blocks(c, g.G), 256, 0, c->stream>>>(g.G, x, pv, sc);
  }
  {
    ProfScope ps_(c, OFDFT_K_VECTOR);
    cg_xclear_kernel<<<1, 1, 0, c->stream>>>(sc);
  }
  CU(cudaGetLastError());
  return OFDFT_OK;
}

// One V-cycle z = M r of the multigrid preconditioner (plan: mg_plan in host.cuh;
// kernels and the cycle's steps: mg_* in kernels.cuh).

// Whether the CG on this grid runs preconditioned; allocates what the cycle needs.
template <typename T>
int mg_prepare(ofdft_ctx* c, const GridDev& g, double h, MgPlan* P) {
  *P = MgPlan{};
  if (c->precond != OFDFT_PRECOND_MG) return OFDFT_OK;
  *P = mg_plan(g, h, sizeof(T), c->mg_omega);
  if (!P->ok) return OFDFT_OK;
  TRY(ensure(c, c->v[V_Z], g.G * sizeof(T)));
  TRY(ensure(c, c->v[V_T], g.G * sizeof(T)));
  TRY(ensure(c, c->mgbuf, std::max<long long>(P->elems, 1) * sizeof(T)));
  TRY(ensure_partials(c, pointwise_blocks(c, g.G), 1));
  {
    using D = MgPU<T>;
    const long long nb = (long long)((g.n1 + D::FX - 1) / D::FX) * ((g.n2 + D::FY - 1) / D::FY) *
                         ((g.n3 + D::FZ - 1) / D::FZ);
    TRY(ensure_partials(c, nb, 1));
  }
  static bool attr_dev[64] = {false};  // per element type and device (a per-device setting)
  if (c->device < 0 || c->device >= 64) return fail(c, OFDFT_EINVAL, "device index out of range");
  if (!attr_dev[c->device]) {
    CU(cudaFuncSetAttribute(mg_coarse_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    CU(cudaFuncSetAttribute(mg_coarse_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr_dev[c->device] = true;
  }
  static bool cattr_dev[64] = {false};  // the cluster kernel's shared memory, only where it is used
  if (c->mg_cluster && P->lq > 0 && !cattr_dev[c->device]) {
    CU(cudaFuncSetAttribute(mg_cluster_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)kMgClusterSmem));
    cattr_dev[c->device] = true;
  }
  return OFDFT_OK;
}

// The damped-Jacobi sweep of a level as radius-1 stencil weights: centre
// 1 - omega, neighbours omega / 6, rounded in T as the row passes round them.
template <typename T>
inline Weights<double> mg_smoother_weights(double omega) {
  Weights<double> W;
  memset(&W, 0, sizeof(W));
  const T om = (T)omega;
  W.c = (double)(T(1) - om);
  W.w[1] = (double)(om / T(6));
  return W;
}
inline GridDev mg_gdev(const MgLevel& d) {
  GridDev g;
  g.n1 = d.n1;
  g.n2 = d.n2;
  g.n3 = d.n3;
  g.G = (long long)d.n1 * d.n2 * d.n3;
  return g;
}

// Whether level l of the V-cycle runs as the two fused passes.
inline bool mg_level_fused(const ofdft_ctx* c, const MgPlan& P, int l) {
  const long long n = mg_nodes(P.d[l]);
  return (c->mg_fuse_nodes >= 0 && n >= c->mg_fuse_nodes) || (l > 0 && n <= c->mg_fuse_below);
}

// z = M r (one V-cycle); the finest level's last pass also forms r.z and the
// PCG scalars (beta, rz).  Every kernel returns at once when the solve is done.
template <typename T>
int mg_vcycle(ofdft_ctx* c, const MgPlan& P, const T* r, T* z, CgScalars* sc) {
  T* cb = static_cast<T*>(c->mgbuf.p);
  T* t0 = vec<T>(c, V_T);
  auto rl = [&](int l) -> T* { return l == 0 ? const_cast<T*>(r) : cb + P.off[l]; };
  auto zl = [&](int l) -> T* { return l == 0 ? z : cb + P.off[l] + mg_nodes(P.d[l]); };
  auto tl = [&](int l) -> T* { return l == 0 ? t0 : cb + P.off[l] + 2 * mg_nodes(P.d[l]); };
  // the plain passes take a warp per x-row: enough blocks for every row, at most 8 per SM
  auto rows_blocks = [&](const MgLevel& d) {
    return (int)std::max<long long>(1, std::min<long long>(((long long)d.n2 * d.n3 + 7) / 8, (long long)c->sms * 8));
  };
  // levels with at least mg_fuse_nodes nodes, and coarser levels with at most
  // mg_fuse_below nodes (whose launches are latency-bound), take the two fused
  // passes (shared-memory tiles); the others the four plain passes
  auto fused = [&](int l) { return mg_level_fused(c, P, l); };
  const T om = (T)c->mg_omega;
  const Weights<double> Wsm = mg_smoother_weights<T>(c->mg_omega);  // the smoother as stencil weights
  // levels whose smoothing passes run as z-streaming stencils: all with
  // mg_zstream, else those of at least mg_zstream_nodes nodes (-1: none)
  auto zs = [&](int l) {
    return c->mg_zstream || (c->mg_zstream_nodes >= 0 && mg_nodes(P.d[l]) >= c->mg_zstream_nodes);
  };
  // mg_finest_smooth == 0: the finest level is not smoothed (its smoother is
  // the scaled identity s r alone): r_c = R r and z = s r + P e_c.  M stays
  // symmetric positive definite (s > 0, R = P^T / 8, M_c SPD).
  const bool smooth0 = c->mg_finest_smooth != 0;
  // levels lq .. lc-1 and the coarse end on one thread-block cluster
  const bool clus = c->mg_cluster && P.lq > 0;
  const int ltop = clus ? P.lq : P.lc;  // levels above run as separate passes
  for (int l = 0; l < ltop; ++l) {
    if (l == 0 && !smooth0) {
      ProfScope ps_(c, OFDFT_K_MG);
      CU(launch_k(c, mg_restrict_kernel<T>, dim3(rows_blocks(P.d[1])), dim3(256), 0, P.d[0], P.d[1], r, rl(1),
                  (const CgScalars*)sc));
      continue;
    }
    if (fused(l)) {
      using D = MgDR<T>;
      const MgLevel& dc = P.d[l + 1];
      const dim3 gr((dc.n1 + D::CX - 1) / D::CX, (dc.n2 + D::CY - 1) / D::CY, (dc.n3 + D::CZ - 1) / D::CZ);
      ProfScope ps_(c, OFDFT_K_MG);
      CU(launch_k(c, mg_down_restrict_kernel<T>, gr, dim3(256), 0, P.d[l], dc, (const T*)rl(l), rl(l + 1), om,
                  (const CgScalars*)sc));
      continue;
    }
    if (zs(l)) {
      TRY((launch_z<T, 1>(c, mg_gdev(P.d[l]), Wsm, LoadPlain<T>{rl(l)}, EpiMgDown<T>{tl(l), sc}, OFDFT_K_MG)));
    } else {
      ProfScope ps_(c, OFDFT_K_MG);
      CU(launch_k(c, mg_down_kernel<T>, dim3(rows_blocks(P.d[l])), dim3(256), 0, P.d[l], (const T*)rl(l), tl(l),
                  om, (const CgScalars*)sc));
    }
    {
      ProfScope ps_(c, OFDFT_K_MG);
      CU(launch_k(c, mg_restrict_kernel<T>, dim3(rows_blocks(P.d[l + 1])), dim3(256), 0, P.d[l], P.d[l + 1],
                  (const T*)tl(l), rl(l + 1), (const CgScalars*)sc));
    }
  }
  double s = P.s0;
  for (int l = 0; l < P.lc; ++l) s *= 4.0;
  if (clus) {
    MgClusterArgs<T> A;
    double sl = P.s0;
    for (int l = 0; l <= P.lc; ++l, sl *= 4.0) {
      if (l >= P.lq) {
        A.L[l] = P.slab[l];
        A.s[l] = (T)sl;
      }
    }
    A.lq = P.lq;
    A.lc = P.lc;
    A.ncoarse = P.nlev - P.lc;
    A.r_in = rl(P.lq);
    A.z_out = zl(P.lq);
    A.r_tail = rl(P.lc);
    A.z_tail = zl(P.lc);
    A.tail_off = P.tail_off;
    A.omega = om;
    A.sweeps = c->mg_sweeps;
    ProfScope ps_(c, OFDFT_K_MG);
    CU(launch_k(c, mg_cluster_kernel<T>, dim3(kMgClusterCtas), dim3(1024), P.csmem, A, sc));
    for (int l = P.lc - 1; l >= P.lq; --l) s *= 0.25;
  }
  if (!clus) {
    ProfScope ps_(c, OFDFT_K_MG);
    const int nl = P.nlev - P.lc;
    if (P.lc == 0)
      CU(launch_k(c, mg_coarse_kernel<T, true>, dim3(1), dim3(1024), P.smem, P.d[P.lc], nl, (const T*)rl(P.lc),
                  zl(P.lc), om, (T)s, c->mg_sweeps, sc));
    else
      CU(launch_k(c, mg_coarse_kernel<T, false>, dim3(1), dim3(1024), P.smem, P.d[P.lc], nl, (const T*)rl(P.lc),
                  zl(P.lc), om, (T)s, c->mg_sweeps, sc));
  }
  for (int l = ltop - 1; l >= 0; --l) {
    s *= 0.25;
    if (l == 0 && !smooth0) {
      ProfScope ps_(c, OFDFT_K_MG);
      CU(launch_k(c, mg_prolong_kernel<T, true>, dim3(pointwise_blocks(c, mg_nodes(P.d[0]))), dim3(256), 0, P.d[0],
                  P.d[1], r, (const T*)zl(1), z, (T)s, sc, red(c)));
      continue;
    }
    if (fused(l)) {
      using D = MgPU<T>;
      const MgLevel& df = P.d[l];
      const dim3 gr((df.n1 + D::FX - 1) / D::FX, (df.n2 + D::FY - 1) / D::FY, (df.n3 + D::FZ - 1) / D::FZ);
      ProfScope ps_(c, OFDFT_K_MG);
      if (l == 0)
        CU(launch_k(c, mg_prolong_up_kernel<T, true>, gr, dim3(256), 0, df, P.d[1], (const T*)r, (const T*)zl(1), z,
                    om, (T)s, sc, red(c)));
      else
        CU(launch_k(c, mg_prolong_up_kernel<T, false>, gr, dim3(256), 0, df, P.d[l + 1], (const T*)rl(l),
                    (const T*)zl(l + 1), zl(l), om, (T)s, sc, red(c)));
      continue;
    }
    {
      ProfScope ps_(c, OFDFT_K_MG);
      CU(launch_k(c, mg_prolong_kernel<T, false>, dim3(rows_blocks(P.d[l])), dim3(256), 0, P.d[l], P.d[l + 1],
                  (const T*)rl(l), (const T*)zl(l + 1), tl(l), (T)s, sc, RedBuf{}));
    }
    if (zs(l)) {
      if (l == 0)
        TRY((launch_z<T, 1>(c, mg_gdev(P.d[0]), Wsm, LoadPlain<T>{t0}, EpiMgUp<T, true>{r, z, (T)s, sc}, OFDFT_K_MG)));
      else
        TRY((launch_z<T, 1>(c, mg_gdev(P.d[l]), Wsm, LoadPlain<T>{tl(l)}, EpiMgUp<T, false>{rl(l), zl(l), (T)s, sc},
                            OFDFT_K_MG)));
      continue;
    }
    ProfScope ps_(c, OFDFT_K_MG);
    if (l == 0)
      CU(launch_k(c, mg_up_kernel<T, true>, dim3(pointwise_blocks(c, mg_nodes(P.d[0]))), dim3(256), 0, P.d[0],
                  (const T*)r, (const T*)t0, z, om, (T)s, sc, red(c)));
    else
      CU(launch_k(c, mg_up_kernel<T, false>, dim3(rows_blocks(P.d[l])), dim3(256), 0, P.d[l], (const T*)rl(l),
                  (const T*)tl(l), zl(l), om, (T)s, sc, red(c)));
  }
  return OFDFT_OK;
}

// V-cycle launches per CG iteration.
inline int mg_launches(const ofdft_ctx* c, const MgPlan& P) {
  if (!P.ok) return 0;
  int n = 1;
  const int ltop = (c->mg_cluster && P.lq > 0) ? P.lq : P.lc;
  for (int l = 0; l < ltop; ++l) n += (l == 0 && !c->mg_finest_smooth) ? 2 : mg_level_fused(c, P, l) ? 2 : 4;
  return n;
}

// Launches one CG iteration (S3): the stencil pass on r with the p/q update and
// p.q (and the previous x update), then the r update with r.r; both kernels
// read and write the CG scalars on the device and return at once when the
// solve is done.
template <typename T, typename X>
int cg_step(ofdft_ctx* c, int R, const GridDev& g, const Weights<double>& Wneg, X* x, T* r, T* pv, T* qv,
            CgScalars* sc, int pb, const MgPlan* mg = nullptr) {
  static_assert(sizeof(X) == sizeof(T), "the iterate has the CG vectors' type");
  const bool fold = cg_fold<T>(c, g);
  const T* dir = r;  // the stencil pass forms p and q from r, or from z = M r (PCG)
  if (mg && mg->ok) {
    T* z = vec<T>(c, V_Z);
    TRY(mg_vcycle<T>(c, *mg, r, z, sc));
    dir = z;
  }
  TRY(cg_stencil<T>(c, R, g, Wneg, reinterpret_cast<T*>(x), dir, pv, qv, sc, fold));
  return cg_update<T>(c, g, reinterpret_cast<T*>(x), r, pv, qv, sc, pb, fold);
}

constexpr int kChunk = 8;  // CG iterations between convergence polls

// Autotuner (S11): picks the number of z chunks of the CG stencil pass for one
// (kernel, grid) by timing candidate splits on scratch vectors (a private CG
// scalar block keeps the solve's state untouched) and caches the choice in the
// context.  The split changes the blocks' partial sums, so it is fixed before
// the solve's first CG pass and the reduction order stays the same afterwards.
template <typename T>
int tune_cg_split(ofdft_ctx* c, int R, const GridDev& g, const Weights<double>& Wneg, const T* r, T* x) {
  if (!c->autotune) return OFDFT_OK;
  T *pv = nullptr, *qv = nullptr;  // scratch p and q (separate allocations, aligned like the solver's)
  const bool fold = cg_fold<T>(c, g);
  const long long vec16 = zvec_ok<T>(g, LoadPlain<T>{r}, EpiCgAX<T>{vec<T>(c, V_P0), vec<T>(c, V_AP), x, nullptr});
  const std::vector<long long> tkey = {(long long)sizeof(T), R, g.n1, g.n2, g.n3, vec16, fold ? 1 : 0};
  for (auto& t : c->ztuned)
    if (t == tkey) return OFDFT_OK;
  const std::vector<int> cand = {0, 1, 2, 3, 4, 5, 6, 7, 8, 10, 12, 14, 16, 20, 24, 32, 48, 64};
  TRY(ensure_partials(c, zshape<T>(c, g, R, 1, 64).nblocks, 1));  // largest candidate
  CU(cudaMalloc(&pv, g.G * sizeof(T)));
  if (cudaMalloc(&qv, g.G * sizeof(T)) != cudaSuccess) {
    cudaFree(pv);
    return fail(c, OFDFT_ENOMEM, "autotune: no room for scratch vectors");
  }
  CgScalars* sc = c->sc + 2;
  CgScalars init;
  memset(&init, 0, sizeof(init));
  init.first = 1;
  init.max_it = 1 << 30;
  const int prof = c->prof;
  const long long launches = c->launches;
  long long kinds[OFDFT_K_COUNT];
  memcpy(kinds, c->kind_launches, sizeof(kinds));
  c->prof = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int best = 0, rc = OFDFT_OK;
  float best_ms = 1e30f;
  std::vector<long long> key;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    rc = fail(c, OFDFT_ECUDA, "autotune: event creation failed");
  for (int nz : cand) {
    if (rc != OFDFT_OK || nz > g.n3) break;
    c->force_nz = nz;
    float ms = 0.0f;
    for (int rep = 0; rep < 4 && rc == OFDFT_OK; ++rep) {
      if (cudaMemcpyAsync(sc, &init, sizeof(init), cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
          cudaEventRecord(e0, c->stream) != cudaSuccess) {
        rc = fail(c, OFDFT_ECUDA, "autotune: enqueue failed");
        break;
      }
      rc = cg_stencil<T>(c, R, g, Wneg, x, r, pv, qv, sc, fold);
      key = c->last_zkey;
      float t = 0.0f;
      if (rc == OFDFT_OK && (cudaEventRecord(e1, c->stream) != cudaSuccess ||
                             cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
        rc = fail(c, OFDFT_ECUDA, "autotune: timing failed");
      if (rep > 0) ms += t;  // the first launch of each split warms up
    }
    if (ms < best_ms) {
      best_ms = ms;
      best = nz;
    }
  }
  c->force_nz = -1;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(c->stream);
  cudaFree(pv);
  cudaFree(qv);
  c->prof = prof;
  c->launches = launches;  // tuning launches are not part of the caller's work
  memcpy(c->kind_launches, kinds, sizeof(kinds));
  if (rc != OFDFT_OK) return rc;
  c->ztune.push_back({key, best});
  c->ztuned.push_back(tkey);
  return OFDFT_OK;
}

// The graph of one chunk of CG iterations for this buffer set, captured on
// first use (the launches bake in pointers, sizes and weights).
// With sample_set = 0 or 1 the graph also records the context's timing events
// gev[sample_set] around the stencil pass of its middle iteration, so that a
// timed run keeps its graphs and times one stencil launch in kChunk.
template <typename T, typename X>
int cg_graph(ofdft_ctx* c, int R, const GridDev& g, double h, const Weights<double>& Wneg, X* x, T* r, T* pv, T* qv,
             CgScalars* sc, int pb, int sample_set, cudaGraphExec_t* out, const MgPlan* mg) {
  const bool pcg = mg && mg->ok;
  const std::vector<long long> key = {(long long)sizeof(T), (long long)sizeof(X), R, g.n1, g.n2, g.n3, (long long)x,
                                      (long long)r,
                                      (long long)pv, (long long)qv, (long long)sc, pb,
                                      (long long)c->partials.p, (long long)(h * 1e12), sample_set, pcg ? 1 : 0,
                                      pcg ? (long long)c->mgbuf.p : 0, pcg ? (long long)c->v[V_Z].p : 0,
                                      pcg ? (long long)c->v[V_T].p : 0};
  if (sample_set >= 0 && !c->gev[sample_set][0]) {
    CU(cudaEventCreate(&c->gev[sample_set][0]));
    CU(cudaEventCreate(&c->gev[sample_set][1]));
  }
  for (auto& e : c->graphs)
    if (e.key == key) {
      *out = e.exec;
      return OFDFT_OK;
    }
  // the launches must not allocate or time themselves while being captured
  const int prof = c->prof;
  c->prof = 0;
  const long long launches = c->launches;
  long long kinds[OFDFT_K_COUNT];
  memcpy(kinds, c->kind_launches, sizeof(kinds));
  TRY((cg_step<T, X>(c, R, g, Wneg, x, r, pv, qv, sc, pb, mg)));  // sets kernel attributes outside capture
  CU(cudaStreamSynchronize(c->stream));
  // capture on the context's private stream (the caller's stream may be the
  // legacy default stream, which cannot be captured); replay on the caller's
  cudaGraph_t graph = nullptr;
  cudaStream_t user = c->stream;
  c->stream = c->gstream;
  cudaError_t eb = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
  int rc = OFDFT_OK;
  if (eb == cudaSuccess)
    for (int i = 0; i < kChunk && rc == OFDFT_OK; ++i) {
      if (sample_set >= 0 && i == kChunk / 2) {
        const T* dir = r;
        if (pcg) {
          rc = mg_vcycle<T>(c, *mg, r, vec<T>(c, V_Z), sc);
          dir = vec<T>(c, V_Z);
        }
        cudaEventRecordWithFlags(c->gev[sample_set][0], c->stream, cudaEventRecordExternal);
        const bool fold = cg_fold<T>(c, g);
        if (rc == OFDFT_OK) rc = cg_stencil<T>(c, R, g, Wneg, reinterpret_cast<T*>(x), dir, pv, qv, sc, fold);
        cudaEventRecordWithFlags(c->gev[sample_set][1], c->stream, cudaEventRecordExternal);
        if (rc == OFDFT_OK) rc = cg_update<T>(c, g, reinterpret_cast<T*>(x), r, pv, qv, sc, pb, fold);
      } else {
        rc = cg_step<T, X>(c, R, g, Wneg, x, r, pv, qv, sc, pb, mg);
      }
    }
  const cudaError_t ec = (eb == cudaSuccess) ? cudaStreamEndCapture(c->stream, &graph) : eb;
  c->stream = user;
  c->prof = prof;
  c->launches = launches;
  memcpy(c->kind_launches, kinds, sizeof(kinds));
  if (rc != OFDFT_OK) return rc;
  if (ec != cudaSuccess) return fail(c, OFDFT_ECUDA, "CG graph capture: %s", cudaGetErrorString(ec));
  cudaGraphExec_t exec = nullptr;
  CU(cudaGraphInstantiate(&exec, graph, 0));
  cudaGraphDestroy(graph);
  c->graphs.push_back({key, exec});
  *out = exec;
  return OFDFT_OK;
}

// The whole CG loop of a solve as one CUDA graph: a WHILE node whose body is
// one iteration (V-cycle, stencil pass, update) followed by cg_cond_kernel, so
// the device iterates until the solve's own `done` flag rises, with no host
// polling and no launches past convergence.  A kernel ahead of the node sets
// the condition from `done` at entry.  Captured once per buffer set (the
// launches bake in pointers, sizes and weights).
template <typename T, typename X>
int cg_while_graph(ofdft_ctx* c, int R, const GridDev& g, double h, const Weights<double>& Wneg, X* x, T* r, T* pv,
                   T* qv, CgScalars* sc, int pb, cudaGraphExec_t* out, const MgPlan* mg) {
  const bool pcg = mg && mg->ok;
  const std::vector<long long> key = {-1, (long long)sizeof(T), (long long)sizeof(X), R, g.n1, g.n2, g.n3,
                                      (long long)x, (long long)r, (long long)pv, (long long)qv, (long long)sc, pb,
                                      (long long)c->partials.p, (long long)(h * 1e12), pcg ? 1 : 0,
                                      pcg ? (long long)c->mgbuf.p : 0, pcg ? (long long)c->v[V_Z].p : 0,
                                      pcg ? (long long)c->v[V_T].p : 0};
  for (auto& e : c->graphs)
    if (e.key == key) {
      *out = e.exec;
      return OFDFT_OK;
    }
  cudaGraph_t graph = nullptr;
  CU(cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle handle;
  int rc = OFDFT_OK;
  cudaError_t e = cudaGraphConditionalHandleCreate(&handle, graph, 0, cudaGraphCondAssignDefault);
  cudaGraphNode_t init = nullptr, loop = nullptr;
  if (e == cudaSuccess) {
    cudaKernelNodeParams kp = {};
    const CgScalars* csc = sc;
    void* args[] = {&handle, &csc};
    kp.func = (void*)cg_cond_kernel;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(1);
    kp.kernelParams = args;
    e = cudaGraphAddKernelNode(&init, graph, nullptr, 0, &kp);
  }
  cudaGraphNodeParams cp = {};
  if (e == cudaSuccess) {
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    e = cudaGraphAddNode(&loop, graph, &init, nullptr, 1, &cp);
  }
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return fail(c, OFDFT_ECUDA, "CG loop graph: %s", cudaGetErrorString(e));
  }
  // the body: one iteration and the condition update, captured on the private stream
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  const int prof = c->prof;
  c->prof = 0;
  const long long launches = c->launches;
  long long kinds[OFDFT_K_COUNT];
  memcpy(kinds, c->kind_launches, sizeof(kinds));
  cudaStream_t user = c->stream;
  c->stream = c->gstream;
  e = cudaStreamBeginCaptureToGraph(c->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    rc = cg_step<T, X>(c, R, g, Wneg, x, r, pv, qv, sc, pb, mg);
    if (rc == OFDFT_OK) {
      cg_cond_kernel<<<1, 1, 0, c->stream>>>(handle, sc);
      if (cudaGetLastError() != cudaSuccess) rc = fail(c, OFDFT_ECUDA, "CG loop graph: condition launch failed");
    }
    cudaGraph_t got = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(c->stream, &got);
    if (rc == OFDFT_OK && ee != cudaSuccess) e = ee;
  }
  c->stream = user;
  c->prof = prof;
  c->launches = launches;
  memcpy(c->kind_launches, kinds, sizeof(kinds));
  cudaGraphExec_t exec = nullptr;
  if (rc == OFDFT_OK && e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (rc != OFDFT_OK) return rc;
  if (e != cudaSuccess) return fail(c, OFDFT_ECUDA, "CG loop graph: %s", cudaGetErrorString(e));
  c->graphs.push_back({key, exec});
  *out = exec;
  return OFDFT_OK;
}

// Persistent CG: one cooperative launch of cg_coop_kernel runs up to kChunk
// iterations (both halves of each, with grid-wide sums between them), so an
// iteration costs no launch gaps and no separate update kernel.  Needs 16-byte
// staging (the kernel's loads bypass L1: other blocks write r within the launch)
// and a grid whose blocks are all co-resident; *used = false otherwise, and the
// caller runs the two-kernel iteration.
template <typename T, int R>
int cg_coop_r(ofdft_ctx* c, const GridDev& g, const Weights<double>& Wneg, T* x, T* r, T* pv, T* qv, CgScalars* sc,
              int max_it, CgScalars* host_sc, bool* used) {
  constexpr int VW = 16 / (int)sizeof(T);
  *used = false;
  // grids whose CG vectors overflow L2 run faster as two kernels with the
  // folded iterate update (at 256^3: 160 against 250 us per iteration)
  if (cg_fold<T>(c, g)) return OFDFT_OK;
  if (!zvec_ok<T>(g, LoadPlain<T>{r}, EpiCgAv<T>{pv, qv, 0, T(0)})) return OFDFT_OK;
  auto* kern = cg_coop_kernel<T, R, VW>;
  constexpr int smem = zsmem_bytes<T, R, VW, EpiCgAv<T>>();
  // co-resident blocks per SM of this instantiation, per device (the shared-memory
  // attribute is a per-device setting; -1: not yet queried on that device)
  static int per_sm_dev[64] = {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1,
                               -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1,
                               -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1,
                               -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1};
  if (c->device < 0 || c->device >= 64) return OFDFT_OK;
  int& per_sm = per_sm_dev[c->device];
  if (per_sm < 0) {
    CU(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int nb = 0;
    CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, NT, smem));
    per_sm = std::max(nb, 0);
  }
  const long long maxb = (long long)per_sm * c->sms;
  const int gx = (g.n1 + BX - 1) / BX, gy = (g.n2 + ZCfg<T>::TY - 1) / ZCfg<T>::TY;
  const long long tiles = (long long)gx * gy;
  if (maxb < 1 || tiles > maxb) return OFDFT_OK;
  // z-split: as many chunks as co-resident blocks allow (at 128^3, FP32: 4 x 4
  // tiles x 19 chunks of 7 planes, 304 blocks, 2 per SM), at least 2 planes each
  int nz = (int)std::min<long long>(maxb / tiles, std::max(1, g.n3 / 2));
  if (c->coop_nz > 0) nz = (int)std::min<long long>(maxb / tiles, c->coop_nz);
  nz = std::max(nz, 1);
  const int zc = (g.n3 + nz - 1) / nz;
  nz = (g.n3 + zc - 1) / zc;
  const int nblocks = (int)(tiles * nz);
  TRY(ensure_partials(c, 2LL * nblocks, 1));
  if (!c->coop_bar) CU(cudaMalloc(&c->coop_bar, 256));
  CU(cudaMemsetAsync(c->coop_bar, 0, sizeof(unsigned int), c->stream));
  *used = true;
  GridDev gg = g;
  Weights<T> W = cast_weights<T>(Wneg);
  int zchunk = zc;
  double* partials = static_cast<double*>(c->partials.p);
  unsigned int* bar = c->coop_bar;
  const dim3 grid(gx, gy, nz), block(BX, BY);
  int launched = 0, chunks = 0;
  while (launched < max_it) {
    int niter = std::min(kChunk, max_it - launched);
    void* args[] = {&gg, &W, &zchunk, &x, &r, &pv, &qv, &sc, &partials, &bar, &niter};
    {
      ProfScope ps_(c, OFDFT_K_CG_PERSISTENT);
      CU(cudaLaunchCooperativeKernel((const void*)kern, grid, block, args, smem, c->stream));
    }
    launched += niter;
    const int slot = chunks & 1;
    CU(cudaMemcpyAsync(&c->ring[slot], sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaEventRecord(c->ring_ev[slot], c->stream));
    if (chunks > 0) {
      CU(cudaEventSynchronize(c->ring_ev[slot ^ 1]));
      if (c->ring[slot ^ 1].err) return fail(c, OFDFT_ETIMEOUT, "persistent CG: a grid barrier timed out");
      if (c->ring[slot ^ 1].done) break;
    }
    ++chunks;
  }
  const int it0 = host_sc->iters;
  TRY(sync_scalars(c, sc, sizeof(CgScalars), host_sc));
  if (host_sc->err) return fail(c, OFDFT_ETIMEOUT, "persistent CG: a grid barrier timed out");
  c->coop_iters += host_sc->iters - it0;
  return OFDFT_OK;
}

template <typename T>
int cg_coop(ofdft_ctx* c, int R, const GridDev& g, const Weights<double>& Wneg, T* x, T* r, T* pv, T* qv,
            CgScalars* sc, int max_it, CgScalars* host_sc, bool* used) {
  switch (R) {
    case 1: return cg_coop_r<T, 1>(c, g, Wneg, x, r, pv, qv, sc, max_it, host_sc, used);
    case 2: return cg_coop_r<T, 2>(c, g, Wneg, x, r, pv, qv, sc, max_it, host_sc, used);
    case 3: return cg_coop_r<T, 3>(c, g, Wneg, x, r, pv, qv, sc, max_it, host_sc, used);
    case 4: return cg_coop_r<T, 4>(c, g, Wneg, x, r, pv, qv, sc, max_it, host_sc, used);
    case 5: return cg_coop_r<T, 5>(c, g, Wneg, x, r, pv, qv, sc, max_it, host_sc, used);
    default: return cg_coop_r<T, 6>(c, g, Wneg, x, r, pv, qv, sc, max_it, host_sc, used);
  }
}

// Plain CG iterations on the prepared scalars `sc` (residual r, iterate x),
// checking the device `done` flag every kChunk iterations.  Chunk k+1 is
// enqueued before the host waits for chunk k's copy of the scalars, so the
// stream never drains; kernels of a converged solve return at once, so an extra
// chunk costs only empty launches.  A chunk is one CUDA graph launch unless the
// CG update is being timed (then every launch is bracketed by events); when
// only the stencil pass is timed, the graphs of alternate chunks carry the two
// sets of sampling events and the host reads chunk k's set while chunk k+1 runs.
template <typename T, typename X = T>
int cg_iterate(ofdft_ctx* c, int R, const GridDev& g, double h, const Weights<double>& Wneg, X* x, T* r,
               CgScalars* sc, int max_it, CgScalars* host_sc) {
  T* pv = vec<T>(c, V_P0);
  T* qv = vec<T>(c, V_AP);
  const bool per_launch = (c->prof & (1 << OFDFT_K_CG_UPDATE)) != 0;  // per-kernel timing asked for
  MgPlan mg;
  TRY(mg_prepare<T>(c, g, h, &mg));
  if (c->coop && !per_launch && !mg.ok) {
    bool used = false;
    TRY(cg_coop<T>(c, R, g, Wneg, reinterpret_cast<T*>(x), r, pv, qv, sc, max_it, host_sc, &used));
    if (used) return OFDFT_OK;
  }
  const int pb = pointwise_blocks(c, g.G);
  TRY(ensure_partials(c, pb, 1));
  TRY(ensure_partials(c, zshape<T>(c, g, R, 32).nblocks, 1));
  TRY(tune_cg_split<T>(c, R, g, Wneg, r, reinterpret_cast<T*>(x)));
  const bool full_timed = (c->prof & (1 << OFDFT_K_CG_UPDATE)) != 0;
  const bool sampled = !full_timed && (c->prof & (1 << OFDFT_K_CG_DIR_STENCIL)) != 0;
  const int nmg = mg_launches(c, mg);  // V-cycle launches per iteration
  if (c->use_graphs && c->cond_graphs && !full_timed && !sampled && max_it > 0) {
    // the whole loop on the device: one eager iteration (it also sets every kernel
    // attribute outside the capture), then the WHILE graph for the rest
    const int it0 = host_sc->iters;
    TRY((cg_step<T, X>(c, R, g, Wneg, x, r, pv, qv, sc, pb, &mg)));
    cudaGraphExec_t wexec = nullptr;
    TRY((cg_while_graph<T, X>(c, R, g, h, Wneg, x, r, pv, qv, sc, pb, &wexec, &mg)));
    CU(cudaGraphLaunch(wexec, c->stream));
    if (cg_fold<T>(c, g)) TRY(cg_flush<T>(c, g, reinterpret_cast<T*>(x), pv, sc));
    TRY(sync_scalars(c, sc, sizeof(CgScalars), host_sc));
    const long long its = std::max(0, host_sc->iters - it0 - 1);  // iterations the graph ran
    c->launches += (2 + nmg + 1) * its + 1;
    c->kind_launches[OFDFT_K_CG_DIR_STENCIL] += its;
    c->kind_launches[OFDFT_K_CG_UPDATE] += its;
    c->kind_launches[OFDFT_K_MG] += nmg * its;
    c->kind_launches[OFDFT_K_VECTOR] += its + 1;
    return OFDFT_OK;
  }
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  if (c->use_graphs && !full_timed && max_it >= kChunk) {
    TRY((cg_graph<T, X>(c, R, g, h, Wneg, x, r, pv, qv, sc, pb, sampled ? 0 : -1, &exec[0], &mg)));
    exec[1] = exec[0];
    if (sampled) TRY((cg_graph<T, X>(c, R, g, h, Wneg, x, r, pv, qv, sc, pb, 1, &exec[1], &mg)));
  }
  bool pending[2] = {false, false};
  auto read_sample = [&](int set) {
    float ms = 0.0f;
    if (pending[set] && cudaEventElapsedTime(&ms, c->gev[set][0], c->gev[set][1]) == cudaSuccess) {
      c->timed_ms[OFDFT_K_CG_DIR_STENCIL] += ms;
      c->timed_launches[OFDFT_K_CG_DIR_STENCIL] += 1;
    }
    pending[set] = false;
  };
  int launched = 0, chunks = 0;
  while (launched < max_it) {
    const int slot = chunks & 1;
    if (exec[0] && launched + kChunk <= max_it) {
      CU(cudaGraphLaunch(exec[slot], c->stream));
      pending[slot] = sampled;
      launched += kChunk;
      c->launches += (2 + nmg) * kChunk;
      c->kind_launches[OFDFT_K_CG_DIR_STENCIL] += kChunk;
      c->kind_launches[OFDFT_K_CG_UPDATE] += kChunk;
      c->kind_launches[OFDFT_K_MG] += nmg * kChunk;
    } else {
      for (int i = 0; i < kChunk && launched < max_it; ++i, ++launched)
        TRY((cg_step<T, X>(c, R, g, Wneg, x, r, pv, qv, sc, pb, &mg)));
    }
    CU(cudaMemcpyAsync(&c->ring[slot], sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaEventRecord(c->ring_ev[slot], c->stream));
    if (chunks > 0) {
      CU(cudaEventSynchronize(c->ring_ev[slot ^ 1]));
      read_sample(slot ^ 1);  // chunk k-1 has finished; chunk k+1 will reuse its events
      if (c->ring[slot ^ 1].done) break;
    }
    ++chunks;
  }
  if (cg_fold<T>(c, g)) TRY(cg_flush<T>(c, g, reinterpret_cast<T*>(x), pv, sc));
  TRY(sync_scalars(c, sc, sizeof(CgScalars), host_sc));
  read_sample(0);
  read_sample(1);
  return OFDFT_OK;
}

// Workspace sizes for a solve (vectors of the prec type, plus FP64 mixed extras).
int ensure_cg_vectors(ofdft_ctx* c, long long G, size_t es, bool mixed) {
  TRY(ensure(c, c->v[V_R], G * es));
  TRY(ensure(c, c->v[V_P0], G * es));
  TRY(ensure(c, c->v[V_P1], G * es));
  TRY(ensure(c, c->v[V_AP], G * es));
  if (mixed) {
    TRY(ensure(c, c->v[V_R64], G * sizeof(double)));
    TRY(ensure(c, c->v[V_E32], G * sizeof(float)));
  }
  return OFDFT_OK;
}

// FP64 Poisson solve: r = 4 pi rho + L phi, then CG.  rho = rho_in or u^2 + b.
// On return r (V_R) holds the final recursive residual; st gets the stats.
int poisson_fp64(ofdft_ctx* c, int R, const GridDev& g, double h, const double* rho, const double* u,
                 const double* b, double* phi, double tol, int max_it, ofdft_cg_stats* st) {
  TRY(ensure_cg_vectors(c, g.G, sizeof(double), false));
  const Weights<double> W = lap_weights(R, h, 1.0), Wneg = lap_weights(R, h, -1.0);
  double* r = vec<double>(c, V_R);
  MgPlan mg;
  TRY(mg_prepare<double>(c, g, h, &mg));
  TRY(launch_z_r<double>(c, R, g, W, LoadPlain<double>{phi},
                         EpiResidual<double>{rho, u, b, r, c->sc, tol, max_it, 1, mg.ok ? 1 : 0}, OFDFT_K_RESIDUAL));
  CgScalars hs;
  TRY(sync_scalars(c, c->sc, sizeof(CgScalars), &hs));
  if (!hs.done) TRY(cg_iterate<double>(c, R, g, h, Wneg, phi, r, c->sc, max_it, &hs));
  if (st) {
    st->iterations = hs.iters;
    st->rel_residual = sqrt(hs.rr / (hs.bb > 0 ? hs.bb : 1.0));
  }
  if (!isfinite(hs.rr)) return fail(c, OFDFT_ENONFINITE, "Poisson residual is not finite");
  if (hs.rr > tol * tol * (hs.bb > 0 ? hs.bb : 1.0))
    return fail(c, OFDFT_ENOTCONV, "Poisson CG reached %d iterations at relative residual %.3e", hs.iters,
                sqrt(hs.rr / (hs.bb > 0 ? hs.bb : 1.0)));
  return OFDFT_OK;
}

// Mixed Poisson solve (S3 + S10): FP32 CG with residual replacement.  The
// potential phi64 stays FP64; r, p, q = A p and the correction e of the current
// round are FP32.  Each round folds e into phi64 and computes the FP64 true
// residual r64 = 4 pi (u^2 + b64) + L_h phi64 with the FP64 stencil; the solve
// ends when it meets tol.  Otherwise r64 replaces the FP32 residual (plain CG
// keeps the search direction after the first round, so no Krylov information is
// lost; preconditioned CG restarts from p = z) and FP32 iterations run until the FP32 residual falls by mixed_inner_tol (1e-4,
// or less when the FP64 test needs less) or refine_every steps.  At the end
// phi32 = (float) phi64.  rho32 (optional) replaces u^2 + b.  b2_valid
// (optional): the caller's flag that V_B2 already holds b64 as float-float
// pairs (the pseudocharge is fixed for a whole ground state, so a solve splits
// it once); set here after a split.
int poisson_mixed(ofdft_ctx* c, int R, const GridDev& g, double h, const float* rho32, const float* u,
                  const double* b64, double* phi64, float* phi32, double tol, int max_it, int refine_every,
                  ofdft_cg_stats* st, int* b2_valid = nullptr) {
  TRY(ensure_cg_vectors(c, g.G, sizeof(float), true));
  const Weights<double> W = lap_weights(R, h, 1.0), Wneg = lap_weights(R, h, -1.0);
  double* r64 = vec<double>(c, V_R64);
  float* r32 = vec<float>(c, V_R);
  float* e32 = vec<float>(c, V_E32);
  const int pb = pointwise_blocks(c, g.G);
  MgPlan mg;
  TRY(mg_prepare<float>(c, g, h, &mg));
  int total = 0, rc = OFDFT_OK;
  CgScalars hs, hs32;
  const int max_rounds = 60;
  CU(cudaMemsetAsync(e32, 0, g.G * sizeof(float), c->stream));
  // float-float residual pass: the potential and the pseudocharge as float-float
  // pairs (phi2, b2), split once here and phi2 kept in step by every fold; the
  // residual itself is written as pairs (r2, in the r64 buffer)
  float2 *phi2 = nullptr, *b2 = nullptr;
  float2* r2 = reinterpret_cast<float2*>(r64);
  c->mixed_ff = c->ff_residual != 0;
  if (c->mixed_ff) {
    TRY(ensure(c, c->v[V_PHI2], g.G * sizeof(float2)));
    phi2 = vec<float2>(c, V_PHI2);
    if (!rho32) {
      TRY(ensure(c, c->v[V_B2], g.G * sizeof(float2)));
      b2 = vec<float2>(c, V_B2);
    }
    const bool split_b = b2 && !(b2_valid && *b2_valid);
    {
      ProfScope ps_(c, OFDFT_K_VECTOR);
      ff_split_kernel<<<pb, 256, 0, c->stream>>>(g.G, phi2, phi64, split_b ? b2 : nullptr, b64);
    }
    CU(cudaGetLastError());
    if (split_b && b2_valid) *b2_valid = 1;
  }
  const float2 fourpi = ff_of(4.0 * kPi);
  for (int round = 0; round <= max_rounds; ++round) {
    if (round > 0) {
      ProfScope ps_(c, OFDFT_K_VECTOR);
      fold_kernel<<<pb, 256, 0, c->stream>>>(g.G, phi64, e32, phi2);
    }
    if (c->mixed_ff) {
      const EpiResidualFF ep{rho32, rho32 ? nullptr : u, b2, r2, c->sc, tol, max_it, 0, fourpi};
      TRY(launch_z_r<float2>(c, R, g, W, LoadPlain<float2>{phi2}, ep, OFDFT_K_RESIDUAL));
    } else {
      const EpiResidual<double, float, double> ep =
          rho32 ? EpiResidual<double, float, double>{rho32, nullptr, nullptr, r64, c->sc, tol, max_it, 1}
                : EpiResidual<double, float, double>{nullptr, u, b64, r64, c->sc, tol, max_it, 1};
      TRY(launch_z_r<double>(c, R, g, W, LoadPlain<double>{phi64}, ep, OFDFT_K_RESIDUAL));
    }
    TRY(sync_scalars(c, c->sc, sizeof(CgScalars), &hs));
    const double bb = hs.bb > 0 ? hs.bb : 1.0;
    if (st) {
      st->iterations = total;
      st->rel_residual = sqrt(hs.rr / bb);
    }
    if (!isfinite(hs.rr)) return fail(c, OFDFT_ENONFINITE, "Poisson residual is not finite");
    if (hs.rr <= tol * tol * bb) break;
    if (total >= max_it || round == max_rounds) {
      rc = fail(c, OFDFT_ENOTCONV, "mixed Poisson reached %d FP32 iterations at relative residual %.3e", total,
                sqrt(hs.rr / bb));
      break;
    }
    const int budget = std::min(refine_every, max_it - total);
    TRY(ensure_partials(c, pb, 1));
    {
      ProfScope ps_(c, OFDFT_K_VECTOR);
      // later rounds keep the search direction (plain CG); preconditioned CG
      // restarts from p = z: the replaced residual is not orthogonal to the old
      // directions, and keeping them let the FP32 PCG diverge on some states
      if (c->mixed_ff)
        refine_replace_kernel<float2><<<pb, 256, 0, c->stream>>>(g.G, r32, r2, c->sc32,
                                                                 mixed_inner_tol(hs.rr, bb, tol), budget,
                                                                 (round == 0 || mg.ok) ? 1 : 0, mg.ok ? 1 : 0, red(c));
      else
        refine_replace_kernel<double><<<pb, 256, 0, c->stream>>>(g.G, r32, r64, c->sc32,
                                                                 mixed_inner_tol(hs.rr, bb, tol), budget,
                                                                 (round == 0 || mg.ok) ? 1 : 0, mg.ok ? 1 : 0, red(c));
    }
    CU(cudaGetLastError());
    TRY(sync_scalars(c, c->sc32, sizeof(CgScalars), &hs32));
    const int before = hs32.iters;
    if (!hs32.done) TRY((cg_iterate<float, float>(c, R, g, h, Wneg, e32, r32, c->sc32, budget, &hs32)));
    if (c->trace)
      fprintf(stderr, "[ofdft] mixed round %d rel64=%.3e its=%d rr32=%.3e rz=%.3e pAp=%.3e alpha=%.3e beta=%.3e pc=%d\n",
              round, sqrt(hs.rr / bb), hs32.iters - before, hs32.rr, hs32.rz, hs32.pAp, hs32.alpha, hs32.beta,
              hs32.pc);
    total += std::max(hs32.iters - before, 1);
  }
  {
    ProfScope ps_(c, OFDFT_K_VECTOR);
    convert_kernel<double, float><<<pb, 256, 0, c->stream>>>(g.G, phi32, phi64);
  }
  CU(cudaGetLastError());
  if (st) st->iterations = total;
  return rc;
}

// ------------------------------------------------------ functional (S4) ---

template <typename T>
int functional_pass(ofdft_ctx* c, int R, const GridDev& g, double h, const ofdft_params* p, const T* u,
                    const T* b, const T* phi, const T* rcg, double eta, double mu, double N,
                    const double* sum_uu_dev, T* G, T* s, const T* d, const T* s_old, EvalOut* out,
                    T* winv = nullptr, const double* phi64 = nullptr, const double* b64 = nullptr,
                    const double* r64 = nullptr, const CgScalars* es_sums = nullptr) {
  const Weights<double> W = lap_weights(R, h, 1.0);
  FuncScalars f;
  f.h3 = h * h * h;
  f.N = N;
  f.eta = eta;
  f.inv_mu = 1.0 / mu;
  f.lambda = p->lambda;
  f.CF = 0.3 * pow(3.0 * kPi * kPi, 2.0 / 3.0);
  f.kin_vw = -p->lambda * W.c;  // -lambda 6 w_0 > 0
  f.terms = p->terms;
  const bool es = p->terms & OFDFT_TERM_ES;
  // split_dots: G.d and G.s_old by a pointwise pass after the functional (which
  // then reads neither d nor s_old) instead of inside it
  const bool split_dots = c->func_split_dots && G && (d || s_old);
  EpiFunctional<T> ep{es ? phi : nullptr, b, es ? rcg : nullptr, split_dots ? nullptr : d,
                      split_dots ? nullptr : s_old, G, s, winv, sum_uu_dev, f, c->scal};
  if (es && es_sums) {
    ep.es_sums = es_sums;
  } else if (es && phi64) {
    ep.phi64 = phi64;
    ep.b64 = b64;
    ep.r64 = r64;
  }
  TRY(launch_z_r<T>(c, R, g, W, LoadPlain<T>{u}, ep, OFDFT_K_FUNCTIONAL));
  if (split_dots) {  // sums 5 and 6 of the functional's row: G.d and G.s_old
    const int pb = pointwise_blocks(c, g.G);
    TRY(ensure_partials(c, pb, 2));
    {
      ProfScope ps_(c, OFDFT_K_VECTOR);
      dot2_kernel<T><<<pb, 256, 0, c->stream>>>(g.G, G, d ? d : G, s_old ? G : nullptr, s_old, c->scal + 5,
                                                red(c));
    }
    CU(cudaGetLastError());
    if (!d) CU(cudaMemsetAsync(c->scal + 5, 0, sizeof(double), c->stream));
  }
  TRY(sync_scalars(c, c->scal, 12 * sizeof(double), out->sums));
  return OFDFT_OK;
}

#define TRY_PLAIN(expr)       \
  do {                        \
    const int rc_ = (expr);   \
    if (rc_ != OFDFT_OK) return rc_; \
  } while (0)

// Brent's minimiser (R. P. Brent, "Algorithms for Minimization without
// Derivatives", Prentice-Hall 1973, ch. 5, the published procedure restated
// here): parabolic steps through the three best points,
// golden-section steps when a parabola is not trusted, on a bracket a < x < b
// (or b < x < a) with f(x) below both ends.  f(t, &value) returns a status;
// rel_tol bounds the final bracket relative to |x|.  Returns the status and
// leaves the best abscissa/value in *xmin / *fmin.
template <class F>
int brent_minimise(F&& f, double a, double x, double b, double fx, double rel_tol, int max_it, double* xmin,
                   double* fmin) {
  constexpr double kGold = 0.38196601125010515;  // (3 - sqrt 5) / 2
  double lo = std::min(a, b), hi = std::max(a, b);
  double second = x, third = x, f2 = fx, f3 = fx;  // second- and third-best points
  double last_step = 0.0, step = 0.0;
  for (int it = 0; it < max_it; ++it) {
    const double mid = 0.5 * (lo + hi);
    const double tol1 = rel_tol * fabs(x) + 1e-12, tol2 = 2.0 * tol1;
    if (fabs(x - mid) <= tol2 - 0.5 * (hi - lo)) break;
    bool parabolic = false;
    if (fabs(last_step) > tol1) {
      const double r = (x - second) * (fx - f3);
      double q = (x - third) * (fx - f2);
      double num = (x - third) * q - (x - second) * r;
      q = 2.0 * (q - r);
      if (q > 0.0) num = -num;
      q = fabs(q);
      const double older = last_step;
      last_step = step;
      // accept the parabola's minimum if it lies inside the bracket and the
      // step is less than half of the step before last
      if (fabs(num) < fabs(0.5 * q * older) && num > q * (lo - x) && num < q * (hi - x)) {
        step = num / q;
        if ((x + step) - lo < tol2 || hi - (x + step) < tol2) step = (x < mid) ? tol1 : -tol1;
        parabolic = true;
      }
    }
    if (!parabolic) {
      last_step = (x >= mid) ? lo - x : hi - x;
      step = kGold * last_step;
    }
    const double t = (fabs(step) >= tol1) ? x + step : x + (step > 0.0 ? tol1 : -tol1);
    double ft = 0.0;
    TRY_PLAIN(f(t, &ft));
    if (ft <= fx) {
      (t >= x ? lo : hi) = x;
      third = second;
      f3 = f2;
      second = x;
      f2 = fx;
      x = t;
      fx = ft;
    } else {
      (t < x ? lo : hi) = t;
      if (ft <= f2 || second == x) {
        third = second;
        f3 = f2;
        second = t;
        f2 = ft;
      } else if (ft <= f3 || third == x || third == second) {
        third = t;
        f3 = ft;
      }
    }
  }
  *xmin = x;
  *fmin = fx;
  return OFDFT_OK;
}

// ------------------------------------------------------------- solve state --
// One energy/gradient evaluation of the solver (S3 + S4): Poisson at u (warm
// start from the state's phi), then the functional.  T is the field type.
template <typename T>
struct Solver {
  ofdft_ctx* c;
  const ofdft_params* p;
  GridDev g;
  double h, N, E_self, ezz;
  int R, M;
  bool mixed;
  T *u, *ut, *phi, *b, *G, *Gt, *s, *st, *sn, *d;
  double* b64;    // mixed: FP64 pseudocharge
  double* phi64;  // mixed: FP64 potential
  double* phi0;   // FP64 potential at the origin of the current line search
  double line_l = 0.0;  // position along d of the last Poisson solve (0: none yet)
  double tol_p = 0.0;   // Poisson tolerance of the next evaluations (adaptive_poisson_tol)
  ofdft_solve_stats* stats;
  ofdft_energy e;  // at the current point
  int trace = 0;   // OFDFT_TRACE=1: one line per evaluation on stderr
  int b2_valid = 0;  // mixed: V_B2 holds b64 as float-float pairs (split by the first Poisson solve)

  int eval(const T* at, T* Gout, T* sout, const T* dd, const T* s_old, double eta, double mu, ofdft_energy* out) {
    const int rc = eval_inner(at, Gout, sout, dd, s_old, eta, mu, out);
    if (trace)
      fprintf(stderr, "[ofdft] eval %d rc=%d L=%.12g E=%.12g C=%.3e gd=%.4e rs=%.4e cg=%d rel=%.2e\n",
              stats->grad_evals, rc, out->L, out->E, out->C, out->gd, out->rs, out->poisson.iterations,
              out->poisson.rel_residual);
    return rc;
  }

  int eval_inner(const T* at, T* Gout, T* sout, const T* dd, const T* s_old, double eta, double mu,
                 ofdft_energy* out) {
    ofdft_cg_stats cs{0, 0.0};
    const bool es = p->terms & OFDFT_TERM_ES;
    const double* sum_uu = &c->sc->sum_uu;
    if (es) {
      int rc;
      if (!mixed)
        rc = poisson_fp64(c, R, g, h, nullptr, (const double*)at, (const double*)b, (double*)phi, tol_p, p->max_cg,
                          &cs);
      else
        rc = poisson_mixed(c, R, g, h, nullptr, (const float*)at, b64, phi64, (float*)phi, tol_p, p->max_cg,
                           std::max(p->refine_every, 1), &cs, &b2_valid);
      if (rc != OFDFT_OK) return rc;
      stats->stencil_apps += cs.iterations + 1;
      stats->cg_iters += cs.iterations;
    } else {
      const int pb = pointwise_blocks(c, g.G);
      TRY(ensure_partials(c, pb, 2));
      {
        ProfScope ps_(c, OFDFT_K_VECTOR);
        dot2_kernel<T><<<pb, 256, 0, c->stream>>>(g.G, at, at, nullptr, nullptr, c->scal + 16, red(c));
      }
      CU(cudaGetLastError());
      sum_uu = c->scal + 16;
    }
    // the phi.r energy term uses the Poisson solve's residual (FP64 in MIXED)
    const T* rcg = (es && !mixed) ? vec<T>(c, V_R) : nullptr;
    EvalOut o;
    T* winv = (p->precond_rank1 && sout) ? vec<T>(c, V_W) : nullptr;
    TRY(functional_pass<T>(c, R, g, h, p, at, b, phi, rcg, eta, mu, N, sum_uu, Gout, sout, dd, s_old, &o, winv,
                           mixed ? phi64 : nullptr, mixed ? b64 : nullptr, mixed ? vec<double>(c, V_R64) : nullptr,
                           (mixed && c->mixed_ff) ? c->sc : nullptr));
    stats->stencil_apps += 2;
    stats->grad_evals += 1;
    fill_energy(o, h, p, E_self, ezz, eta, mu, out);
    if (winv) {
      // exact inverse of diag + (4 h^3/mu) u u^T (Sherman-Morrison) applied to r = -G
      const double cpen = 4.0 * h * h * h / mu;
      const double gamma = cpen * o.sums[10] / (1.0 + cpen * o.sums[11]);
      {
        ProfScope ps_(c, OFDFT_K_VECTOR);
        rank1_kernel<T><<<pointwise_blocks(c, g.G), 256, 0, c->stream>>>(g.G, sout, winv, gamma);
      }
      CU(cudaGetLastError());
      out->rs_pc -= h * h * h * gamma * o.sums[10];
    }
    out->poisson = cs;
    return OFDFT_OK;
  }

  // Warm start of the Poisson solves of a line search: phi(u + a d) is close to
  // phi0 + (a / l) (phi_l - phi0) (rho = u^2 + b is smooth in a), a better start
  // than phi_l alone.  line_start records phi0 at the origin; line_guess(a)
  // rewrites the FP64 potential (phi_l, from the solve at position l) in place.
  double* master() { return mixed ? phi64 : reinterpret_cast<double*>(phi); }
  int line_start() {
    CU(cudaMemcpyAsync(phi0, master(), g.G * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    line_l = 0.0;
    return OFDFT_OK;
  }
  int line_guess(double a) {
    if (line_l != 0.0 && (p->terms & OFDFT_TERM_ES)) {
      ProfScope ps_(c, OFDFT_K_VECTOR);
      extrap_kernel<<<pointwise_blocks(c, g.G), 256, 0, c->stream>>>(g.G, master(), phi0, a / line_l - 1.0);
    }
    CU(cudaGetLastError());
    line_l = a;
    return OFDFT_OK;
  }

  int dots(const T* a, const T* bb, const T* cc, const T* ee, double* r2) {
    const int pb = pointwise_blocks(c, g.G);
    TRY(ensure_partials(c, pb, 2));
    {
      ProfScope ps_(c, OFDFT_K_VECTOR);
      dot2_kernel<T><<<pb, 256, 0, c->stream>>>(g.G, a, bb, cc, ee, c->scal + 16, red(c));
    }
    CU(cudaGetLastError());
    TRY(sync_scalars(c, c->scal + 16, 2 * sizeof(double), r2));
    return OFDFT_OK;
  }

  int axpy_abs(T* out, const T* a, const T* bb, double alpha) {
    {
      ProfScope ps_(c, OFDFT_K_VECTOR);
      axpy_abs_kernel<T><<<pointwise_blocks(c, g.G), 256, 0, c->stream>>>(g.G, out, a, bb, alpha);
    }
    CU(cudaGetLastError());
    return OFDFT_OK;
  }

  int direction(double beta) {
    {
      ProfScope ps_(c, OFDFT_K_VECTOR);
      direction_kernel<T><<<pointwise_blocks(c, g.G), 256, 0, c->stream>>>(g.G, d, s, beta);
    }
    CU(cudaGetLastError());
    return OFDFT_OK;
  }

  // Polak-Ribiere nonlinear CG with a secant line search and the Jacobi
  // preconditioner, u <- |u| after every update (Sec. 4), on L(., eta, mu).
  int nlcg(double eta, double mu, int* converged) {
    *converged = 0;
    const double h3 = h * h * h;
    const double tol_in = p->tol_inner * M;
    TRY(eval(u, G, s, nullptr, nullptr, eta, mu, &e));
    TRY(direction(0.0));  // d = s
    double delta_new = e.rs_pc;
    int k = 0;
    for (int it = 0; it < p->max_nlcg; ++it) {
      if (e.rs < tol_in) {
        *converged = 1;
        break;
      }
      tol_p = adaptive_poisson_tol(p, e.rs, M);
      if (!isfinite(e.L) || !isfinite(e.rs)) return fail(c, OFDFT_ENONFINITE, "augmented Lagrangian is not finite");
      stats->nlcg_iters++;
      T* s_old = s;
      double gdd[2];
      TRY(dots(G, d, d, d, gdd));
      double g0 = h3 * gdd[0];
      double dd = h3 * gdd[1];
      if (!(g0 < 0.0)) {  // not a descent direction: restart along s
        TRY(direction(0.0));
        k = 0;
        TRY(dots(G, d, d, d, gdd));
        g0 = h3 * gdd[0];
        dd = h3 * gdd[1];
      }
      // trial point at sig along d (sigma0, capped to an RMS change of trial_max_rel of u)
      if (!std::isfinite(g0) || !std::isfinite(dd))
        return fail(c, OFDFT_ENONFINITE, "search direction is not finite (g.d = %g, d.d = %g)", g0, dd);
      double sig = p->sigma0;
      if (p->trial_max_rel > 0.0 && dd > 0.0) sig = std::min(sig, p->trial_max_rel * sqrt(N / dd));
      if (trace) fprintf(stderr, "[ofdft] nlcg it %d g0=%.6e dd=%.6e sig=%.6e\n", it, g0, dd, sig);
      TRY(line_start());
      TRY(line_guess(sig));
      TRY(axpy_abs(ut, u, d, sig));
      ofdft_energy et;
      const double tol_keep = tol_p;
      tol_p = trial_poisson_tol(p, tol_p);
      TRY(eval(ut, Gt, st, d, s_old, eta, mu, &et));
      tol_p = tol_keep;
      double alpha = -sig, gprev = et.gd, gcur = g0;
      if (!((gcur - gprev) / alpha > 0.0)) {
        // no positive curvature between 0 and sigma0: keep the trial point
        std::swap(u, ut);
        std::swap(G, Gt);
        std::swap(s, st);
        e = et;
      } else {
        T* snew = sn;
        const double L0 = e.L + l_resolution(e, mixed);
        double pos = 0.0;  // position of u along d
        for (int j = 1; j <= p->max_secant; ++j) {
          alpha = alpha * gcur / (gprev - gcur);
          // candidate written beside u so that a rejected step can be halved
          TRY(line_guess(pos + alpha));
          TRY(axpy_abs(ut, u, d, alpha));
          TRY(eval(ut, G, snew, d, s_old, eta, mu, &e));
          for (int bt = 0; bt < p->max_backtrack && !(e.L <= L0); ++bt) {
            alpha *= 0.5;
            TRY(line_guess(pos + alpha));
            TRY(axpy_abs(ut, u, d, alpha));
            TRY(eval(ut, G, snew, d, s_old, eta, mu, &e));
          }
          std::swap(u, ut);
          pos += alpha;
          gprev = gcur;
          gcur = e.gd;
          if (j == p->max_secant || alpha * alpha * dd <= p->eps_secant * p->eps_secant * N) break;
          if (!((gcur - gprev) / alpha > 0.0)) break;
        }
        // the new s lives in snew; the old s buffer becomes spare
        sn = s;
        s = snew;
      }
      const double delta_old = delta_new;
      const double delta_mid = -e.gs_old;
      delta_new = e.rs_pc;
      const double beta = (delta_new - delta_mid) / delta_old;
      ++k;
      if (trace) fprintf(stderr, "[ofdft] nlcg beta=%.6e delta_old=%.6e delta_new=%.6e delta_mid=%.6e\n", beta,
                         delta_old, delta_new, delta_mid);
      if (k >= p->restart_every || !(beta > 0.0) || !std::isfinite(beta)) {
        TRY(direction(0.0));
        k = 0;
      } else {
        TRY(direction(beta));
      }
    }
    if (!*converged && e.rs < tol_in) *converged = 1;
    return OFDFT_OK;
  }

  // ---- Lagrange-multiplier method (Sec. 5.3.2) --------------------------------
  int lincomb(T* out, const T* a, double ca, const T* bb, double cb, int take_abs) {
    {
      ProfScope ps_(c, OFDFT_K_VECTOR);
      lincomb_kernel<T><<<pointwise_blocks(c, g.G), 256, 0, c->stream>>>(g.G, out, a, ca, bb, cb, take_abs);
    }
    CU(cudaGetLastError());
    return OFDFT_OK;
  }

  // Energy E_h at `at` (no gradient); L = E with eta = 0 and 1/mu = 0.
  int energy_at(const T* at, ofdft_energy* out) {
    TRY(eval(at, nullptr, nullptr, nullptr, nullptr, 0.0, INFINITY, out));
    stats->energy_evals++;
    stats->grad_evals--;  // counted as an energy evaluation
    return OFDFT_OK;
  }

  // PR nonlinear CG on the sphere h^3 sum u^2 = N: the energy gradient G_E at u,
  // eta = G_E.u / (2 u.u), g = G_E - 2 eta u, s = -g / diag projected orthogonal
  // to u, the Polak-Ribiere direction projected the same way, and a Brent line
  // search on the angle t of u(t) = |cos t u + sin t d^|, d^ = d sqrt(N) / |d|,
  // which keeps the norm.  Buffers: G holds g, s the direction of steepest
  // preconditioned descent, sn the previous s, st the scaled direction d^, Gt
  // the line's origin u0, ut the trial point.
  int lm_stall = 0;  // 1: the LM line search found no lower energy along a descent direction

  int lm(double* eta_out, int* converged) {
    *converged = 0;
    const double h3 = h * h * h;
    const double tol_in = p->tol_inner * M;
    const int pb = pointwise_blocks(c, g.G);
    TRY(ensure_partials(c, pb, 2));
    double r2[2];
    // start on the sphere
    TRY(dots(u, u, nullptr, nullptr, r2));
    TRY(lincomb(u, u, sqrt(N / (h3 * r2[0])), nullptr, 0.0, 0));
    CU(cudaMemsetAsync(sn, 0, g.G * sizeof(T), c->stream));
    FuncScalars f;
    const Weights<double> W = lap_weights(R, h, 1.0);
    f.h3 = h3;
    f.N = N;
    f.inv_mu = 0.0;
    f.lambda = p->lambda;
    f.CF = 0.3 * pow(3.0 * kPi * kPi, 2.0 / 3.0);
    f.kin_vw = -p->lambda * W.c;
    f.terms = p->terms;
    const bool es = p->terms & OFDFT_TERM_ES;
    double eta = 0.0, delta = 0.0;
    int k = 0;
    T* u0 = Gt;
    T* dh = st;
    for (int it = 0; it <= p->max_nlcg; ++it) {
      // G_E at u and G_E.u (the functional pass's <G, d> with d = u)
      TRY(eval(u, G, nullptr, u, nullptr, 0.0, INFINITY, &e));
      if (!isfinite(e.E)) return fail(c, OFDFT_ENONFINITE, "energy is not finite");
      const double uu_h3 = e.C + N;  // h^3 u.u
      eta = e.gd / (2.0 * uu_h3);
      f.eta = eta;
      {
        ProfScope ps_(c, OFDFT_K_VECTOR);
        lm_precond_kernel<T><<<pb, 256, 0, c->stream>>>(g.G, G, s, u, es ? phi : nullptr, f, c->scal + 16, red(c));
      }
      CU(cudaGetLastError());
      TRY(sync_scalars(c, c->scal + 16, 2 * sizeof(double), r2));
      const double uu = r2[1];
      TRY(lincomb(s, s, 1.0, u, -r2[0] / uu, 0));  // s orthogonal to u
      TRY(dots(G, s, G, sn, r2));
      const double rs = -h3 * r2[0], rs_mid = -h3 * r2[1];
      e.rs = rs;
      e.rs_pc = rs;
      if (trace) fprintf(stderr, "[ofdft] lm it %d E=%.12g eta=%.9f rs=%.4e\n", it, e.E, eta, rs);
      if (rs < tol_in) {
        if (tol_p > p->tol_poisson) {  // confirm at the full Poisson tolerance
          tol_p = p->tol_poisson;
          continue;
        }
        *converged = 1;
        break;
      }
      if (it == p->max_nlcg) break;
      tol_p = adaptive_poisson_tol(p, rs, M);
      stats->nlcg_iters++;
      const double beta = (it == 0) ? 0.0 : (rs - rs_mid) / delta;
      delta = rs;
      ++k;
      const bool restart = (it == 0 || k >= p->restart_every || !(beta > 0.0));
      if (restart) k = 0;
      TRY(direction(restart ? 0.0 : beta));
      TRY(dots(d, u, nullptr, nullptr, r2));
      TRY(lincomb(d, d, 1.0, u, -r2[0] / uu, 0));  // d orthogonal to u
      TRY(dots(G, d, d, d, r2));
      double gdot = r2[0], dd = r2[1];
      if (!(gdot < 0.0)) {  // not a descent direction: restart along s
        TRY(direction(0.0));
        k = 0;
        TRY(dots(d, d, nullptr, nullptr, r2));
        dd = r2[0];
      }
      std::swap(s, sn);  // this s is the next iteration's s_old
      const double dnorm = sqrt(h3 * dd);
      if (!(dnorm > 0.0)) break;
      TRY(lincomb(dh, d, sqrt(N) / dnorm, nullptr, 0.0, 0));
      CU(cudaMemcpyAsync(u0, u, g.G * sizeof(T), cudaMemcpyDeviceToDevice, c->stream));
      auto E_at = [&](double t, double* val) -> int {
        TRY(lincomb(ut, u0, cos(t), dh, sin(t), 1));
        ofdft_energy et;
        TRY(energy_at(ut, &et));
        if (!isfinite(et.E)) return fail(c, OFDFT_ENONFINITE, "energy is not finite on the line search");
        *val = et.E;
        return OFDFT_OK;
      };
      // bracket the minimum along t, then Brent
      double ta = 0.0, fa = e.E;
      double tb = std::min(dnorm / sqrt(N), 0.3), fb = 0.0;
      TRY(E_at(tb, &fb));
      for (int sh = 0; sh < 30 && fb >= fa; ++sh) {
        tb *= 0.25;
        TRY(E_at(tb, &fb));
      }
      if (fb >= fa) {  // no decrease along d: stop where we are (phi back at u for the forces)
        TRY(eval(u, G, nullptr, u, nullptr, 0.0, INFINITY, &e));
        e.rs = rs;
        lm_stall = 1;
        break;
      }
      double tc = 2.0 * tb, fc = 0.0;
      TRY(E_at(tc, &fc));
      for (int gr = 0; gr < 40 && fc < fb; ++gr) {
        ta = tb;
        fa = fb;
        tb = tc;
        fb = fc;
        tc = 1.618034 * tb;
        TRY(E_at(tc, &fc));
      }
      double tmin = tb, fmin = fb;
      TRY(brent_minimise(E_at, ta, tb, tc, fb, 1e-4, 60, &tmin, &fmin));
      TRY(lincomb(u, u0, cos(tmin), dh, sin(tmin), 1));
    }
    *eta_out = eta;
    return OFDFT_OK;
  }
};


// Copies atoms to a device scratch buffer (V_ATOM0): R (3M) then Z (M).
int upload_atoms(ofdft_ctx* c, const double* R_host, const double* Z_host, int M, AtomArgs* A,
                 const ofdft_grid* g, double sigma, double rc) {
  TRY(ensure(c, c->v[V_ATOM0], (size_t)4 * M * sizeof(double)));
  double* dR = vec<double>(c, V_ATOM0);
  CU(cudaMemcpyAsync(dR, R_host, 3 * M * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  CU(cudaMemcpyAsync(dR + 3 * M, Z_host, M * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  A->R = dR;
  A->Z = dR + 3 * M;
  A->M = M;
  A->h = g ? g->h : 1.0;
  A->ox = g ? g->origin[0] : 0.0;
  A->oy = g ? g->origin[1] : 0.0;
  A->oz = g ? g->origin[2] : 0.0;
  A->sigma = sigma;
  A->rc = rc;
  return OFDFT_OK;
}

int check_atoms(ofdft_ctx* c, const double* R, const double* Z, int M) {
  if (M < 1 || !R || !Z) return fail(c, OFDFT_EINVAL, "need M >= 1 atoms with positions and charges");
  for (int i = 0; i < 3 * M; ++i)
    if (!isfinite(R[i])) return fail(c, OFDFT_ENONFINITE, "atom coordinate %d is not finite", i);
  for (int i = 0; i < M; ++i)
    if (!isfinite(Z[i])) return fail(c, OFDFT_ENONFINITE, "charge %d is not finite", i);
  return OFDFT_OK;
}

// Per-atom tables (S1, S9): box of lattice nodes whose centre can lie within r_c
// of the atom, plus one node of slack; b_J is tabulated on the box grown by R
// (bdim) and V_J on the box grown by 2R (vdim).
struct AtomTables {
  int rb, box, bdim, vdim, batch;
  long long vper, bper;
};

inline AtomTables atom_tables(double rc, double h, int R, int M, size_t budget) {
  AtomTables t;
  t.rb = (int)ceil(rc / h) + 1;
  t.box = 2 * t.rb + 1;
  t.bdim = t.box + 2 * R;
  t.vdim = t.box + 4 * R;
  t.vper = (long long)t.vdim * t.vdim * t.vdim;
  t.bper = (long long)t.bdim * t.bdim * t.bdim;
  t.batch = (int)std::max<long long>(1, std::min<long long>(M, (long long)budget / ((t.vper + t.bper) * 8)));
  return t;
}

inline void atom_box_lo(const double* R_host, int a0, int na, const ofdft_grid* gr, int rb, std::vector<int>& lo) {
  for (int a = 0; a < na; ++a)
    for (int d = 0; d < 3; ++d)
      lo[3 * a + d] = (int)floor((R_host[3 * (a0 + a) + d] - gr->origin[d]) / gr->h - 0.5) - rb + 1;
}

template <typename T, int R>
int launch_force_boxes(ofdft_ctx* c, const AtomArgs& A, int a0, int na, int vdim, int bdim, const int* lo,
                       const Weights<double>& W, double* vbox, double* bbox);

// Identity of the b_J tables of a geometry: everything they depend on.
inline std::vector<double> btab_key(const ofdft_grid* gr, int R, const double* R_host, const double* Z_host, int M,
                                    double sigma, double rc) {
  std::vector<double> k = {(double)M, (double)R, gr->h, gr->origin[0], gr->origin[1], gr->origin[2],
                           (double)gr->n[0], (double)gr->n[1], (double)gr->n[2], sigma, rc};
  k.insert(k.end(), R_host, R_host + 3 * (size_t)M);
  k.insert(k.end(), Z_host, Z_host + (size_t)M);
  return k;
}
constexpr size_t kBtabMaxBytes = (size_t)4 << 30;  // b_J tables kept for the forces up to this size

// b = sum_J b_J and E_self (Sec. 4): the atoms' V_J and b_J tables are built for
// ranges of at most 512 atoms, then every node gathers the b_J of the atoms whose
// box holds it, in atom order (FP64 running sums across ranges).  With `keep`
// the b_J tables of all atoms go to V_BTAB (at most kBtabMaxBytes) and stay
// there for the forces of the same geometry (device_forces), which then skip
// rebuilding them.
template <typename T, int R>
int pseudocharge_tables(ofdft_ctx* c, const ofdft_grid* gr, const GridDev& g, const AtomArgs& A,
                        const double* R_host, const double* Z_host, int M, T* b, double* es_dev, bool keep) {
  const Weights<double> W = lap_weights(R, gr->h, 1.0);
  AtomTables t = atom_tables(A.rc, gr->h, R, M, (size_t)768 << 20);
  if (t.vdim > 1024) return fail(c, OFDFT_EINVAL, "r_c / h = %g is too large for the atom tables", A.rc / gr->h);
  t.batch = std::min(t.batch, 512);
  c->btab_key.clear();
  keep = keep && (size_t)M * t.bper * sizeof(double) <= kBtabMaxBytes;
  if (keep) TRY(ensure(c, c->v[V_BTAB], (size_t)M * t.bper * sizeof(double)));
  TRY(ensure(c, c->v[V_ATOM1], (size_t)t.batch * (t.vper + (keep ? 0 : t.bper)) * sizeof(double)));
  TRY(ensure(c, c->v[V_ATOM2], (size_t)t.batch * 3 * sizeof(int) + 64));
  const bool multi = M > t.batch;
  if (multi) TRY(ensure(c, c->v[V_BACC], g.G * sizeof(double)));
  double* vbox = vec<double>(c, V_ATOM1);
  double* btab = keep ? vec<double>(c, V_BTAB) : nullptr;
  int* lo_dev = vec<int>(c, V_ATOM2);
  double* bacc = multi ? vec<double>(c, V_BACC) : nullptr;
  std::vector<int> lo((size_t)3 * t.batch);
  const dim3 grid((g.n1 + AT - 1) / AT, (g.n2 + AT - 1) / AT, (g.n3 + AT - 1) / AT);
  TRY(ensure_partials(c, (long long)grid.x * grid.y * grid.z, 1));
  CU(cudaMemsetAsync(es_dev, 0, sizeof(double), c->stream));
  for (int a0 = 0; a0 < M; a0 += t.batch) {
    const int na = std::min(t.batch, M - a0);
    double* bbox = keep ? btab + (size_t)a0 * t.bper : vbox + (size_t)t.batch * t.vper;
    atom_box_lo(R_host, a0, na, gr, t.rb, lo);
    CU(cudaMemcpyAsync(lo_dev, lo.data(), 3 * na * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    TRY((launch_force_boxes<T, R>(c, A, a0, na, t.vdim, t.bdim, lo_dev, W, vbox, bbox)));
    {
      ProfScope ps_(c, OFDFT_K_ATOMS);
      pseudocharge_gather_kernel<T><<<grid, dim3(AT, AT, AT), 0, c->stream>>>(
          g, A, a0, na, t.box, t.bdim, t.vdim, R, lo_dev, vbox, bbox, bacc, a0 == 0 ? 1 : 0,
          a0 + na >= M ? 1 : 0, b, es_dev, red(c));
    }
    CU(cudaGetLastError());
  }
  if (keep) c->btab_key = btab_key(gr, R, R_host, Z_host, M, A.sigma, A.rc);
  return OFDFT_OK;
}

template <typename T>
int device_pseudocharge(ofdft_ctx* c, const ofdft_grid* gr, int R, const double* R_host, const double* Z_host,
                        int M, double sigma, double rc, T* b, double* E_self, bool keep_tables) {
  AtomArgs A;
  TRY(upload_atoms(c, R_host, Z_host, M, &A, gr, sigma, rc));
  const GridDev g = gdev(gr);
  double* es_dev = c->scal + 20;
  switch (R) {
#define PSC_CASE(RR)                                                                                         \
  case RR:                                                                                                   \
    TRY((pseudocharge_tables<T, RR>(c, gr, g, A, R_host, Z_host, M, b, es_dev, keep_tables)));              \
    break;
    PSC_CASE(1)
    PSC_CASE(2)
    PSC_CASE(3)
    PSC_CASE(4)
    PSC_CASE(5)
    PSC_CASE(6)
#undef PSC_CASE
    default: return fail(c, OFDFT_EINVAL, "stencil radius %d", R);
  }
  double es;
  TRY(sync_scalars(c, es_dev, sizeof(double), &es));
  *E_self = 0.5 * gr->h * gr->h * gr->h * es;
  return OFDFT_OK;
}

template <typename T>
int device_guess(ofdft_ctx* c, const ofdft_grid* gr, const double* R_host, const double* Z_host, int M,
                 double gsig, double gcut, double N, T* u) {
  AtomArgs A;
  TRY(upload_atoms(c, R_host, Z_host, M, &A, gr, 1.0, 1.0));
  const GridDev g = gdev(gr);
  dim3 grid((g.n1 + AT - 1) / AT, (g.n2 + AT - 1) / AT, (g.n3 + AT - 1) / AT);
  TRY(ensure_partials(c, (long long)grid.x * grid.y * grid.z, 1));
  {
    ProfScope ps_(c, OFDFT_K_ATOMS);
    guess_kernel<T><<<grid, dim3(AT, AT, AT), 0, c->stream>>>(g, A, gsig, gcut, u, c->scal + 21, red(c));
  }
  CU(cudaGetLastError());
  {
    ProfScope ps_(c, OFDFT_K_ATOMS);
    normalise_kernel<T><<<pointwise_blocks(c, g.G), 256, 0, c->stream>>>(g.G, u, c->scal + 21,
                                                                        gr->h * gr->h * gr->h, N);
  }
  CU(cudaGetLastError());
  return OFDFT_OK;
}

template <typename T, int R>
int launch_force_boxes(ofdft_ctx* c, const AtomArgs& A, int a0, int na, int vdim, int bdim, const int* lo,
                       const Weights<double>& W, double* vbox, double* bbox) {
  // one block row per atom, about eight blocks per SM in total
  auto grid_for = [&](long long per) {
    const long long bx = std::max<long long>(1, std::min<long long>((per + 255) / 256, ((long long)c->sms * 8 + na - 1) / na));
    return dim3((unsigned)bx, (unsigned)na);
  };
  {
    ProfScope ps_(c, OFDFT_K_ATOMS);
    force_vbox_kernel<<<grid_for((long long)vdim * vdim * vdim), 256, 0, c->stream>>>(A, a0, vdim, R, lo, vbox);
  }
  CU(cudaGetLastError());
  {
    ProfScope ps_(c, OFDFT_K_ATOMS);
    force_bbox_kernel<R><<<grid_for((long long)bdim * bdim * bdim), 256, 0, c->stream>>>(A, a0, vdim, bdim, lo, W,
                                                                                        vbox, bbox);
  }
  CU(cudaGetLastError());
  return OFDFT_OK;
}

template <typename T, int R>
int launch_force_ball(ofdft_ctx* c, const GridDev& g, const AtomArgs& A, int a0, int na, int bdim, int box,
                      const int* lo, const Weights<double>& W, const Weights<double>& Wt, const double* bbox,
                      const T* phi, int exact, double* partial, int nblk) {
  {
    ProfScope ps_(c, OFDFT_K_ATOMS);
    force_ball_kernel<T, R><<<dim3(nblk, na), 256, 0, c->stream>>>(g, A, a0, bdim, box, lo, W, Wt, bbox, phi, exact,
                                                                    partial);
  }
  CU(cudaGetLastError());
  return OFDFT_OK;
}

template <typename T>
int device_forces(ofdft_ctx* c, const ofdft_grid* gr, int R, const double* R_host, const double* Z_host, int M,
                  double sigma, double rc, int variant, const T* phi, double* F) {
  AtomArgs A;
  TRY(upload_atoms(c, R_host, Z_host, M, &A, gr, sigma, rc));
  const GridDev g = gdev(gr);
  const double h = gr->h;
  // per-atom box: nodes whose centre can lie within r_c, plus one node of slack
  const int rb = (int)ceil(rc / h) + 1;
  const int box = 2 * rb + 1;
  const int bdim = box + 2 * R, vdim = box + 4 * R;
  const long long vper = (long long)vdim * vdim * vdim, bper = (long long)bdim * bdim * bdim;
  const bool exact = (variant == OFDFT_FORCE_EXACT);
  // atoms per batch: keep the box scratch near 256 MB
  if (vdim > 1024) return fail(c, OFDFT_EINVAL, "r_c / h = %g is too large for the atom tables", rc / h);
  int batch = (int)std::max<long long>(1, std::min<long long>(M, (256ll << 20) / ((vper + bper) * 8)));
  batch = std::min(batch, 16384);  // atoms of one launch (one block row each)
  if (exact) batch = std::min(M, 4096);
  const int nblk = std::max(1, std::min(64, (int)((long long)box * box * box / 2048) + 1));
  // the b_J tables of this very geometry, kept by the solve's pseudocharge pass
  const bool kept = !exact && !c->btab_key.empty() && c->btab_key == btab_key(gr, R, R_host, Z_host, M, sigma, rc);
  if (kept) batch = std::min(M, 4096);
  TRY(ensure(c, c->v[V_ATOM1], (exact || kept) ? 256 : (size_t)batch * (vper + bper) * sizeof(double)));
  TRY(ensure(c, c->v[V_ATOM2], (size_t)batch * (3 + nblk * 3) * sizeof(double) + (size_t)batch * 3 * sizeof(int) +
                                  (size_t)3 * M * sizeof(double) + 64));
  double* vbox = vec<double>(c, V_ATOM1);
  double* bbox = vbox + (size_t)batch * vper;
  double* partial = vec<double>(c, V_ATOM2);
  double* Fdev = partial + (size_t)batch * nblk * 3;
  int* lo_dev = (int*)(Fdev + (size_t)3 * M);
  std::vector<int> lo((size_t)3 * batch);
  const Weights<double> W = lap_weights(R, h, 1.0), Wt = grad_weights(R, h);
  for (int a0 = 0; a0 < M; a0 += batch) {
    const int na = std::min(batch, M - a0);
    for (int a = 0; a < na; ++a)
      for (int d = 0; d < 3; ++d)
        lo[3 * a + d] = (int)floor((R_host[3 * (a0 + a) + d] - gr->origin[d]) / h - 0.5) - rb + 1;
    CU(cudaMemcpyAsync(lo_dev, lo.data(), 3 * na * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    if (kept) bbox = vec<double>(c, V_BTAB) + (size_t)a0 * bper;
    if (!exact && !kept) {
      switch (R) {
        case 1: TRY((launch_force_boxes<T, 1>(c, A, a0, na, vdim, bdim, lo_dev, W, vbox, bbox))); break;
        case 2: TRY((launch_force_boxes<T, 2>(c, A, a0, na, vdim, bdim, lo_dev, W, vbox, bbox))); break;
        case 3: TRY((launch_force_boxes<T, 3>(c, A, a0, na, vdim, bdim, lo_dev, W, vbox, bbox))); break;
        case 4: TRY((launch_force_boxes<T, 4>(c, A, a0, na, vdim, bdim, lo_dev, W, vbox, bbox))); break;
        case 5: TRY((launch_force_boxes<T, 5>(c, A, a0, na, vdim, bdim, lo_dev, W, vbox, bbox))); break;
        case 6: TRY((launch_force_boxes<T, 6>(c, A, a0, na, vdim, bdim, lo_dev, W, vbox, bbox))); break;
      }
    }
    switch (R) {
      case 1: TRY((launch_force_ball<T, 1>(c, g, A, a0, na, bdim, box, lo_dev, W, Wt, bbox, phi, exact, partial, nblk))); break;
      case 2: TRY((launch_force_ball<T, 2>(c, g, A, a0, na, bdim, box, lo_dev, W, Wt, bbox, phi, exact, partial, nblk))); break;
      case 3: TRY((launch_force_ball<T, 3>(c, g, A, a0, na, bdim, box, lo_dev, W, Wt, bbox, phi, exact, partial, nblk))); break;
      case 4: TRY((launch_force_ball<T, 4>(c, g, A, a0, na, bdim, box, lo_dev, W, Wt, bbox, phi, exact, partial, nblk))); break;
      case 5: TRY((launch_force_ball<T, 5>(c, g, A, a0, na, bdim, box, lo_dev, W, Wt, bbox, phi, exact, partial, nblk))); break;
      case 6: TRY((launch_force_ball<T, 6>(c, g, A, a0, na, bdim, box, lo_dev, W, Wt, bbox, phi, exact, partial, nblk))); break;
    }
    {
      ProfScope ps_(c, OFDFT_K_ATOMS);
      force_sum_kernel<<<(na + 127) / 128, 128, 0, c->stream>>>(a0, na, nblk, h * h * h, partial, Fdev);
    }
    CU(cudaGetLastError());
  }
  CU(cudaMemcpyAsync(F, Fdev, 3 * M * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return OFDFT_OK;
}

int device_ezz(ofdft_ctx* c, const double* R_host, const double* Z_host, int M, double sigma, double* E,
               double* F) {
  AtomArgs A;
  TRY(upload_atoms(c, R_host, Z_host, M, &A, nullptr, sigma, 1.0));
  TRY(ensure(c, c->v[V_ATOM2], (size_t)4 * M * sizeof(double) + 64));
  double* eI = vec<double>(c, V_ATOM2);
  double* Fd = eI + M;
  {
    ProfScope ps_(c, OFDFT_K_ATOMS);
    ezz_kernel<<<(M + 127) / 128, 128, 0, c->stream>>>(A, eI, Fd);
  }
  CU(cudaGetLastError());
  std::vector<double> e(M), f(3 * (size_t)M);
  CU(cudaMemcpyAsync(e.data(), eI, M * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaMemcpyAsync(f.data(), Fd, 3 * M * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  double s = 0.0;
  for (int i = 0; i < M; ++i) s += e[i];
  *E = s;
  if (F)
    for (int i = 0; i < 3 * M; ++i) F[i] = f[i];
  return OFDFT_OK;
}

// Results of a solve at its final state: energy, stats, forces at phi* (S9).
template <typename T>
int finish_solve(ofdft_ctx* c, Solver<T>& S, const ofdft_grid* gr, int R, const double* R_host, const double* Z_host,
                 int M, const ofdft_params* p, void* u_out, void* phi_out, double* energy, double* forces,
                 ofdft_solve_stats* st, int converged, const double* Fz, const char* notconv) {
  const size_t es = sizeof(T);
  st->E = S.e.E;
  st->C = S.e.C;
  st->parts = S.e;
  st->converged = converged;
  st->grid = *gr;
  *energy = S.e.E;
  if (forces) {
    // MIXED: the forces take the FP64 potential of the last Poisson solve's
    // residual correction (phi in the field type is its float rounding)
    if (S.phi64)
      TRY(device_forces<double>(c, gr, R, R_host, Z_host, M, p->sigma, p->rc, p->force_variant, S.phi64, forces));
    else
      TRY(device_forces<T>(c, gr, R, R_host, Z_host, M, p->sigma, p->rc, p->force_variant, S.phi, forces));
    if (p->ezz_correction)
      for (int i = 0; i < 3 * M; ++i) forces[i] += Fz[i];
  }
  if (u_out) CU(cudaMemcpyAsync(u_out, S.u, S.g.G * es, cudaMemcpyDeviceToDevice, c->stream));
  if (phi_out) CU(cudaMemcpyAsync(phi_out, S.phi, S.g.G * es, cudaMemcpyDeviceToDevice, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  TRY(zstream_fault_check(c));
  return converged ? OFDFT_OK : fail(c, OFDFT_ENOTCONV, "%s", notconv);
}

template <typename T>
int solve_impl(ofdft_ctx* c, const ofdft_grid* gr, const double* R_host, const double* Z_host, int M,
               const ofdft_params* p, void* u_out, void* phi_out, double* energy, double* forces,
               ofdft_solve_stats* st, const void* u_in = nullptr, const void* phi_in = nullptr) {
  const bool mixed = (p->precision == OFDFT_PREC_MIXED);
  const GridDev g = gdev(gr);
  const int R = p->fd_order / 2;
  const size_t es = sizeof(T);
  // workspace
  for (int v : {V_U, V_UT, V_PHI, V_B, V_G, V_GT, V_S, V_ST, V_SN, V_D}) TRY(ensure(c, c->v[v], g.G * es));
  if (p->precond_rank1) TRY(ensure(c, c->v[V_W], g.G * es));
  TRY(ensure_cg_vectors(c, g.G, es, mixed));
  if (mixed) {
    TRY(ensure(c, c->v[V_B64], g.G * sizeof(double)));
    TRY(ensure(c, c->v[V_PHI64], g.G * sizeof(double)));
  }
  double N = 0.0;
  for (int J = 0; J < M; ++J) N += Z_host[J];
  Solver<T> S;
  S.c = c;
  S.p = p;
  S.g = g;
  S.h = gr->h;
  S.N = N;
  S.R = R;
  S.M = M;
  S.mixed = mixed;
  S.stats = st;
  S.trace = getenv("OFDFT_TRACE") && getenv("OFDFT_TRACE")[0] == '1';
  S.u = vec<T>(c, V_U);
  S.ut = vec<T>(c, V_UT);
  S.phi = vec<T>(c, V_PHI);
  S.b = vec<T>(c, V_B);
  S.G = vec<T>(c, V_G);
  S.Gt = vec<T>(c, V_GT);
  S.s = vec<T>(c, V_S);
  S.st = vec<T>(c, V_ST);
  S.sn = vec<T>(c, V_SN);
  S.d = vec<T>(c, V_D);
  S.b64 = mixed ? vec<double>(c, V_B64) : nullptr;
  S.phi64 = mixed ? vec<double>(c, V_PHI64) : nullptr;
  TRY(ensure(c, c->v[V_PHI0], g.G * sizeof(double)));
  S.phi0 = vec<double>(c, V_PHI0);
  S.tol_p = (p->poisson_adapt > 0.0) ? std::max(p->tol_poisson, 1e-4) : p->tol_poisson;  // first solve from phi = 0
  // S1: pseudocharge (FP64 for the mixed path too), starting guess, phi = 0
  if (!mixed) {
    TRY(device_pseudocharge<double>(c, gr, R, R_host, Z_host, M, p->sigma, p->rc, (double*)S.b, &S.E_self, true));
  } else {
    TRY(device_pseudocharge<double>(c, gr, R, R_host, Z_host, M, p->sigma, p->rc, S.b64, &S.E_self, true));
    {
      ProfScope ps_(c, OFDFT_K_VECTOR);
      convert_kernel<double, float><<<pointwise_blocks(c, g.G), 256, 0, c->stream>>>(g.G, (float*)S.b, S.b64);
    }
    CU(cudaGetLastError());
    CU(cudaMemsetAsync(S.phi64, 0, g.G * sizeof(double), c->stream));
  }
  if (u_in) {
    // warm start: the given density amplitude, rescaled to h^3 sum u^2 = N
    CU(cudaMemcpyAsync(S.u, u_in, g.G * es, cudaMemcpyDeviceToDevice, c->stream));
    const int pb = pointwise_blocks(c, g.G);
    TRY(ensure_partials(c, pb, 2));
    {
      ProfScope ps_(c, OFDFT_K_VECTOR);
      dot2_kernel<T><<<pb, 256, 0, c->stream>>>(g.G, S.u, S.u, nullptr, nullptr, c->scal + 16, red(c));
    }
    {
      ProfScope ps_(c, OFDFT_K_VECTOR);
      normalise_kernel<T><<<pb, 256, 0, c->stream>>>(g.G, S.u, c->scal + 16, gr->h * gr->h * gr->h, N);
    }
    CU(cudaGetLastError());
  } else {
    TRY(device_guess<T>(c, gr, R_host, Z_host, M, p->guess_sigma, p->guess_cut, N, S.u));
  }
  if (phi_in) {
    // warm start of the Poisson solves
    CU(cudaMemcpyAsync(S.phi, phi_in, g.G * es, cudaMemcpyDeviceToDevice, c->stream));
    if (mixed) {
      ProfScope ps_(c, OFDFT_K_VECTOR);
      convert_kernel<float, double><<<pointwise_blocks(c, g.G), 256, 0, c->stream>>>(g.G, S.phi64,
                                                                                      (const float*)phi_in);
    }
    CU(cudaGetLastError());
  } else {
    CU(cudaMemsetAsync(S.phi, 0, g.G * es, c->stream));
  }
  S.ezz = 0.0;
  std::vector<double> Fz(3 * (size_t)M, 0.0);
  if (p->ezz_correction) TRY(device_ezz(c, R_host, Z_host, M, p->sigma, &S.ezz, Fz.data()));
  int converged = 0;
  if (p->method == OFDFT_METHOD_LM) {
    double eta_lm = 0.0;
    TRY(S.lm(&eta_lm, &converged));
    st->eta = eta_lm;
    st->outer_iters = 1;
    return finish_solve(c, S, gr, R, R_host, Z_host, M, p, u_out, phi_out, energy, forces, st, converged,
                        Fz.data(),
                        S.lm_stall ? "the Lagrange-multiplier line search found no lower energy before h^3 r.s "
                                     "reached tol_inner (energy resolution of the precision)"
                                   : "the Lagrange-multiplier method reached max_nlcg");
  }
  // Algorithm 1
  double eta = (p->method == OFDFT_METHOD_PENALTY) ? 0.0 : p->eta0;
  double mu = p->mu0;
  TRY(S.eval(S.u, S.G, S.s, nullptr, nullptr, eta, mu, &S.e));
  double E_prev = S.e.E;
  const double tolE = p->tol_E * M;
  for (int q = 0; q < p->max_outer; ++q) {
    int inner_ok = 0;
    TRY(S.nlcg(eta, mu, &inner_ok));
    st->outer_iters++;
    const double E = S.e.E, C = S.e.C;
    if (!isfinite(E) || !isfinite(C)) return fail(c, OFDFT_ENONFINITE, "energy or constraint is not finite");
    const double eta_eff = eta - C / mu;  // multiplier update of Algorithm 1
    st->eta = eta_eff;
    if (p->method == OFDFT_METHOD_AL) eta = eta_eff;
    mu = p->kappa * mu;
    if (fabs(E - E_prev) < tolE) {
      converged = 1;
      break;
    }
    E_prev = E;
  }
  if (S.tol_p > p->tol_poisson) {
    // the last potential may come from a loose solve (poisson_adapt): the
    // reported energy and the forces use one solved to tol_poisson
    S.tol_p = p->tol_poisson;
    TRY(S.eval(S.u, nullptr, nullptr, nullptr, nullptr, eta, mu, &S.e));
  }
  return finish_solve(c, S, gr, R, R_host, Z_host, M, p, u_out, phi_out, energy, forces, st, converged, Fz.data(),
                      "Algorithm 1 reached max_outer");
}

int check_params(ofdft_ctx* c, const ofdft_params* p) {
  if (!p) return fail(c, OFDFT_EINVAL, "params is NULL");
  TRY(check_order(c, p->fd_order));
  TRY(check_prec(c, p->precision));
  if (p->method != OFDFT_METHOD_AL && p->method != OFDFT_METHOD_PENALTY && p->method != OFDFT_METHOD_LM)
    return fail(c, OFDFT_EINVAL, "method must be OFDFT_METHOD_AL, OFDFT_METHOD_PENALTY or OFDFT_METHOD_LM");
  if (!(p->mu0 > 0.0) || !(p->kappa > 0.0 && p->kappa < 1.0))
    return fail(c, OFDFT_EINVAL, "Algorithm 1 needs mu0 > 0 and 0 < kappa < 1");
  if (!(p->poisson_adapt >= 0.0)) return fail(c, OFDFT_EINVAL, "poisson_adapt must be >= 0");
  if (!(p->trial_poisson_loosen >= 1.0)) return fail(c, OFDFT_EINVAL, "trial_poisson_loosen must be >= 1");
  if (!(p->tol_poisson > 0.0) || p->max_cg < 1 || p->max_nlcg < 0 || p->max_outer < 1 || p->max_secant < 1)
    return fail(c, OFDFT_EINVAL, "tolerances must be positive and iteration caps >= 1");
  if (!(p->sigma > 0.0) || !(p->rc > 0.0)) return fail(c, OFDFT_EINVAL, "sigma and rc must be positive");
  return OFDFT_OK;
}

template int device_pseudocharge<double>(ofdft_ctx*, const ofdft_grid*, int, const double*, const double*, int,
                                         double, double, double*, double*, bool);
template int device_pseudocharge<float>(ofdft_ctx*, const ofdft_grid*, int, const double*, const double*, int,
                                        double, double, float*, double*, bool);
template int device_guess<double>(ofdft_ctx*, const ofdft_grid*, const double*, const double*, int, double, double,
                                  double, double*);
template int device_guess<float>(ofdft_ctx*, const ofdft_grid*, const double*, const double*, int, double, double,
                                 double, float*);
template int device_forces<double>(ofdft_ctx*, const ofdft_grid*, int, const double*, const double*, int, double,
                                   double, int, const double*, double*);
template int device_forces<float>(ofdft_ctx*, const ofdft_grid*, int, const double*, const double*, int, double,
                                  double, int, const float*, double*);

}  // namespace ofd

using namespace ofd;

// ===================================================================== C ABI
extern "C" {

void ofdft_default_params(ofdft_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->fd_order = 12;
  p->terms = OFDFT_TERM_ALL;
  p->method = OFDFT_METHOD_AL;
  p->precision = OFDFT_PREC_FP64;
  p->lambda = 0.2;
  p->eta0 = -0.2;
  p->mu0 = 1.0;
  p->kappa = 0.1;
  p->sigma = 1.0;
  p->rc = 7.0;
  p->guess_sigma = 2.0;
  p->guess_cut = 8.0;
  p->tol_E = 1e-6;
  p->tol_inner = 1e-8;
  p->tol_poisson = 1e-8;
  p->max_outer = 30;
  p->max_nlcg = 2000;
  p->max_cg = 20000;
  p->max_secant = 1;
  p->sigma0 = 0.5;
  p->eps_secant = 1e-7;
  p->restart_every = 20;
  p->force_variant = OFDFT_FORCE_PAPER;
  p->ezz_correction = 0;
  p->vacuum = 8.0;
  p->round_to = 16;
  p->refine_every = 200;
  p->trial_max_rel = 0.2;
  p->max_backtrack = 2;
  p->precond_rank1 = 1;
  p->poisson_adapt = 1.0;
  p->trial_poisson_loosen = 1.0;
}

int ofdft_create(ofdft_ctx** out, int device, void* stream) {
  if (!out) return OFDFT_EINVAL;
  *out = nullptr;
  ofdft_ctx* c = new ofdft_ctx();
  c->device = device;
  c->stream = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) {
    delete c;
    return OFDFT_ECUDA;
  }
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
  if (cudaMalloc(&c->counter, 64) != cudaSuccess || cudaMemset(c->counter, 0, 64) != cudaSuccess ||
      cudaMalloc(&c->sc, 3 * sizeof(CgScalars)) != cudaSuccess ||
      cudaMalloc(&c->scal, 64 * sizeof(double)) != cudaSuccess ||
      cudaMallocHost(&c->host_scal, 64 * sizeof(double)) != cudaSuccess ||
      cudaMallocHost(&c->ring, 2 * sizeof(CgScalars)) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ring_ev[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ring_ev[1], cudaEventDisableTiming) != cudaSuccess) {
    delete c;
    return OFDFT_ENOMEM;
  }
  c->sc32 = c->sc + 1;
  if (cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking) != cudaSuccess) c->use_graphs = 0;
  const char* at = getenv("OFDFT_AUTOTUNE");
  c->autotune = !(at && at[0] == '0');
  const char* co = getenv("OFDFT_COOP");  // 1: persistent cooperative CG iterations where they apply
  c->coop = (co && co[0] == '1') ? 1 : 0;
  const char* pcn = getenv("OFDFT_PRECOND");  // 0: plain Poisson CG (ofdft_set_poisson_precond)
  c->precond = (pcn && pcn[0] == '0') ? OFDFT_PRECOND_NONE : OFDFT_PRECOND_MG;
  c->trace = getenv("OFDFT_TRACE") && getenv("OFDFT_TRACE")[0] == '1';  // per-round lines of the mixed Poisson
  c->mg_omega = kMgOmega;
  c->mg_sweeps = kMgSweeps;
  const char* mo = getenv("OFDFT_MG_OMEGA");  // multigrid experiments: Jacobi weight, bottom sweeps
  if (mo && atof(mo) > 0.0 && atof(mo) < 1.0) c->mg_omega = atof(mo);
  const char* ms = getenv("OFDFT_MG_SWEEPS");
  if (ms && atoi(ms) >= 1) c->mg_sweeps = atoi(ms);
  const char* cz = getenv("OFDFT_COOP_NZ");  // launch-shape experiments: z-chunks of the persistent CG grid
  c->coop_nz = cz ? atoi(cz) : 0;
  const char* fsd = getenv("OFDFT_FUNC_SPLIT_DOTS");  // 1: G.d, G.s_old after the functional pass
  if (fsd) c->func_split_dots = atoi(fsd) != 0;
  const char* mzs = getenv("OFDFT_MG_ZSTREAM");  // 1: level smoothing passes as z-streaming stencils
  if (mzs) c->mg_zstream = atoi(mzs) != 0;
  const char* mzn = getenv("OFDFT_MG_ZSTREAM_NODES");  // levels of at least this many nodes: z-streaming smoothing
  if (mzn) c->mg_zstream_nodes = atoll(mzn);
  const char* mcl = getenv("OFDFT_MG_CLUSTER");  // 1: coarse multigrid levels on one thread-block cluster
  if (mcl) c->mg_cluster = atoi(mcl) != 0;
  const char* fbl = getenv("OFDFT_MG_FUSE_BELOW");  // coarser levels of at most this many nodes take the fused passes
  if (fbl) c->mg_fuse_below = atoll(fbl);
  const char* m0 = getenv("OFDFT_MG_FINEST_SMOOTH");  // 0: no smoothing on the finest multigrid level
  if (m0) c->mg_finest_smooth = atoi(m0) != 0;
  const char* pdl = getenv("OFDFT_PDL");  // 1: programmatic dependent launch in the CG loop
  c->pdl = (pdl && pdl[0] == '1') ? 1 : 0;
  const char* tma = getenv("OFDFT_TMA");  // 1: TMA staging in the FP32 z-streaming passes that allow it
  c->tma = (tma && tma[0] == '1') ? 1 : 0;
  const char* cgr = getenv("OFDFT_COND_GRAPHS");  // 0: CG chunks of eight iterations polled by the host
  c->cond_graphs = !(cgr && cgr[0] == '0');
  const char* ffr = getenv("OFDFT_FF_RESIDUAL");  // 0: FP64 stencil in the mixed residual pass
  c->ff_residual = !(ffr && ffr[0] == '0');
  const char* mf = getenv("OFDFT_MG_FUSE_NODES");  // levels of at least this many nodes take the fused passes
  if (mf) c->mg_fuse_nodes = atoll(mf);          // (-1: none)
  const char* fb = getenv("OFDFT_CG_FOLD_BYTES");  // CG working set above which the iterate update is folded
  if (fb && atof(fb) >= 0.0) c->cg_fold_bytes = atof(fb);
  const char* pw = getenv("OFDFT_POINTWISE_BLOCKS_PER_SM");  // launch-shape experiments (default 4)
  if (pw && atoi(pw) >= 1 && atoi(pw) <= 16) c->pw_per_sm = atoi(pw);
  cudaMemset(c->sc, 0, 3 * sizeof(CgScalars));
  cudaMemset(c->scal, 0, 64 * sizeof(double));
  cudaDeviceSynchronize();
  *out = c;
  return OFDFT_OK;
}

int ofdft_destroy(ofdft_ctx* c) {
  if (!c) return OFDFT_OK;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  cudaDeviceSynchronize();
  harvest(c);
  for (auto& e : c->graphs) cudaGraphExecDestroy(e.exec);
  if (c->gstream) cudaStreamDestroy(c->gstream);
  if (c->coop_bar) cudaFree(c->coop_bar);
  for (auto& s : c->gev)
    for (auto& e : s)
      if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : c->free_events) cudaEventDestroy(e);
  cudaFree(c->partials.p);
  for (auto& b : c->v) cudaFree(b.p);
  cudaFree(c->mgbuf.p);
  cudaFree(c->counter);
  cudaFree(c->sc);
  cudaFree(c->scal);
  cudaFreeHost(c->host_scal);
  cudaFreeHost(c->ring);
  for (cudaEvent_t e : c->ring_ev)
    if (e) cudaEventDestroy(e);
  delete c;
  return OFDFT_OK;
}

const char* ofdft_last_error(const ofdft_ctx* c) { return c ? c->err.c_str() : "null context"; }

int ofdft_set_poisson_precond(ofdft_ctx* c, int kind) {
  if (!c) return OFDFT_EINVAL;
  if (kind != OFDFT_PRECOND_NONE && kind != OFDFT_PRECOND_MG)
    return fail(c, OFDFT_EINVAL, "unknown Poisson preconditioner %d", kind);
  c->precond = kind;
  return OFDFT_OK;
}

int ofdft_profile(ofdft_ctx* c, int kind_mask) {
  if (!c) return OFDFT_EINVAL;
  c->prof = kind_mask;
  return OFDFT_OK;
}

int ofdft_get_counters(ofdft_ctx* c, ofdft_counters* out) {
  if (!c || !out) return OFDFT_EINVAL;
  CU(cudaSetDevice(c->device));
  CU(cudaStreamSynchronize(c->stream));
  harvest(c);
  out->launches = c->launches;
  for (int k = 0; k < OFDFT_K_COUNT; ++k) {
    out->kind_launches[k] = c->kind_launches[k];
    out->timed_launches[k] = c->timed_launches[k];
    out->timed_ms[k] = c->timed_ms[k];
  }
  out->persistent_cg_iters = c->coop_iters;
  out->tma_launches = c->tma_launches;
  return OFDFT_OK;
}

int ofdft_reset_counters(ofdft_ctx* c) {
  if (!c) return OFDFT_EINVAL;
  CU(cudaSetDevice(c->device));
  CU(cudaStreamSynchronize(c->stream));
  harvest(c);
  c->launches = 0;
  for (int k = 0; k < OFDFT_K_COUNT; ++k) {
    c->kind_launches[k] = 0;
    c->timed_launches[k] = 0;
    c->timed_ms[k] = 0.0;
  }
  c->coop_iters = 0;
  c->tma_launches = 0;
  return OFDFT_OK;
}

int ofdft_grid_for_atoms(const double* R, int M, double h, double vacuum, int round_to, ofdft_grid* g) {
  if (!R || M < 1 || !g || !(h > 0.0) || round_to < 1 || !(vacuum >= 0.0)) return OFDFT_EINVAL;
  for (int d = 0; d < 3; ++d) {
    double lo = R[d], hi = R[d];
    for (int J = 1; J < M; ++J) {
      lo = std::min(lo, R[3 * J + d]);
      hi = std::max(hi, R[3 * J + d]);
    }
    if (!isfinite(lo) || !isfinite(hi)) return OFDFT_ENONFINITE;
    lo -= vacuum;
    hi += vacuum;
    const double L = hi - lo;
    long long n = (long long)ceil(L / h - 1e-9);
    if (n < 1) n = 1;
    n = ((n + round_to - 1) / round_to) * round_to;
    if (n > (1 << 16)) return OFDFT_EINVAL;
    g->n[d] = (int)n;
    g->origin[d] = lo - 0.5 * ((double)n * h - L);
  }
  g->h = h;
  return OFDFT_OK;
}

long long ofdft_struct_bytes(const char* name) {
  if (!name) return -1;
  const std::string n(name);
  if (n == "ofdft_grid") return (long long)sizeof(ofdft_grid);
  if (n == "ofdft_params") return (long long)sizeof(ofdft_params);
  if (n == "ofdft_cg_stats") return (long long)sizeof(ofdft_cg_stats);
  if (n == "ofdft_energy") return (long long)sizeof(ofdft_energy);
  if (n == "ofdft_solve_stats") return (long long)sizeof(ofdft_solve_stats);
  if (n == "ofdft_counters") return (long long)sizeof(ofdft_counters);
  if (n == "ofdft_relax_stats") return (long long)sizeof(ofdft_relax_stats);
  if (n == "ofdft_batch_stats") return (long long)sizeof(ofdft_batch_stats);
  return -1;
}

int ofdft_mg_plan(const ofdft_grid* g, int prec, int* levels, int* coarse_level, int* dims, long long* bytes) {
  if (!g || !levels || !coarse_level) return OFDFT_EINVAL;
  if (g->n[0] < 1 || g->n[1] < 1 || g->n[2] < 1 || !(g->h > 0.0)) return OFDFT_EINVAL;
  const size_t es = (prec == OFDFT_PREC_MIXED) ? 4 : 8;
  const GridDev gd = gdev(g);
  const MgPlan P = mg_plan(gd, g->h, es);
  *levels = P.nlev;
  *coarse_level = P.ok ? P.lc : -1;
  if (dims)
    for (int l = 0; l < P.nlev; ++l) {
      dims[3 * l] = P.d[l].n1;
      dims[3 * l + 1] = P.d[l].n2;
      dims[3 * l + 2] = P.d[l].n3;
    }
  if (bytes) *bytes = P.ok ? (long long)((2 * gd.G + P.elems) * (long long)es) : 0;
  return OFDFT_OK;
}

long long ofdft_workspace_bytes(const ofdft_grid* g, int fd_order, int prec) {
  if (!g) return -1;
  const long long G = (long long)g->n[0] * g->n[1] * g->n[2];
  const long long es = (prec == OFDFT_PREC_MIXED) ? 4 : 8;
  long long bytes = G * es * 14;                 // solve state, NLCG and CG vectors
  if (prec == OFDFT_PREC_MIXED) bytes += G * 8 * 3 + G * 4;  // r64, phi64, b64, e32
  bytes += G * 8;                                // potential at the line-search origin
  bytes += G * es * 3;                           // multigrid: z, finest scratch, coarser levels (3/7 G)
  (void)fd_order;
  return bytes;
}

int ofdft_stencil(ofdft_ctx* c, const ofdft_grid* g, int fd_order, int prec, const void* f, void* out) {
  if (!c) return OFDFT_EINVAL;
  c->err.clear();
  TRY(check_grid(c, g));
  TRY(check_order(c, fd_order));
  TRY(check_prec(c, prec));
  if (!f || !out) return fail(c, OFDFT_EINVAL, "null field pointer");
  if (f == out) return fail(c, OFDFT_EINVAL, "in-place stencil is not supported");
  CU(cudaSetDevice(c->device));
  const GridDev gd = gdev(g);
  const Weights<double> W = lap_weights(fd_order / 2, g->h, 1.0);
  if (prec == OFDFT_PREC_FP64)
    return launch_z_r<double>(c, fd_order / 2, gd, W, LoadPlain<double>{(const double*)f}, EpiStore<double>{(double*)out}, OFDFT_K_STENCIL);
  return launch_z_r<float>(c, fd_order / 2, gd, W, LoadPlain<float>{(const float*)f}, EpiStore<float>{(float*)out}, OFDFT_K_STENCIL);
}

int ofdft_pseudocharge(ofdft_ctx* c, const ofdft_grid* g, int fd_order, const double* R, const double* Z, int M,
                       double sigma, double rc, int prec, void* b, double* E_self) {
  if (!c) return OFDFT_EINVAL;
  c->err.clear();
  TRY(check_grid(c, g));
  TRY(check_order(c, fd_order));
  TRY(check_prec(c, prec));
  TRY(check_atoms(c, R, Z, M));
  if (!b || !E_self) return fail(c, OFDFT_EINVAL, "null output pointer");
  if (!(sigma > 0.0) || !(rc > 0.0)) return fail(c, OFDFT_EINVAL, "sigma and rc must be positive");
  CU(cudaSetDevice(c->device));
  if (prec == OFDFT_PREC_FP64)
    return device_pseudocharge<double>(c, g, fd_order / 2, R, Z, M, sigma, rc, (double*)b, E_self);
  return device_pseudocharge<float>(c, g, fd_order / 2, R, Z, M, sigma, rc, (float*)b, E_self);
}

int ofdft_initial_guess(ofdft_ctx* c, const ofdft_grid* g, const double* R, const double* Z, int M,
                        double guess_sigma, double guess_cut, double N, int prec, void* u) {
  if (!c) return OFDFT_EINVAL;
  c->err.clear();
  TRY(check_grid(c, g));
  TRY(check_prec(c, prec));
  TRY(check_atoms(c, R, Z, M));
  if (!u) return fail(c, OFDFT_EINVAL, "null output pointer");
  if (!(guess_sigma > 0.0) || !(guess_cut > 0.0) || !(N > 0.0)) return fail(c, OFDFT_EINVAL, "bad guess parameters");
  CU(cudaSetDevice(c->device));
  if (prec == OFDFT_PREC_FP64) return device_guess<double>(c, g, R, Z, M, guess_sigma, guess_cut, N, (double*)u);
  return device_guess<float>(c, g, R, Z, M, guess_sigma, guess_cut, N, (float*)u);
}

int ofdft_poisson(ofdft_ctx* c, const ofdft_grid* g, int fd_order, int prec, const void* rho, const void* u,
                  const void* b, void* phi, double tol, int max_it, ofdft_cg_stats* st) {
  if (!c) return OFDFT_EINVAL;
  c->err.clear();
  TRY(check_grid(c, g));
  TRY(check_order(c, fd_order));
  TRY(check_prec(c, prec));
  if (!phi || (!rho && (!u || !b))) return fail(c, OFDFT_EINVAL, "need phi and either rho or (u, b)");
  if (!(tol > 0.0) || max_it < 0) return fail(c, OFDFT_EINVAL, "need tol > 0 and max_it >= 0");
  CU(cudaSetDevice(c->device));
  const GridDev gd = gdev(g);
  ofdft_cg_stats tmp;
  if (!st) st = &tmp;
  if (prec == OFDFT_PREC_FP64) {
    const int rc = poisson_fp64(c, fd_order / 2, gd, g->h, (const double*)rho, (const double*)u, (const double*)b,
                                (double*)phi, tol, max_it, st);
    TRY(zstream_fault_check(c));
    return rc;
  }
  // mixed: FP64 copies of b and phi live in the context for the call
  TRY(ensure(c, c->v[V_PHI64], gd.G * sizeof(double)));
  TRY(ensure(c, c->v[V_B64], gd.G * sizeof(double)));
  const int pb = pointwise_blocks(c, gd.G);
  {
    ProfScope ps_(c, OFDFT_K_VECTOR);
    convert_kernel<float, double><<<pb, 256, 0, c->stream>>>(gd.G, vec<double>(c, V_PHI64), (const float*)phi);
  }
  if (!rho) {
    ProfScope ps_(c, OFDFT_K_VECTOR);
    convert_kernel<float, double><<<pb, 256, 0, c->stream>>>(gd.G, vec<double>(c, V_B64), (const float*)b);
  }
  CU(cudaGetLastError());
  ofdft_params dp;
  ofdft_default_params(&dp);
  const int rc = poisson_mixed(c, fd_order / 2, gd, g->h, (const float*)rho, (const float*)u, vec<double>(c, V_B64),
                               vec<double>(c, V_PHI64), (float*)phi, tol, max_it, dp.refine_every, st);
  TRY(zstream_fault_check(c));
  return rc;
}

int ofdft_energy_grad(ofdft_ctx* c, const ofdft_grid* g, const ofdft_params* p, const void* u, const void* b,
                      void* phi, double E_self, double eta, double mu, double N, int solve_poisson, void* grad,
                      void* s, const void* d, const void* s_old, ofdft_energy* out) {
  if (!c) return OFDFT_EINVAL;
  c->err.clear();
  TRY(check_grid(c, g));
  TRY(check_params(c, p));
  if (!u || !out || ((p->terms & OFDFT_TERM_ES) && (!b || !phi))) return fail(c, OFDFT_EINVAL, "null pointer");
  if (!(mu > 0.0) || !isfinite(eta) || !isfinite(N)) return fail(c, OFDFT_EINVAL, "need mu > 0, finite eta and N");
  CU(cudaSetDevice(c->device));
  const GridDev gd = gdev(g);
  const int R = p->fd_order / 2;
  const bool mixed = p->precision == OFDFT_PREC_MIXED;
  const bool es = p->terms & OFDFT_TERM_ES;
  memset(out, 0, sizeof(*out));
  ofdft_cg_stats cs{0, 0.0};
  const double* sum_uu = &c->sc->sum_uu;
  TRY(ensure_cg_vectors(c, gd.G, mixed ? 4 : 8, mixed));
  if (es) {
    if (!mixed) {
      // residual at the incoming phi (and CG if asked): gives r for the energy and sum u^2
      const int rc = poisson_fp64(c, R, gd, g->h, nullptr, (const double*)u, (const double*)b, (double*)phi,
                                  p->tol_poisson, solve_poisson ? p->max_cg : 0, &cs);
      if (rc != OFDFT_OK && !(rc == OFDFT_ENOTCONV && !solve_poisson)) return rc;
      c->err.clear();
    } else {
      TRY(ensure(c, c->v[V_PHI64], gd.G * sizeof(double)));
      TRY(ensure(c, c->v[V_B64], gd.G * sizeof(double)));
      const int pb = pointwise_blocks(c, gd.G);
      {
        ProfScope ps_(c, OFDFT_K_VECTOR);
        convert_kernel<float, double><<<pb, 256, 0, c->stream>>>(gd.G, vec<double>(c, V_PHI64), (const float*)phi);
      }
      {
        ProfScope ps_(c, OFDFT_K_VECTOR);
        convert_kernel<float, double><<<pb, 256, 0, c->stream>>>(gd.G, vec<double>(c, V_B64), (const float*)b);
      }
      CU(cudaGetLastError());
      int rc = poisson_mixed(c, R, gd, g->h, nullptr, (const float*)u, vec<double>(c, V_B64), vec<double>(c, V_PHI64),
                             (float*)phi, p->tol_poisson, solve_poisson ? p->max_cg : 0, std::max(p->refine_every, 1),
                             &cs);
      if (rc != OFDFT_OK && !(rc == OFDFT_ENOTCONV && !solve_poisson)) return rc;
      c->err.clear();
    }
  } else {
    const int pb = pointwise_blocks(c, gd.G);
    TRY(ensure_partials(c, pb, 2));
    if (mixed)
      {
        ProfScope ps_(c, OFDFT_K_VECTOR);
        dot2_kernel<float><<<pb, 256, 0, c->stream>>>(gd.G, (const float*)u, (const float*)u, nullptr, nullptr, c->scal + 16, red(c));
      }
    else
      {
        ProfScope ps_(c, OFDFT_K_VECTOR);
        dot2_kernel<double><<<pb, 256, 0, c->stream>>>(gd.G, (const double*)u, (const double*)u, nullptr, nullptr, c->scal + 16, red(c));
      }
    CU(cudaGetLastError());
    sum_uu = c->scal + 16;
  }
  EvalOut o;
  const bool r1 = p->precond_rank1 && s;
  if (r1) TRY(ensure(c, c->v[V_W], gd.G * (mixed ? 4 : 8)));
  if (!mixed)
    TRY(functional_pass<double>(c, R, gd, g->h, p, (const double*)u, (const double*)b, (const double*)phi,
                                es ? vec<double>(c, V_R) : nullptr, eta, mu, N, sum_uu, (double*)grad, (double*)s,
                                (const double*)d, (const double*)s_old, &o, r1 ? vec<double>(c, V_W) : nullptr));
  else
    TRY(functional_pass<float>(c, R, gd, g->h, p, (const float*)u, (const float*)b, (const float*)phi, nullptr, eta,
                               mu, N, sum_uu, (float*)grad, (float*)s, (const float*)d, (const float*)s_old, &o,
                               r1 ? vec<float>(c, V_W) : nullptr, es ? vec<double>(c, V_PHI64) : nullptr,
                               es ? vec<double>(c, V_B64) : nullptr, es ? vec<double>(c, V_R64) : nullptr,
                               (es && c->mixed_ff) ? c->sc : nullptr));
  fill_energy(o, g->h, p, E_self, 0.0, eta, mu, out);
  if (r1) {
    // the preconditioned residual includes the exact inverse of the rank-one term (4 h^3/mu) u u^T
    const double h3 = g->h * g->h * g->h;
    const double cpen = 4.0 * h3 / mu;
    const double gamma = cpen * o.sums[10] / (1.0 + cpen * o.sums[11]);
    {
      ProfScope ps_(c, OFDFT_K_VECTOR);
      if (!mixed)
        rank1_kernel<double><<<pointwise_blocks(c, gd.G), 256, 0, c->stream>>>(gd.G, (double*)s, vec<double>(c, V_W), gamma);
      else
        rank1_kernel<float><<<pointwise_blocks(c, gd.G), 256, 0, c->stream>>>(gd.G, (float*)s, vec<float>(c, V_W), gamma);
    }
    CU(cudaGetLastError());
    out->rs_pc -= h3 * gamma * o.sums[10];
  }
  out->poisson = cs;
  TRY(zstream_fault_check(c));
  if (!isfinite(out->L)) return fail(c, OFDFT_ENONFINITE, "augmented Lagrangian is not finite");
  return OFDFT_OK;
}

int ofdft_overlap_correction(ofdft_ctx* c, const ofdft_grid* g, int fd_order, const double* R, const double* Z,
                             int M, double sigma, double rc, double sigma_ref, double rc_ref, double tol, double* E_c,
                             double* F_c) {
  if (!c) return OFDFT_EINVAL;
  c->err.clear();
  TRY(check_grid(c, g));
  TRY(check_order(c, fd_order));
  TRY(check_atoms(c, R, Z, M));
  if (!E_c || !F_c) return fail(c, OFDFT_EINVAL, "null output pointer");
  if (!(sigma > 0.0) || !(rc > 0.0) || !(sigma_ref > 0.0) || !(rc_ref > 0.0) || !(tol > 0.0))
    return fail(c, OFDFT_EINVAL, "sigma, rc, sigma_ref, rc_ref and tol must be positive");
  for (int i = 0; i < M; ++i)  // the reference charges must not overlap (App. A)
    for (int j = i + 1; j < M; ++j) {
      const double dx = R[3 * i] - R[3 * j], dy = R[3 * i + 1] - R[3 * j + 1], dz = R[3 * i + 2] - R[3 * j + 2];
      const double d = sqrt(dx * dx + dy * dy + dz * dz);
      if (!(d > 2.0 * rc_ref))
        return fail(c, OFDFT_EINVAL, "reference charges of atoms %d and %d overlap (distance %g <= 2 rc_ref = %g)", i,
                    j, d, 2.0 * rc_ref);
    }
  CU(cudaSetDevice(c->device));
  const GridDev gd = gdev(g);
  const int Rr = fd_order / 2;
  TRY(ensure(c, c->v[V_OC], 4 * (size_t)gd.G * sizeof(double)));
  double* b = vec<double>(c, V_OC);
  double* bt = b + gd.G;
  double* V = bt + gd.G;
  double* Vt = V + gd.G;
  double es = 0.0, est = 0.0;
  TRY(device_pseudocharge<double>(c, g, Rr, R, Z, M, sigma, rc, b, &es));
  TRY(device_pseudocharge<double>(c, g, Rr, R, Z, M, sigma_ref, rc_ref, bt, &est));
  CU(cudaMemsetAsync(V, 0, 2 * (size_t)gd.G * sizeof(double), c->stream));
  ofdft_cg_stats st{0, 0.0};
  TRY(poisson_fp64(c, Rr, gd, g->h, b, nullptr, nullptr, V, tol, 20000, &st));
  TRY(poisson_fp64(c, Rr, gd, g->h, bt, nullptr, nullptr, Vt, tol, 20000, &st));
  // (b~ + b).(V~ - V) = b~.V~ - b~.V + b.V~ - b.V
  const int pb = pointwise_blocks(c, gd.G);
  TRY(ensure_partials(c, pb, 2));
  double d1[2], d2[2];
  {
    ProfScope ps_(c, OFDFT_K_VECTOR);
    dot2_kernel<double><<<pb, 256, 0, c->stream>>>(gd.G, bt, Vt, bt, V, c->scal + 16, red(c));
  }
  CU(cudaGetLastError());
  TRY(sync_scalars(c, c->scal + 16, 2 * sizeof(double), d1));
  {
    ProfScope ps_(c, OFDFT_K_VECTOR);
    dot2_kernel<double><<<pb, 256, 0, c->stream>>>(gd.G, b, Vt, b, V, c->scal + 16, red(c));
  }
  CU(cudaGetLastError());
  TRY(sync_scalars(c, c->scal + 16, 2 * sizeof(double), d2));
  const double h3 = g->h * g->h * g->h;
  *E_c = 0.5 * h3 * ((d1[0] - d1[1]) + (d2[0] - d2[1])) + es - est;
  std::vector<double> Ft(3 * (size_t)M), Fb(3 * (size_t)M);
  TRY(device_forces<double>(c, g, Rr, R, Z, M, sigma_ref, rc_ref, OFDFT_FORCE_PAPER, Vt, Ft.data()));
  TRY(device_forces<double>(c, g, Rr, R, Z, M, sigma, rc, OFDFT_FORCE_PAPER, V, Fb.data()));
  for (size_t k = 0; k < Ft.size(); ++k) F_c[k] = Ft[k] - Fb[k];
  return OFDFT_OK;
}

int ofdft_forces(ofdft_ctx* c, const ofdft_grid* g, int fd_order, const double* R, const double* Z, int M,
                 double sigma, double rc, int variant, int prec, const void* phi, double* F) {
  if (!c) return OFDFT_EINVAL;
  c->err.clear();
  TRY(check_grid(c, g));
  TRY(check_order(c, fd_order));
  TRY(check_prec(c, prec));
  TRY(check_atoms(c, R, Z, M));
  if (!phi || !F) return fail(c, OFDFT_EINVAL, "null pointer");
  if (variant != OFDFT_FORCE_PAPER && variant != OFDFT_FORCE_EXACT) return fail(c, OFDFT_EINVAL, "bad force variant");
  CU(cudaSetDevice(c->device));
  if (prec == OFDFT_PREC_FP64)
    return device_forces<double>(c, g, fd_order / 2, R, Z, M, sigma, rc, variant, (const double*)phi, F);
  return device_forces<float>(c, g, fd_order / 2, R, Z, M, sigma, rc, variant, (const float*)phi, F);
}

int ofdft_solve_from(ofdft_ctx* c, const ofdft_grid* grid, const double* R, const double* Z, int M, double h,
                     const ofdft_params* p, const void* u_in, const void* phi_in, void* u_out, void* phi_out,
                     double* energy, double* forces, ofdft_solve_stats* st) {
  if (!c) return OFDFT_EINVAL;
  c->err.clear();
  if ((u_in || phi_in) && !grid) return fail(c, OFDFT_EINVAL, "a warm start needs the grid it was computed on");
  TRY(check_params(c, p));
  TRY(check_atoms(c, R, Z, M));
  if (!energy) return fail(c, OFDFT_EINVAL, "energy pointer is NULL");
  ofdft_solve_stats tmp;
  if (!st) st = &tmp;
  memset(st, 0, sizeof(*st));
  ofdft_grid g;
  if (grid) {
    g = *grid;
  } else {
    const int rc = ofdft_grid_for_atoms(R, M, h, p->vacuum, p->round_to > 0 ? p->round_to : 1, &g);
    if (rc != OFDFT_OK) return fail(c, rc, "box rule failed for h=%g vacuum=%g", h, p->vacuum);
  }
  TRY(check_grid(c, &g));
  CU(cudaSetDevice(c->device));
  if (p->precision == OFDFT_PREC_FP64)
    return solve_impl<double>(c, &g, R, Z, M, p, u_out, phi_out, energy, forces, st, u_in, phi_in);
  return solve_impl<float>(c, &g, R, Z, M, p, u_out, phi_out, energy, forces, st, u_in, phi_in);
}

int ofdft_solve(ofdft_ctx* c, const ofdft_grid* grid, const double* R, const double* Z, int M, double h,
                const ofdft_params* p, void* u_out, void* phi_out, double* energy, double* forces,
                ofdft_solve_stats* st) {
  if (!c) return OFDFT_EINVAL;
  c->err.clear();
  TRY(check_params(c, p));
  TRY(check_atoms(c, R, Z, M));
  if (!energy) return fail(c, OFDFT_EINVAL, "energy pointer is NULL");
  ofdft_solve_stats tmp;
  if (!st) st = &tmp;
  memset(st, 0, sizeof(*st));
  ofdft_grid g;
  if (grid) {
    g = *grid;
  } else {
    const int rc = ofdft_grid_for_atoms(R, M, h, p->vacuum, p->round_to > 0 ? p->round_to : 1, &g);
    if (rc != OFDFT_OK) return fail(c, rc, "box rule failed for h=%g vacuum=%g", h, p->vacuum);
  }
  TRY(check_grid(c, &g));
  CU(cudaSetDevice(c->device));
  if (p->precision == OFDFT_PREC_FP64) return solve_impl<double>(c, &g, R, Z, M, p, u_out, phi_out, energy, forces, st);
  return solve_impl<float>(c, &g, R, Z, M, p, u_out, phi_out, energy, forces, st);
}

int ofdft_relax(ofdft_ctx* c, const ofdft_grid* grid, double* R, const double* Z, int M, double h,
                const ofdft_params* p, int max_steps, double f_tol, double max_move, double* energy,
                double* forces, ofdft_relax_stats* rst) {
  if (!c) return OFDFT_EINVAL;
  c->err.clear();
  TRY(check_params(c, p));
  TRY(check_atoms(c, R, Z, M));
  if (!energy || !forces) return fail(c, OFDFT_EINVAL, "energy and forces are required");
  if (max_steps < 0 || !(f_tol > 0.0) || !(max_move > 0.0))
    return fail(c, OFDFT_EINVAL, "need max_steps >= 0, f_tol > 0 and max_move > 0");
  ofdft_relax_stats tmp;
  if (!rst) rst = &tmp;
  memset(rst, 0, sizeof(*rst));
  // one grid for the whole relaxation: the caller's, or the box rule at the start
  ofdft_grid g;
  if (grid) {
    g = *grid;
  } else {
    const int rc = ofdft_grid_for_atoms(R, M, h, p->vacuum, p->round_to > 0 ? p->round_to : 1, &g);
    if (rc != OFDFT_OK) return fail(c, rc, "box rule failed for h=%g vacuum=%g", h, p->vacuum);
  }
  TRY(check_grid(c, &g));
  CU(cudaSetDevice(c->device));
  const size_t es = (p->precision == OFDFT_PREC_FP64) ? 8 : 4;
  const long long G = (long long)g.n[0] * g.n[1] * g.n[2];
  // u* and phi* of the last ground state: the warm start of the next one
  DevBuf bu, bphi;
  TRY(ensure(c, bu, G * es));
  TRY(ensure(c, bphi, G * es));
  struct Free {
    DevBuf *a, *b;
    ~Free() {
      cudaFree(a->p);
      cudaFree(b->p);
    }
  } free_bufs{&bu, &bphi};
  const int n = 3 * M;
  std::vector<double> F(n), Ft(n), Rt(n), d(n, 0.0), gold(n, 0.0);
  // a warm start also resumes Algorithm 1 where the previous ground state ended:
  // eta0 = its eta*, mu0 = the last penalty weight it used
  ofdft_params pw = *p;
  auto ground = [&](const double* Rx, double* Ex, double* Fx, bool warm) -> int {
    ofdft_solve_stats st;
    const int rc = ofdft_solve_from(c, &g, Rx, Z, M, h, warm ? &pw : p, warm ? bu.p : nullptr,
                                    warm ? bphi.p : nullptr, bu.p, bphi.p, Ex, Fx, &st);
    rst->solves++;
    rst->cg_iters += st.cg_iters;
    if (rc == OFDFT_OK && p->method == OFDFT_METHOD_AL) {
      pw.eta0 = st.eta;
      pw.mu0 = p->mu0 * pow(p->kappa, std::max(st.outer_iters - 1, 0));
    }
    return rc;
  };
  auto fmax_of = [&](const std::vector<double>& Fx) {
    double m = 0.0;
    for (int J = 0; J < M; ++J)
      m = std::max(m, sqrt(Fx[3 * J] * Fx[3 * J] + Fx[3 * J + 1] * Fx[3 * J + 1] + Fx[3 * J + 2] * Fx[3 * J + 2]));
    return m;
  };
  double E = 0.0;
  TRY(ground(R, &E, F.data(), false));
  double gg_old = 0.0;
  // Polak-Ribiere CG on E(R) with g = -F, a secant step on the directional
  // derivative -F.d between R and a trial geometry whose largest atomic move is
  // max_move, and a halved step when the energy rises
  for (int step = 0; step < max_steps; ++step) {
    rst->max_force = fmax_of(F);
    if (rst->max_force < f_tol) {
      rst->converged = 1;
      break;
    }
    double gg = 0.0, gdg = 0.0;
    for (int i = 0; i < n; ++i) {
      gg += F[i] * F[i];
      gdg += -F[i] * (-F[i] - gold[i]);
    }
    double beta = (step == 0 || gg_old <= 0.0) ? 0.0 : std::max(0.0, gdg / gg_old);
    double dg = 0.0;
    for (int i = 0; i < n; ++i) {
      d[i] = F[i] + beta * d[i];
      dg += -F[i] * d[i];
    }
    if (!(dg < 0.0)) {  // not a descent direction: steepest descent
      for (int i = 0; i < n; ++i) d[i] = F[i];
      dg = -gg;
    }
    for (int i = 0; i < n; ++i) gold[i] = -F[i];
    gg_old = gg;
    double dmax = 0.0;
    for (int J = 0; J < M; ++J)
      dmax = std::max(dmax, sqrt(d[3 * J] * d[3 * J] + d[3 * J + 1] * d[3 * J + 1] + d[3 * J + 2] * d[3 * J + 2]));
    if (!(dmax > 0.0)) break;
    const double a0 = max_move / dmax;
    for (int i = 0; i < n; ++i) Rt[i] = R[i] + a0 * d[i];
    double Et = 0.0;
    TRY(ground(Rt.data(), &Et, Ft.data(), true));
    double g1 = 0.0;
    for (int i = 0; i < n; ++i) g1 += -Ft[i] * d[i];
    // secant on the directional derivative: dg at 0, g1 at a0
    double a = (g1 > dg) ? a0 * dg / (dg - g1) : 2.0 * a0;
    a = std::min(std::max(a, 0.1 * a0), 4.0 * a0);
    for (int i = 0; i < n; ++i) Rt[i] = R[i] + a * d[i];
    double En = 0.0;
    TRY(ground(Rt.data(), &En, Ft.data(), true));
    if (En > E && Et < E) {  // the secant overshot: take the trial geometry instead
      for (int i = 0; i < n; ++i) Rt[i] = R[i] + a0 * d[i];
      TRY(ground(Rt.data(), &En, Ft.data(), true));
    }
    for (int i = 0; i < n; ++i) {
      R[i] = Rt[i];
      F[i] = Ft[i];
    }
    E = En;
    rst->steps++;
  }
  rst->max_force = fmax_of(F);
  if (rst->max_force < f_tol) rst->converged = 1;
  rst->energy = E;
  *energy = E;
  for (int i = 0; i < n; ++i) forces[i] = F[i];
  return rst->converged ? OFDFT_OK : fail(c, OFDFT_ENOTCONV, "relaxation reached %d steps (max force %.3e)",
                                          max_steps, rst->max_force);
}

}  // extern "C"
