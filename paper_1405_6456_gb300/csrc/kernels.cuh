// CUDA kernels of the library (sm_103a).  Every stencil-shaped pass of the
// method (S2 stencil, S3 CG, S4 fused functional) is one instance of the
// z-streaming kernel below with its own loader (what the stencil is applied to)
// and epilogue (what is done with the result at each node).
#pragma once

#include <cuda.h>  // CUtensorMap (the type only; no driver call is made from here)
#include <math.h>

#include <cooperative_groups.h>

#include "common.cuh"

namespace ofd {

constexpr int BX = 32;  // threads along x (one warp per row)
constexpr int BY = 8;   // thread rows per block
constexpr int NT = BX * BY;

// Tile shape of the z-streaming passes per element type: each thread computes
// RY consecutive rows (register blocking: the y-neighbours of its own rows come
// from its registers, and the staging and synchronisation of a plane are shared
// by RY outputs), so a block covers BX x TY nodes.  ZD = planes staged ahead of
// use.  FP64 takes fewer rows and a shallower pipeline to keep two blocks per SM.
template <typename T>
struct ZCfg {
  static constexpr int CX = sizeof(T) == 4 ? 2 : 1;  // adjacent columns per thread (packed FP32 pairs)
  static constexpr int RY = 2;                       // rows per thread
  static constexpr int THX = BX / CX;                // threads along a tile row
  static constexpr int TY = (NT / THX) * RY;         // rows per tile
  static constexpr int ZD = sizeof(T) == 4 ? 3 : 2;
};

// Double-float32 ("float-float") numbers: an unevaluated sum hi + lo of two
// floats with |lo| <= ulp(hi) / 2, about 48 significant bits.  Error-free
// transformations: Knuth's TwoSum for the sum of two floats, Dekker's Fast2Sum
// to renormalise, and the FMA for the exact rounding error of a product
// (Dekker 1971; Hida, Li and Bailey 2001 for the double-double forms these
// follow).  Every operation runs on the FP32 pipes, which on this GPU issue at
// many times the FP64 rate; an add or multiply has an absolute error of a few
// units of 2^-48 of its operands' magnitudes.
__device__ __forceinline__ float2 ff_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return make_float2(s, (a - (s - bb)) + (b - bb));
}
__device__ __forceinline__ float2 ff_fast_two_sum(float a, float b) {  // needs |a| >= |b| or a == 0
  const float s = a + b;
  return make_float2(s, b - (s - a));
}
__device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
  const float2 s = ff_two_sum(a.x, b.x);
  return ff_fast_two_sum(s.x, s.y + (a.y + b.y));
}
__device__ __forceinline__ float2 ff_mul(float2 w, float2 a) {
  const float p = w.x * a.x;
  float e = fmaf(w.x, a.x, -p);  // exact rounding error of w.hi a.hi
  e = fmaf(w.x, a.y, fmaf(w.y, a.x, e));
  return ff_fast_two_sum(p, e);
}
// The same without the closing renormalisation: the pair stays an unevaluated
// sum hi + lo whose lo may exceed ulp(hi) / 2 by the few roundings of the
// chain it came from.  TwoSum and the FMA product are exact for any operands,
// so a chain of these keeps the error bound of the normalised forms (a few
// units of 2^-48 of its terms per operation) while skipping a Fast2Sum per
// step; the chain's result is renormalised once, with a TwoSum.
__device__ __forceinline__ float2 ff_add_lazy(float2 a, float2 b) {
  const float2 s = ff_two_sum(a.x, b.x);
  return make_float2(s.x, s.y + (a.y + b.y));
}
__device__ __forceinline__ float2 ff_mul_lazy(float2 w, float2 a) {
  const float p = w.x * a.x;
  const float e = fmaf(w.x, a.x, -p);
  return make_float2(p, fmaf(w.x, a.y, fmaf(w.y, a.x, e)));
}

template <typename T>
__host__ __device__ __forceinline__ T zero_of() { return T(0); }
template <>
__host__ __device__ __forceinline__ float2 zero_of<float2>() { return make_float2(0.0f, 0.0f); }

// Arithmetic on a thread's CX adjacent columns: one FP64 value, or an FP32 pair
// computed with the packed FP32x2 instructions (each lane rounds as the scalar
// operation does, so results equal the one-column code's bit for bit).
template <typename T, int CX>
struct Lanes;
template <typename T>
struct Lanes<T, 1> {
  using V = T;
  __device__ static V ld(const T* p) { return *p; }
  __device__ static V add(V a, V b) { return a + b; }
  __device__ static V mul(T w, V a) { return w * a; }
  __device__ static V fma(T w, V a, V c) { return ::fma(w, a, c); }
  __device__ static V make(const T* v) { return v[0]; }
  __device__ static T lane(V v, int) { return v; }
};
// float-float values (float2 = hi, lo), one column per thread; the stencil's
// sums run unnormalised (the lazy forms) and the consumer renormalises the
// result once
template <>
struct Lanes<float2, 1> {
  using V = float2;
  __device__ static V ld(const float2* p) { return *p; }
  __device__ static V add(V a, V b) { return ff_add_lazy(a, b); }
  __device__ static V mul(float2 w, V a) { return ff_mul_lazy(w, a); }
  __device__ static V fma(float2 w, V a, V c) { return ff_add_lazy(ff_mul_lazy(w, a), c); }
  __device__ static V make(const float2* v) { return v[0]; }
  __device__ static float2 lane(V v, int) { return v; }
};
template <>
struct Lanes<float, 2> {
  using V = float2;
  __device__ static V ld(const float* p) { return *reinterpret_cast<const float2*>(p); }
  __device__ static V add(V a, V b) { return __fadd2_rn(a, b); }
  __device__ static V mul(float w, V a) { return __fmul2_rn(make_float2(w, w), a); }
  __device__ static V fma(float w, V a, V c) { return __ffma2_rn(make_float2(w, w), a, c); }
  __device__ static V make(const float* v) { return make_float2(v[0], v[1]); }
  __device__ static float lane(V v, int l) { return l == 0 ? v.x : v.y; }
};

// ---------------------------------------------------------------------------
// Device scalars of one CG solve (S3).  Written only by the last block of a
// reduction, read by every thread of the next kernel.
struct CgScalars {
  double rr;      // r.r of the current residual
  double bb;      // ||4 pi rho||^2
  double pAp;     // p.(A p)
  double alpha;   // rr / pAp
  double beta;    // rr_new / rr
  double tol2;    // tol^2 (relative, squared)
  double sum_uu;  // sum u^2 (from the residual pass, for C_h)
  double rr0;     // rr at the start of the solve (or at the last residual replacement)
  double rr_prev; // r.r of the previous iteration (beta after a residual replacement)
  int iters;      // CG iterations done
  int max_it;
  int done;       // 1 once converged or out of iterations
  int first;      // 1 until the first search direction is formed
  int xdefer;     // 1 while x += alpha p of the last iteration is still to be applied
  int err;        // 1 when a grid barrier of the persistent CG kernel timed out
  int pc;         // 1: preconditioned CG (alpha = rz / pAp, beta from the preconditioner pass)
  double rz;      // r.z of the preconditioned residual z = M r (PCG)
  double es_rho_phi;  // sum (u^2 + b) phi at the residual pass's phi (float-float residual pass)
  double es_phi_r;    // sum phi r, r the residual it writes
};

// ---------------------------------------------------------------------------
// z-streaming radius-R star stencil (Sec. 4, Eq. FD:Laplacian).
//
// A block owns a BX x TY column of nodes and a z-range [z0, z1).  It walks the
// range one plane at a time: the plane (with an R-wide x/y halo) is staged in
// shared memory, the 2R+1 values of the block's own column along z live in a
// register queue, so every node's 6R neighbours come from shared memory or
// registers.  Every index outside the grid reads 0 (zero Dirichlet, Sec. 4).
//
// Loader: T value(idx) (pure; used for halo nodes and for nodes of other
//         z-ranges) and T own(idx) (called once per node of this block's range;
//         may store a side product, e.g. the new CG direction).
// Epi:    static constexpr int K (number of FP64 partial sums), bool skip(),
//         void apply(idx, centre, lap, acc[K]), and fin(sums[K]) run once by
//         the last block.
// Epilogue accumulators: plain doubles, or DotAcc (compensated for FP32).
__device__ __forceinline__ double to_double(double v) { return v; }
template <typename T>
__device__ __forceinline__ double to_double(const DotAcc<T>& a) { return a.value(); }

// Accumulator of the functional pass's sums: plain FP64 for FP64 fields; for
// FP32 fields the compensated FP32 pair of DotAcc (no FP64 arithmetic per node),
// with add_d for the terms formed in FP64 (the electrostatic sums of MIXED).
template <typename T>
struct FAcc;
template <>
struct FAcc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double a, double b) { s += a * b; }
  __device__ __forceinline__ void add_fast(double a, double b) { s += a * b; }
  __device__ __forceinline__ void add_d(double v) { s += v; }
  __device__ __forceinline__ double value() const { return s; }
};
template <>
struct FAcc<float> {
  DotAcc<float> a;
  __device__ __forceinline__ void add(float x, float y) { a.add(x, y); }
  // plain FP32 accumulation (one FMA) for sums that only steer the line search
  // and the stopping tests, where the FP32 relative accuracy of a thread's
  // partial sum is enough; the pair's low part stays zero
  __device__ __forceinline__ void add_fast(float x, float y) { a.hi = fmaf(x, y, a.hi); }
  __device__ __forceinline__ void add_d(double v) {
    const float hi = (float)v;
    a.add(hi, 1.0f);
    a.add((float)(v - (double)hi), 1.0f);
  }
  __device__ __forceinline__ double value() const { return a.value(); }
};
template <typename T>
__device__ __forceinline__ double to_double(const FAcc<T>& a) { return a.value(); }

// Asynchronous global -> shared copy of BYTES = 4, 8 or 16 bytes (16: both
// addresses 16-byte aligned; bypasses L1).  src_valid == false fills the
// destination with zeros (the zero Dirichlet value of every out-of-grid node)
// and reads nothing.
template <int BYTES>
__device__ __forceinline__ void cp_async_bytes(void* dst, const void* src, bool src_valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int n = src_valid ? BYTES : 0;
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
  else if constexpr (BYTES == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Staging granularity V (elements per copy): 1, or 16 / sizeof(T) when the
// grid's rows and the arrays are 16-byte aligned (zvec_ok).  The x-halo is
// staged RA = R rounded up to a multiple of V and of CX wide, so a staged row is
// BX + 2 RA elements, every copy stays aligned and a thread's column pair starts
// on an even element.
template <typename T, int R, int V>
constexpr int zhalo_x() {
  constexpr int m = V > ZCfg<T>::CX ? V : ZCfg<T>::CX;
  return ((R + m - 1) / m) * m;
}
// Shared-memory ring of R + ZD stencil planes (tile plus x/y halo).
template <typename T, int R, int V>
constexpr int zring_bytes() {
  return (R + ZCfg<T>::ZD) * (ZCfg<T>::TY + 2 * R) * (BX + 2 * zhalo_x<T, R, V>()) * (int)sizeof(T);
}
// TMA staging applies when every staged slot starts on a 128-byte boundary:
// FP32, 16-byte vectors, and a slot size that is a multiple of 128 bytes.
template <typename T, int R, int V>
constexpr bool ztma_fits() {
  return sizeof(T) == 4 && V == 4 &&
         ((ZCfg<T>::TY + 2 * R) * (BX + 2 * zhalo_x<T, R, V>()) * (int)sizeof(T)) % 128 == 0;
}
// Dynamic shared memory of a z-streaming pass: the stencil-input ring plus a
// ring of ZD planes for each pointwise input the epilogue declares (NIN).
template <typename T, int R, int V, class Epi>
constexpr int zsmem_bytes() {
  return zring_bytes<T, R, V>() + ZCfg<T>::ZD * Epi::NIN * ZCfg<T>::TY * BX * (int)sizeof(T);
}

// ---------------------------------------------------------------------------
// TMA staging (the tensor memory accelerator of sm_100-class GPUs): one thread
// issues a tiled bulk copy of a whole staged plane (tile plus halo) from a
// tensor map, the hardware fills every out-of-grid element with zero (the zero
// Dirichlet values) and signals an mbarrier when the bytes have landed; the
// other threads wait on that barrier.  Every wait is bounded: if a copy never
// arrives the waiting thread raises zstream_fault and carries on, and the host
// reports OFDFT_ETIMEOUT.
__device__ int zstream_fault;

struct ZTmaMaps {
  const CUtensorMap* f;      // stencil input: box {SX, SY, 1}
  const CUtensorMap* in[3];  // epilogue inputs: box {BX, TY, 1}
};

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for phase `parity` of bar to complete, at most ~2^22 polls.
__device__ __forceinline__ void mbar_wait_bounded(unsigned long long* bar, unsigned parity) {
  for (int i = 0; i < (1 << 22); ++i)
    if (mbar_try_wait(bar, parity)) return;
  atomicExch(&zstream_fault, 1);
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];\n" ::"r"(smem_addr(dst)),
      "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
      : "memory");
}

// One block's share of a z-streaming pass: tile (bx, by) of BX x TY columns,
// planes [z0, z1).  Planes are staged (tile plus an R-wide x/y halo) in a
// shared-memory ring of R + ZD slots by cp.async, ZD planes ahead of use; each
// thread owns CX adjacent columns times RY rows, whose values along z live in
// register queues fed from the ring.  No register ever holds an in-flight load,
// so global latency overlaps compute.  The staging work is a flat list over the
// staged plane whose in-plane offsets and validity each thread computes once;
// per plane only the plane offset changes.  nblocks / bid describe the reduction
// this block takes part in (the whole grid for a single solve, one grid of a
// batch otherwise).  f is the stencil input.  The epilogue's NIN pointwise
// inputs (ep.input(j)) at the block's own nodes travel in the same pipeline, so
// the epilogue never waits on a global load.  In-plane offsets are 32-bit
// (n1 * n2 < 2^31).
template <typename T, int R, int V, class Epi, bool TMA = false>
__device__ __forceinline__ void zstream_tile(const GridDev& g, const Weights<T>& W, int bx, int by, int z0, int z1,
                                             const T* __restrict__ f, const Epi& ep_in, const RedBuf& red,
                                             int nblocks, int bid, double* block_out = nullptr,
                                             const ZTmaMaps* tm = nullptr) {
  Epi ep = ep_in;  // block-local copy: load() caches the epilogue's device scalars in registers
  constexpr int CX = ZCfg<T>::CX, RY = ZCfg<T>::RY, THX = ZCfg<T>::THX, TY = ZCfg<T>::TY, ZD = ZCfg<T>::ZD;
  using L = Lanes<T, CX>;
  using VT = typename L::V;
  constexpr int NS = R + ZD;
  constexpr int RA = zhalo_x<T, R, V>();
  constexpr int SY = TY + 2 * R, SX = BX + 2 * RA, SP = SY * SX;
  constexpr int CH = SX / V;                 // copies per staged row
  constexpr int NE = (SY * CH + NT - 1) / NT;  // stencil copies per thread and plane
  constexpr int ICH = TY * BX / V;           // copies per input plane
  constexpr int NI = ICH / NT;               // input copies per thread, input and plane
  constexpr int NIN = Epi::NIN;
  constexpr int RE = ((R + CX - 1) / CX) * CX;  // x-window half width (a multiple of CX)
  constexpr int NWIN = 2 * RE + CX;             // x-window of a row: columns x0 - RE .. x0 + CX - 1 + RE
  static_assert(NE <= 32 && NI * (NIN > 0 ? NIN : 1) <= 32, "staging masks hold 32 entries");
  static_assert(ICH % NT == 0, "input planes split evenly over the threads");
  static_assert(RE <= RA, "the x-window stays inside the staged halo");
  static_assert(!TMA || (sizeof(T) == 4 && V == 4), "TMA staging: FP32 fields with 16-byte rows");
  extern __shared__ __align__(128) unsigned char zsm_raw[];
  __shared__ __align__(8) unsigned long long zbar[TMA ? R + ZCfg<T>::ZD : 1];  // one barrier per ring slot
  unsigned zphase = 0;  // bit s: parity of ring slot s's next completion
  // TMA destinations must be 128-byte aligned: the launch adds 128 bytes of room
  unsigned char* zsm = zsm_raw;
  if constexpr (TMA) zsm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(zsm_raw) + 127) & ~uintptr_t(127));
  T(*ring)[SP] = reinterpret_cast<T(*)[SP]>(zsm);
  T(*pin)[NIN > 0 ? NIN : 1][TY * BX] =
      reinterpret_cast<T(*)[NIN > 0 ? NIN : 1][TY * BX]>(zsm + zring_bytes<T, R, V>());
  __shared__ double red_smem[(Epi::K > 0 ? Epi::K : 1) * (NT / 32)];
  const int tid = threadIdx.y * BX + threadIdx.x;
  const int tx = tid % THX, ty = tid / THX;  // column group and row group of this thread
  const int x0 = bx * BX + CX * tx, y0 = by * TY + ty * RY;  // first column and first row
  const long long plane = (long long)g.n1 * g.n2;
  unsigned node_ok = 0;  // bit i * CX + l: node (x0 + l, y0 + i) is inside the grid
#pragma unroll
  for (int i = 0; i < RY; ++i)
#pragma unroll
    for (int l = 0; l < CX; ++l)
      if (x0 + l < g.n1 && y0 + i < g.n2) node_ok |= 1u << (i * CX + l);

  // this thread's share of a staged plane: copies e = tid + j NT of V
  // elements, row e / CH and column V (e % CH) of the SY x SX tile-with-halo
  // (shared offset V e), at in-plane offset soff[j] when inside the grid.  A
  // copy lies wholly inside or wholly outside the grid (n1 % V == 0).
  int soff[NE];
  unsigned smask = 0;
#pragma unroll
  for (int j = 0; j < NE; ++j) {
    const int e = tid + j * NT;
    const int sy = e / CH, cx = e - sy * CH;
    const int gx = bx * BX - RA + cx * V, gy = by * TY - R + sy;
    const bool ok = e < SY * CH && gx >= 0 && gx + V <= g.n1 && gy >= 0 && gy < g.n2;
    soff[j] = ok ? gy * g.n1 + gx : 0;
    if (ok) smask |= 1u << j;
  }
  // and of each epilogue input plane: copies e = tid + m NT of the TY x BX tile
  int ioff[NI > 0 ? NI : 1];
  unsigned imask = 0;
#pragma unroll
  for (int m = 0; m < NI; ++m) {
    const int e = tid + m * NT;
    const int row = e / (BX / V), cx = e - row * (BX / V);
    const int gx = bx * BX + cx * V, gy = by * TY + row;
    const bool ok = gx + V <= g.n1 && gy < g.n2;
    ioff[m] = ok ? gy * g.n1 + gx : 0;
    if (ok) imask |= 1u << m;
  }

  // stage plane p into ring slot sl and (for p - R inside the chunk) the
  // epilogue inputs of plane p - R into input slot isl; one commit group per call
  auto stage = [&](int p, int sl, int isl) {
    if constexpr (TMA) {
      if (tid == 0) {
        const int pp = p - R;
        const bool inputs = NIN > 0 && pp >= z0 && pp < z1;
        // the slot was last read through the generic proxy (ordered by the
        // caller's __syncthreads); order those reads before the async writes
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        mbar_expect_tx(&zbar[sl], (unsigned)(SP * sizeof(T) + (inputs ? NIN * TY * BX * sizeof(T) : 0)));
        tma_load_3d(ring[sl], tm->f, bx * BX - RA, by * TY - R, p, &zbar[sl]);
        if constexpr (NIN > 0) {
          if (inputs)
#pragma unroll
            for (int j = 0; j < NIN; ++j) tma_load_3d(&pin[isl][j][0], tm->in[j], bx * BX, by * TY, pp, &zbar[sl]);
        }
      }
      return;
    }
    const bool pv = (p >= 0) && (p < g.n3);
    const T* fp = f + plane * (long long)(pv ? p : 0);
    T* dst = ring[sl];
#pragma unroll
    for (int j = 0; j < NE; ++j) {
      const int e = tid + j * NT;
      if (j < NE - 1 || e < SY * CH) {
        const bool ok = pv && ((smask >> j) & 1u);
        cp_async_bytes<V * (int)sizeof(T)>(dst + V * e, ok ? fp + soff[j] : f, ok);
      }
    }
    if constexpr (NIN > 0) {
      const int pp = p - R;
      if (pp >= z0 && pp < z1) {
        const long long o = plane * (long long)pp;
#pragma unroll
        for (int j = 0; j < NIN; ++j) {
          const T* src = ep.input(j);
#pragma unroll
          for (int m = 0; m < NI; ++m) {
            const bool v = ((imask >> m) & 1u) && src != nullptr;
            cp_async_bytes<V * (int)sizeof(T)>(&pin[isl][j][V * (tid + m * NT)], v ? src + o + ioff[m] : f, v);
          }
        }
      }
    }
    cp_async_commit();
  };

  // register queues of the own nodes along z (planes k-R .. k+R); the planes
  // below the chunk and the first R of it come from plain loads
  VT q[RY][2 * R + 1];
#pragma unroll
  for (int i = 0; i < RY; ++i)
#pragma unroll
    for (int m = 0; m < 2 * R; ++m) {
      const int kk = z0 - R + m;
      T v[CX];
#pragma unroll
      for (int l = 0; l < CX; ++l)
        v[l] = (((node_ok >> (i * CX + l)) & 1u) && kk >= 0 && kk < g.n3)
                   ? __ldcg(&f[(long long)g.n1 * (y0 + i) + x0 + l + plane * kk])  // L2: other blocks may have written it
                   : zero_of<T>();
      q[i][m] = L::make(v);
    }
  // ring slots advance by one per plane (no integer division in the loop):
  // stencil plane p lives in slot (p - z0) mod NS, input plane p in (p - z0) mod ZD
  int s_stage = 0, i_stage = (ZD - R % ZD) % ZD;
  auto bump = [](int v, int n) { return v + 1 == n ? 0 : v + 1; };
  if constexpr (TMA) {
    if (tid == 0) {
#pragma unroll
      for (int sl = 0; sl < NS; ++sl) mbar_init(&zbar[sl], 1);
      asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
  }
  // waits (TMA staging) for the copies of the slots a block issued but never
  // consumed, so that no copy lands after the block has exited
  auto drain = [&](int first_plane, int count) {
    if constexpr (TMA) {
      for (int p = first_plane; p < first_plane + count; ++p) {
        const int sl = (p - z0) % NS;
        mbar_wait_bounded(&zbar[sl], (zphase >> sl) & 1u);
        zphase ^= 1u << sl;
      }
    }
  };
  for (int p = z0; p < z0 + R + ZD - 1; ++p) {
    stage(p, s_stage, i_stage);
    s_stage = bump(s_stage, NS);
    i_stage = bump(i_stage, ZD);
  }

  // the epilogue's device scalars (and whether the pass has anything to do)
  // are read while the first planes are in flight
  if (ep.skip()) {
    cp_async_wait<0>();  // no copy may land in shared memory after the block exits
    drain(z0, R + ZD - 1);
    return;
  }
  ep.load();
  // TMA: the first R planes of the chunk are read (as plane k) before the loop
  // waits on them as plane k + R, so wait for them here; the loop then waits for
  // planes z0 + R .. z1 - 1 + R and the end for the rest
  drain(z0, R);

  typename Epi::Acc acc[Epi::K > 0 ? Epi::K : 1];
#pragma unroll
  for (int i = 0; i < (Epi::K > 0 ? Epi::K : 1); ++i) acc[i] = typename Epi::Acc();

  const int cb = ty * RY * SX + CX * tx + RA;  // ring offset of this thread's first column, lowest y-halo row
  int sk = 0, sf = R % NS, ik = 0;            // slots of plane k, plane k + R, inputs of plane k
  for (int k = z0; k < z1; ++k) {
    __syncthreads();                          // every thread is done with plane k-1's slot
    stage(k + R + ZD - 1, s_stage, i_stage);  // refills that slot
    s_stage = bump(s_stage, NS);
    i_stage = bump(i_stage, ZD);
    if constexpr (TMA) {
      mbar_wait_bounded(&zbar[sf], (zphase >> sf) & 1u);  // plane k + R and the inputs of plane k
      zphase ^= 1u << sf;
    } else {
      cp_async_wait<ZD - 1>();  // planes <= k + R have landed (this thread's copies)
      __syncthreads();          // ... and every other thread's
    }
    const T* pk = ring[sk] + cb;  // (row offset m, first column) of plane k at pk[m * SX]
#pragma unroll
    for (int i = 0; i < RY; ++i) q[i][2 * R] = L::ld(ring[sf] + cb + (i + R) * SX);
    // y-neighbours: the R rows below and above the own rows in plane k; the own
    // rows' values are q[i][R]
    auto ycol = [&](int m) -> VT { return (m >= R && m < RY + R) ? q[m - R][R] : L::ld(pk + m * SX); };
    // nodes outside the grid read zeros and are computed but not applied
    VT lap[RY];
#pragma unroll
    for (int i = 0; i < RY; ++i) lap[i] = L::mul(W.c, q[i][R]);
#pragma unroll
    for (int i = 0; i < RY; ++i) {
      // x-window of row i: columns x0 - RE .. x0 + CX - 1 + RE (the centre is q[i][R])
      const T* row = pk + (i + R) * SX;
      T win[NWIN];
#pragma unroll
      for (int c = 0; c < NWIN; c += CX) {
        if (CX == 1 && c == RE) continue;
        const VT t = L::ld(row + c - RE);
#pragma unroll
        for (int l = 0; l < CX; ++l) win[c + l] = L::lane(t, l);
      }
      // one weighted sum per axis: three independent FMA chains per row
      VT ax = L::mul(W.w[1], L::add(L::make(win + RE + 1), L::make(win + RE - 1)));
      VT ay = L::mul(W.w[1], L::add(ycol(i + R + 1), ycol(i + R - 1)));
      VT az = L::mul(W.w[1], L::add(q[i][R + 1], q[i][R - 1]));
#pragma unroll
      for (int p = 2; p <= R; ++p) {
        ax = L::fma(W.w[p], L::add(L::make(win + RE + p), L::make(win + RE - p)), ax);
        ay = L::fma(W.w[p], L::add(ycol(i + R + p), ycol(i + R - p)), ay);
        az = L::fma(W.w[p], L::add(q[i][R + p], q[i][R - p]), az);
      }
      lap[i] = L::add(L::add(L::add(lap[i], ax), ay), az);
    }
    const long long base = plane * k + (long long)g.n1 * y0 + x0;
#pragma unroll
    for (int i = 0; i < RY; ++i)
#pragma unroll
      for (int l = 0; l < CX; ++l) {
        if ((node_ok >> (i * CX + l)) & 1u) {
          T vin[NIN > 0 ? NIN : 1];
#pragma unroll
          for (int j = 0; j < NIN; ++j) vin[j] = pin[ik][j][(ty * RY + i) * BX + CX * tx + l];
          ep.apply(base + (long long)g.n1 * i + l, L::lane(q[i][R], l), L::lane(lap[i], l), vin, acc);
        }
      }
#pragma unroll
    for (int i = 0; i < RY; ++i)
#pragma unroll
      for (int m = 0; m < 2 * R; ++m) q[i][m] = q[i][m + 1];
    sk = bump(sk, NS);
    sf = bump(sf, NS);
    ik = bump(ik, ZD);
  }
  cp_async_wait<0>();
  drain(z1 + R, ZD - 1);
  if constexpr (Epi::K > 0) {
    double accd[Epi::K];
#pragma unroll
    for (int i = 0; i < Epi::K; ++i) accd[i] = to_double(acc[i]);
    if (block_out) {  // the block's sums only (valid in thread 0); the caller combines blocks
      block_sum<Epi::K, NT>(accd, red_smem, tid);
      if (tid == 0)
#pragma unroll
        for (int i = 0; i < Epi::K; ++i) block_out[i] = accd[i];
      return;
    }
    Epi fin = ep;
    grid_sum<Epi::K, NT>(accd, red_smem, red, nblocks, bid, tid, fin);
  }
}

// ---------------------------------------------------------------------------
// Persistent CG (S3) for one grid: a cooperative launch whose blocks (all
// co-resident) run up to niter CG iterations, each the z-streaming pass on r
// (q = A r + beta q, p = r + beta p, p.q) and the x / r update of the block's
// own nodes (r.r), with a grid-wide sum after each half.  Every block sums the
// blocks' partials in the same order, so all blocks hold identical alpha, beta
// and convergence decisions without a second pass; block 0 publishes the CG
// scalars for the host.  Saves the launch gaps and the separate update kernel
// of the two-kernel iteration.

// CG epilogue with beta and `first` given as values (no device scalars).
template <typename T>
struct EpiCgAv {
  static constexpr int K = 1;
  static constexpr int NIN = 2;
  using Acc = DotAcc<T>;
  T* p;
  T* q;
  int first_;
  T beta_;
  __device__ __forceinline__ bool skip() const { return false; }
  __device__ __forceinline__ void load() {}
  __host__ __device__ __forceinline__ const T* input(int j) const { return j == 0 ? p : q; }
  __device__ __forceinline__ void apply(long long i, T rc, T ar, const T* vin, Acc* acc) const {
    T pc, qc;
    if (first_) {
      pc = rc;
      qc = ar;
    } else {
      pc = fma(beta_, vin[0], rc);
      qc = fma(beta_, vin[1], ar);
    }
    p[i] = pc;
    q[i] = qc;
    acc[0].add(pc, qc);
  }
  __device__ __forceinline__ void operator()(double*) const {}
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide sum over co-resident blocks: each block's thread 0 publishes the
// block total `v` (valid in thread 0), arrives at a counting barrier and waits
// (at most ~2 s, then raises *err); afterwards every block sums all partials in
// block order.  Returns the total in every thread; false after a timeout.
// `bar` counts arrivals over the whole solve (reset by the host before it), so
// the target of this barrier is the next multiple of nblocks.
template <int NT>
__device__ __forceinline__ bool coop_sum(double& v, double* smem, double* partials, unsigned int* bar, int* err,
                                         int nblocks, int bid, int tid) {
  __shared__ int ok_s;
  __shared__ double tot_s;
  if (tid == 0) {
    partials[bid] = v;
    __threadfence();
    const unsigned int t = atomicAdd(bar, 1u);
    const unsigned int target = (t / (unsigned)nblocks + 1u) * (unsigned)nblocks;
    const unsigned long long t0 = global_ns();
    int ok = 1;
    while ((int)(*(volatile unsigned int*)bar - target) < 0) {
      if (*(volatile int*)err || global_ns() - t0 > 2000000000ull) {
        atomicExch(err, 1);
        ok = 0;
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  double t[1] = {0.0};
  for (int b = tid; b < nblocks; b += NT) t[0] += __ldcg(&partials[b]);
  block_sum<1, NT>(t, smem, tid);
  if (tid == 0) tot_s = t[0];
  __syncthreads();
  v = tot_s;
  const bool ok = ok_s != 0;
  __syncthreads();
  return ok;
}

template <typename T, int R, int V>
__global__ void __launch_bounds__(NT, 2) cg_coop_kernel(GridDev g, Weights<T> W, int zchunk, T* __restrict__ x,
                                                        T* __restrict__ r, T* __restrict__ p, T* __restrict__ q,
                                                        CgScalars* sc, double* partials, unsigned int* bar,
                                                        int niter) {
  constexpr int CX = ZCfg<T>::CX, RY = ZCfg<T>::RY, THX = ZCfg<T>::THX, TY = ZCfg<T>::TY;
  __shared__ double smem[NT / 32];
  const int nblocks = gridDim.x * gridDim.y * gridDim.z;
  const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  const int tid = threadIdx.y * BX + threadIdx.x;
  const int z0 = blockIdx.z * zchunk, z1 = min(z0 + zchunk, g.n3);
  // the CG state, identical in every block (all read it before any block writes)
  double rr = sc->rr, beta = sc->beta, tol2 = sc->tol2, bb = sc->bb, alpha = sc->alpha, pAp = sc->pAp;
  int first = sc->first, iters = sc->iters, max_it = sc->max_it, done = sc->done;
  const double thr = tol2 * (bb > 0.0 ? bb : 1.0);
  __syncthreads();
  int* err = &sc->err;
  double* partA = partials;            // p.q of the blocks
  double* partB = partials + nblocks;  // r.r of the blocks
  const int tx = tid % THX, ty = tid / THX;
  const int x0 = blockIdx.x * BX + CX * tx, y0 = blockIdx.y * TY + ty * RY;
  const long long plane = (long long)g.n1 * g.n2;
  bool ok = true;
  for (int it = 0; it < niter && !done && ok; ++it) {
    // first half: the stencil pass
    double v = 0.0;
    zstream_tile<T, R, V>(g, W, blockIdx.x, blockIdx.y, z0, z1, r, EpiCgAv<T>{p, q, first, (T)beta}, RedBuf{},
                          nblocks, bid, &v);
    ok = coop_sum<NT>(v, smem, partA, bar, err, nblocks, bid, tid);
    if (!ok) break;
    pAp = v;
    alpha = (pAp != 0.0) ? rr / pAp : 0.0;
    first = 0;
    // second half: x += alpha p, r -= alpha q on this block's own nodes
    const T al = (T)alpha;
    DotAcc<T> dacc;
    for (int k = z0; k < z1; ++k)
#pragma unroll
      for (int i = 0; i < RY; ++i) {
        const int y = y0 + i;
        if (y >= g.n2) continue;
        const long long o = plane * k + (long long)g.n1 * y;
#pragma unroll
        for (int l = 0; l < CX; ++l) {
          const int xx = x0 + l;
          if (xx < g.n1) {
            const T xi = fma(al, p[o + xx], x[o + xx]);
            const T ri = fma(-al, q[o + xx], r[o + xx]);
            x[o + xx] = xi;
            r[o + xx] = ri;
            dacc.add(ri, ri);
          }
        }
      }
    double w[1] = {dacc.value()};
    block_sum<1, NT>(w, smem, tid);
    v = w[0];
    ok = coop_sum<NT>(v, smem, partB, bar, err, nblocks, bid, tid);
    if (!ok) break;
    const double rr_new = v;
    beta = (rr != 0.0) ? rr_new / rr : 0.0;
    const double rr_prev = rr;
    rr = rr_new;
    iters += 1;
    if (rr_new <= thr || iters >= max_it || !(rr_new == rr_new)) done = 1;
    if (bid == 0 && tid == 0) {
      sc->pAp = pAp;
      sc->alpha = alpha;
      sc->first = 0;
      sc->beta = beta;
      sc->rr_prev = rr_prev;
      sc->rr = rr;
      sc->iters = iters;
      sc->done = done;
    }
  }
}

// Single grid: blocks tile (x, y) and split z into chunks of `zchunk` planes.
template <typename T, int R, int V, class Loader, class Epi>
__global__ void __launch_bounds__(NT, 2) zstream_kernel(GridDev g, Weights<T> W, int zchunk,
                                                     Loader ld, Epi ep, RedBuf red) {
  pdl_enter();
  const int z0 = blockIdx.z * zchunk;
  const int z1 = min(z0 + zchunk, g.n3);
  const int nblocks = gridDim.x * gridDim.y * gridDim.z;
  const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  zstream_tile<T, R, V>(g, W, blockIdx.x, blockIdx.y, z0, z1, ld.f, ep, red, nblocks, bid);
}

// Single grid with TMA staging (FP32, rows of whole 16-byte vectors): the
// tensor maps travel as kernel parameters.
template <typename T, int R, int V, class Loader, class Epi>
__global__ void __launch_bounds__(NT, 2) zstream_tma_kernel(const __grid_constant__ CUtensorMap tmf,
                                                            const __grid_constant__ CUtensorMap tm0,
                                                            const __grid_constant__ CUtensorMap tm1,
                                                            const __grid_constant__ CUtensorMap tm2, GridDev g,
                                                            Weights<T> W, int zchunk, Loader ld, Epi ep, RedBuf red) {
  pdl_enter();
  const int z0 = blockIdx.z * zchunk;
  const int z1 = min(z0 + zchunk, g.n3);
  const int nblocks = gridDim.x * gridDim.y * gridDim.z;
  const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  const ZTmaMaps maps{&tmf, {&tm0, &tm1, &tm2}};
  zstream_tile<T, R, V, Epi, true>(g, W, blockIdx.x, blockIdx.y, z0, z1, ld.f, ep, red, nblocks, bid, nullptr,
                                   &maps);
}

// Batched: uneven grids packed into one launch (S11).  Block b works on
// tiles[b] of grid slots[tiles[b].slot]; each grid reduces into its own scratch.
struct ZTile {
  int slot, bx, by, z0, z1, bid;
};

template <typename T, class Loader, class Epi>
struct ZSlot {
  GridDev g;
  Weights<T> W;
  Loader ld;
  Epi ep;
  RedBuf red;
  int nblocks;
};

template <typename T, int R, int V, class Loader, class Epi>
__global__ void __launch_bounds__(NT, 2) zbatch_kernel(const ZTile* __restrict__ tiles,
                                                    const ZSlot<T, Loader, Epi>* __restrict__ slots) {
  const ZTile t = tiles[blockIdx.x];
  const ZSlot<T, Loader, Epi>* S = slots + t.slot;
  const GridDev g = S->g;
  const Weights<T> W = S->W;
  const Epi ep = S->ep;
  const RedBuf red = S->red;
  zstream_tile<T, R, V>(g, W, t.bx, t.by, t.z0, t.z1, S->ld.f, ep, red, S->nblocks, t.bid);
}

// Batched pointwise pass: block b works on elements [begin, end) of grid
// segs[b].slot with that grid's operation; per-grid deterministic reductions.
struct PSeg {
  int slot;
  int bid;
  long long begin, end;
};

template <class Op>
__global__ void __launch_bounds__(256) pbatch_kernel(const PSeg* __restrict__ segs, const Op* __restrict__ ops) {
  const PSeg sg = segs[blockIdx.x];
  Op op = ops[sg.slot];
  if (op.skip()) return;
  op.load();  // the op's device scalars, once per block
  __shared__ double smem[(Op::K > 0 ? Op::K : 1) * (256 / 32)];
  typename Op::Acc acc[Op::K > 0 ? Op::K : 1];
#pragma unroll
  for (int i = 0; i < (Op::K > 0 ? Op::K : 1); ++i) acc[i] = typename Op::Acc();
  for (long long i = sg.begin + threadIdx.x; i < sg.end; i += 256) op.apply(i, acc);
  if constexpr (Op::K > 0) {
    double accd[Op::K];
#pragma unroll
    for (int i = 0; i < Op::K; ++i) accd[i] = to_double(acc[i]);
    Op fin = op;
    grid_sum<Op::K, 256>(accd, smem, op.red, op.nblocks, sg.bid, threadIdx.x, fin);
  }
}

// ----------------------------------------------------------------- loaders --
template <typename T>
struct LoadPlain {
  const T* f;
  __device__ __forceinline__ T value(long long i) const { return f[i]; }
  __device__ __forceinline__ T own(long long i) const { return f[i]; }
};

// ---------------------------------------------------------------- epilogues --
// out = lap (S2).
template <typename T>
struct EpiStore {
  static constexpr int K = 0;
  static constexpr int NIN = 0;
  using Acc = double;
  T* out;
  __device__ __forceinline__ bool skip() const { return false; }
  __device__ __forceinline__ void load() {}
  __host__ __device__ __forceinline__ const T* input(int) const { return nullptr; }
  __device__ __forceinline__ void apply(long long i, T, T lap, const T*, Acc*) const { out[i] = lap; }
  __device__ __forceinline__ void operator()(double*) const {}
};

// CG step, first half (S3).  The stencil is applied to the residual r (a plain
// array): with p = r + beta p_old and q = A p, linearity gives
// q = A r + beta q_old, so p and q are updated in place at each node and only r
// is read with a halo.  Reduces p.q; the last block sets alpha = rr / p.q.  The
// weights carry the minus sign of A = -L_h.
template <typename T>
struct EpiCgA {
  static constexpr int K = 1;
  static constexpr int NIN = 2;  // p_old, q_old at the node, staged by the pipeline
  using Acc = DotAcc<T>;
  T* p;
  T* q;
  CgScalars* sc;
  int first_ = 0;  // copies of the CG scalars, read once per block by load()
  T beta_ = T(0);
  __device__ __forceinline__ bool skip() const { return sc->done != 0; }
  __device__ __forceinline__ void load() {
    first_ = sc->first;
    beta_ = (T)sc->beta;
  }
  __host__ __device__ __forceinline__ const T* input(int j) const { return j == 0 ? p : q; }
  __device__ __forceinline__ void apply(long long i, T rc, T ar, const T* vin, Acc* acc) const {
    T pc, qc;
    if (first_) {
      pc = rc;
      qc = ar;
    } else {
      pc = fma(beta_, vin[0], rc);
      qc = fma(beta_, vin[1], ar);
    }
    p[i] = pc;
    q[i] = qc;
    acc[0].add(pc, qc);
  }
  __device__ __forceinline__ void operator()(double* t) const {
    sc->pAp = t[0];
    sc->alpha = (t[0] != 0.0) ? (sc->pc ? sc->rz : sc->rr) / t[0] : 0.0;
    sc->first = 0;
  }
};

// EpiCgA with the iterate update folded in: x += alpha p of the previous
// iteration (p = the staged p_old, alpha = the previous alpha) is applied here,
// at the nodes this pass already visits, instead of in the update kernel, which
// then only moves r and q (cg_update_r_kernel).  xdefer says whether an update
// is pending; the last block clears it.  NIN = 3: p_old, q_old, x.
template <typename T>
struct EpiCgAX {
  static constexpr int K = 1;
  static constexpr int NIN = 3;
  using Acc = DotAcc<T>;
  T* p;
  T* q;
  T* x;
  CgScalars* sc;
  int first_ = 0, xd_ = 0;
  T beta_ = T(0), alpha_ = T(0);
  __device__ __forceinline__ bool skip() const { return sc->done != 0; }
  __device__ __forceinline__ void load() {
    first_ = sc->first;
    xd_ = sc->xdefer;
    beta_ = (T)sc->beta;
    alpha_ = (T)sc->alpha;
  }
  __host__ __device__ __forceinline__ const T* input(int j) const { return j == 0 ? p : (j == 1 ? q : x); }
  __device__ __forceinline__ void apply(long long i, T rc, T ar, const T* vin, Acc* acc) const {
    if (xd_) x[i] = fma(alpha_, vin[0], vin[2]);
    T pc, qc;
    if (first_) {
      pc = rc;
      qc = ar;
    } else {
      pc = fma(beta_, vin[0], rc);
      qc = fma(beta_, vin[1], ar);
    }
    p[i] = pc;
    q[i] = qc;
    acc[0].add(pc, qc);
  }
  __device__ __forceinline__ void operator()(double* t) const {
    sc->pAp = t[0];
    sc->alpha = (t[0] != 0.0) ? (sc->pc ? sc->rz : sc->rr) / t[0] : 0.0;
    sc->first = 0;
    sc->xdefer = 0;
  }
};

// Initial residual of a Poisson solve (S3, S5): rhs = 4 pi rho with
// rho = rho_in or u^2 + b; r = rhs + L_h phi (= rhs - (-L_h) phi); reduces
// sum u^2 (for C_h), ||rhs||^2 and ||r||^2 and sets up the CG scalars.
template <typename T, typename U = T, typename V = U>
struct EpiResidual {
  static constexpr int K = 3;
  static constexpr int NIN = 0;
  using Acc = double;
  const U* rho;
  const U* u;
  const V* b;
  T* r;
  CgScalars* sc;
  double tol;
  int max_it;
  int want_r;
  int pc = 0;  // the CG that follows is preconditioned
  __device__ __forceinline__ bool skip() const { return false; }
  __device__ __forceinline__ void load() {}
  __host__ __device__ __forceinline__ const T* input(int) const { return nullptr; }
  __device__ __forceinline__ void apply(long long i, T, T lap, const T*, double* acc) const {
    T uu = T(0);
    if (u) {
      const T ui = (T)u[i];
      uu = ui * ui;
      acc[0] += (double)ui * (double)ui;
    }
    if (want_r) {
      const T rh = (T)(4.0 * kPi) * (rho ? (T)rho[i] : uu + (T)b[i]);
      const T ri = rh + lap;
      r[i] = ri;
      acc[1] += (double)rh * (double)rh;
      acc[2] += (double)ri * (double)ri;
    }
  }
  __device__ __forceinline__ void operator()(double* t) const {
    sc->sum_uu = t[0];
    sc->bb = t[1];
    sc->rr = t[2];
    sc->rr0 = t[2];
    sc->tol2 = tol * tol;
    sc->iters = 0;
    sc->max_it = max_it;
    sc->first = 1;
    sc->beta = 0.0;
    sc->xdefer = 0;
    sc->err = 0;
    sc->pc = pc;
    const double thr = tol * tol * (t[1] > 0.0 ? t[1] : 1.0);
    sc->done = (!want_r || t[2] <= thr || max_it <= 0) ? 1 : 0;
  }
};

// The residual pass of the mixed Poisson rounds with the potential in
// float-float form (phi64 = hi + lo, staged as float2): the stencil runs in
// float-float arithmetic on the FP32 pipes (replacing 37 FP64 FMAs per node,
// which bound the FP64 pass), and so does the epilogue:
//   rho = u^2 + b (u^2 exact from an FMA, b as float-float pairs) or rho_in,
//   r = 4 pi rho + L_h phi, written as float-float pairs,
// with compensated FP32 sums (DotAcc) of u.u, ||4 pi rho||^2, ||r||^2 and, for
// the variational electrostatic energy of the functional that follows, of
// (u^2 + b) phi and phi r.  Accuracy: about 2^-48 of the magnitudes of the
// stencil's terms (the FP64 pass: 2^-53).
__device__ __forceinline__ float2 ff_prod(float a, float b) {  // a b exactly
  const float p = a * b;
  return make_float2(p, fmaf(a, b, -p));
}

struct EpiResidualFF {
  static constexpr int K = 5;
  static constexpr int NIN = 1;  // b at the node (float-float pairs), staged by the pipeline
  using Acc = DotAcc<float>;
  const float* rho;  // explicit density, or NULL for u^2 + b
  const float* u;
  const float2* b2;
  float2* r2;
  CgScalars* sc;
  double tol;
  int max_it;
  int pc = 0;  // the CG that follows is preconditioned
  float2 fourpi;
  __device__ __forceinline__ bool skip() const { return false; }
  __device__ __forceinline__ void load() {}
  __host__ __device__ __forceinline__ const float2* input(int) const { return rho ? nullptr : b2; }
  __device__ __forceinline__ void apply(long long i, float2 ph, float2 lap_raw, const float2* vin, Acc* acc) const {
    // the stencil's float-float sum comes unnormalised (lazy chain): renormalise
    const float2 lap = ff_two_sum(lap_raw.x, lap_raw.y);
    float2 rr;
    if (rho) {
      rr = make_float2(rho[i], 0.0f);
    } else {
      const float ui = u[i];
      acc[0].add(ui, ui);
      rr = ff_add(ff_prod(ui, ui), vin[0]);
    }
    const float2 rh = ff_mul(fourpi, rr);
    const float2 r = ff_add(rh, lap);
    r2[i] = r;
    acc[1].add(rh.x, rh.x);
    acc[2].add(r.x, r.x);
    acc[3].add(rr.x, ph.x);
    acc[3].add(rr.x, ph.y);
    acc[3].add(rr.y, ph.x);
    acc[4].add(ph.x, r.x);
    acc[4].add(ph.x, r.y);
    acc[4].add(ph.y, r.x);
  }
  __device__ __forceinline__ void operator()(double* t) const {
    sc->sum_uu = t[0];
    sc->bb = t[1];
    sc->rr = t[2];
    sc->rr0 = t[2];
    sc->es_rho_phi = t[3];
    sc->es_phi_r = t[4];
    sc->tol2 = tol * tol;
    sc->iters = 0;
    sc->max_it = max_it;
    sc->first = 1;
    sc->beta = 0.0;
    sc->xdefer = 0;
    sc->err = 0;
    sc->pc = pc;
    const double thr = tol * tol * (t[1] > 0.0 ? t[1] : 1.0);
    sc->done = (t[2] <= thr || max_it <= 0) ? 1 : 0;
  }
};

// phi2 = phi64 and b2 = b64 (if b2 is not NULL) split into float-float pairs
// (hi = nearest float, lo = nearest float of the remainder).
static __global__ void __launch_bounds__(256) ff_split_kernel(long long G, float2* phi2, const double* phi64,
                                                              float2* b2, const double* b64) {
  for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < G; i += (long long)gridDim.x * 256) {
    const double v = phi64[i];
    const float hi = (float)v;
    phi2[i] = make_float2(hi, (float)(v - (double)hi));
    if (b2) {
      const double w = b64[i];
      const float bh = (float)w;
      b2[i] = make_float2(bh, (float)(w - (double)bh));
    }
  }
}

// ------------------------------------------------------------- functional ---
// LDA exchange-correlation of Sec. 2 / Sec. 3 (Ceperley-Alder form), density
// floor u^2 < 1e-30 -> 0.  c13 = u^(2/3) = rho^(1/3) is passed in (the caller
// already has cbrt(u) for the Thomas-Fermi term); one reciprocal per branch
// replaces the divisions.
template <typename T>
__device__ __forceinline__ void xc_eval(T u, T rho13, T& eps, T& v) {
  const T rho = u * u;
  if (!(rho >= (T)1e-30)) {
    eps = T(0);
    v = T(0);
    return;
  }
  const T g1 = (T)-0.1423, b1 = (T)1.0529, b2 = (T)0.3334;
  const T A1 = (T)0.0311, B1 = (T)-0.048, C1 = (T)0.002, D1 = (T)-0.0116;
  const T c3pi = (T)0.98474502184269641;  // (3/pi)^{1/3}
  const T ex = (T)-0.75 * c3pi * rho13;
  const T vx = -c3pi * rho13;
  const T rs = (T)0.62035049089940009 / rho13;  // (3/(4 pi))^{1/3} / rho^{1/3}
  T ec, vc;
  if (rs >= T(1)) {
    const T srs = sqrt(rs);
    const T iden = T(1) / (T(1) + b1 * srs + b2 * rs);
    ec = g1 * iden;
    vc = (g1 + (T)(7.0 / 6.0) * g1 * b1 * srs + (T)(4.0 / 3.0) * g1 * b2 * rs) * (iden * iden);
  } else {
    const T lr = log(rs);
    ec = A1 * lr + B1 + C1 * rs * lr + D1 * rs;
    vc = (A1 + (T)(2.0 / 3.0) * C1 * rs) * lr + (B1 - A1 / T(3)) + (T)(1.0 / 3.0) * (T(2) * D1 - C1) * rs;
  }
  eps = ex + ec;
  v = vx + vc;
}
template <typename T>
__device__ __forceinline__ void xc_eval(T u, T& eps, T& v) {
  xc_eval<T>(u, cbrt(u * u), eps, v);
}

struct FuncScalars {
  double h3, N, eta, inv_mu, lambda, CF, kin_vw;
  int terms;
};

// Fused energy + gradient pass (S4): lap = L_h u from the stencil, then at each
// node the TF, vW, XC and electrostatic energy densities, the gradient
//   G = -lambda L_h u + 2 (V_K + V_xc + phi) u + 2 (-eta + C/mu) u,
// the Jacobi diagonal and s = -G / diag, and nine FP64 partial sums.
template <typename T>
struct EpiFunctional {
  static constexpr int K = 11;
  // staged by the pipeline: phi and b at the node, and in FP32 also the search
  // direction d (the third input ring still leaves two blocks per SM; with the
  // pseudocharge's electrostatic sums taken from the residual pass b is not read)
  static constexpr int NIN = sizeof(T) == 4 ? 3 : 2;
  using Acc = FAcc<T>;
  const T* phi;
  const T* b;
  const T* rcg;
  const T* d;
  const T* s_old;
  T* G;
  T* s;
  T* winv;               // optional: u / diag (rank-one correction of the preconditioner)
  const double* sum_uu;  // device sum of u^2 (C_h = h^3 sum_uu - N)
  FuncScalars f;
  double* out;  // 11 sums + C
  T mult_ = T(0);  // -eta + C/mu, from the device sum of u^2 (load())
  T cf_ = T(0), vk_ = T(0), lam_ = T(0), kvw_ = T(0);  // FuncScalars in the field type (load())
  // MIXED: the FP64 potential, pseudocharge and Poisson residual.  With them the
  // electrostatic energy sums use the same FP64 phi and rho = u^2 + b as the FP64
  // residual of the Poisson solve (no FP32 rounding of phi in the variational
  // form); the gradient still takes (float) phi.
  const double* phi64 = nullptr;
  const double* b64 = nullptr;
  const double* r64 = nullptr;
  // MIXED with the float-float residual pass: that pass already summed (u^2 + b) phi
  // and phi r in compensated arithmetic; the functional takes them from here
  const CgScalars* es_sums = nullptr;
  __device__ __forceinline__ bool skip() const { return false; }
  __device__ __forceinline__ void load() {
    const double C = f.h3 * *sum_uu - f.N;
    mult_ = (T)(-f.eta + C * f.inv_mu);
    cf_ = (T)f.CF;
    vk_ = (T)(5.0 / 3.0 * f.CF);
    lam_ = (T)(-f.lambda);
    kvw_ = (T)f.kin_vw;
  }
  __host__ __device__ __forceinline__ const T* input(int j) const {
    if (j == 0) return (f.terms & 8) ? phi : nullptr;
    if (j == 1) return ((f.terms & 8) && !es_sums) ? b : nullptr;
    return d;
  }
  __device__ __forceinline__ void apply(long long i, T uc, T lap, const T* vin, Acc* acc) const {
    const T mult = mult_;
    const bool tf = f.terms & 1, vw = f.terms & 2, xc = f.terms & 4, es = f.terms & 8;
    const T ux = fabs(uc);
    T vk = T(0), vxc = T(0), exc = T(0), ph = T(0);
    const T c = (tf || xc) ? cbrt(ux) : T(0);
    const T c2 = c * c;  // u^(2/3) = rho^(1/3)
    if (tf) {
      const T u43 = c2 * c2;
      vk = vk_ * u43;
      acc[0].add(cf_ * u43, ux * ux);
    }
    if (vw) acc[1].add(uc, lap);
    if (xc) {
      xc_eval<T>(ux, c2, exc, vxc);
      acc[2].add(exc, ux * ux);
    }
    if (es) {
      if (es_sums) {
        ph = vin[0];
      } else if (phi64) {
        const double phd = phi64[i];
        ph = (T)phd;
        acc[3].add_d(((double)uc * (double)uc + b64[i]) * phd);
        if (r64) acc[4].add_d(phd * r64[i]);
      } else {
        ph = vin[0];
        const T rho = uc * uc + vin[1];
        acc[3].add(rho, ph);
        if (rcg) acc[4].add(ph, rcg[i]);
      }
    }
    const T gx = (vw ? lam_ * lap : T(0)) + T(2) * (vk + vxc + ph) * uc + T(2) * mult * uc;
    const T kin = (vw ? kvw_ : T(0)) + (T)(14.0 / 3.0) * vk;
    T md = kin + T(2) * (vxc + ph + mult);
    md = fmax(md, (T)0.25 * kin);
    md = fmax(md, (T)1e-10);
    const T inv = T(1) / md;
    const T sx = -gx * inv;
    const T wv = uc * inv;
    if (G) G[i] = gx;
    if (s) s[i] = sx;
    if (winv) winv[i] = wv;
    // sums of terms of one sign (the stopping test's g^2 / diag, g.g, u^2 /
    // diag) in plain FP32 per thread: no cancellation, so a thread's partial sum
    // keeps FP32 relative accuracy; the sums of mixed-sign terms (line search,
    // Polak-Ribiere beta, the rank-one correction's u.s), whose totals can be
    // far smaller than their terms, stay compensated like the energy sums
    if (d) {
      if constexpr (NIN == 3)
        acc[5].add(gx, vin[2]);
      else
        acc[5].add(gx, d[i]);
    }
    if (s_old) acc[6].add(gx, s_old[i]);
    acc[7].add_fast(gx, -sx);  // g^2 / diag
    acc[8].add_fast(gx, gx);
    acc[9].add(uc, sx);
    acc[10].add_fast(uc, wv);  // u^2 / diag
  }
  __device__ __forceinline__ void operator()(double* t) const {
#pragma unroll
    for (int k = 0; k < 9; ++k) out[k] = t[k];
    if (es_sums && (f.terms & 8)) {
      out[3] = es_sums->es_rho_phi;
      out[4] = es_sums->es_phi_r;
    }
    out[9] = f.h3 * *sum_uu - f.N;
    out[10] = t[9];
    out[11] = t[10];
  }
};

// ------------------------------------------------------- CG second half ---
// x += alpha p, r -= alpha q, reduces r.r; the last block sets beta, counts the
// iteration and raises `done` at convergence or at the iteration cap.  X is the
// iterate's type: T, or double for the mixed CG (FP32 r, p, q, FP64 iterate).
// 16-byte vector of T (the wide path of the pointwise CG update).
template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
  __device__ static void get(const type& v, float* o) { o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w; }
  __device__ static type make(const float* o) { return make_float4(o[0], o[1], o[2], o[3]); }
};
template <>
struct Vec16<double> {
  using type = double2;
  __device__ static void get(const type& v, double* o) { o[0] = v.x; o[1] = v.y; }
  __device__ static type make(const double* o) { return make_double2(o[0], o[1]); }
};

// WIDE: every array 16-byte aligned, G a multiple of 16 / sizeof(T) and X == T;
// each thread then moves whole 16-byte vectors (two per pass).
template <typename T, typename X = T, bool WIDE = false>
__global__ void __launch_bounds__(256) cg_update_kernel(long long G, X* __restrict__ phi,
                                                        T* __restrict__ r, const T* __restrict__ p,
                                                        const T* __restrict__ Ap, CgScalars* sc,
                                                        RedBuf red) {
  pdl_enter();
  __shared__ double smem[256 / 32];
  DotAcc<T> dacc;
  if constexpr (WIDE) {
    static_assert(sizeof(X) == sizeof(T), "the wide update needs X == T");
    using VT = typename Vec16<T>::type;
    constexpr int VW = 16 / (int)sizeof(T);
    const long long nv = G / VW;
    const VT* p4 = reinterpret_cast<const VT*>(p);
    const VT* a4 = reinterpret_cast<const VT*>(Ap);
    VT* x4 = reinterpret_cast<VT*>(phi);
    VT* r4 = reinterpret_cast<VT*>(r);
    constexpr int UV = 2;  // vectors per thread and pass: all loads of a pass in flight together
    const long long stride = (long long)gridDim.x * 256 * UV;
    // the first pass's loads are issued together with the loads of the CG
    // scalars (reading is harmless when the solve is already done)
    bool first = true;
    int done = 0;
    T alpha = T(0);
    for (long long v0 = (long long)blockIdx.x * 256 * UV + threadIdx.x; v0 < nv; v0 += stride) {
      VT pv[UV], av[UV], xv[UV], rv[UV];
#pragma unroll
      for (int u = 0; u < UV; ++u) {
        const long long v = v0 + 256 * u;
        if (v < nv) {
          pv[u] = p4[v];
          av[u] = a4[v];
          xv[u] = x4[v];
          rv[u] = r4[v];
        }
      }
      if (first) {
        done = sc->done;
        alpha = (T)sc->alpha;
        first = false;
        if (done) return;
      }
#pragma unroll
      for (int u = 0; u < UV; ++u) {
        const long long v = v0 + 256 * u;
        if (v < nv) {
          T pe[VW], ae[VW], xe[VW], re[VW];
          Vec16<T>::get(pv[u], pe);
          Vec16<T>::get(av[u], ae);
          Vec16<T>::get(xv[u], xe);
          Vec16<T>::get(rv[u], re);
#pragma unroll
          for (int l = 0; l < VW; ++l) {
            xe[l] = fma(alpha, pe[l], xe[l]);
            re[l] = fma(-alpha, ae[l], re[l]);
            dacc.add(re[l], re[l]);
          }
          x4[v] = Vec16<T>::make(xe);
          r4[v] = Vec16<T>::make(re);
        }
      }
    }
    if (first && sc->done) return;  // threads without elements take the same exit
  } else {
    if (sc->done) return;
    const T alpha = (T)sc->alpha;
    const X alpha_x = (X)sc->alpha;
    // four independent elements per thread and pass keep several loads in flight
    const long long stride = (long long)gridDim.x * 1024;
    for (long long i0 = (long long)blockIdx.x * 1024 + threadIdx.x; i0 < G; i0 += stride) {
      T pv[4], av[4], rv[4];
      X xv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const long long i = i0 + 256 * u;
        if (i < G) {
          pv[u] = p[i];
          av[u] = Ap[i];
          xv[u] = phi[i];
          rv[u] = r[i];
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const long long i = i0 + 256 * u;
        if (i < G) {
          phi[i] = fma(alpha_x, (X)pv[u], xv[u]);
          const T ri = fma(-alpha, av[u], rv[u]);
          r[i] = ri;
          dacc.add(ri, ri);
        }
      }
    }
  }
  double acc[1] = {dacc.value()};
  struct Fin {
    CgScalars* sc;
    __device__ void operator()(double* t) const {
      const double rr_new = t[0];
      if (!sc->pc) sc->beta = (sc->rr != 0.0) ? rr_new / sc->rr : 0.0;
      sc->rr_prev = sc->rr;
      sc->rr = rr_new;
      sc->iters += 1;
      const double thr = sc->tol2 * (sc->bb > 0.0 ? sc->bb : 1.0);
      if (rr_new <= thr || sc->iters >= sc->max_it || !(rr_new == rr_new)) sc->done = 1;
    }
  } fin{sc};
  grid_sum<1, 256>(acc, smem, red, gridDim.x, blockIdx.x, threadIdx.x, fin);
}

// CG second half when the iterate update is folded into the next stencil pass
// (EpiCgAX): r -= alpha q and r.r only; the last block sets beta, counts the
// iteration, raises `done` and marks x += alpha p as pending (xdefer).
template <typename T, bool WIDE = false>
__global__ void __launch_bounds__(256) cg_update_r_kernel(long long G, T* __restrict__ r, const T* __restrict__ Ap,
                                                          CgScalars* sc, RedBuf red) {
  pdl_enter();
  __shared__ double smem[256 / 32];
  DotAcc<T> dacc;
  if constexpr (WIDE) {
    using VT = typename Vec16<T>::type;
    constexpr int VW = 16 / (int)sizeof(T);
    constexpr int UV = 4;  // vectors per thread and pass
    const long long nv = G / VW;
    const VT* a4 = reinterpret_cast<const VT*>(Ap);
    VT* r4 = reinterpret_cast<VT*>(r);
    const long long stride = (long long)gridDim.x * 256 * UV;
    bool first = true;
    T alpha = T(0);
    for (long long v0 = (long long)blockIdx.x * 256 * UV + threadIdx.x; v0 < nv; v0 += stride) {
      VT av[UV], rv[UV];
#pragma unroll
      for (int u = 0; u < UV; ++u) {
        const long long v = v0 + 256 * u;
        if (v < nv) {
          av[u] = a4[v];
          rv[u] = r4[v];
        }
      }
      if (first) {  // the CG scalars arrive with the first loads
        const int done = sc->done;
        alpha = (T)sc->alpha;
        first = false;
        if (done) return;
      }
#pragma unroll
      for (int u = 0; u < UV; ++u) {
        const long long v = v0 + 256 * u;
        if (v < nv) {
          T ae[VW], re[VW];
          Vec16<T>::get(av[u], ae);
          Vec16<T>::get(rv[u], re);
#pragma unroll
          for (int l = 0; l < VW; ++l) {
            re[l] = fma(-alpha, ae[l], re[l]);
            dacc.add(re[l], re[l]);
          }
          r4[v] = Vec16<T>::make(re);
        }
      }
    }
    if (first && sc->done) return;  // threads without elements take the same exit
  } else {
    if (sc->done) return;
    const T alpha = (T)sc->alpha;
    const long long stride = (long long)gridDim.x * 1024;
    for (long long i0 = (long long)blockIdx.x * 1024 + threadIdx.x; i0 < G; i0 += stride) {
      T av[4], rv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const long long i = i0 + 256 * u;
        if (i < G) {
          av[u] = Ap[i];
          rv[u] = r[i];
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const long long i = i0 + 256 * u;
        if (i < G) {
          const T ri = fma(-alpha, av[u], rv[u]);
          r[i] = ri;
          dacc.add(ri, ri);
        }
      }
    }
  }
  double acc[1] = {dacc.value()};
  struct Fin {
    CgScalars* sc;
    __device__ void operator()(double* t) const {
      const double rr_new = t[0];
      if (!sc->pc) sc->beta = (sc->rr != 0.0) ? rr_new / sc->rr : 0.0;
      sc->rr_prev = sc->rr;
      sc->rr = rr_new;
      sc->iters += 1;
      sc->xdefer = 1;
      const double thr = sc->tol2 * (sc->bb > 0.0 ? sc->bb : 1.0);
      if (rr_new <= thr || sc->iters >= sc->max_it || !(rr_new == rr_new)) sc->done = 1;
    }
  } fin{sc};
  grid_sum<1, 256>(acc, smem, red, gridDim.x, blockIdx.x, threadIdx.x, fin);
}

// Condition of the device-side CG loop (a CUDA graph WHILE node): keep
// iterating while the solve is not done.  `done` is raised by the CG kernels
// themselves at convergence, at the iteration cap or on a non-finite residual,
// so the loop always ends.
static __global__ void cg_cond_kernel(cudaGraphConditionalHandle h, const CgScalars* sc) {
  cudaGraphSetConditional(h, sc->done ? 0u : 1u);
}

// Condition of the batched CG loop graph: keep iterating while any of the n
// solves base[idx[i]] is not done.
static __global__ void batch_cond_kernel(cudaGraphConditionalHandle h, const CgScalars* base, const int* idx, int n) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    if (!base[idx[i]].done) any = 1;
  __syncthreads();
  if (threadIdx.x == 0) cudaGraphSetConditional(h, any ? 1u : 0u);
}

// Applies a pending x += alpha p (xdefer) after the last CG iteration of a call.
template <typename T>
__global__ void __launch_bounds__(256) cg_xflush_kernel(long long G, T* __restrict__ x, const T* __restrict__ p,
                                                        const CgScalars* sc) {
  if (!sc->xdefer) return;
  const T alpha = (T)sc->alpha;
  for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < G; i += (long long)gridDim.x * 256)
    x[i] = fma(alpha, p[i], x[i]);
}
static __global__ void cg_xclear_kernel(CgScalars* sc) { sc->xdefer = 0; }

// Residual replacement of the mixed CG: r32 = (float) r64 (the FP64 true
// residual).  On the first round the CG starts from scratch (p = r); later
// rounds keep the search direction and rescale beta to the replaced residual.
// The FP32 iterations of a round stop when r.r falls by inner_tol^2.
__device__ __forceinline__ float nearest_float(double v) { return (float)v; }
__device__ __forceinline__ float nearest_float(float2 v) { return v.x; }  // hi is the nearest float of hi + lo

template <typename RS>
__global__ void __launch_bounds__(256) refine_replace_kernel(long long G, float* r32, const RS* r64,
                                                                    CgScalars* sc, double inner_tol, int budget,
                                                                    int restart, int pc, RedBuf red) {
  __shared__ double smem[256 / 32];
  DotAcc<float> rr;
  for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < G; i += (long long)gridDim.x * 256) {
    const float v = nearest_float(r64[i]);
    r32[i] = v;
    rr.add(v, v);
  }
  double acc[1] = {rr.value()};
  struct Fin {
    CgScalars* sc;
    double tol;
    int budget, restart, pc;
    __device__ void operator()(double* t) const {
      sc->pc = pc;  // with a preconditioner the next pass forms beta from r.z
      if (restart) {
        sc->first = 1;
        sc->beta = 0.0;
        sc->iters = 0;
      } else {
        sc->beta = (sc->rr_prev != 0.0) ? t[0] / sc->rr_prev : 0.0;
      }
      sc->rr = t[0];
      sc->rr0 = t[0];
      sc->bb = t[0];
      sc->xdefer = 0;
      sc->err = 0;
      sc->tol2 = tol * tol;
      sc->max_it = sc->iters + budget;
      sc->done = (t[0] == 0.0 || budget <= 0) ? 1 : 0;
    }
  } fin{sc, inner_tol, budget, restart, pc};
  grid_sum<1, 256>(acc, smem, red, gridDim.x, blockIdx.x, threadIdx.x, fin);
}

// ------------------------------------------------- multigrid preconditioner ---
// Preconditioner of the Poisson CG (S3).  The paper's Poisson solver is a
// Krylov method without a stated preconditioner; the multigrid cycle here is a
// solver choice of this implementation and leaves the solution (phi to the
// same residual tolerance) unchanged.  M is one V(1,1)-cycle for the
// second-order 7-point operator A7 f = (6 f - sum of the 6 neighbours) / H^2
// with zero Dirichlet values: coarse node I of a level sits on fine node
// 2I + 1 (n_c = floor(n / 2) per axis, H doubles), damped Jacobi smoothing
// with weight omega (diagonal 6 / H^2), full-weighting restriction R = P^T / 8
// and trilinear prolongation P (1D weights 1/2, 1, 1/2; zero outside), and on
// the bottom level (smallest extent below 4) a fixed number of Jacobi sweeps
// from zero.  The same smoother before and after the coarse correction makes
// M a fixed symmetric positive definite operator, so CG with z = M r stays
// CG; A7 is spectrally equivalent to the high-order stencil (equal at low
// frequency, within a factor 2.5 at the grid's highest), so the iteration
// count stays nearly flat as the grid grows.
//
// With s = omega H^2 / 6 the cycle's steps on one level are
//   down:   z1 = s r,  t = r - A7 z1 = (1 - omega) r + (omega / 6) sum_nb r
//   coarse: r_c = R t
//   up:     y = z1 + P e_c,  z = y + (omega / D)(r - A7 y)
//             = (1 - omega) y + s r + (omega / 6) sum_nb y
// and on the bottom level  z <- (1 - omega) z + s r + (omega / 6) sum_nb z.
struct MgLevel {
  int n1, n2, n3;
};
constexpr int kMgMaxLevels = 24;

template <typename T>
__device__ __forceinline__ T mg_nb_sum(const T* f, int i, int j, int k, const MgLevel& d, long long idx,
                                       long long plane) {
  T s = T(0);
  if (i > 0) s += f[idx - 1];
  if (i + 1 < d.n1) s += f[idx + 1];
  if (j > 0) s += f[idx - d.n1];
  if (j + 1 < d.n2) s += f[idx + d.n1];
  if (k > 0) s += f[idx - plane];
  if (k + 1 < d.n3) s += f[idx + plane];
  return s;
}

// (i, j, k) of linear index idx on level d; every level holds fewer than 2^31
// nodes (mg_plan), so 32-bit unsigned divisions suffice.
__device__ __forceinline__ void mg_ijk(long long idx, const MgLevel& d, int& i, int& j, int& k) {
  const unsigned q = (unsigned)idx;
  const unsigned jk = q / (unsigned)d.n1;
  i = (int)(q - jk * (unsigned)d.n1);
  const unsigned kk = jk / (unsigned)d.n2;
  k = (int)kk;
  j = (int)(jk - kk * (unsigned)d.n2);
}

// Coarse node c = I of one axis: full-weighting sum over fine 2I, 2I+1, 2I+2.
template <typename T>
__device__ __forceinline__ T mg_restrict_at(const T* t, const MgLevel& f, int I, int J, int K) {
  const long long fplane = (long long)f.n1 * f.n2;
  T acc = T(0);
#pragma unroll
  for (int dk = 0; dk < 3; ++dk) {
    const int kk = 2 * K + dk;
    if (kk >= f.n3) continue;
    const T wz = dk == 1 ? T(0.5) : T(0.25);
#pragma unroll
    for (int dj = 0; dj < 3; ++dj) {
      const int jj = 2 * J + dj;
      if (jj >= f.n2) continue;
      const T wy = dj == 1 ? T(0.5) : T(0.25);
      const T* row = t + fplane * kk + (long long)f.n1 * jj;
      const int ii = 2 * I;
      T sx = T(0.25) * row[ii] + T(0.5) * row[ii + 1];
      if (ii + 2 < f.n1) sx += T(0.25) * row[ii + 2];
      acc += wz * wy * sx;
    }
  }
  return acc;
}

// Trilinear prolongation of the coarse field e (dims c) at fine node (i, j, k):
// per axis, odd q takes coarse (q - 1) / 2 with weight 1, even q the mean of
// coarse q / 2 - 1 and q / 2 (zero outside).  Missing terms get weight 0 at a
// clamped (valid) index, so the 8 loads need no branches.
template <typename T>
__device__ __forceinline__ void mg_axis(int q, int n, int& c0, int& c1, T& w0, T& w1) {
  if (q & 1) {
    c0 = c1 = (q - 1) >> 1;
    w0 = T(1);
    w1 = T(0);
  } else {
    const int lo = (q >> 1) - 1, hi = q >> 1;
    c0 = lo >= 0 ? lo : 0;
    w0 = lo >= 0 ? T(0.5) : T(0);
    c1 = hi < n ? hi : n - 1;
    w1 = hi < n ? T(0.5) : T(0);
  }
}

template <typename T>
__device__ __forceinline__ T mg_prolong_at(const T* e, const MgLevel& c, int i, int j, int k) {
  int x0, x1, y0, y1, z0, z1;
  T wx0, wx1, wy0, wy1, wz0, wz1;
  mg_axis(i, c.n1, x0, x1, wx0, wx1);
  mg_axis(j, c.n2, y0, y1, wy0, wy1);
  mg_axis(k, c.n3, z0, z1, wz0, wz1);
  const long long cplane = (long long)c.n1 * c.n2;
  const T* r00 = e + cplane * z0 + (long long)c.n1 * y0;
  const T* r01 = e + cplane * z0 + (long long)c.n1 * y1;
  const T* r10 = e + cplane * z1 + (long long)c.n1 * y0;
  const T* r11 = e + cplane * z1 + (long long)c.n1 * y1;
  const T a00 = wx0 * r00[x0] + wx1 * r00[x1];
  const T a01 = wx0 * r01[x0] + wx1 * r01[x1];
  const T a10 = wx0 * r10[x0] + wx1 * r10[x1];
  const T a11 = wx0 * r11[x0] + wx1 * r11[x1];
  return wz0 * (wy0 * a00 + wy1 * a01) + wz1 * (wy0 * a10 + wy1 * a11);
}

// The single-grid passes of the cycle walk x-rows: each warp takes one (j, k)
// row at a time, its lanes the row's nodes (coalesced, one division per row).
// down: t = (1 - omega) r + (omega / 6) sum_nb r on one level.
template <typename T>
__global__ void __launch_bounds__(256) mg_down_kernel(MgLevel d, const T* __restrict__ r, T* __restrict__ t,
                                                      T omega, const CgScalars* sc) {
  pdl_enter();
  if (sc->done) return;
  const long long plane = (long long)d.n1 * d.n2;
  const int rows = d.n2 * d.n3;
  const T a = T(1) - omega, b = omega / T(6);
  const int lane = threadIdx.x & 31;
  for (int row = blockIdx.x * 8 + (threadIdx.x >> 5); row < rows; row += gridDim.x * 8) {
    const int k = row / d.n2, j = row - k * d.n2;
    const long long o = (long long)row * d.n1;
    for (int i = lane; i < d.n1; i += 32) t[o + i] = a * r[o + i] + b * mg_nb_sum(r, i, j, k, d, o + i, plane);
  }
}

// coarse: r_c = R t.
template <typename T>
__global__ void __launch_bounds__(256) mg_restrict_kernel(MgLevel f, MgLevel c, const T* __restrict__ t,
                                                          T* __restrict__ rc, const CgScalars* sc) {
  pdl_enter();
  if (sc->done) return;
  const int rows = c.n2 * c.n3;
  const int lane = threadIdx.x & 31;
  for (int row = blockIdx.x * 8 + (threadIdx.x >> 5); row < rows; row += gridDim.x * 8) {
    const int K = row / c.n2, J = row - K * c.n2;
    const long long o = (long long)row * c.n1;
    for (int I = lane; I < c.n1; I += 32) rc[o + I] = mg_restrict_at(t, f, I, J, K);
  }
}

// The PCG scalars after z = M r: beta = (r.z) / (r.z of the previous
// iteration), unless the next direction is the first.
struct MgFin {
  CgScalars* sc;
  __device__ void operator()(double* t) const {
    const double rz = t[0];
    sc->beta = (sc->first || sc->rz == 0.0) ? 0.0 : rz / sc->rz;
    sc->rz = rz;
  }
};

// The smoothing passes of a level as z-streaming stencils: the 7-point sum
// (1 - omega) f + (omega / 6) sum_nb f is the radius-1 star stencil with
// centre weight 1 - omega and neighbour weight omega / 6, so the pipelined
// stencil kernel (planes staged through shared memory, register z-queues)
// runs them at the memory roofline instead of the row-per-warp passes.
// down: t = stencil(r).
template <typename T>
struct EpiMgDown {
  static constexpr int K = 0;
  static constexpr int NIN = 0;
  using Acc = double;
  T* t;
  const CgScalars* sc;
  __device__ __forceinline__ bool skip() const { return sc->done != 0; }
  __device__ __forceinline__ void load() {}
  __host__ __device__ __forceinline__ const T* input(int) const { return nullptr; }
  __device__ __forceinline__ void apply(long long i, T, T lap, const T*, Acc*) const { t[i] = lap; }
  __device__ __forceinline__ void operator()(double*) const {}
};
// up: z = stencil(y) + s r (r staged with the stencil input); on the finest
// level (DOT) also r.z and the PCG scalars.
template <typename T, bool DOT>
struct EpiMgUp {
  static constexpr int K = DOT ? 1 : 0;
  static constexpr int NIN = 1;
  using Acc = DotAcc<T>;
  const T* r;
  T* z;
  T s;
  CgScalars* sc;
  __device__ __forceinline__ bool skip() const { return sc->done != 0; }
  __device__ __forceinline__ void load() {}
  __host__ __device__ __forceinline__ const T* input(int) const { return r; }
  __device__ __forceinline__ void apply(long long i, T, T lap, const T* vin, Acc* acc) const {
    const T zi = fma(s, vin[0], lap);
    z[i] = zi;
    if constexpr (DOT) acc[0].add(vin[0], zi);
  }
  __device__ __forceinline__ void operator()(double* t) const {
    if constexpr (DOT) MgFin{sc}(t);
  }
};

// up, first half: y = s r + P e_c.  With DOT this is the whole up step of a
// level that is not smoothed (the finest level with mg_finest_smooth = 0:
// z = s r + P e_c), with r.z and the PCG scalars.
template <typename T, bool DOT>
__global__ void __launch_bounds__(256) mg_prolong_kernel(MgLevel f, MgLevel c, const T* __restrict__ r,
                                                         const T* __restrict__ ec, T* __restrict__ y, T s,
                                                         CgScalars* sc, RedBuf red) {
  pdl_enter();
  __shared__ double smem[256 / 32];
  if (sc->done) return;
  const int rows = f.n2 * f.n3;
  const int lane = threadIdx.x & 31;
  DotAcc<T> acc;
  for (int row = blockIdx.x * 8 + (threadIdx.x >> 5); row < rows; row += gridDim.x * 8) {
    const int k = row / f.n2, j = row - k * f.n2;
    const long long o = (long long)row * f.n1;
    for (int i = lane; i < f.n1; i += 32) {
      const T ri = r[o + i];
      const T yi = s * ri + mg_prolong_at(ec, c, i, j, k);
      y[o + i] = yi;
      if constexpr (DOT) acc.add(ri, yi);
    }
  }
  if constexpr (DOT) {
    double v[1] = {acc.value()};
    MgFin fin{sc};
    grid_sum<1, 256>(v, smem, red, gridDim.x, blockIdx.x, threadIdx.x, fin);
  }
}

// up, second half: z = (1 - omega) y + s r + (omega / 6) sum_nb y; on the
// finest level (DOT) also r.z and the PCG scalars.
template <typename T, bool DOT>
__global__ void __launch_bounds__(256) mg_up_kernel(MgLevel d, const T* __restrict__ r, const T* __restrict__ y,
                                                    T* __restrict__ z, T omega, T s, CgScalars* sc, RedBuf red) {
  pdl_enter();
  __shared__ double smem[256 / 32];
  if (sc->done) return;
  const long long plane = (long long)d.n1 * d.n2;
  const int rows = d.n2 * d.n3;
  const T a = T(1) - omega, b = omega / T(6);
  const int lane = threadIdx.x & 31;
  DotAcc<T> acc;
  for (int row = blockIdx.x * 8 + (threadIdx.x >> 5); row < rows; row += gridDim.x * 8) {
    const int k = row / d.n2, j = row - k * d.n2;
    const long long o = (long long)row * d.n1;
    for (int i = lane; i < d.n1; i += 32) {
      const T ri = r[o + i];
      const T zi = a * y[o + i] + s * ri + b * mg_nb_sum(y, i, j, k, d, o + i, plane);
      z[o + i] = zi;
      if constexpr (DOT) acc.add(ri, zi);
    }
  }
  if constexpr (DOT) {
    double v[1] = {acc.value()};
    MgFin fin{sc};
    grid_sum<1, 256>(v, smem, red, gridDim.x, blockIdx.x, threadIdx.x, fin);
  }
}

// Fused passes of one level (the single-solve V-cycle): each block works on a
// 3-D tile through shared memory, so the smoothed residual t and the
// prolongated correction y never go to global memory and a level costs two
// launches instead of four.  The arithmetic, and its order, are those of the
// separate passes above (zero-filled out-of-grid values add exact zeros).
//
// down + restrict: r_c = R t with t = (1 - omega) r + (omega / 6) sum_nb r, for
// a tile of MgDR::CX x CY x CZ coarse nodes: r on the fine nodes 2 I0 - 1 ..
// 2 (I0 + C) + 1 of each axis, t on 2 I0 .. 2 (I0 + C), both in shared memory.
template <typename T>
struct MgDR {  // at most 48 KB of static shared memory: 39.6 KB in FP32, 31.8 KB in FP64
  static constexpr int CX = sizeof(T) == 4 ? 16 : 8, CY = 8, CZ = sizeof(T) == 4 ? 3 : 2;
  static constexpr int TX = 2 * CX + 1, TY = 2 * CY + 1, TZ = 2 * CZ + 1;
  static constexpr int RX = TX + 2, RY = TY + 2, RZ = TZ + 2;
};

template <typename T>
__global__ void __launch_bounds__(256) mg_down_restrict_kernel(MgLevel f, MgLevel c, const T* __restrict__ r,
                                                               T* __restrict__ rc, T omega, const CgScalars* sc) {
  pdl_enter();
  using D = MgDR<T>;
  __shared__ T rs[D::RZ * D::RY * D::RX];
  __shared__ T ts[D::TZ * D::TY * D::TX];
  if (sc->done) return;
  const int I0 = blockIdx.x * D::CX, J0 = blockIdx.y * D::CY, K0 = blockIdx.z * D::CZ;
  const int fx0 = 2 * I0 - 1, fy0 = 2 * J0 - 1, fz0 = 2 * K0 - 1;
  for (int q = threadIdx.x; q < D::RX * D::RY * D::RZ; q += 256) {
    const int x = q % D::RX, yz = q / D::RX, y = yz % D::RY, z = yz / D::RY;
    const int gx = fx0 + x, gy = fy0 + y, gz = fz0 + z;
    T v = T(0);
    if (gx >= 0 && gx < f.n1 && gy >= 0 && gy < f.n2 && gz >= 0 && gz < f.n3)
      v = r[((long long)gz * f.n2 + gy) * f.n1 + gx];
    rs[q] = v;
  }
  __syncthreads();
  const T a = T(1) - omega, b = omega / T(6);
  constexpr int SY = D::RX, SZ = D::RX * D::RY;
  for (int q = threadIdx.x; q < D::TX * D::TY * D::TZ; q += 256) {
    const int x = q % D::TX, yz = q / D::TX, y = yz % D::TY, z = yz / D::TY;
    T v = T(0);
    if (fx0 + 1 + x < f.n1 && fy0 + 1 + y < f.n2 && fz0 + 1 + z < f.n3) {
      const int o = (z + 1) * SZ + (y + 1) * SY + (x + 1);
      v = a * rs[o] + b * (rs[o - 1] + rs[o + 1] + rs[o - SY] + rs[o + SY] + rs[o - SZ] + rs[o + SZ]);
    }
    ts[q] = v;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < D::CX * D::CY * D::CZ; q += 256) {
    const int x = q % D::CX, yz = q / D::CX, y = yz % D::CY, z = yz / D::CY;
    const int I = I0 + x, J = J0 + y, K = K0 + z;
    if (I >= c.n1 || J >= c.n2 || K >= c.n3) continue;
    T acc = T(0);
#pragma unroll
    for (int dk = 0; dk < 3; ++dk) {
      const T wz = dk == 1 ? T(0.5) : T(0.25);
#pragma unroll
      for (int dj = 0; dj < 3; ++dj) {
        const T wy = dj == 1 ? T(0.5) : T(0.25);
        const T* row = ts + (2 * z + dk) * D::TY * D::TX + (2 * y + dj) * D::TX + 2 * x;
        const T sx = T(0.25) * row[0] + T(0.5) * row[1] + T(0.25) * row[2];
        acc += wz * wy * sx;
      }
    }
    rc[((long long)K * c.n2 + J) * c.n1 + I] = acc;
  }
}

// prolong + up: y = s r + P e_c on a tile of MgPU::FX x FY x FZ fine nodes and
// a one-node halo, then z = (1 - omega) y + s r + (omega / 6) sum_nb y on the
// tile; on the finest level (DOT) also r.z and the PCG scalars.
template <typename T>
struct MgPU {
  static constexpr int FX = 32, FY = 8, FZ = sizeof(T) == 4 ? 8 : 4;
  static constexpr int YX = FX + 2, YY = FY + 2, YZ = FZ + 2;          // y and r: fine x0 - 1 .. x0 + FX
  static constexpr int EX = FX / 2 + 2, EY = FY / 2 + 2, EZ = FZ / 2 + 2;  // coarse x0/2 - 1 .. x0/2 + FX/2
};

template <typename T, bool DOT>
__global__ void __launch_bounds__(256) mg_prolong_up_kernel(MgLevel f, MgLevel c, const T* __restrict__ r,
                                                            const T* __restrict__ ec, T* __restrict__ z, T omega,
                                                            T s, CgScalars* sc, RedBuf red) {
  pdl_enter();
  using D = MgPU<T>;
  __shared__ T rs[D::YZ * D::YY * D::YX];
  __shared__ T ys[D::YZ * D::YY * D::YX];
  __shared__ T es[D::EZ * D::EY * D::EX];
  __shared__ double smem[256 / 32];
  if (sc->done) return;
  const int x0 = blockIdx.x * D::FX, y0 = blockIdx.y * D::FY, z0 = blockIdx.z * D::FZ;
  const int cx0 = x0 / 2 - 1, cy0 = y0 / 2 - 1, cz0 = z0 / 2 - 1;
  for (int q = threadIdx.x; q < D::EX * D::EY * D::EZ; q += 256) {
    const int x = q % D::EX, yz = q / D::EX, y = yz % D::EY, zz = yz / D::EY;
    const int gx = cx0 + x, gy = cy0 + y, gz = cz0 + zz;
    T v = T(0);
    if (gx >= 0 && gx < c.n1 && gy >= 0 && gy < c.n2 && gz >= 0 && gz < c.n3)
      v = ec[((long long)gz * c.n2 + gy) * c.n1 + gx];
    es[q] = v;
  }
  for (int q = threadIdx.x; q < D::YX * D::YY * D::YZ; q += 256) {
    const int x = q % D::YX, yz = q / D::YX, y = yz % D::YY, zz = yz / D::YY;
    const int gx = x0 - 1 + x, gy = y0 - 1 + y, gz = z0 - 1 + zz;
    T v = T(0);
    if (gx >= 0 && gx < f.n1 && gy >= 0 && gy < f.n2 && gz >= 0 && gz < f.n3)
      v = r[((long long)gz * f.n2 + gy) * f.n1 + gx];
    rs[q] = v;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < D::YX * D::YY * D::YZ; q += 256) {
    const int x = q % D::YX, yz = q / D::YX, y = yz % D::YY, zz = yz / D::YY;
    const int gx = x0 - 1 + x, gy = y0 - 1 + y, gz = z0 - 1 + zz;
    T v = T(0);
    if (gx >= 0 && gx < f.n1 && gy >= 0 && gy < f.n2 && gz >= 0 && gz < f.n3) {
      int ax0, ax1, ay0, ay1, az0, az1;
      T wx0, wx1, wy0, wy1, wz0, wz1;
      mg_axis(gx, c.n1, ax0, ax1, wx0, wx1);
      mg_axis(gy, c.n2, ay0, ay1, wy0, wy1);
      mg_axis(gz, c.n3, az0, az1, wz0, wz1);
      const T* r00 = es + ((az0 - cz0) * D::EY + (ay0 - cy0)) * D::EX - cx0;
      const T* r01 = es + ((az0 - cz0) * D::EY + (ay1 - cy0)) * D::EX - cx0;
      const T* r10 = es + ((az1 - cz0) * D::EY + (ay0 - cy0)) * D::EX - cx0;
      const T* r11 = es + ((az1 - cz0) * D::EY + (ay1 - cy0)) * D::EX - cx0;
      const T a00 = wx0 * r00[ax0] + wx1 * r00[ax1];
      const T a01 = wx0 * r01[ax0] + wx1 * r01[ax1];
      const T a10 = wx0 * r10[ax0] + wx1 * r10[ax1];
      const T a11 = wx0 * r11[ax0] + wx1 * r11[ax1];
      v = s * rs[q] + (wz0 * (wy0 * a00 + wy1 * a01) + wz1 * (wy0 * a10 + wy1 * a11));
    }
    ys[q] = v;
  }
  __syncthreads();
  const T a = T(1) - omega, b = omega / T(6);
  constexpr int SY = D::YX, SZ = D::YX * D::YY;
  DotAcc<T> acc;
  for (int q = threadIdx.x; q < D::FX * D::FY * D::FZ; q += 256) {
    const int x = q % D::FX, yz = q / D::FX, y = yz % D::FY, zz = yz / D::FY;
    const int gx = x0 + x, gy = y0 + y, gz = z0 + zz;
    if (gx >= f.n1 || gy >= f.n2 || gz >= f.n3) continue;
    const int o = (zz + 1) * SZ + (y + 1) * SY + (x + 1);
    const T ri = rs[o];
    const T zi = a * ys[o] + s * ri + b * (ys[o - 1] + ys[o + 1] + ys[o - SY] + ys[o + SY] + ys[o - SZ] + ys[o + SZ]);
    z[((long long)gz * f.n2 + gy) * f.n1 + gx] = zi;
    if constexpr (DOT) acc.add(ri, zi);
  }
  if constexpr (DOT) {
    double v[1] = {acc.value()};
    MgFin fin{sc};
    const int nb = gridDim.x * gridDim.y * gridDim.z;
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    grid_sum<1, 256>(v, smem, red, nb, bid, threadIdx.x, fin);
  }
}

// The coarse end of the cycle in one block, every level in shared memory:
// from level d0 (r in global memory) down to the bottom level, `sweeps`
// Jacobi sweeps there, and back up to z of level d0 (global memory).  nlev
// counts d0 and the levels below it.  With DOT (the whole grid is this small)
// the block also forms r.z and the PCG scalars.
template <typename T, bool DOT>
__device__ __forceinline__ void mg_coarse_body(MgLevel d0, int nlev, const T* __restrict__ r, T* __restrict__ z,
                                               T omega, T s0, int sweeps, CgScalars* sc,
                                               unsigned char* smbase = nullptr) {
  extern __shared__ __align__(16) unsigned char mg_sm[];
  __shared__ double red_sm[1024 / 32];
  if (sc->done) return;
  const int tid = threadIdx.x;
  constexpr int NTH = 1024;
  MgLevel d[kMgMaxLevels];
  T* Rl[kMgMaxLevels];
  T* Zl[kMgMaxLevels];
  T* Wl[kMgMaxLevels];
  T* p = reinterpret_cast<T*>(smbase ? smbase : mg_sm);
  d[0] = d0;
  for (int l = 0; l < nlev; ++l) {
    if (l > 0) d[l] = MgLevel{d[l - 1].n1 / 2, d[l - 1].n2 / 2, d[l - 1].n3 / 2};
    const int G = d[l].n1 * d[l].n2 * d[l].n3;
    Rl[l] = p;
    Zl[l] = p + G;
    Wl[l] = p + 2 * G;
    p += 3 * G;
  }
  const T a = T(1) - omega, b = omega / T(6);
  {
    const int G = d0.n1 * d0.n2 * d0.n3;
    for (int q = tid; q < G; q += NTH) Rl[0][q] = r[q];
  }
  __syncthreads();
  T s = s0;
  for (int l = 0; l + 1 < nlev; ++l, s *= T(4)) {
    const MgLevel& dl = d[l];
    const long long plane = (long long)dl.n1 * dl.n2;
    const int G = dl.n1 * dl.n2 * dl.n3;
    for (int q = tid; q < G; q += NTH) {
      int i, j, k;
      mg_ijk(q, dl, i, j, k);
      Wl[l][q] = a * Rl[l][q] + b * mg_nb_sum(Rl[l], i, j, k, dl, q, plane);
    }
    __syncthreads();
    const MgLevel& dc = d[l + 1];
    const int Gc = dc.n1 * dc.n2 * dc.n3;
    for (int q = tid; q < Gc; q += NTH) {
      int I, J, K;
      mg_ijk(q, dc, I, J, K);
      Rl[l + 1][q] = mg_restrict_at(Wl[l], dl, I, J, K);
    }
    __syncthreads();
  }
  {  // bottom: Jacobi sweeps from zero, alternating between Z and W
    const int l = nlev - 1;
    const MgLevel& dl = d[l];
    const long long plane = (long long)dl.n1 * dl.n2;
    const int G = dl.n1 * dl.n2 * dl.n3;
    T* cur = Zl[l];
    T* nxt = Wl[l];
    for (int q = tid; q < G; q += NTH) cur[q] = s * Rl[l][q];
    __syncthreads();
    for (int it = 1; it < sweeps; ++it) {
      for (int q = tid; q < G; q += NTH) {
        int i, j, k;
        mg_ijk(q, dl, i, j, k);
        nxt[q] = a * cur[q] + s * Rl[l][q] + b * mg_nb_sum(cur, i, j, k, dl, q, plane);
      }
      __syncthreads();
      T* tmp = cur;
      cur = nxt;
      nxt = tmp;
    }
    if (cur != Zl[l]) {
      for (int q = tid; q < G; q += NTH) Zl[l][q] = cur[q];
      __syncthreads();
    }
  }
  for (int l = nlev - 2; l >= 0; --l) {
    s *= T(0.25);
    const MgLevel& dl = d[l];
    const long long plane = (long long)dl.n1 * dl.n2;
    const int G = dl.n1 * dl.n2 * dl.n3;
    for (int q = tid; q < G; q += NTH) {
      int i, j, k;
      mg_ijk(q, dl, i, j, k);
      Wl[l][q] = s * Rl[l][q] + mg_prolong_at(Zl[l + 1], d[l + 1], i, j, k);
    }
    __syncthreads();
    for (int q = tid; q < G; q += NTH) {
      int i, j, k;
      mg_ijk(q, dl, i, j, k);
      Zl[l][q] = a * Wl[l][q] + s * Rl[l][q] + b * mg_nb_sum(Wl[l], i, j, k, dl, q, plane);
    }
    __syncthreads();
  }
  const int G0 = d0.n1 * d0.n2 * d0.n3;
  DotAcc<T> acc;
  for (int q = tid; q < G0; q += NTH) {
    const T zq = Zl[0][q];
    z[q] = zq;
    if constexpr (DOT) acc.add(Rl[0][q], zq);
  }
  if constexpr (DOT) {
    double v[1] = {acc.value()};
    block_sum<1, NTH>(v, red_sm, tid);
    if (tid == 0) MgFin{sc}(v);
  }
}

template <typename T, bool DOT>
__global__ void __launch_bounds__(1024) mg_coarse_kernel(MgLevel d0, int nlev, const T* __restrict__ r,
                                                         T* __restrict__ z, T omega, T s0, int sweeps,
                                                         CgScalars* sc) {
  pdl_enter();
  mg_coarse_body<T, DOT>(d0, nlev, r, z, omega, s0, sweeps, sc);
}

// The coarse end of the V-cycle on one thread-block cluster (single grids).
// Levels lq .. lc-1, each small enough that its launches are latency-bound,
// live in the distributed shared memory of kMgClusterCtas blocks: level l's
// three arrays (r, w = t or y, z) are split by z-planes, block q of the
// cluster holding planes [q P_l, (q + 1) P_l) at the same offset of its own
// shared memory, and every pass reads its neighbours (other blocks' planes
// included) through the cluster's shared-memory window.  A cluster barrier
// (hardware, all blocks co-scheduled) separates the passes.  Levels lc and
// below run as the one-block coarse end in block 0 (global r and z of level
// lc).  Every node's formulas, in their order, are those of the separate
// level passes (mg_down / restrict / prolong / up) and of mg_coarse_kernel; the
// cycle agrees with theirs to rounding (the compiler is free to contract a
// product into an FMA differently in the two kernels).
constexpr int kMgClusterCtas = 8;  // the portable cluster size
struct MgSlab {
  MgLevel d;
  int P;         // z-planes per block
  unsigned off;  // element offset of the level's arrays in each block's shared memory
};
template <typename T>
struct MgClusterArgs {
  MgSlab L[kMgMaxLevels];
  T s[kMgMaxLevels];  // the cycle's scale s at each level, as the host forms it
  int lq, lc, ncoarse;  // first cluster level, the coarse-end level, levels of the coarse end
  const T* r_in;      // r of level lq (global)
  T* z_out;           // z of level lq (global)
  T* r_tail;          // r of level lc (global)
  T* z_tail;          // z of level lc (global)
  unsigned tail_off;  // byte offset of block 0's coarse-end arrays
  T omega;
  int sweeps;
};

// Rows (fixed j, k; contiguous in x) of array a of a cluster level, wherever
// in the cluster they live.
template <typename T>
struct MgRows {
  T* sm;  // this block's shared memory (element type)
  MgSlab L;
  int a;
  __device__ __forceinline__ T* operator()(int j, int k) const {
    namespace cg = cooperative_groups;
    const int q = k / L.P;
    T* local = sm + L.off + (size_t)a * L.P * L.d.n1 * L.d.n2 + ((size_t)(k - q * L.P) * L.d.n2 + j) * L.d.n1;
    return cg::this_cluster().map_shared_rank(local, q);
  }
};

// The level passes' per-node formulas over row accessors, in the order of
// mg_nb_sum, mg_restrict_at and mg_prolong_at.
template <typename T, class Rows>
__device__ __forceinline__ T mgc_nb_sum(const Rows& f, int i, int j, int k, const MgLevel& d) {
  const T* row = f(j, k);
  T s = T(0);
  if (i > 0) s += row[i - 1];
  if (i + 1 < d.n1) s += row[i + 1];
  if (j > 0) s += f(j - 1, k)[i];
  if (j + 1 < d.n2) s += f(j + 1, k)[i];
  if (k > 0) s += f(j, k - 1)[i];
  if (k + 1 < d.n3) s += f(j, k + 1)[i];
  return s;
}
template <typename T, class Rows>
__device__ __forceinline__ T mgc_restrict_at(const Rows& t, const MgLevel& f, int I, int J, int K) {
  T acc = T(0);
#pragma unroll
  for (int dk = 0; dk < 3; ++dk) {
    const int kk = 2 * K + dk;
    if (kk >= f.n3) continue;
    const T wz = dk == 1 ? T(0.5) : T(0.25);
#pragma unroll
    for (int dj = 0; dj < 3; ++dj) {
      const int jj = 2 * J + dj;
      if (jj >= f.n2) continue;
      const T wy = dj == 1 ? T(0.5) : T(0.25);
      const T* row = t(jj, kk);
      const int ii = 2 * I;
      T sx = T(0.25) * row[ii] + T(0.5) * row[ii + 1];
      if (ii + 2 < f.n1) sx += T(0.25) * row[ii + 2];
      acc += wz * wy * sx;
    }
  }
  return acc;
}
template <typename T, class Rows>
__device__ __forceinline__ T mgc_prolong_at(const Rows& e, const MgLevel& c, int i, int j, int k) {
  int x0, x1, y0, y1, z0, z1;
  T wx0, wx1, wy0, wy1, wz0, wz1;
  mg_axis(i, c.n1, x0, x1, wx0, wx1);
  mg_axis(j, c.n2, y0, y1, wy0, wy1);
  mg_axis(k, c.n3, z0, z1, wz0, wz1);
  const T* r00 = e(y0, z0);
  const T* r01 = e(y1, z0);
  const T* r10 = e(y0, z1);
  const T* r11 = e(y1, z1);
  const T a00 = wx0 * r00[x0] + wx1 * r00[x1];
  const T a01 = wx0 * r01[x0] + wx1 * r01[x1];
  const T a10 = wx0 * r10[x0] + wx1 * r10[x1];
  const T a11 = wx0 * r11[x0] + wx1 * r11[x1];
  return wz0 * (wy0 * a00 + wy1 * a01) + wz1 * (wy0 * a10 + wy1 * a11);
}
// rows of a global level array
template <typename T>
struct MgGlobalRows {
  T* f;
  MgLevel d;
  __device__ __forceinline__ T* operator()(int j, int k) const {
    return f + (long long)d.n1 * d.n2 * k + (long long)d.n1 * j;
  }
};

template <typename T>
__global__ void __cluster_dims__(kMgClusterCtas, 1, 1) __launch_bounds__(1024)
    mg_cluster_kernel(MgClusterArgs<T> A, CgScalars* sc) {
  pdl_enter();
  namespace cg = cooperative_groups;
  extern __shared__ __align__(16) unsigned char mgc_sm[];
  cg::cluster_group cluster = cg::this_cluster();
  if (sc->done) return;  // the same flag for every block: the whole cluster returns
  const int q = (int)cluster.block_rank();
  const int tid = threadIdx.x;
  T* sm = reinterpret_cast<T*>(mgc_sm);
  const T a = T(1) - A.omega, b = A.omega / T(6);
  // this block's nodes of level l: planes [q P, min((q + 1) P, n3))
  auto own = [&](const MgSlab& L, int& k0, int& k1) {
    k0 = min(q * L.P, L.d.n3);
    k1 = min(k0 + L.P, L.d.n3);
  };
  {  // r of level lq from global memory
    const MgSlab& L = A.L[A.lq];
    int k0, k1;
    own(L, k0, k1);
    const int plane = L.d.n1 * L.d.n2;
    const T* src = A.r_in + (long long)plane * k0;
    T* dst = sm + L.off;
    for (int e = tid; e < plane * (k1 - k0); e += 1024) dst[e] = src[e];
  }
  cluster.sync();
  for (int l = A.lq; l < A.lc; ++l) {
    const MgSlab& L = A.L[l];
    const MgRows<T> R{sm, L, 0}, Wr{sm, L, 1};
    int k0, k1;
    own(L, k0, k1);
    const int n1 = L.d.n1, n2 = L.d.n2;
    for (int e = tid; e < n1 * n2 * (k1 - k0); e += 1024) {  // down: w = (1 - omega) r + (omega / 6) sum_nb r
      const int i = e % n1, jk = e / n1, j = jk % n2, k = k0 + jk / n2;
      Wr(j, k)[i] = a * R(j, k)[i] + b * mgc_nb_sum<T>(R, i, j, k, L.d);
    }
    cluster.sync();
    const MgLevel& dc = A.L[l + 1].d;
    if (l + 1 < A.lc) {  // restrict into the next cluster level's r
      const MgSlab& C = A.L[l + 1];
      const MgRows<T> Rc{sm, C, 0};
      int c0, c1;
      own(C, c0, c1);
      for (int e = tid; e < dc.n1 * dc.n2 * (c1 - c0); e += 1024) {
        const int I = e % dc.n1, JK = e / dc.n1, J = JK % dc.n2, K = c0 + JK / dc.n2;
        Rc(J, K)[I] = mgc_restrict_at<T>(Wr, L.d, I, J, K);
      }
    } else {  // restrict into the coarse end's r (global), split over the blocks by planes
      const MgGlobalRows<T> Rg{A.r_tail, dc};
      const int Pc = (dc.n3 + kMgClusterCtas - 1) / kMgClusterCtas;
      const int c0 = min(q * Pc, dc.n3), c1 = min(c0 + Pc, dc.n3);
      for (int e = tid; e < dc.n1 * dc.n2 * (c1 - c0); e += 1024) {
        const int I = e % dc.n1, JK = e / dc.n1, J = JK % dc.n2, K = c0 + JK / dc.n2;
        Rg(J, K)[I] = mgc_restrict_at<T>(Wr, L.d, I, J, K);
      }
    }
    cluster.sync();
  }
  // the coarse end in block 0 (levels lc and below, its own shared memory)
  if (q == 0)
    mg_coarse_body<T, false>(A.L[A.lc].d, A.ncoarse, A.r_tail, A.z_tail, A.omega, A.s[A.lc], A.sweeps, sc,
                             mgc_sm + A.tail_off);
  cluster.sync();
  for (int l = A.lc - 1; l >= A.lq; --l) {
    const MgSlab& L = A.L[l];
    const MgRows<T> R{sm, L, 0}, Y{sm, L, 1}, Z{sm, L, 2};
    const T s = A.s[l];
    int k0, k1;
    own(L, k0, k1);
    const int n1 = L.d.n1, n2 = L.d.n2;
    const MgLevel& dc = A.L[l + 1].d;
    if (l + 1 < A.lc) {  // prolong: y = s r + P e_c
      const MgRows<T> Ec{sm, A.L[l + 1], 2};
      for (int e = tid; e < n1 * n2 * (k1 - k0); e += 1024) {
        const int i = e % n1, jk = e / n1, j = jk % n2, k = k0 + jk / n2;
        Y(j, k)[i] = s * R(j, k)[i] + mgc_prolong_at<T>(Ec, dc, i, j, k);
      }
    } else {
      const MgGlobalRows<T> Ec{A.z_tail, dc};
      for (int e = tid; e < n1 * n2 * (k1 - k0); e += 1024) {
        const int i = e % n1, jk = e / n1, j = jk % n2, k = k0 + jk / n2;
        Y(j, k)[i] = s * R(j, k)[i] + mgc_prolong_at<T>(Ec, dc, i, j, k);
      }
    }
    cluster.sync();
    // up: z = (1 - omega) y + s r + (omega / 6) sum_nb y; level lq's z goes to global memory
    T* zg = (l == A.lq) ? A.z_out : nullptr;
    for (int e = tid; e < n1 * n2 * (k1 - k0); e += 1024) {
      const int i = e % n1, jk = e / n1, j = jk % n2, k = k0 + jk / n2;
      const T zi = a * Y(j, k)[i] + s * R(j, k)[i] + b * mgc_nb_sum<T>(Y, i, j, k, L.d);
      if (zg)
        zg[((long long)k * n2 + j) * n1 + i] = zi;
      else
        Z(j, k)[i] = zi;
    }
    cluster.sync();
  }
}

// The coarse end for several grids of a batch (S11): block b takes job b.
template <typename T>
struct MgCoarseJob {
  MgLevel d0;
  int nlev;
  const T* r;
  T* z;
  T s0;
  CgScalars* sc;
};

template <typename T, bool DOT>
__global__ void __launch_bounds__(1024) mg_coarse_batch_kernel(const MgCoarseJob<T>* __restrict__ jobs, T omega,
                                                               int sweeps) {
  const MgCoarseJob<T> j = jobs[blockIdx.x];
  mg_coarse_body<T, DOT>(j.d0, j.nlev, j.r, j.z, omega, j.s0, sweeps, j.sc);
}

// ----------------------------------------------------------- vector ops ---
// s -= gamma w (rank-one correction of the preconditioned residual).
template <typename T>
__global__ void __launch_bounds__(256) rank1_kernel(long long G, T* s, const T* w, double gamma) {
  const T ga = (T)gamma;
  for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < G; i += (long long)gridDim.x * 256)
    s[i] = fma(-ga, w[i], s[i]);
}

// out = |a + alpha b| (trial point and secant update of Sec. 4, u <- |u|).
template <typename T>
__global__ void __launch_bounds__(256) axpy_abs_kernel(long long G, T* out, const T* a, const T* b,
                                                       double alpha) {
  const T al = (T)alpha;
  for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < G; i += (long long)gridDim.x * 256)
    out[i] = fabs(fma(al, b[i], a[i]));
}

// d = s + beta d (Polak-Ribiere direction), or d = s when beta == 0.
template <typename T>
__global__ void __launch_bounds__(256) direction_kernel(long long G, T* d, const T* s, double beta) {
  const T be = (T)beta;
  for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < G; i += (long long)gridDim.x * 256)
    d[i] = (beta == 0.0) ? s[i] : fma(be, d[i], s[i]);
}

// out[0] = a.b, out[1] = c.e (c may be NULL).  Per-thread sums in DotAcc: FP64
// for double fields, compensated FP32 pairs for float fields (the FP64 pipe
// issues at a small fraction of the FP32 rate here).
template <typename T>
__global__ void __launch_bounds__(256) dot2_kernel(long long G, const T* a, const T* b, const T* c,
                                                   const T* e, double* out, RedBuf red) {
  __shared__ double smem[2 * (256 / 32)];
  DotAcc<T> d0, d1;
  for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < G; i += (long long)gridDim.x * 256) {
    d0.add(a[i], b[i]);
    if (c) d1.add(c[i], e[i]);
  }
  double acc[2] = {d0.value(), d1.value()};
  struct Fin {
    double* out;
    __device__ void operator()(double* t) const {
      out[0] = t[0];
      out[1] = t[1];
    }
  } fin{out};
  grid_sum<2, 256>(acc, smem, red, gridDim.x, blockIdx.x, threadIdx.x, fin);
}

// out = ca a + cb b (b may be NULL), |.| when take_abs: the projections,
// scalings and the norm-preserving rotation |cos t u0 + sin t dh| of the
// Lagrange-multiplier method.  out may alias a or b.
template <typename T>
__global__ void __launch_bounds__(256) lincomb_kernel(long long G, T* out, const T* a, double ca, const T* b,
                                                      double cb, int take_abs) {
  const T xa = (T)ca, xb = (T)cb;
  for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < G; i += (long long)gridDim.x * 256) {
    T v = xa * a[i];
    if (b) v = fma(xb, b[i], v);
    out[i] = take_abs ? fabs(v) : v;
  }
}

// Preconditioned projected gradient of the Lagrange-multiplier method (Sec. 5.3.2)
// from the energy gradient G_E at u: g = G_E - 2 eta u (written over G), the
// Jacobi diagonal of the functional pass with multiplier term -eta, s = -g / diag.
// out[0] = s.u, out[1] = u.u (the caller projects s orthogonal to u).
template <typename T>
__global__ void __launch_bounds__(256) lm_precond_kernel(long long G, T* g, T* s, const T* u, const T* phi,
                                                         FuncScalars f, double* out, RedBuf red) {
  __shared__ double smem[2 * (256 / 32)];
  double acc[2] = {0.0, 0.0};
  const bool tf = f.terms & 1, vw = f.terms & 2, xc = f.terms & 4, es = f.terms & 8;
  const T eta = (T)f.eta;
  for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < G; i += (long long)gridDim.x * 256) {
    const T uc = u[i], ux = fabs(uc);
    T vk = T(0), vxc = T(0), exc = T(0);
    if (tf) {
      const T c = cbrt(ux);
      vk = (T)(5.0 / 3.0 * f.CF) * ((c * c) * (c * c));
    }
    if (xc) xc_eval<T>(ux, exc, vxc);
    const T ph = es ? phi[i] : T(0);
    const T gi = fma(T(-2) * eta, uc, g[i]);
    const T kin = (vw ? (T)f.kin_vw : T(0)) + (T)(14.0 / 3.0) * vk;
    T md = kin + T(2) * (vxc + ph - eta);
    md = fmax(md, (T)0.25 * kin);
    md = fmax(md, (T)1e-10);
    const T si = -gi / md;
    g[i] = gi;
    s[i] = si;
    acc[0] += (double)si * (double)uc;
    acc[1] += (double)uc * (double)uc;
  }
  struct Fin {
    double* out;
    __device__ void operator()(double* t) const {
      out[0] = t[0];
      out[1] = t[1];
    }
  } fin{out};
  grid_sum<2, 256>(acc, smem, red, gridDim.x, blockIdx.x, threadIdx.x, fin);
}

// u *= scale where scale = sqrt(N / (h^3 sum)) from the device sum (initial guess).
template <typename T>
__global__ void __launch_bounds__(256) normalise_kernel(long long G, T* u, const double* sum, double h3,
                                                        double N) {
  const double sc = (*sum > 0.0) ? sqrt(N / (h3 * *sum)) : 0.0;
  for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < G; i += (long long)gridDim.x * 256)
    u[i] = (T)(sc * (double)u[i]);
}

// phi64 += e; e = 0 (folds a round's FP32 correction into the FP64 potential).
static __global__ void __launch_bounds__(256) fold_kernel(long long G, double* phi64, float* e, float2* phi2) {
  for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < G; i += (long long)gridDim.x * 256) {
    const double v = phi64[i] + (double)e[i];
    phi64[i] = v;
    e[i] = 0.0f;
    if (phi2) {
      const float hi = (float)v;
      phi2[i] = make_float2(hi, (float)(v - (double)hi));
    }
  }
}

// phi += t (phi - phi0): linear extrapolation of the potential along a line
// search (warm start of the next Poisson solve).
static __global__ void __launch_bounds__(256) extrap_kernel(long long G, double* phi, const double* phi0, double t) {
  for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < G; i += (long long)gridDim.x * 256)
    phi[i] = fma(t, phi[i] - phi0[i], phi[i]);
}

template <typename S, typename D>
__global__ void __launch_bounds__(256) convert_kernel(long long G, D* out, const S* in) {
  for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < G; i += (long long)gridDim.x * 256)
    out[i] = (D)in[i];
}

// ------------------------------------------------- batched pointwise ops ---
// CG second half on one grid of a batch (same arithmetic as cg_update_kernel).
// CG second half with the iterate update folded into the next stencil pass
// (same arithmetic as cg_update_r_kernel).
template <typename T>
struct OpCgUpdateR {
  static constexpr int K = 1;
  T* r;
  const T* q;
  CgScalars* sc;
  RedBuf red;
  int nblocks;
  using Acc = DotAcc<T>;
  T al_ = T(0);
  __device__ __forceinline__ bool skip() const { return sc->done != 0; }
  __device__ __forceinline__ void load() { al_ = (T)sc->alpha; }
  __device__ __forceinline__ void apply(long long i, Acc* acc) const {
    const T ri = fma(-al_, q[i], r[i]);
    r[i] = ri;
    acc[0].add(ri, ri);
  }
  __device__ __forceinline__ void operator()(double* t) const {
    const double rr_new = t[0];
    sc->beta = (sc->rr != 0.0) ? rr_new / sc->rr : 0.0;
    sc->rr_prev = sc->rr;
    sc->rr = rr_new;
    sc->iters += 1;
    sc->xdefer = 1;
    const double thr = sc->tol2 * (sc->bb > 0.0 ? sc->bb : 1.0);
    if (rr_new <= thr || sc->iters >= sc->max_it || !(rr_new == rr_new)) sc->done = 1;
  }
};

// Pending x += alpha p of one grid after its CG loop (as cg_xflush_kernel); the
// last block clears xdefer.
template <typename T>
struct OpXFlush {
  static constexpr int K = 1;
  T* x;
  const T* p;
  CgScalars* sc;
  RedBuf red;
  int nblocks;
  using Acc = double;
  int on_ = 0;
  T al_ = T(0);
  __device__ __forceinline__ bool skip() const { return false; }
  __device__ __forceinline__ void load() {
    on_ = sc->xdefer;
    al_ = (T)sc->alpha;
  }
  __device__ __forceinline__ void apply(long long i, Acc*) const {
    if (on_) x[i] = fma(al_, p[i], x[i]);
  }
  __device__ __forceinline__ void operator()(double*) const { sc->xdefer = 0; }
};

template <typename T, typename X = T>
struct OpCgUpdate {
  static constexpr int K = 1;
  X* x;
  T* r;
  const T* p;
  const T* q;
  CgScalars* sc;
  RedBuf red;
  int nblocks;
  using Acc = DotAcc<T>;
  T al_ = T(0);
  X alx_ = X(0);
  __device__ __forceinline__ bool skip() const { return sc->done != 0; }
  __device__ __forceinline__ void load() {
    al_ = (T)sc->alpha;
    alx_ = (X)sc->alpha;
  }
  __device__ __forceinline__ void apply(long long i, Acc* acc) const {
    x[i] = fma(alx_, (X)p[i], x[i]);
    const T ri = fma(-al_, q[i], r[i]);
    r[i] = ri;
    acc[0].add(ri, ri);
  }
  __device__ __forceinline__ void operator()(double* t) const {
    const double rr_new = t[0];
    sc->beta = (sc->rr != 0.0) ? rr_new / sc->rr : 0.0;
    sc->rr_prev = sc->rr;
    sc->rr = rr_new;
    sc->iters += 1;
    const double thr = sc->tol2 * (sc->bb > 0.0 ? sc->bb : 1.0);
    if (rr_new <= thr || sc->iters >= sc->max_it || !(rr_new == rr_new)) sc->done = 1;
  }
};

// Multigrid passes of one grid of a batch (S11), element i a node of the
// op's level; same arithmetic as mg_down/restrict/prolong/up_kernel.
template <typename T>
struct OpMgDown {
  static constexpr int K = 0;
  using Acc = double;
  MgLevel d;
  const T* r;
  T* t;
  T om;
  const CgScalars* sc;
  RedBuf red;
  int nblocks;
  __device__ __forceinline__ bool skip() const { return sc->done != 0; }
  __device__ __forceinline__ void load() {}
  __device__ __forceinline__ void apply(long long idx, Acc*) const {
    int i, j, k;
    mg_ijk(idx, d, i, j, k);
    const long long plane = (long long)d.n1 * d.n2;
    t[idx] = (T(1) - om) * r[idx] + (om / T(6)) * mg_nb_sum(r, i, j, k, d, idx, plane);
  }
  __device__ __forceinline__ void operator()(double*) const {}
};

template <typename T>
struct OpMgRestrict {
  static constexpr int K = 0;
  using Acc = double;
  MgLevel f, c;
  const T* t;
  T* rc;
  const CgScalars* sc;
  RedBuf red;
  int nblocks;
  __device__ __forceinline__ bool skip() const { return sc->done != 0; }
  __device__ __forceinline__ void load() {}
  __device__ __forceinline__ void apply(long long idx, Acc*) const {
    int I, J, K3;
    mg_ijk(idx, c, I, J, K3);
    rc[idx] = mg_restrict_at(t, f, I, J, K3);
  }
  __device__ __forceinline__ void operator()(double*) const {}
};

template <typename T>
struct OpMgProlong {
  static constexpr int K = 0;
  using Acc = double;
  MgLevel f, c;
  const T* r;
  const T* ec;
  T* y;
  T s;
  const CgScalars* sc;
  RedBuf red;
  int nblocks;
  __device__ __forceinline__ bool skip() const { return sc->done != 0; }
  __device__ __forceinline__ void load() {}
  __device__ __forceinline__ void apply(long long idx, Acc*) const {
    int i, j, k;
    mg_ijk(idx, f, i, j, k);
    y[idx] = s * r[idx] + mg_prolong_at(ec, c, i, j, k);
  }
  __device__ __forceinline__ void operator()(double*) const {}
};

template <typename T, bool DOT>
struct OpMgUp {
  static constexpr int K = DOT ? 1 : 0;
  using Acc = DotAcc<T>;
  MgLevel d;
  const T* r;
  const T* y;
  T* z;
  T om, s;
  CgScalars* sc;
  RedBuf red;
  int nblocks;
  __device__ __forceinline__ bool skip() const { return sc->done != 0; }
  __device__ __forceinline__ void load() {}
  __device__ __forceinline__ void apply(long long idx, Acc* acc) const {
    int i, j, k;
    mg_ijk(idx, d, i, j, k);
    const long long plane = (long long)d.n1 * d.n2;
    const T ri = r[idx];
    const T zi = (T(1) - om) * y[idx] + s * ri + (om / T(6)) * mg_nb_sum(y, i, j, k, d, idx, plane);
    z[idx] = zi;
    if constexpr (DOT) acc[0].add(ri, zi);
  }
  __device__ __forceinline__ void operator()(double* t) const {
    if constexpr (DOT) MgFin{sc}(t);
  }
};

// out = |a + alpha b| (trial point / secant update, u <- |u|).
template <typename T>
struct OpAxpyAbs {
  static constexpr int K = 0;
  T* out;
  const T* a;
  const T* b;
  double alpha;
  using Acc = double;
  __device__ __forceinline__ void load() {}
  __device__ __forceinline__ bool skip() const { return false; }
  __device__ __forceinline__ void apply(long long i, double*) const { out[i] = fabs(fma((T)alpha, b[i], a[i])); }
  __device__ __forceinline__ void operator()(double*) const {}
};

// d = s + beta d (Polak-Ribiere), d = s when beta == 0.
template <typename T>
struct OpDirection {
  static constexpr int K = 0;
  T* d;
  const T* s;
  double beta;
  using Acc = double;
  __device__ __forceinline__ void load() {}
  __device__ __forceinline__ bool skip() const { return false; }
  __device__ __forceinline__ void apply(long long i, double*) const {
    d[i] = (beta == 0.0) ? s[i] : fma((T)beta, d[i], s[i]);
  }
  __device__ __forceinline__ void operator()(double*) const {}
};

// out[0] = a.b, out[1] = c.e (FP64 accumulation).
template <typename T>
struct OpDot2 {
  static constexpr int K = 2;
  const T* a;
  const T* b;
  const T* c;
  const T* e;
  double* out;
  RedBuf red;
  int nblocks;
  using Acc = double;
  __device__ __forceinline__ void load() {}
  __device__ __forceinline__ bool skip() const { return false; }
  __device__ __forceinline__ void apply(long long i, double* acc) const {
    acc[0] += (double)a[i] * (double)b[i];
    acc[1] += (double)c[i] * (double)e[i];
  }
  __device__ __forceinline__ void operator()(double* t) const {
    out[0] = t[0];
    out[1] = t[1];
  }
};

// s -= gamma w (rank-one correction of the preconditioner).
template <typename T>
struct OpRank1 {
  static constexpr int K = 0;
  T* s;
  const T* w;
  double gamma;
  using Acc = double;
  __device__ __forceinline__ void load() {}
  __device__ __forceinline__ bool skip() const { return false; }
  __device__ __forceinline__ void apply(long long i, double*) const { s[i] = fma(-(T)gamma, w[i], s[i]); }
  __device__ __forceinline__ void operator()(double*) const {}
};

// Residual replacement of the mixed CG on one grid (see refine_replace_kernel).
struct OpRefineReplace {
  static constexpr int K = 1;
  float* r32;
  const double* r64;
  CgScalars* sc;
  double tol;
  int budget, restart;
  RedBuf red;
  int nblocks;
  int pc = 0;  // the FP32 CG is preconditioned
  using Acc = double;
  __device__ __forceinline__ void load() {}
  __device__ __forceinline__ bool skip() const { return false; }
  __device__ __forceinline__ void apply(long long i, double* acc) const {
    const float v = (float)r64[i];
    r32[i] = v;
    acc[0] += (double)v * (double)v;
  }
  __device__ __forceinline__ void operator()(double* t) const {
    sc->pc = pc;
    if (restart) {
      sc->first = 1;
      sc->beta = 0.0;
      sc->iters = 0;
    } else {
      sc->beta = (sc->rr_prev != 0.0) ? t[0] / sc->rr_prev : 0.0;
    }
    sc->rr = t[0];
    sc->rr0 = t[0];
    sc->bb = t[0];
    sc->xdefer = 0;
    sc->err = 0;
    sc->tol2 = tol * tol;
    sc->max_it = sc->iters + budget;
    sc->done = (t[0] == 0.0 || budget <= 0) ? 1 : 0;
  }
};

// phi64 += e; e = 0 on one grid of a batch.
struct OpFold {
  static constexpr int K = 0;
  double* phi64;
  float* e;
  using Acc = double;
  __device__ __forceinline__ void load() {}
  __device__ __forceinline__ bool skip() const { return false; }
  __device__ __forceinline__ void apply(long long i, double*) const {
    phi64[i] += (double)e[i];
    e[i] = 0.0f;
  }
  __device__ __forceinline__ void operator()(double*) const {}
};

// Warm start of a line search's Poisson solves on one grid: t == 0 records
// phi0 = phi (the origin), otherwise phi += t (phi - phi0) (as extrap_kernel).
struct OpLine {
  static constexpr int K = 0;
  double* phi;
  double* phi0;
  double t;
  using Acc = double;
  __device__ __forceinline__ void load() {}
  __device__ __forceinline__ bool skip() const { return false; }
  __device__ __forceinline__ void apply(long long i, double*) const {
    if (t == 0.0)
      phi0[i] = phi[i];
    else
      phi[i] = fma(t, phi[i] - phi0[i], phi[i]);
  }
  __device__ __forceinline__ void operator()(double*) const {}
};

template <typename S, typename D>
struct OpConvert {
  static constexpr int K = 0;
  D* out;
  const S* in;
  using Acc = double;
  __device__ __forceinline__ void load() {}
  __device__ __forceinline__ bool skip() const { return false; }
  __device__ __forceinline__ void apply(long long i, double*) const { out[i] = (D)in[i]; }
  __device__ __forceinline__ void operator()(double*) const {}
};

// ------------------------------------------------------------ atom kernels --
// Node-to-atom offsets and distances computed with explicitly rounded IEEE
// operations (no FMA contraction), so that every "is this node inside the
// ball" decision is taken exactly as plain FP64 arithmetic takes it.
__device__ __forceinline__ double node_off(double origin, int i, double h, double Ra) {
  return __dsub_rn(__dadd_rn(origin, __dmul_rn(__dadd_rn((double)i, 0.5), h)), Ra);
}
__device__ __forceinline__ double dist3(double x, double y, double z) {
  return __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z)));
}
__device__ __forceinline__ double dist3_sq(double x, double y, double z) {
  return __dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z));
}

// Gaussian nucleus V(r) = -Z erf(r/sigma)/r and its r -> 0 limit.  From
// r = 6 sigma on, 1 - erf(r/sigma) = erfc(r/sigma) < 2.2e-17 is below half a
// unit in the last place of 1.0 (2^-54), so erf rounds to exactly 1 and
// V = -Z/r; that skips the erf on most of an atom's table (r up to r_c + n h).
__device__ __forceinline__ double gauss_v(double Z, double inv_sigma, double r) {
  if (r < 1e-12 / inv_sigma) return -2.0 * Z * inv_sigma * 0.56418958354775628;  // 1/sqrt(pi)
  const double x = r * inv_sigma;
  if (x >= 6.0) return -Z / r;
  return -Z * erf(x) / r;
}

// Conservative FP32 screen of node-to-atom distances.  The offset of a box's
// first node is formed in FP64 once, then node i of an axis sits at
// x0 + i h in FP32: on boxes of up to a few thousand nodes and offsets of up
// to a few hundred bohr its error stays below 1e-4 bohr, so a node whose
// screened distance exceeds r (1 + 1e-4) + 1e-3 is farther than r in exact
// arithmetic too.  Nodes that pass take the unchanged FP64 path, so every
// value and every inside/outside decision is the one the FP64 code takes;
// the screen only skips FP64 work (a small fraction of the FP32 rate here) on
// nodes that cannot contribute.
struct DistScreen {
  float x0, y0, z0, h, r2;
  __device__ __forceinline__ bool maybe_within(int i, int j, int k) const {
    const float x = fmaf((float)i, h, x0), y = fmaf((float)j, h, y0), z = fmaf((float)k, h, z0);
    return x * x + y * y + z * z <= r2;
  }
};
__device__ __forceinline__ float screen_r2(double r) {
  const float rs = (float)(r * (1.0 + 1e-4) + 1e-3);
  return rs * rs;
}

struct AtomArgs {
  const double* R;  // M x 3
  const double* Z;  // M
  int M;
  double h, ox, oy, oz;  // spacing and origin
  double sigma, rc;
};

constexpr int AT = 8;  // atom-kernel tile edge (AT^3 = 512 threads)

// Ordered list (in atom order) of the atoms of [a0, a0+512) whose ball of radius
// `reach` meets the tile's box; returns the count.  Deterministic order.
__device__ __forceinline__ int tile_atoms(const AtomArgs& A, int a0, double cx, double cy, double cz,
                                          double half, double reach, int* list, int* warp_cnt) {
  const int tid = threadIdx.x + AT * (threadIdx.y + AT * threadIdx.z);
  const int lane = tid & 31, warp = tid >> 5;
  const int a = a0 + tid;
  bool hit = false;
  if (a < A.M) {
    const double dx = fmax(fabs(A.R[3 * a] - cx) - half, 0.0);
    const double dy = fmax(fabs(A.R[3 * a + 1] - cy) - half, 0.0);
    const double dz = fmax(fabs(A.R[3 * a + 2] - cz) - half, 0.0);
    hit = dx * dx + dy * dy + dz * dz < reach * reach;
  }
  const unsigned m = __ballot_sync(0xffffffffu, hit);
  if (lane == 0) warp_cnt[warp] = __popc(m);
  __syncthreads();
  int off = 0, total = 0;
  for (int w = 0; w < 16; ++w) {
    if (w < warp) off += warp_cnt[w];
    total += warp_cnt[w];
  }
  if (hit) list[off + __popc(m & ((1u << lane) - 1u))] = a;
  __syncthreads();
  return total;
}

// rho_0 = sum_J Z_J (2 pi s^2)^{-3/2} exp(-r^2/(2 s^2)) (r < cut); writes
// sqrt(rho_0) and reduces sum rho_0 (starting guess, Sec. 4).
template <typename T>
__global__ void __launch_bounds__(512) guess_kernel(GridDev g, AtomArgs A, double gsig, double gcut,
                                                    T* u, double* sum_out, RedBuf red) {
  __shared__ int list[512];
  __shared__ int warp_cnt[16];
  __shared__ double smem[512 / 32];
  const int x = blockIdx.x * AT + threadIdx.x, y = blockIdx.y * AT + threadIdx.y,
            z = blockIdx.z * AT + threadIdx.z;
  const int tid = threadIdx.x + AT * (threadIdx.y + AT * threadIdx.z);
  const bool inside = x < g.n1 && y < g.n2 && z < g.n3;
  const double half = 0.5 * AT * A.h;
  const double cx = A.ox + (blockIdx.x * AT) * A.h + half, cy = A.oy + (blockIdx.y * AT) * A.h + half,
               cz = A.oz + (blockIdx.z * AT) * A.h + half;
  const double norm = pow(2.0 * kPi * gsig * gsig, -1.5);
  // FP32 screen of the node's distance to each listed atom (see DistScreen):
  // node x sits at ox + (x + 1/2) h
  const float fx = (float)(A.ox + (x + 0.5) * A.h), fy = (float)(A.oy + (y + 0.5) * A.h),
              fz = (float)(A.oz + (z + 0.5) * A.h);
  const float cut2 = screen_r2(gcut);
  double rho = 0.0;
  for (int a0 = 0; a0 < A.M; a0 += 512) {
    const int cnt = tile_atoms(A, a0, cx, cy, cz, half, gcut + A.h, list, warp_cnt);
    if (inside) {
      for (int t = 0; t < cnt; ++t) {
        const int J = list[t];
        const float dx = fx - (float)A.R[3 * J], dy = fy - (float)A.R[3 * J + 1], dz = fz - (float)A.R[3 * J + 2];
        if (dx * dx + dy * dy + dz * dz > cut2) continue;
        const double rx = node_off(A.ox, x, A.h, A.R[3 * J]), ry = node_off(A.oy, y, A.h, A.R[3 * J + 1]),
                     rz = node_off(A.oz, z, A.h, A.R[3 * J + 2]);
        const double r2 = dist3_sq(rx, ry, rz);
        if (r2 < __dmul_rn(gcut, gcut)) rho += A.Z[J] * norm * exp(-r2 / (2.0 * gsig * gsig));
      }
    }
    __syncthreads();
  }
  if (inside) u[lin(g, x, y, z)] = (T)sqrt(rho);
  double acc[1] = {inside ? rho : 0.0};
  struct Fin {
    double* out;
    __device__ void operator()(double* t) const { out[0] = t[0]; }
  } fin{sum_out};
  const int nb = gridDim.x * gridDim.y * gridDim.z;
  const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  grid_sum<1, 512>(acc, smem, red, nb, bid, tid, fin);
}

// Per-atom box of lattice nodes [lo, lo + dim) (may extend outside the grid).
struct AtomBox {
  int lo[3];
  int dim[3];
};

// V_J tabulated on the atom's box grown by 2R: vbox[a][...], one block row per
// atom (blockIdx.y).  Only nodes within r_c + R h of the atom are ever read
// (the stencil neighbours of the nodes of its ball, where b_J is nonzero), so
// V_J is evaluated there only and the rest of the cube holds 0.
static __global__ void __launch_bounds__(256) force_vbox_kernel(AtomArgs A, int a0, int vdim, int R,
                                                         const int* __restrict__ lo, double* vbox) {
  const int a = blockIdx.y;
  const int J = a0 + a;
  const unsigned per = (unsigned)vdim * vdim * vdim;
  const double reach = A.rc + R * A.h + 1e-9 * (A.rc + A.h);
  const int bx = lo[3 * a] - 2 * R, by = lo[3 * a + 1] - 2 * R, bz = lo[3 * a + 2] - 2 * R;
  const double Rx = A.R[3 * J], Ry = A.R[3 * J + 1], Rz = A.R[3 * J + 2];
  const DistScreen sc{(float)node_off(A.ox, bx, A.h, Rx), (float)node_off(A.oy, by, A.h, Ry),
                      (float)node_off(A.oz, bz, A.h, Rz), (float)A.h, screen_r2(reach)};
  double* out = vbox + (size_t)a * per;
  for (unsigned e = blockIdx.x * 256 + threadIdx.x; e < per; e += gridDim.x * 256) {
    const unsigned jk = e / (unsigned)vdim;
    const int i = (int)(e - jk * (unsigned)vdim);
    const int k = (int)(jk / (unsigned)vdim);
    const int j = (int)(jk - (unsigned)k * (unsigned)vdim);
    double v = 0.0;
    if (sc.maybe_within(i, j, k)) {
      const double r = dist3(node_off(A.ox, bx + i, A.h, Rx), node_off(A.oy, by + j, A.h, Ry),
                             node_off(A.oz, bz + k, A.h, Rz));
      if (r <= reach) v = gauss_v(A.Z[J], 1.0 / A.sigma, r);
    }
    out[e] = v;
  }
}

// Pseudocharge from the atoms' tables (S1): for every node of a tile, the atoms
// of [a0, a0 + na) (na <= 512) whose ball can reach the tile, in atom order,
// add b_J (bbox, -(1/4 pi) L_h V_J inside r_c, 0 outside) to the node's running
// FP64 sum (bacc, carried across launches of successive atom ranges) and
// b_J V_J to the self-energy sum (added into es_out[0]).  The last range writes
// b in the field type.
template <typename T>
__global__ void __launch_bounds__(512) pseudocharge_gather_kernel(GridDev g, AtomArgs A, int a0, int na, int box,
                                                                  int bdim, int vdim, int R,
                                                                  const int* __restrict__ lo,
                                                                  const double* __restrict__ vbox,
                                                                  const double* __restrict__ bbox, double* bacc,
                                                                  int first, int last, T* b, double* es_out,
                                                                  RedBuf red) {
  __shared__ int list[512];
  __shared__ int warp_cnt[16];
  __shared__ double smem[512 / 32];
  const int x = blockIdx.x * AT + threadIdx.x, y = blockIdx.y * AT + threadIdx.y,
            z = blockIdx.z * AT + threadIdx.z;
  const int tid = threadIdx.x + AT * (threadIdx.y + AT * threadIdx.z);
  const bool inside = x < g.n1 && y < g.n2 && z < g.n3;
  const double half = 0.5 * AT * A.h;
  const double cx = A.ox + (blockIdx.x * AT) * A.h + half, cy = A.oy + (blockIdx.y * AT) * A.h + half,
               cz = A.oz + (blockIdx.z * AT) * A.h + half;
  AtomArgs Ar = A;
  Ar.M = a0 + na;  // the list covers this range only
  const int cnt = tile_atoms(Ar, a0, cx, cy, cz, half, A.rc + A.h, list, warp_cnt);
  const long long bper = (long long)bdim * bdim * bdim, vper = (long long)vdim * vdim * vdim;
  double es = 0.0;
  if (inside) {
    const long long node = lin(g, x, y, z);
    double bsum = first ? 0.0 : bacc[node];
    for (int t = 0; t < cnt; ++t) {
      const int a = list[t] - a0;
      const int ix = x - lo[3 * a], iy = y - lo[3 * a + 1], iz = z - lo[3 * a + 2];
      if (ix < 0 || iy < 0 || iz < 0 || ix >= box || iy >= box || iz >= box) continue;
      const double bj = bbox[a * bper + (ix + R) + (long long)bdim * ((iy + R) + (long long)bdim * (iz + R))];
      if (bj == 0.0) continue;
      bsum += bj;
      es += bj * vbox[a * vper + (ix + 2 * R) + (long long)vdim * ((iy + 2 * R) + (long long)vdim * (iz + 2 * R))];
    }
    if (last)
      b[node] = (T)bsum;
    else
      bacc[node] = bsum;
  }
  double acc[1] = {es};
  struct Fin {
    double* out;
    __device__ void operator()(double* t) const { out[0] += t[0]; }
  } fin{es_out};
  const int nb = gridDim.x * gridDim.y * gridDim.z;
  const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  grid_sum<1, 512>(acc, smem, red, nb, bid, tid, fin);
}

// b_J on the atom's box grown by R: -(1/4 pi) L_h V_J inside r_c, 0 outside;
// one block row per atom (blockIdx.y).
template <int R>
__global__ void __launch_bounds__(256) force_bbox_kernel(AtomArgs A, int a0, int vdim, int bdim,
                                                         const int* __restrict__ lo, Weights<double> W,
                                                         const double* __restrict__ vbox, double* bbox) {
  const int a = blockIdx.y;
  const int J = a0 + a;
  const unsigned per = (unsigned)bdim * bdim * bdim;
  const size_t vper = (size_t)vdim * vdim * vdim;
  const int bx = lo[3 * a] - R, by = lo[3 * a + 1] - R, bz = lo[3 * a + 2] - R;
  const double Rx = A.R[3 * J], Ry = A.R[3 * J + 1], Rz = A.R[3 * J + 2];
  const DistScreen sc{(float)node_off(A.ox, bx, A.h, Rx), (float)node_off(A.oy, by, A.h, Ry),
                      (float)node_off(A.oz, bz, A.h, Rz), (float)A.h, screen_r2(A.rc)};
  const double* v = vbox + (size_t)a * vper;
  double* out = bbox + (size_t)a * per;
  const long long sy = vdim, sz = (long long)vdim * vdim;
  for (unsigned e = blockIdx.x * 256 + threadIdx.x; e < per; e += gridDim.x * 256) {
    const unsigned jk = e / (unsigned)bdim;
    const int i = (int)(e - jk * (unsigned)bdim);
    const int k = (int)(jk / (unsigned)bdim);
    const int j = (int)(jk - (unsigned)k * (unsigned)bdim);
    double val = 0.0;
    if (sc.maybe_within(i, j, k) &&
        dist3(node_off(A.ox, bx + i, A.h, Rx), node_off(A.oy, by + j, A.h, Ry), node_off(A.oz, bz + k, A.h, Rz)) <
            A.rc) {
      const long long c = (long long)(i + R) + sy * (j + R) + sz * (k + R);
      double lap = W.c * v[c];
#pragma unroll
      for (int p = 1; p <= R; ++p)
        lap = fma(W.w[p], ((v[c + p] + v[c - p]) + (v[c + p * sy] + v[c - p * sy])) + (v[c + p * sz] + v[c - p * sz]), lap);
      val = -lap / (4.0 * kPi);
    }
    out[e] = val;
  }
}

// Force of atom a0+blockIdx.y: h^3 sum over in-grid ball nodes of
// grad(b_J) (phi - V_J); paper form uses the FD gradient (weights wt) of the
// tabulated b_J, exact form uses -(1/4 pi) L_h grad V_J (analytic grad V).
// One block row per atom; partial sums reduced per atom by force_sum_kernel.
template <typename T, int R>
__global__ void __launch_bounds__(256) force_ball_kernel(GridDev g, AtomArgs A, int a0, int bdim,
                                                         int box, const int* __restrict__ lo,
                                                         Weights<double> W, Weights<double> Wt,
                                                         const double* __restrict__ bbox,
                                                         const T* __restrict__ phi, int exact,
                                                         double* partial) {
  __shared__ double smem[3 * (256 / 32)];
  const int a = blockIdx.y;
  const int J = a0 + a;
  const long long per = (long long)box * box * box;
  const long long bper = (long long)bdim * bdim * bdim;
  const double inv_s = 1.0 / A.sigma;
  const DistScreen sc{(float)node_off(A.ox, lo[3 * a], A.h, A.R[3 * J]),
                      (float)node_off(A.oy, lo[3 * a + 1], A.h, A.R[3 * J + 1]),
                      (float)node_off(A.oz, lo[3 * a + 2], A.h, A.R[3 * J + 2]), (float)A.h, screen_r2(A.rc)};
  double acc[3] = {0.0, 0.0, 0.0};
  for (unsigned t = blockIdx.x * 256 + threadIdx.x; t < (unsigned)per; t += gridDim.x * 256) {
    const unsigned jk = t / (unsigned)box;
    const int i = (int)(t - jk * (unsigned)box);
    const int k = (int)(jk / (unsigned)box);
    const int j = (int)(jk - (unsigned)k * (unsigned)box);
    const int gi = lo[3 * a] + i, gj = lo[3 * a + 1] + j, gk = lo[3 * a + 2] + k;
    if (gi < 0 || gj < 0 || gk < 0 || gi >= g.n1 || gj >= g.n2 || gk >= g.n3) continue;
    if (!sc.maybe_within(i, j, k)) continue;
    const double rx = node_off(A.ox, gi, A.h, A.R[3 * J]);
    const double ry = node_off(A.oy, gj, A.h, A.R[3 * J + 1]);
    const double rz = node_off(A.oz, gk, A.h, A.R[3 * J + 2]);
    const double r = dist3(rx, ry, rz);
    if (!(r < A.rc)) continue;
    const double pv = (double)phi[lin(g, gi, gj, gk)] - gauss_v(A.Z[J], inv_s, r);
    double gx = 0.0, gy = 0.0, gz = 0.0;
    if (!exact) {
      const double* bb = bbox + (long long)a * bper;
      const long long c = (long long)(i + R) + (long long)bdim * ((j + R) + (long long)bdim * (k + R));
      const long long sy = bdim, sz = (long long)bdim * bdim;
#pragma unroll
      for (int p = 1; p <= R; ++p) {
        gx = fma(Wt.w[p], bb[c + p] - bb[c - p], gx);
        gy = fma(Wt.w[p], bb[c + p * sy] - bb[c - p * sy], gy);
        gz = fma(Wt.w[p], bb[c + p * sz] - bb[c - p * sz], gz);
      }
    } else {
      // -(1/4 pi) L_h grad V_J with grad V analytic: dV/dr = Z erf(r/s)/r^2 - Z (2/(s sqrt pi)) e^{-r^2/s^2}/r
      double lx = 0.0, ly = 0.0, lz = 0.0;
      for (int p = -R; p <= R; ++p) {
        for (int ax = 0; ax < 3; ++ax) {
          if (p == 0 && ax > 0) continue;
          const double ex = rx + (ax == 0 ? p * A.h : 0.0);
          const double ey = ry + (ax == 1 ? p * A.h : 0.0);
          const double ez = rz + (ax == 2 ? p * A.h : 0.0);
          const double rr = sqrt(ex * ex + ey * ey + ez * ez);
          double gvx = 0.0, gvy = 0.0, gvz = 0.0;
          if (rr > 1e-12 * A.sigma) {
            const double x = rr * inv_s;
            const double dVdr = A.Z[J] * erf(x) / (rr * rr) -
                                A.Z[J] * 2.0 * inv_s * 0.56418958354775628 * exp(-x * x) / rr;
            gvx = dVdr * ex / rr;
            gvy = dVdr * ey / rr;
            gvz = dVdr * ez / rr;
          }
          const double wp = (p == 0) ? W.c : W.w[p < 0 ? -p : p];
          lx = fma(wp, gvx, lx);
          ly = fma(wp, gvy, ly);
          lz = fma(wp, gvz, lz);
        }
      }
      gx = -lx / (4.0 * kPi);
      gy = -ly / (4.0 * kPi);
      gz = -lz / (4.0 * kPi);
    }
    acc[0] = fma(gx, pv, acc[0]);
    acc[1] = fma(gy, pv, acc[1]);
    acc[2] = fma(gz, pv, acc[2]);
  }
  block_sum<3, 256>(acc, smem, threadIdx.x);
  if (threadIdx.x == 0) {
    const long long o = ((long long)a * gridDim.x + blockIdx.x) * 3;
    partial[o] = acc[0];
    partial[o + 1] = acc[1];
    partial[o + 2] = acc[2];
  }
}

// F[J] = h^3 * (sum of the per-block partials of atom J, in block order).
static __global__ void force_sum_kernel(int a0, int na, int nblk, double h3, const double* partial, double* F) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= na) return;
  double f[3] = {0.0, 0.0, 0.0};
  for (int b = 0; b < nblk; ++b)
    for (int d = 0; d < 3; ++d) f[d] += partial[((long long)a * nblk + b) * 3 + d];
  for (int d = 0; d < 3; ++d) F[3 * (a0 + a) + d] = h3 * f[d];
}

// Gaussian-overlap repulsion correction (Appendix A in closed form):
// E_c = sum_{I<J} Z_I Z_J erfc(R_IJ/(sqrt2 sigma))/R_IJ and its forces.  One
// thread per atom I sums over all J != I (half the pair energy each).
static __global__ void ezz_kernel(AtomArgs A, double* eI, double* F) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= A.M) return;
  const double a = 0.70710678118654752 / A.sigma;
  double e = 0.0, f[3] = {0.0, 0.0, 0.0};
  for (int J = 0; J < A.M; ++J) {
    if (J == I) continue;
    const double dx = A.R[3 * I] - A.R[3 * J], dy = A.R[3 * I + 1] - A.R[3 * J + 1],
                 dz = A.R[3 * I + 2] - A.R[3 * J + 2];
    const double r2 = dx * dx + dy * dy + dz * dz, r = sqrt(r2);
    const double zz = A.Z[I] * A.Z[J];
    e += 0.5 * zz * erfc(a * r) / r;
    const double dEdr = zz * (-erfc(a * r) / r2 - 2.0 * a * 0.56418958354775628 * exp(-a * a * r2) / r);
    f[0] -= dEdr * dx / r;
    f[1] -= dEdr * dy / r;
    f[2] -= dEdr * dz / r;
  }
  eI[I] = e;
  F[3 * I] = f[0];
  F[3 * I + 1] = f[1];
  F[3 * I + 2] = f[2];
}

}  // namespace ofd
