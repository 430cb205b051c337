// Device-side building blocks shared by every kernel of the library:
// grid description, stencil weights, deterministic block and grid reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ofd {

constexpr int kMaxR = 6;  // stencil radius n <= 6 (FD order <= 12)
constexpr double kPi = 3.14159265358979323846;

struct GridDev {
  int n1, n2, n3;
  long long G;  // n1 n2 n3
};

__host__ __device__ inline long long lin(const GridDev& g, int x, int y, int z) {
  return (long long)x + (long long)g.n1 * ((long long)y + (long long)g.n2 * z);
}

// Radius-R star-stencil weights: centre coefficient c (= 6 w_0 of Sec. 4, times a
// scale) and w[1..R] (the w_p of Eq. FD:Laplacian, times the same scale).
template <typename T>
struct Weights {
  T c;
  T w[kMaxR + 1];
};

// Scratch used by the last-block-done grid reduction: one row of K partial sums
// per block and an arrival counter that the last block resets to zero.
struct RedBuf {
  double* partials;
  unsigned int* counter;
};

// Per-thread accumulator of a dot product.  FP64 fields accumulate with FP64
// FMAs.  FP32 fields accumulate as an unevaluated pair hi + lo of floats with
// error-free transformations (the product's rounding error from an FMA, the
// sum's from TwoSum), so the per-thread partial carries FP64-level accuracy
// without any FP64 instruction per element (FP64 issues at 1/64 of the FP32
// rate on this GPU); the pair is converted to FP64 once, for the cross-thread
// FP64 reduction.
template <typename T>
struct DotAcc {
  double s = 0.0;
  __device__ __forceinline__ void add(T a, T b) { s = fma((double)a, (double)b, s); }
  __device__ __forceinline__ double value() const { return s; }
};
template <>
struct DotAcc<float> {
  float hi = 0.0f, lo = 0.0f;
  __device__ __forceinline__ void add(float a, float b) {
    const float p = a * b;
    const float pe = fmaf(a, b, -p);  // exact rounding error of the product
    const float t = hi + p;           // TwoSum(hi, p)
    const float bp = t - hi;
    const float se = (hi - (t - bp)) + (p - bp);
    hi = t;
    lo += se + pe;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Programmatic dependent launch (sm_90 and later).  pdl_wait() blocks until
// every kernel this grid depends on has completed and its memory is visible (a
// no-op for a grid launched without the programmatic attribute);
// pdl_launch_dependents() lets the next grid of the stream be scheduled once
// every block of this one has called it or exited.  Kernels call both first,
// in that order, so at most two grids overlap and none reads early.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}
__device__ __forceinline__ void pdl_enter() {
  pdl_wait();
  pdl_launch_dependents();
}

// Sum K per-thread doubles over the block; the result is valid in thread 0.
// NT is the block size (a multiple of 32); smem holds K * NT/32 doubles.
template <int K, int NT>
__device__ __forceinline__ void block_sum(double (&v)[K], double* smem, int tid) {
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double s = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) smem[k * (NT / 32) + warp] = s;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double s = (lane < NT / 32) ? smem[k * (NT / 32) + lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      v[k] = s;
    }
  }
  __syncthreads();
}

// Grid-wide deterministic reduction of K doubles.  Every block calls it once
// with its threads' partial sums (tid = the thread's linear index in the block,
// NT threads, warps made of consecutive tids).  Block partials go to red.partials; the last
// block to arrive sums the rows in block order (a fixed order, so the result does
// not depend on scheduling) and calls fin(sums) from its thread 0, then resets
// the counter.  Returns nothing; fin runs exactly once per launch.
template <int K, int NT, class Fin>
__device__ __forceinline__ void grid_sum(double (&v)[K], double* smem, const RedBuf& red,
                                         int nblocks, int block_id, int tid, Fin& fin) {
  block_sum<K, NT>(v, smem, tid);
  __shared__ bool is_last;
  if (tid == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) red.partials[(long long)block_id * K + k] = v[k];
    __threadfence();
    const unsigned int prev = atomicAdd(red.counter, 1u);
    is_last = (prev == (unsigned int)(nblocks - 1));
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  double t[K];
#pragma unroll
  for (int k = 0; k < K; ++k) t[k] = 0.0;
  for (int b = tid; b < nblocks; b += NT) {
#pragma unroll
    for (int k = 0; k < K; ++k) t[k] += __ldcg(&red.partials[(long long)b * K + k]);
  }
  block_sum<K, NT>(t, smem, tid);
  if (tid == 0) {
    fin(t);
    *red.counter = 0u;
  }
}

}  // namespace ofd
