// ofdft_poisson_noalloc: the FP64 Poisson CG of ofdft_poisson for callers that
// cannot allocate device memory (a framework that owns every allocation of the
// process, code that must not call cudaMalloc on a latency-critical path).  It
// needs no context: its CG vectors, reduction scratch and CG scalars live in
// one file-scope device array of fixed size, so no call allocates anything.
#include "host.cuh"

#include <mutex>

namespace {

using namespace ofd;

// Largest grid the array holds: 64^3 nodes (three FP64 CG vectors of 2 MiB).
constexpr long long kMaxPoints = 64LL * 64 * 64;
constexpr long long kPartialsBytes = 64 * 1024;  // per-block partial sums of the reductions
constexpr long long kVecBytes = kMaxPoints * (long long)sizeof(double);
constexpr long long kScratchBytes = 3 * kVecBytes + kPartialsBytes + 256 + 256;

// One array per device that loads the library, held until the process exits.
// In host code this name is only a host-side stand-in: kernels get the device
// address that cudaGetSymbolAddress returns.
static __device__ __align__(256) unsigned char noalloc_scratch[kScratchBytes];

std::mutex g_mutex;

// Per-device set-up, done once by the first call on each device: the array's
// device address, the SM count (launch split) and the dynamic shared-memory
// limits of the kernels this entry point launches (a per-device attribute).
struct DevSetup {
  void* addr = nullptr;
  int sms = 0;
};
DevSetup g_dev[256];

template <int R>
cudaError_t set_smem_attrs() {
  cudaError_t e = cudaFuncSetAttribute(zstream_kernel<double, R, 1, LoadPlain<double>, EpiResidual<double>>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       zsmem_bytes<double, R, 1, EpiResidual<double>>());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(zstream_kernel<double, R, 1, LoadPlain<double>, EpiCgA<double>>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, zsmem_bytes<double, R, 1, EpiCgA<double>>());
}

int fail_na(const char* msg) {
  fprintf(stderr, "[ofdft_poisson_noalloc] %s\n", msg);
  return OFDFT_EINVAL;
}

// The current device's set-up (performed on its first call).
int device_setup(DevSetup* out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return OFDFT_ECUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  DevSetup& d = g_dev[dev];
  if (!d.addr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, noalloc_scratch) != cudaSuccess || !p) return OFDFT_ECUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
      return OFDFT_ECUDA;
    if (set_smem_attrs<1>() != cudaSuccess || set_smem_attrs<2>() != cudaSuccess ||
        set_smem_attrs<3>() != cudaSuccess || set_smem_attrs<4>() != cudaSuccess ||
        set_smem_attrs<5>() != cudaSuccess || set_smem_attrs<6>() != cudaSuccess)
      return OFDFT_ECUDA;
    d.sms = sms;
    d.addr = p;
  }
  *out = d;
  return OFDFT_OK;
}

template <int R>
cudaError_t launch_stencil_pass(dim3 grid, int zchunk, const GridDev& g, const Weights<double>& W,
                                const double* f, EpiResidual<double> ep, RedBuf red, cudaStream_t s) {
  constexpr int smem = zsmem_bytes<double, R, 1, EpiResidual<double>>();
  zstream_kernel<double, R, 1, LoadPlain<double>, EpiResidual<double>>
      <<<grid, dim3(BX, BY), smem, s>>>(g, W, zchunk, LoadPlain<double>{f}, ep, red);
  return cudaGetLastError();
}

}  // namespace

extern "C" int ofdft_poisson_noalloc(const ofdft_grid* gr, int fd_order, const double* rho, double* phi,
                                     double tol, int max_it, void* cuda_stream, ofdft_cg_stats* st) {
  if (!gr || !rho || !phi) return fail_na("null grid, rho or phi");
  for (int d = 0; d < 3; ++d)
    if (gr->n[d] < 1) return fail_na("grid dimensions must be positive");
  const long long G = (long long)gr->n[0] * gr->n[1] * gr->n[2];
  if (G > kMaxPoints) return fail_na("grid exceeds the fixed scratch (at most 262144 = 64^3 nodes)");
  if (fd_order < 2 || fd_order > 2 * kMaxR || (fd_order & 1)) return fail_na("fd_order must be even in [2, 12]");
  if (!(tol > 0.0) || max_it < 0 || !(gr->h > 0.0)) return fail_na("need tol > 0, max_it >= 0, h > 0");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  DevSetup dv;
  int rc = device_setup(&dv);
  if (rc != OFDFT_OK) return rc;
  char* p = static_cast<char*>(dv.addr);
  double* r = reinterpret_cast<double*>(p);
  double* pv = reinterpret_cast<double*>(p + kVecBytes);
  double* qv = reinterpret_cast<double*>(p + 2 * kVecBytes);
  double* partials = reinterpret_cast<double*>(p + 3 * kVecBytes);
  unsigned int* counter = reinterpret_cast<unsigned int*>(p + 3 * kVecBytes + kPartialsBytes);
  CgScalars* sc = reinterpret_cast<CgScalars*>(p + 3 * kVecBytes + kPartialsBytes + 256);
  // the array keeps the previous call's contents: the reduction counter must start at zero
  if (cudaMemsetAsync(counter, 0, sizeof(unsigned int), s) != cudaSuccess) return OFDFT_ECUDA;
  const RedBuf red{partials, counter};
  const GridDev g{gr->n[0], gr->n[1], gr->n[2], G};
  const int R = fd_order / 2;
  const Weights<double> W = lap_weights(R, gr->h, 1.0), Wneg = lap_weights(R, gr->h, -1.0);
  // launch shape of the library's single-grid passes: about four blocks per SM
  const int gx = (g.n1 + BX - 1) / BX, gy = (g.n2 + ZCfg<double>::TY - 1) / ZCfg<double>::TY;
  int nz = std::max(1, (4 * dv.sms + gx * gy - 1) / (gx * gy));
  nz = std::min(nz, std::max(1, g.n3 / std::max(2 * R, 4)));
  const int zc = (g.n3 + nz - 1) / nz;
  nz = (g.n3 + zc - 1) / zc;
  const dim3 zgrid(gx, gy, nz);
  if ((long long)gx * gy * nz * 3 * 8 > kPartialsBytes) return fail_na("launch needs more partial sums than fit");
  const int pb = (int)std::min<long long>(std::max<long long>(1, (G + 255) / 256), 1024);
  cudaError_t e = cudaSuccess;
  // r = 4 pi rho + L phi, CG scalars initialised by the last block
  EpiResidual<double> res{rho, nullptr, nullptr, r, sc, tol, max_it, 1};
  switch (R) {
    case 1: e = launch_stencil_pass<1>(zgrid, zc, g, W, phi, res, red, s); break;
    case 2: e = launch_stencil_pass<2>(zgrid, zc, g, W, phi, res, red, s); break;
    case 3: e = launch_stencil_pass<3>(zgrid, zc, g, W, phi, res, red, s); break;
    case 4: e = launch_stencil_pass<4>(zgrid, zc, g, W, phi, res, red, s); break;
    case 5: e = launch_stencil_pass<5>(zgrid, zc, g, W, phi, res, red, s); break;
    case 6: e = launch_stencil_pass<6>(zgrid, zc, g, W, phi, res, red, s); break;
  }
  if (e != cudaSuccess) return OFDFT_ECUDA;
  CgScalars hs;
  int launched = 0;
  for (;;) {
    if (cudaMemcpyAsync(&hs, sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, s) != cudaSuccess) return OFDFT_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return OFDFT_ECUDA;
    if (hs.done || launched >= max_it) break;
    for (int i = 0; i < 8 && launched < max_it; ++i, ++launched) {
      switch (R) {
#define NA_CG(RR)                                                                                                \
  case RR: {                                                                                                     \
    constexpr int smem = zsmem_bytes<double, RR, 1, EpiCgA<double>>();                                         \
    zstream_kernel<double, RR, 1, LoadPlain<double>, EpiCgA<double>>                                             \
        <<<zgrid, dim3(BX, BY), smem, s>>>(g, cast_weights<double>(Wneg), zc, LoadPlain<double>{r},             \
                                          EpiCgA<double>{pv, qv, sc}, red);                                      \
  } break;
        NA_CG(1)
        NA_CG(2)
        NA_CG(3)
        NA_CG(4)
        NA_CG(5)
        NA_CG(6)
#undef NA_CG
      }
      cg_update_kernel<double><<<pb, 256, 0, s>>>(G, phi, r, pv, qv, sc, red);
      if (cudaGetLastError() != cudaSuccess) return OFDFT_ECUDA;
    }
  }
  const double bb = hs.bb > 0 ? hs.bb : 1.0;
  if (st) {
    st->iterations = hs.iters;
    st->rel_residual = sqrt(hs.rr / bb);
  }
  if (!isfinite(hs.rr)) return OFDFT_ENONFINITE;
  return hs.rr <= tol * tol * bb ? OFDFT_OK : OFDFT_ENOTCONV;
}
