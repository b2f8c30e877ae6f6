// Lanczos kernels: extreme eigenvalues (spectral scale), one step of the
// outer Lanczos on the walk Laplacian, exp of the tridiagonal, combination.
#define WL_LANCZOS_KERNELS
#define WL_LANCZOS2_KERNELS
#include "wl_host.h"
#include "wl_lanczos2.cuh"

namespace wl {

#define WL_FOR_K(X) X(1) X(2) X(4) X(8) X(16) X(32) X(64)

static const void* step_fn(int K) {
  switch (K) {
#define LS(k) \
  case k:     \
    return (const void*)lanczos_step<k>;
    WL_FOR_K(LS)
#undef LS
  }
  return nullptr;
}

int lanczos_ext_grid() { return coop_grid((const void*)lanczos_extreme, 2); }

int lanczos_step_grid(int K) {
  const void* f = step_fn(K);
  return f ? coop_grid(f, 4) : 0;
}

cudaError_t launch_lanczos_extreme(const LanczosExtArgs& a, int G, cudaStream_t s) {
  return coop_launch((const void*)lanczos_extreme, G, a, s);
}

cudaError_t launch_lanczos_step(int K, const LanczosStepArgs& a, int G, cudaStream_t s) {
  const void* f = step_fn(K);
  if (!f) return cudaErrorInvalidValue;
  return coop_launch(f, G, a, s);
}

cudaError_t launch_tridiag_exp(const TridiagArgs& a, int K, cudaStream_t s) {
  tridiag_exp<<<dim3(K, a.ntau), kBlock, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_combine(int K, const CombineArgs& a, cudaStream_t s) {
  int64_t blocks = ((int64_t)a.n * K + kBlock - 1) / kBlock;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  switch (K) {
#define CB(k)                                                   \
  case k:                                                       \
    combine<k><<<(unsigned)blocks, kBlock, 0, s>>>(a);          \
    break;
    WL_FOR_K(CB)
#undef CB
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

int lz_blocks() {
  int nb = 0, dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void*)lz_s, kPhaseBlock, 0);
  return (nb < 1 ? 1 : nb) * sms;
}

cudaError_t launch_lanczos2(const LzArgs& a0, int j0, int m, int check, int grid_s, int grid_u, cudaStream_t s) {
  LzArgs a = a0;
  a.j = 0;
  if (j0 == 0)
    lz_init<<<grid_u, kPhaseBlock, 0, s>>>(a);
  else
    lz_resume<<<1, 32, 0, s>>>(a.st);
  for (int j = j0; j < m; ++j) {
    a.j = j;
    lz_s<<<grid_s, kPhaseBlock, 0, s>>>(a);
    lz_u<<<grid_u, kPhaseBlock, 0, s>>>(a, j == m - 1 ? 1 : 0);
  }
  lz_eig<<<1, 4 * kEigT, 0, s>>>(a.st, check);
  return cudaGetLastError();
}

}  // namespace wl
