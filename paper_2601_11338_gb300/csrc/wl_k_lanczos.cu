// Lanczos kernels: one step of the outer Lanczos on the walk Laplacian,
// exp of the tridiagonal, combination.
#define WL_LANCZOS_KERNELS
#include "wl_host.h"

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

int lanczos_step_grid(int K) {
  const void* f = step_fn(K);
  return f ? coop_grid(f, 4) : 0;
}

cudaError_t launch_lanczos_step(int K, const LanczosStepArgs& a, int G, cudaStream_t s) {
  const void* f = step_fn(K);
  if (!f) return cudaErrorInvalidValue;
  return coop_launch(f, G, a, s);
}

// a warp per (column, tau) when every column has at most kWarpRows steps
// (mmax is the host's bound on the steps), else a CTA per pair
cudaError_t launch_tridiag_exp(const TridiagArgs& a, int K, int mmax, cudaStream_t s) {
  if (mmax <= kWarpRows) {
    const int pairs = K * a.ntau;
    tridiag_exp_warp<<<(pairs + 3) / 4, 128, 0, s>>>(a, K);
  } else {
    const cudaError_t e = cudaFuncSetAttribute(tridiag_exp, cudaFuncAttributeMaxDynamicSharedMemorySize, kTridiagSmem);
    if (e != cudaSuccess) return e;
    tridiag_exp<<<dim3(K, a.ntau), kBlock, kTridiagSmem, s>>>(a);
  }
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

}  // namespace wl
