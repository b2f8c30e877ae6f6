// FP32 instances of the CG phase kernels (inner solves of the refined form
// and of the sketch), K = 1, 2, 4, ..., 64 columns.
#include <algorithm>

#include "wl_cg2.cuh"
#include "wl_host.h"

namespace wl {

#define WL_FOR_K(X) X(1) X(2) X(4) X(8) X(16) X(32) X(64)

// L2 residency of the gathered vector. The S kernel gathers rows of r at
// random, each about nnz / n times per iteration, while x, p, q and the index
// arrays stream through once; the access-policy window asks the L2 to keep r
// (persisting) and to let the streams pass (the L2 set-aside for persisting
// lines is a limit of this process's context, sized once per device).
static size_t l2_persist_bytes() {
  static int dev_done[64] = {0};
  static size_t bytes[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return 0;
  if (!dev_done[dev]) {
    int maxp = 0;
    cudaDeviceGetAttribute(&maxp, cudaDevAttrMaxPersistingL2CacheSize, dev);
    if (maxp > 0 && cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, (size_t)maxp) == cudaSuccess)
      bytes[dev] = (size_t)maxp;
    (void)cudaGetLastError();
    dev_done[dev] = 1;
  }
  return bytes[dev];
}

template <typename Kern, typename... Args>
static cudaError_t launch_with_window(Kern k, int grid, cudaStream_t s, const void* win, size_t win_bytes,
                                      Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kPhaseBlock);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  const size_t persist = l2_persist_bytes();
  if (persist > 0 && win_bytes > 0) {
    int maxw = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&maxw, cudaDevAttrMaxAccessPolicyWindowSize, dev);
    const size_t nb = std::min(win_bytes, (size_t)maxw);
    attr[0].id = cudaLaunchAttributeAccessPolicyWindow;
    attr[0].val.accessPolicyWindow.base_ptr = const_cast<void*>(win);
    attr[0].val.accessPolicyWindow.num_bytes = nb;
    attr[0].val.accessPolicyWindow.hitRatio = (float)std::min(1.0, (double)persist / (double)nb);
    attr[0].val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
    attr[0].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  return cudaLaunchKernelEx(&cfg, k, args...);
}

template <int K>
static cudaError_t run_cg32(const PhaseArgs<float>& a, int grid_s, int grid_u, int mode, int chunk, cudaStream_t s) {
  const size_t rb = (size_t)a.g.n * K * sizeof(float);
  if (mode == 0) {
    cg_u_phase<float, K><<<grid_u, kPhaseBlock, 0, s>>>(a, 1);
  } else if (mode == 1) {
    for (int i = 0; i < chunk; ++i) {
      cudaError_t e = launch_with_window(cg_s_phase<float, K>, grid_s, s, a.r, rb, a);
      if (e == cudaSuccess) e = launch_with_window(cg_u_phase<float, K>, grid_u, s, a.r, rb, a, 0);
      if (e != cudaSuccess) return e;
    }
  } else {
    cg_f_phase<float, K><<<grid_u, kPhaseBlock, 0, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_cg_phases_f32(int K, const PhaseArgs<float>& a, int grid_s, int grid_u, int mode, int chunk,
                                 cudaStream_t s) {
  switch (K) {
#define C32(k) \
  case k:      \
    return run_cg32<k>(a, grid_s, grid_u, mode, chunk, s);
    WL_FOR_K(C32)
#undef C32
  }
  return cudaErrorInvalidValue;
}

int phase_blocks_f32(int K) {
  const void* f = nullptr;
  switch (K) {
#define F32(k)                                   \
  case k:                                        \
    f = (const void*)cg_s_phase<float, k>;       \
    break;
    WL_FOR_K(F32)
#undef F32
  }
  int nb = 0, dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, kPhaseBlock, 0);
  return (nb < 1 ? 1 : nb) * sms;
}

void thresholds_f32(int K, int* Tw, int* Tc) {
  switch (K) {
#define T32(k)                   \
  case k:                        \
    *Tw = Cfg<float, k>::Tw;     \
    *Tc = Cfg<float, k>::Tc;     \
    return;
    WL_FOR_K(T32)
#undef T32
  }
  *Tw = *Tc = 0;
}

}  // namespace wl
