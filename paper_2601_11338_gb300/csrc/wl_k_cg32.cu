// FP32 instances of the CG phase kernels (inner solves of the refined form
// and of the sketch), K = 1, 2, 4, ..., 64 columns.
#include "wl_cg2.cuh"
#include "wl_host.h"

namespace wl {

#define WL_FOR_K(X) X(1) X(2) X(4) X(8) X(16) X(32) X(64)

template <int K>
static cudaError_t run_cg32(const PhaseArgs<float>& a, int grid_s, int grid_u, int mode, int chunk, cudaStream_t s) {
  if (mode == 0) {
    cg_u_phase<float, K><<<grid_u, kPhaseBlock, 0, s>>>(a, 1);
  } else if (mode == 1) {
    for (int i = 0; i < chunk; ++i) {
      if (a.dshift)
        cg_s_phase<float, K, true><<<grid_s, kPhaseBlock, 0, s>>>(a);
      else
        cg_s_phase<float, K><<<grid_s, kPhaseBlock, 0, s>>>(a);
      cg_u_phase<float, K><<<grid_u, kPhaseBlock, 0, s>>>(a, 0);
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
