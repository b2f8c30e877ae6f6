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

// Start of a solve whose residual norms are already in st->gamma (written by
// the double-float residual that produced r): the state the init phase would
// set, without its pass over r. Column c is done when its norm is zero or not
// finite, or skip[c] is set.
__global__ void cg_state_restart(CgState* st, const int* skip, int K) {
  const int c = threadIdx.x;
  __shared__ int s_any;
  if (c == 0) s_any = 0;
  __syncthreads();
  if (c < K) {
    const double gn = st->gamma[c];
    st->b2[c] = gn;
    st->alpha[c] = 0.0;
    st->beta[c] = 0.0;
    int status = 0, done = !(gn > 0.0) || (skip && skip[c]);
    if (!isfinite(gn)) { done = 1; status = WL_ERR_NONFINITE; }
    st->status[c] = status;
    st->done[c] = done;
    if (!done) atomicOr(&s_any, 1);
  }
  __syncthreads();
  if (c == 0) {
    st->iters = 0;
    st->ticket = 0;
    st->active = s_any;
  }
}

cudaError_t launch_cg_state_restart(CgState* st, const int* skip, int K, cudaStream_t s) {
  cg_state_restart<<<1, 64, 0, s>>>(st, skip, K);
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
