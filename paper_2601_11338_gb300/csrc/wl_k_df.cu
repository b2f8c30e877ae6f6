// Double-float kernels of the refined form (refinement residual, outer
// Lanczos step and basis combination), K = 1, 2, 4, ..., 64.
#define WL_EXPDF_KERNELS
#define WL_EXPS_KERNELS
#include <algorithm>

#include "wl_expdf.cuh"
#include "wl_host.h"
#include "wl_res.cuh"
#include "wl_exps.cuh"

namespace wl {

#define WL_FOR_K(X) X(1) X(2) X(4) X(8) X(16) X(32) X(64)

cudaError_t launch_df_res(int K, const DfResArgs& a, int grid, bool full, cudaStream_t s) {
  switch (K) {
#define DR(k)                                                      \
  case k:                                                          \
    if (full && a.dsh_h)                                           \
      df_res<k, true, true><<<grid, kPhaseBlock, 0, s>>>(a);       \
    else if (full)                                                 \
      df_res<k, true><<<grid, kPhaseBlock, 0, s>>>(a);             \
    else if (a.dsh_h)                                              \
      df_res<k, false, true><<<grid, kPhaseBlock, 0, s>>>(a);      \
    else                                                           \
      df_res<k, false><<<grid, kPhaseBlock, 0, s>>>(a);            \
    return cudaGetLastError();
    WL_FOR_K(DR)
#undef DR
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_df_from_f64(int K, const double* b, double scale, int64_t n, float* bh, float* bl, float* r32,
                               double* part, CgState* st, double* b2, int grid, cudaStream_t s) {
  switch (K) {
#define DC(k)                                                                               \
  case k:                                                                                   \
    df_from_f64<k><<<grid, kPhaseBlock, 0, s>>>(b, scale, n, bh, bl, r32, part, st, b2);    \
    return cudaGetLastError();
    WL_FOR_K(DC)
#undef DC
  }
  return cudaErrorInvalidValue;
}

int df_res_blocks(int K) {
  const void* f = nullptr;
  switch (K) {
#define DB(k)                                  \
  case k:                                      \
    f = (const void*)df_res<k, false>;         \
    break;
    WL_FOR_K(DB)
#undef DB
  }
  int nb = 0, dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, kPhaseBlock, 0);
  return (nb < 1 ? 1 : nb) * sms;
}

static const void* df_step_fn(int K) {
  switch (K) {
#define SF(k) \
  case k:     \
    return (const void*)df_lanczos_step<k>;
    WL_FOR_K(SF)
#undef SF
  }
  return nullptr;
}

int df_lanczos_grid(int K) {
  const void* f = df_step_fn(K);
  return f ? coop_grid(f, 4) : 0;
}

cudaError_t launch_df_lanczos_step(int K, const DfLanczosArgs& a, int G, cudaStream_t s) {
  const void* f = df_step_fn(K);
  if (!f) return cudaErrorInvalidValue;
  return coop_launch(f, G, a, s);
}

cudaError_t launch_df_combine(int K, const DfCombineArgs& a, cudaStream_t s) {
  const int64_t blocks = std::min<int64_t>(((int64_t)a.n * K + kBlock - 1) / kBlock, 152 * 16);
  switch (K) {
#define CB(k)                                                                  \
  case k:                                                                      \
    df_combine<k><<<(unsigned)std::max<int64_t>(blocks, 1), kBlock, 0, s>>>(a); \
    return cudaGetLastError();
    WL_FOR_K(CB)
#undef CB
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_df_scale_cols(const double* X, int64_t n, int K, const double* nrm, float* hi, float* lo,
                                 cudaStream_t s) {
  const int64_t blocks = std::min<int64_t>(((int64_t)n * K + kBlock - 1) / kBlock, 152 * 16);
  df_scale_cols<<<(unsigned)std::max<int64_t>(blocks, 1), kBlock, 0, s>>>(X, n, K, nrm, hi, lo);
  return cudaGetLastError();
}

cudaError_t launch_exp_term(int K, const ExpArgs& a, int grid, cudaStream_t s) {
  switch (K) {
#define ET(k)                                            \
  case k:                                                \
    exp_term<k><<<grid, kPhaseBlock, 0, s>>>(a);         \
    return cudaGetLastError();
    WL_FOR_K(ET)
#undef ET
  }
  return cudaErrorInvalidValue;
}

int exp_blocks(int K) {
  const void* f = nullptr;
  switch (K) {
#define EB(k)                              \
  case k:                                  \
    f = (const void*)exp_term<k>;          \
    break;
    WL_FOR_K(EB)
#undef EB
  }
  int nb = 0, dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, kPhaseBlock, 0);
  return (nb < 1 ? 1 : nb) * sms;
}

cudaError_t launch_df_split(const double* x, size_t total, float* hi, float* lo, cudaStream_t s) {
  const int64_t blocks = std::min<int64_t>(((int64_t)total + kBlock - 1) / kBlock, 152 * 16);
  df_split<<<(unsigned)std::max<int64_t>(blocks, 1), kBlock, 0, s>>>(x, total, hi, lo);
  return cudaGetLastError();
}

}  // namespace wl
