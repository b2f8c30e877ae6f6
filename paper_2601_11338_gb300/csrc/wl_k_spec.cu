// Spectral-scale Lanczos kernels (k = 1, double-float basis): launchers.
#define WL_SPEC_KERNELS
#include "wl_host.h"
#include "wl_spec.cuh"

namespace wl {

int sp_blocks() {
  int nb = 0, dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void*)sp_s, kPhaseBlock, 0);
  return (nb < 1 ? 1 : nb) * sms;
}

cudaError_t launch_sp_start(const SpArgs& a, int mode, int grid_u, cudaStream_t s) {
  if (mode == 0)
    sp_init<<<grid_u, kPhaseBlock, 0, s>>>(a);
  else
    sp_restart<<<1, 32, 0, s>>>(a.st, mode == 2 ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_sp_steps(const SpArgs& a0, int j0, int j1, int cap, int check, double rtol, int grid_s,
                            int grid_u, cudaStream_t s) {
  SpArgs a = a0;
  for (int j = j0; j < j1; ++j) {
    a.j = j;
    sp_s<<<grid_s, kPhaseBlock, 0, s>>>(a);
    sp_u<<<grid_u, kPhaseBlock, 0, s>>>(a, j == cap - 1 ? 1 : 0);
    if ((j + 1) % check == 0 || j + 1 == j1) sp_eig<<<1, 2 * kSpEigT, 0, s>>>(a.st, rtol);
  }
  return cudaGetLastError();
}

cudaError_t launch_sp_ritz(const SpArgs& a, int grid_u, cudaStream_t s) {
  sp_ritz<<<grid_u, kPhaseBlock, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_sp_round(const SpJob* jobs, const int* off_s, const int* off_u, int np, int grid_s, int grid_u,
                            int steps, int check, unsigned eig_mask, bool any_ritz, bool any_init, SpOut* out,
                            cudaStream_t s) {
  if (np <= 0) return cudaSuccess;
  if (any_ritz) sp_ritz_multi<<<grid_u, kPhaseBlock, 0, s>>>(jobs, off_u, np);
  sp_prep_multi<<<np, 128, 0, s>>>(jobs, np);
  if (any_init) sp_init_multi<<<grid_u, kPhaseBlock, 0, s>>>(jobs, off_u, np);
  for (int st = 0; st < steps; ++st) {
    sp_s_multi<<<grid_s, kPhaseBlock, 0, s>>>(jobs, off_s, np, st);
    sp_u_multi<<<grid_u, kPhaseBlock, 0, s>>>(jobs, off_u, np, st);
    if (eig_mask >> st & 1u) sp_eig_multi<<<np, 2 * kSpEigT, 0, s>>>(jobs, np, st, check);
  }
  sp_pack_multi<<<(np + 127) / 128, 128, 0, s>>>(jobs, np, out);
  return cudaGetLastError();
}

}  // namespace wl
