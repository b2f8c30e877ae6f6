// FP64 instances of the lockstep CG kernel and the FP64 residual of the
// iterative refinement (K = 1, 2, 4, ..., 64 columns).
#include "wl_host.h"

namespace wl {

#define WL_FOR_K(X) X(1) X(2) X(4) X(8) X(16) X(32) X(64)

static const void* cg64_fn(int K) {
  switch (K) {
#define C64(k) \
  case k:      \
    return (const void*)cg_persistent<double, k>;
    WL_FOR_K(C64)
#undef C64
  }
  return nullptr;
}

static const void* res_fn(int K) {
  switch (K) {
#define R64(k) \
  case k:      \
    return (const void*)residual64<k>;
    WL_FOR_K(R64)
#undef R64
  }
  return nullptr;
}

static int g_cap_per_sm = 4;

int cg_grid_f64(int K) {
  const void* f = cg64_fn(K);
  return f ? coop_grid(f, g_cap_per_sm) : 0;
}

int res_grid(int K) {
  const void* f = res_fn(K);
  return f ? coop_grid(f, g_cap_per_sm) : 0;
}

cudaError_t launch_cg_f64(int K, const CgArgs<double>& a, int G, cudaStream_t s) {
  const void* f = cg64_fn(K);
  if (!f) return cudaErrorInvalidValue;
  return coop_launch(f, G, a, s);
}

cudaError_t launch_residual64(int K, const ResArgs& a, int G, cudaStream_t s) {
  const void* f = res_fn(K);
  if (!f) return cudaErrorInvalidValue;
  return coop_launch(f, G, a, s);
}

void thresholds_f64(int K, int* Tw, int* Tc) {
  switch (K) {
#define T64(k)                    \
  case k:                         \
    *Tw = Cfg<double, k>::Tw;     \
    *Tc = Cfg<double, k>::Tc;     \
    return;
    WL_FOR_K(T64)
#undef T64
  }
  *Tw = *Tc = 0;
}

}  // namespace wl
