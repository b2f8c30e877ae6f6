// FP32 instances of the lockstep CG kernel (inner solves of the refined
// form and of the sketch), K = 1, 2, 4, ..., 64 columns.
#include "wl_host.h"

namespace wl {

#define WL_FOR_K(X) X(1) X(2) X(4) X(8) X(16) X(32) X(64)

static const void* cg32_fn(int K) {
  switch (K) {
#define C32(k) \
  case k:      \
    return (const void*)cg_persistent<float, k>;
    WL_FOR_K(C32)
#undef C32
  }
  return nullptr;
}

static int g_cap_per_sm = 4;

int cg_grid_f32(int K) {
  const void* f = cg32_fn(K);
  return f ? coop_grid(f, g_cap_per_sm) : 0;
}

cudaError_t launch_cg_f32(int K, const CgArgs<float>& a, int G, cudaStream_t s) {
  const void* f = cg32_fn(K);
  if (!f) return cudaErrorInvalidValue;
  return coop_launch(f, G, a, s);
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

#ifdef WL_PHASE_TIMING
extern "C" int wl_debug_stamps(unsigned long long* out, int count) {
  return (int)cudaMemcpyFromSymbol(out, wl::g_stamps, sizeof(unsigned long long) * count);
}
#endif
