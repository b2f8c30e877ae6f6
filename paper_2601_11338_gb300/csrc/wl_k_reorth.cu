// Launch sequence of the basis reorthogonalisation (two classical
// Gram-Schmidt passes, then normalisation); kernels in wl_reorth.cuh.
#define WL_REORTH_KERNELS
#include <algorithm>

#include "wl_host.h"

namespace wl {

namespace {
constexpr int kRoMaxCtas = 152 * 8;

int ro_update_blocks(size_t blk) {
  const size_t b = (blk + kRoBlock - 1) / kRoBlock;
  return (int)std::max<size_t>(1, std::min<size_t>(b, kRoMaxCtas));
}
}  // namespace

// Row chunks of ro_dots for nb earlier blocks: about four waves of CTAs in
// total, at most 64 chunks (the partial sums stay nb * 64 * K doubles).
int reorth_chunks(int nb, size_t blk) {
  const int groups = (nb + kRoIB - 1) / kRoIB;
  int R = std::max(1, (152 * 4) / std::max(groups, 1));
  R = std::min(R, 64);
  const size_t maxR = std::max<size_t>(1, blk / kRoBlock);
  return (int)std::min<size_t>((size_t)R, maxR);
}

size_t reorth_part_doubles(int nb, int K, size_t blk) {
  return (size_t)nb * reorth_chunks(nb, blk) * K + (size_t)nb * K + (size_t)kRoMaxCtas * K + 64;
}

// a.part must hold reorth_part_doubles(a.nb, a.K, a.blk) doubles; a.h,
// a.npart and a.scale are carved from it here.
cudaError_t launch_reorth(ReorthArgs a, bool df, cudaStream_t s) {
  if (a.nb <= 0 || a.K <= 0 || a.K > 64 || kRoBlock % a.K != 0) return cudaErrorInvalidValue;
  a.R = reorth_chunks(a.nb, a.blk);
  a.nupd = ro_update_blocks(a.blk);
  double* base = a.part;
  a.h = base + (size_t)a.nb * a.R * a.K;
  a.npart = a.h + (size_t)a.nb * a.K;
  a.scale = a.npart + (size_t)kRoMaxCtas * a.K;
  const dim3 gd(a.R, (a.nb + kRoIB - 1) / kRoIB);
  const int nred = (a.nb * a.K + 255) / 256;
  for (int pass = 0; pass < 2; ++pass) {
    if (df) {
      ro_dots<true><<<gd, kRoBlock, 0, s>>>(a);
      ro_reduce<<<nred, 256, 0, s>>>(a);
      ro_update<true><<<a.nupd, kRoBlock, 0, s>>>(a);
    } else {
      ro_dots<false><<<gd, kRoBlock, 0, s>>>(a);
      ro_reduce<<<nred, 256, 0, s>>>(a);
      ro_update<false><<<a.nupd, kRoBlock, 0, s>>>(a);
    }
  }
  ro_norm<<<1, 64, 0, s>>>(a);
  if (df)
    ro_scale<true><<<a.nupd, kRoBlock, 0, s>>>(a);
  else
    ro_scale<false><<<a.nupd, kRoBlock, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace wl
