// Element-wise kernels of the shift-and-invert Lanczos on the resolvent walk
// Laplacian (Sec. 4.4: a rational Krylov space for exp(-t L) needs solves
// with L + sigma I; Sec. 4.2: L = D_f - a M^{-1} with the sparse M).
//
// With Dt = D_f + sigma I, (L + sigma I) x = v is equivalent to
//   (M - a Dt^{-1}) z = Dt^{-1} v ,  x = M z :
// substituting x = M z gives (Dt M - a I) z = v. The matrix M - a Dt^{-1} is
// the Schur complement of the positive definite block [[M, sqrt(a) I],
// [sqrt(a) I, Dt]] (its other Schur complement is L + sigma I, positive
// definite for sigma > 0), so it is symmetric positive definite and one CG
// solve with the CG kernels' M plus the per-row diagonal -a / (D_f + sigma)
// gives each shifted solve, without an inner solve inside the outer one.
//
//   si_prep   the diagonal -a / (D_f + sigma) and 1 / (D_f + sigma), FP64
//             and as double-float pairs
//   si_rhs64  B = Dt^{-1} V (FP64 form)
//   si_rhs_df (bh, bl) = Dt^{-1} (vh, vl) in double-float, per-CTA partial
//             sums of |B|^2 per column; si_colsum adds them in fixed order
//   si_mz     the product M z without a gather: with the solve's residual
//             r = B - (M - a Dt^{-1}) z, M z = (B - r) + a Dt^{-1} z; written
//             negated (-R v, the operand of the Lanczos step kernels)
#include <algorithm>

#include "wl_df.cuh"
#include "wl_host.h"

namespace wl {

namespace {
unsigned blocks_for(int64_t work, int cap = 152 * 16) {
  int64_t b = (work + 255) / 256;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, cap));
}
}  // namespace

__global__ void si_prep(const double* Df, int64_t n, double a, double sigma, double* dsh64, float* dsh_h,
                        float* dsh_l, double* inv64, float* inv_h, float* inv_l) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double inv = 1.0 / (Df[i] + sigma);
    const double d = -a * inv;
    dsh64[i] = d;
    inv64[i] = inv;
    const df dd = df_from_double(d), ii = df_from_double(inv);
    dsh_h[i] = dd.hi;
    dsh_l[i] = dd.lo;
    inv_h[i] = ii.hi;
    inv_l[i] = ii.lo;
  }
}

__global__ void si_rhs64(const double* V, const double* inv, int64_t n, int K, double* B) {
  const int64_t total = n * K;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    B[e] = V[e] * inv[e / K];
}

// one thread per element; block size 256 is a multiple of K, so thread t
// always meets column t % K; the squares are summed in FP32 with the
// rounding error of every add kept (the norm needs a few digits)
__global__ void si_rhs_df(const float* vh, const float* vl, const float* inv_h, const float* inv_l, int64_t n, int K,
                          int kshift, float* bh, float* bl, double* part) {
  __shared__ double s[256];
  const int64_t total = n * K;
  float acc = 0.f, cmp = 0.f;
  for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < total; e += (int64_t)gridDim.x * 256) {
    const int64_t row = e >> kshift;
    const df b = df_mul(df{vh[e], vl[e]}, df{__ldg(inv_h + row), __ldg(inv_l + row)});
    bh[e] = b.hi;
    bl[e] = b.lo;
    df_acc(acc, cmp, b.hi * b.hi);
  }
  s[threadIdx.x] = (double)acc + (double)cmp;
  __syncthreads();
  if ((int)threadIdx.x < K) {
    double t = 0.0;
    for (int u = threadIdx.x; u < 256; u += K) t += s[u];
    part[(size_t)blockIdx.x * K + threadIdx.x] = t;
  }
}

// column sums of G x K partials: 256 threads, column c summed by threads
// c, c + K, ... in a fixed order, then combined in shared memory
__global__ void si_colsum(const double* part, int G, int K, double* out) {
  __shared__ double s[256];
  const int t = threadIdx.x, c = t % K, j = t / K, J = 256 / K;
  double acc = 0.0;
  for (int g = j; g < G; g += J) acc += part[(size_t)g * K + c];
  s[t] = acc;
  __syncthreads();
  if (t < K) {
    double tot = 0.0;
    for (int u = 0; u < J; ++u) tot += s[u * K + t];
    out[t] = tot;
  }
}

// (yh, yl) = -((bh, bl) - (rh, rl) + a (inv_h, inv_l) (zh, zl)) in double-float
// (y may alias r)
__global__ void si_mz_df(const float* bh, const float* bl, const float* rh, const float* rl, const float* zh,
                         const float* zl, const float* inv_h, const float* inv_l, df a, int64_t n, int kshift,
                         float* yh, float* yl) {
  const int64_t total = n << kshift;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = e >> kshift;
    const df w = df_mul(df_mul(a, df{__ldg(inv_h + row), __ldg(inv_l + row)}), df{zh[e], zl[e]});
    const df y = df_add(df_sub(df{bh[e], bl[e]}, df{rh[e], rl[e]}), w);
    yh[e] = -y.hi;
    yl[e] = -y.lo;
  }
}

// X = -((B - R) + a inv z) in FP64
__global__ void si_mz64(const double* B, const double* R, const double* Z, const double* inv, double a, int64_t n,
                        int kshift, double* X) {
  const int64_t total = n << kshift;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    X[e] = -((B[e] - R[e]) + a * inv[e >> kshift] * Z[e]);
}

cudaError_t launch_si_prep(const double* Df, int64_t n, double a, double sigma, double* dsh64, float* dsh_h,
                           float* dsh_l, double* inv64, float* inv_h, float* inv_l, cudaStream_t s) {
  si_prep<<<blocks_for(n), 256, 0, s>>>(Df, n, a, sigma, dsh64, dsh_h, dsh_l, inv64, inv_h, inv_l);
  return cudaGetLastError();
}

cudaError_t launch_si_rhs64(const double* V, const double* inv, int64_t n, int K, double* B, cudaStream_t s) {
  si_rhs64<<<blocks_for(n * K), 256, 0, s>>>(V, inv, n, K, B);
  return cudaGetLastError();
}

int si_rhs_blocks(int64_t n, int K) { return (int)blocks_for(n * K, 152 * 8); }

static int log2k(int K) {
  int k = 0;
  while ((1 << k) < K) ++k;
  return k;
}

cudaError_t launch_si_rhs_df(const float* vh, const float* vl, const float* inv_h, const float* inv_l, int64_t n,
                             int K, float* bh, float* bl, double* part, double* bn2, cudaStream_t s) {
  if (K < 1 || K > 64 || (K & (K - 1)) != 0) return cudaErrorInvalidValue;
  const int G = si_rhs_blocks(n, K);
  si_rhs_df<<<G, 256, 0, s>>>(vh, vl, inv_h, inv_l, n, K, log2k(K), bh, bl, part);
  si_colsum<<<1, 256, 0, s>>>(part, G, K, bn2);
  return cudaGetLastError();
}

cudaError_t launch_si_mz_df(const float* bh, const float* bl, const float* rh, const float* rl, const float* zh,
                            const float* zl, const float* inv_h, const float* inv_l, double a, int64_t n, int K,
                            float* yh, float* yl, cudaStream_t s) {
  if (K < 1 || K > 64 || (K & (K - 1)) != 0) return cudaErrorInvalidValue;
  si_mz_df<<<blocks_for(n * K), 256, 0, s>>>(bh, bl, rh, rl, zh, zl, inv_h, inv_l, df_from_double(a), n, log2k(K),
                                            yh, yl);
  return cudaGetLastError();
}

cudaError_t launch_si_mz64(const double* B, const double* R, const double* Z, const double* inv, double a, int64_t n,
                           int K, double* X, cudaStream_t s) {
  if (K < 1 || K > 64 || (K & (K - 1)) != 0) return cudaErrorInvalidValue;
  si_mz64<<<blocks_for(n * K), 256, 0, s>>>(B, R, Z, inv, a, n, log2k(K), X);
  return cudaGetLastError();
}

}  // namespace wl
