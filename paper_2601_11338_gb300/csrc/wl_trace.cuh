// XNysTrace of phi (Alg. 1, step "XNysTrace(Y, Omega)") on the device.
//
//  philox_sketch : Omega (n x M, bfloat16) from Philox4x32-10 (Salmon et al.,
//                  SC'11): element e = i M + j uses counter block e / 4 with key
//                  = seed; words (x0, x1) and (x2, x3) give two Box-Muller pairs
//                  r = sqrt(-2 ln u_a), (r cos 2 pi u_b, r sin 2 pi u_b),
//                  u = (x + 0.5) 2^-32, evaluated in FP64 and rounded to bf16
//                  to nearest even.
//  sketch_rhs    : B = a Omega as FP32 n x K (zero-padded columns), the
//                  right-hand side of Y = phi Omega = M^{-1} (a Omega).
//  gram_cc       : per-CTA partial Grams H = Omega^T Y and G = Y^T Y over a
//                  contiguous row chunk (FP32 products and sums inside a
//                  chunk, FP64 across chunks in gram_reduce).
//  nys_core      : with P = H^{-1} (Cholesky, FP64), the leave-one-out
//                  estimates t_i = tr(P G) + (1 - (P G P)_ii) / P_ii, which
//                  equal tr(A_hat_(i)) + w_i^T (A - A_hat_(i)) w_i for the
//                  Nystrom approximation A_hat_(i) = Y_-i (Omega_-i^T Y_-i)^{-1}
//                  Y_-i^T built without column i (Schur-complement identities
//                  for (H_-i)^{-1}); estimate mean(t), error std(t)/sqrt(M).
#pragma once
#include <stdint.h>

#include "wl_common.cuh"

namespace wl {

constexpr int kMaxSketch = 64;

__device__ __forceinline__ void philox4x32_10(uint32_t (&c)[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
    const uint32_t n0 = hi1 ^ c[1] ^ k0;
    const uint32_t n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

// FP64 -> bfloat16 bits, round to nearest even, for finite normal-range inputs
__device__ __forceinline__ uint16_t f64_to_bf16_rne(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 63);
  int e = (int)((b >> 52) & 0x7FF);
  const unsigned long long m = b & ((1ull << 52) - 1);
  if (e == 0) return (uint16_t)(sign << 15);  // zero (and FP64 subnormals) -> signed zero
  unsigned long long keep = m >> 45;
  const unsigned long long rest = m & ((1ull << 45) - 1), half = 1ull << 44;
  if (rest > half || (rest == half && (keep & 1ull))) ++keep;
  if (keep == 128ull) {
    keep = 0;
    ++e;
  }
  int fe = e - 1023 + 127;
  if (fe <= 0) return (uint16_t)(sign << 15);
  if (fe >= 255) return (uint16_t)((sign << 15) | 0x7F80u);
  return (uint16_t)((sign << 15) | ((unsigned)fe << 7) | (unsigned)keep);
}

__device__ __forceinline__ float bf16_to_f32(uint16_t h) { return __uint_as_float(((uint32_t)h) << 16); }

#ifdef WL_TRACE_KERNELS
__global__ void philox_sketch(uint16_t* omega, int64_t total, uint64_t seed) {
  const int64_t nblk = (total + 3) / 4;
  const uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFull), k1 = (uint32_t)(seed >> 32);
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += (int64_t)gridDim.x * blockDim.x) {
    uint32_t c[4] = {(uint32_t)((uint64_t)b & 0xFFFFFFFFull), (uint32_t)((uint64_t)b >> 32), 0u, 0u};
    philox4x32_10(c, k0, k1);
    const double s = 1.0 / 4294967296.0;
    const double u0 = ((double)c[0] + 0.5) * s, u1 = ((double)c[1] + 0.5) * s;
    const double u2 = ((double)c[2] + 0.5) * s, u3 = ((double)c[3] + 0.5) * s;
    const double two_pi = 6.283185307179586;
    const double r01 = sqrt(-2.0 * log(u0)), r23 = sqrt(-2.0 * log(u2));
    double z[4];
    z[0] = r01 * cos(two_pi * u1);
    z[1] = r01 * sin(two_pi * u1);
    z[2] = r23 * cos(two_pi * u3);
    z[3] = r23 * sin(two_pi * u3);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t e = b * 4 + q;
      if (e < total) omega[e] = f64_to_bf16_rne(z[q]);
    }
  }
}

// B[i, j] = a * Omega[i, j] (j < M), 0 for M <= j < K
__global__ void sketch_rhs(const uint16_t* omega, int64_t n, int M, int K, float a, float* B) {
  const int64_t total = n * K;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / K;
    const int j = (int)(e % K);
    B[e] = (j < M) ? a * bf16_to_f32(omega[i * M + j]) : 0.0f;
  }
}

// Omega as an FP64 n x K block (zero-padded columns): the start block of the
// return-probability Lanczos
__global__ void sketch_block_f64(const uint16_t* omega, int64_t n, int M, int K, double* B) {
  const int64_t total = n * K;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / K;
    const int j = (int)(e % K);
    B[e] = (j < M) ? (double)bf16_to_f32(omega[i * M + j]) : 0.0;
  }
}

// FP64 -> FP32 (the Gram of the estimator takes FP32 Y)
__global__ void to_f32(const double* X, int64_t total, float* Y) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    Y[e] = (float)X[e];
}

// ---------------------------------------------------------------- Gram on CUDA cores
// Grid of G CTAs of kGramThreads, CTA g sums rows [g * chunk, min(n, (g+1) *
// chunk)) of the 2M x M block [Omega Y]^T Y (M <= 64). Thread (tr, tc) =
// (t / 8, t % 8) owns the 8 x 8 outputs of X columns 8 tr .. 8 tr + 7 (X =
// [Omega Y], 128 columns) and Y columns 8 tc .. 8 tc + 7: per staged row it
// reads two float4 of X and two of Y from shared memory for 64 FMAs. Tiles
// of kGramRows rows alternate between two buffers; the next tile's loads are
// issued into registers before the current tile's products.
constexpr int kGramRows = 32;     // rows staged per tile
constexpr int kGramThreads = 128;
constexpr int kGramLoads = kGramRows * kMaxSketch / kGramThreads;  // elements of Omega (and of Y) per thread and tile

__global__ void __launch_bounds__(kGramThreads) gram_cc(const uint16_t* omega, const float* Y, int64_t n, int M,
                                                        int K, int64_t chunk, float* partial /* G x 2M x M */) {
  __shared__ __align__(16) float sX[2][kGramRows][2 * kMaxSketch];  // [Omega_i, Y_i]
  const int tid = threadIdx.x;
  const int tr = tid >> 3, tc = tid & 7;
  const int64_t r0 = (int64_t)blockIdx.x * chunk;
  const int64_t r1 = min(n, r0 + chunk);
  float acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
  float po[kGramLoads], py[kGramLoads];  // the next tile, in flight
  auto fetch = [&](int64_t base) {
#pragma unroll
    for (int u = 0; u < kGramLoads; ++u) {
      const int e = tid + u * kGramThreads, i = e / kMaxSketch, j = e % kMaxSketch;
      const int64_t r = base + i;
      float om = 0.f, y = 0.f;
      if (r < r1 && j < M) {
        om = bf16_to_f32(omega[r * M + j]);
        y = Y[r * K + j];
      }
      po[u] = om;
      py[u] = y;
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int u = 0; u < kGramLoads; ++u) {
      const int e = tid + u * kGramThreads, i = e / kMaxSketch, j = e % kMaxSketch;
      sX[buf][i][j] = po[u];
      sX[buf][i][kMaxSketch + j] = py[u];
    }
  };
  if (r0 < r1) fetch(r0);
  int buf = 0;
  for (int64_t base = r0; base < r1; base += kGramRows) {
    const int rows = (int)min((int64_t)kGramRows, r1 - base);
    stash(buf);
    __syncthreads();
    if (base + kGramRows < r1) fetch(base + kGramRows);
    for (int i = 0; i < rows; ++i) {
      const float4 x0 = *reinterpret_cast<const float4*>(&sX[buf][i][8 * tr]);
      const float4 x1 = *reinterpret_cast<const float4*>(&sX[buf][i][8 * tr + 4]);
      const float4 y0 = *reinterpret_cast<const float4*>(&sX[buf][i][kMaxSketch + 8 * tc]);
      const float4 y1 = *reinterpret_cast<const float4*>(&sX[buf][i][kMaxSketch + 8 * tc + 4]);
      const float xv[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
      const float yv[8] = {y0.x, y0.y, y0.z, y0.w, y1.x, y1.y, y1.z, y1.w};
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(xv[a], yv[b], acc[a][b]);
    }
    buf ^= 1;  // the other buffer is written next: no barrier needed before it
  }
  // rows of the 2M block: index rr in [0, 128): rr < 64 -> Omega column rr, else Y column rr - 64
  float* out = partial + (size_t)blockIdx.x * (2 * kMaxSketch) * kMaxSketch;
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) out[(8 * tr + a) * kMaxSketch + (8 * tc + b)] = acc[a][b];
}

// out[r * 64 + c] = sum_g partial[g][r][c] in FP64, fixed order
__global__ void gram_reduce(const float* partial, int G, double* out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 2 * kMaxSketch * kMaxSketch) return;
  double s = 0.0;
  for (int g = 0; g < G; ++g) s += (double)partial[(size_t)g * 2 * kMaxSketch * kMaxSketch + e];
  out[e] = s;
}

// ---------------------------------------------------------------- Gram in FP64 (CUDA cores)
// The same block [Omega Y]^T Y from an FP64 Y (the FP64 and refined forms of
// the estimators): FP64 products and sums throughout, partial per CTA in
// the layout of gram_cc (doubles), summed by gram_reduce_f64.
constexpr int kGramRows64 = 16;  // rows staged per tile

__global__ void __launch_bounds__(256) gram_f64(const uint16_t* omega, const double* Y, int64_t n, int M, int K,
                                                int64_t chunk, double* partial /* G x 2M x M */) {
  __shared__ double sX[kGramRows64][2 * kMaxSketch];  // [Omega_i, Y_i]
  const int tid = threadIdx.x;
  const int rt = tid / 16, ct = tid % 16;
  const int64_t r0 = (int64_t)blockIdx.x * chunk;
  const int64_t r1 = min(n, r0 + chunk);
  double acc[8][4];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  for (int64_t base = r0; base < r1; base += kGramRows64) {
    const int rows = (int)min((int64_t)kGramRows64, r1 - base);
    __syncthreads();
    for (int e = tid; e < kGramRows64 * kMaxSketch; e += 256) {
      const int i = e / kMaxSketch, j = e % kMaxSketch;
      double om = 0.0, y = 0.0;
      if (i < rows && j < M) {
        om = (double)bf16_to_f32(omega[(base + i) * M + j]);
        y = Y[(base + i) * K + j];
      }
      sX[i][j] = om;
      sX[i][kMaxSketch + j] = y;
    }
    __syncthreads();
    for (int i = 0; i < rows; ++i) {
      double xv[8], yv[4];
#pragma unroll
      for (int a = 0; a < 8; ++a) xv[a] = sX[i][rt + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) yv[b] = sX[i][kMaxSketch + ct + 16 * b];
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(xv[a], yv[b], acc[a][b]);
    }
  }
  double* out = partial + (size_t)blockIdx.x * (2 * kMaxSketch) * kMaxSketch;
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) out[(rt + 16 * a) * kMaxSketch + (ct + 16 * b)] = acc[a][b];
}

__global__ void gram_reduce_f64(const double* partial, int G, double* out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 2 * kMaxSketch * kMaxSketch) return;
  double s = 0.0;
  for (int g = 0; g < G; ++g) s += partial[(size_t)g * 2 * kMaxSketch * kMaxSketch + e];
  out[e] = s;
}

// ---------------------------------------------------------------- FP64 leave-one-out core
// gram: 128 x 64 doubles, rows 0..63 = Omega^T Y (H), rows 64..127 = Y^T Y (G).
// out[0] = estimate, out[1] = error estimate, out[2] = status (0 ok, 1 not PD), out[8 + i] = t_i
__global__ void __launch_bounds__(256) nys_core(const double* gram, int M, double* out) {
  extern __shared__ double sm[];
  double* H = sm;                        // M x M (Cholesky factor in the lower triangle)
  double* Gm = H + kMaxSketch * kMaxSketch;  // M x M
  double* P = Gm + kMaxSketch * kMaxSketch;  // M x M inverse
  double* W = P + kMaxSketch * kMaxSketch;   // M x M
  __shared__ double s_t[kMaxSketch];
  __shared__ int s_bad;
  const int tid = threadIdx.x;
  constexpr int LD = kMaxSketch;
  if (tid == 0) s_bad = 0;
  for (int e = tid; e < M * M; e += 256) {
    const int r = e / M, c = e % M;
    H[r * LD + c] = 0.5 * (gram[r * kMaxSketch + c] + gram[c * kMaxSketch + r]);
    Gm[r * LD + c] = 0.5 * (gram[(kMaxSketch + r) * kMaxSketch + c] + gram[(kMaxSketch + c) * kMaxSketch + r]);
  }
  __syncthreads();
  // right-looking Cholesky H = L L^T (lower triangle)
  for (int k = 0; k < M; ++k) {
    if (tid == 0) {
      const double d = H[k * LD + k];
      if (!(d > 0.0)) s_bad = 1;
      H[k * LD + k] = sqrt(fmax(d, 1e-300));
    }
    __syncthreads();
    const double dk = H[k * LD + k];
    for (int i = k + 1 + tid; i < M; i += 256) H[i * LD + k] /= dk;
    __syncthreads();
    for (int e = tid; e < (M - k - 1) * (M - k - 1); e += 256) {
      const int i = k + 1 + e / (M - k - 1), j = k + 1 + e % (M - k - 1);
      if (j <= i) H[i * LD + j] -= H[i * LD + k] * H[j * LD + k];
    }
    __syncthreads();
  }
  // P = H^{-1}: thread c solves L L^T p = e_c
  for (int c = tid; c < M; c += 256) {
    for (int i = 0; i < M; ++i) {  // forward: L z = e_c, z stored in P[i][c]
      double s = (i == c) ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) s -= H[i * LD + k] * P[k * LD + c];
      P[i * LD + c] = s / H[i * LD + i];
    }
    for (int i = M - 1; i >= 0; --i) {  // backward: L^T p = z
      double s = P[i * LD + c];
      for (int k = i + 1; k < M; ++k) s -= H[k * LD + i] * P[k * LD + c];
      P[i * LD + c] = s / H[i * LD + i];
    }
  }
  __syncthreads();
  // W = G P
  for (int e = tid; e < M * M; e += 256) {
    const int r = e / M, c = e % M;
    double s = 0.0;
    for (int k = 0; k < M; ++k) s += Gm[r * LD + k] * P[k * LD + c];
    W[r * LD + c] = s;
  }
  __syncthreads();
  // S = tr(P G) = sum_r (P W')... tr(P G) = sum_{r,k} P_rk G_kr = sum_r (G P)_rr = sum_r W_rr
  // q_i = (P G P)_ii = sum_k P_ki W_ki
  if (tid < M) {
    double q = 0.0;
    for (int k = 0; k < M; ++k) q += P[k * LD + tid] * W[k * LD + tid];
    double S = 0.0;
    for (int r = 0; r < M; ++r) S += W[r * LD + r];
    s_t[tid] = S + (1.0 - q) / P[tid * LD + tid];
  }
  __syncthreads();
  if (tid == 0) {
    double mean = 0.0;
    for (int i = 0; i < M; ++i) mean += s_t[i];
    mean /= M;
    double var = 0.0;
    for (int i = 0; i < M; ++i) var += (s_t[i] - mean) * (s_t[i] - mean);
    var /= (M - 1);
    out[0] = mean;
    out[1] = sqrt(var / M);
    out[2] = s_bad ? 1.0 : 0.0;
  }
  if (tid < M) out[8 + tid] = s_t[tid];
}

#endif  // WL_TRACE_KERNELS

}  // namespace wl
