// Reorthogonalisation of the outer Lanczos basis on the walk Laplacian
// (Sec. 4.1: the Lanczos process builds an orthonormal basis of the Krylov
// space; in floating point the three-term recurrence loses that
// orthogonality once Ritz values converge, which repeats Ritz values and
// lengthens the run).
//
// A new basis block v = v_{j+1} (K columns, one per lockstep recurrence) is
// made orthogonal to the earlier blocks v_0 .. v_j of its own column by
// classical Gram-Schmidt applied twice: h_i = (v_i, v), v <- v - sum_i h_i
// v_i, then again, then v <- v / |v| and beta_j <- beta_j |v| (the
// recurrence's beta_j v_{j+1} = w keeps its meaning). Columns with mask 0
// are left untouched.
//
// Two storages of the basis:
//   FP64          block i at basis + i * blk (doubles)
//   double-float  hi terms at (float*) basis + 2 i blk, lo terms right after
// In the double-float form the dot products take both terms of each value
// in FP64; the corrections h_i v_i are small (h is at the level of the lost
// orthogonality) and are formed from the hi terms in FP32; the subtraction
// from v is an error-free double-float update.
//
// Kernels (element-parallel; element e = row * K + c belongs to column c):
//   ro_dots    partial sums of (v_i, v) per (block, row chunk, column)
//   ro_reduce  h_i per column (fixed-order sum over the row chunks; 0 where
//              the mask is 0)
//   ro_update  v -= sum_i h_i v_i, partial sums of |v|^2 per CTA
//   ro_norm    |v| per column, beta_j update, scale factor 1 / |v|
//   ro_scale   v *= 1 / |v|
#pragma once
#include "wl_common.cuh"
#include "wl_df.cuh"

namespace wl {

constexpr int kRoBlock = 256;  // threads per CTA (a multiple of every K)
constexpr int kRoIB = 8;       // basis blocks per CTA of ro_dots

struct ReorthArgs {
  const void* basis;  // earlier blocks (see storage above)
  void* v;            // FP64: the new block (doubles); double-float: its hi terms
  float* vlo;         // double-float: lo terms of the new block (else NULL)
  int64_t n;
  int K;
  int nb;             // number of earlier blocks v_0 .. v_{nb-1}
  size_t blk;         // n * K
  int R;              // row chunks of ro_dots (gridDim.x)
  double* part;       // nb * R * K partial dots
  double* h;          // nb * K coefficients
  double* npart;      // gridDim.x (of ro_update) * K partial |v|^2
  int nupd;           // CTAs of ro_update
  const int* mask;    // K: 1 = reorthogonalise this column
  double* scale;      // K: 1 / |v| (1 where mask is 0)
  double* Tb;         // K x ldT off-diagonals; Tb[c * ldT + j] *= |v|
  int* done;          // K Lanczos column flags (2 = breakdown)
  int j;
  int ldT;
};

#ifdef WL_REORTH_KERNELS
// Basis and new-block values as FP64 (a double-float pair hi + lo is exact
// in FP64): the dot products need the lo terms, since the lost
// orthogonality they measure lies far below the FP32 rounding of the hi terms.
template <bool DF>
__device__ __forceinline__ double ro_load(const ReorthArgs& a, int i, size_t e) {
  if constexpr (DF) {
    const float* b = (const float*)a.basis + (size_t)2 * i * a.blk + e;
    return (double)__ldcg(b) + (double)__ldcg(b + a.blk);
  } else {
    return __ldcg((const double*)a.basis + (size_t)i * a.blk + e);
  }
}

template <bool DF>
__device__ __forceinline__ double ro_vload(const ReorthArgs& a, size_t e) {
  if constexpr (DF)
    return (double)__ldcg((const float*)a.v + e) + (double)__ldcg(a.vlo + e);
  else
    return __ldcg((const double*)a.v + e);
}

// grid (R, ceil(nb / kRoIB)): CTA (r, g) sums (v_i, v) over its row chunk
// for blocks i = g kRoIB .. g kRoIB + kRoIB - 1
template <bool DF>
__global__ void __launch_bounds__(kRoBlock) ro_dots(ReorthArgs a) {
  __shared__ double s[kRoIB][kRoBlock];
  const int tid = threadIdx.x, r = blockIdx.x, i0 = blockIdx.y * kRoIB;
  const int nib = min(kRoIB, a.nb - i0);
  // chunk of whole CTA strides: every thread keeps one column c = tid % K
  const size_t per = ((a.blk + (size_t)a.R * kRoBlock - 1) / ((size_t)a.R * kRoBlock)) * kRoBlock;
  const size_t e0 = (size_t)r * per, e1 = min(a.blk, e0 + per);
  double acc[kRoIB];
#pragma unroll
  for (int b = 0; b < kRoIB; ++b) acc[b] = 0.0;
  for (size_t e = e0 + tid; e < e1; e += kRoBlock) {
    const double x = ro_vload<DF>(a, e);
#pragma unroll
    for (int b = 0; b < kRoIB; ++b)
      if (b < nib) acc[b] += ro_load<DF>(a, i0 + b, e) * x;
  }
#pragma unroll
  for (int b = 0; b < kRoIB; ++b) s[b][tid] = acc[b];
  __syncthreads();
  const int K = a.K;
  for (int t = tid; t < nib * K; t += kRoBlock) {
    const int b = t / K, c = t % K;
    double sum = 0.0;
    for (int u = c; u < kRoBlock; u += K) sum += s[b][u];
    a.part[((size_t)(i0 + b) * a.R + r) * K + c] = sum;
  }
}

__global__ void ro_reduce(ReorthArgs a) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.nb * a.K) return;
  const int i = t / a.K, c = t % a.K;
  double sum = 0.0;
  if (a.mask[c] && !a.done[c])
    for (int r = 0; r < a.R; ++r) sum += a.part[((size_t)i * a.R + r) * a.K + c];
  a.h[t] = sum;
}

// v -= sum_i h_i v_i for every element; per-CTA |v|^2 per column
template <bool DF>
__global__ void __launch_bounds__(kRoBlock) ro_update(ReorthArgs a) {
  __shared__ double s[kRoBlock];
  const int tid = threadIdx.x, K = a.K, c = tid % K;
  double nrm = 0.0;
  for (size_t e = (size_t)blockIdx.x * kRoBlock + tid; e < a.blk; e += (size_t)gridDim.x * kRoBlock) {
    if constexpr (DF) {
      float corr = 0.f;
      for (int i = 0; i < a.nb; ++i) {
        const float hi = (float)a.h[(size_t)i * K + c];
        if (hi != 0.f) corr = __fmaf_rn(hi, __ldcg((const float*)a.basis + (size_t)2 * i * a.blk + e), corr);
      }
      float* vh = (float*)a.v;
      const df x = df_add_f(df{vh[e], a.vlo[e]}, -corr);
      vh[e] = x.hi;
      a.vlo[e] = x.lo;
      const double xd = (double)x.hi + (double)x.lo;
      nrm += xd * xd;
    } else {
      double corr = 0.0;
      for (int i = 0; i < a.nb; ++i) {
        const double hi = a.h[(size_t)i * K + c];
        if (hi != 0.0) corr = fma(hi, __ldcg((const double*)a.basis + (size_t)i * a.blk + e), corr);
      }
      double* v = (double*)a.v;
      const double x = v[e] - corr;
      v[e] = x;
      nrm += x * x;
    }
  }
  s[tid] = nrm;
  __syncthreads();
  if (tid < K) {
    double sum = 0.0;
    for (int u = tid; u < kRoBlock; u += K) sum += s[u];
    a.npart[(size_t)blockIdx.x * K + tid] = sum;
  }
}

// one thread per column: |v|, beta_j <- beta_j |v|, scale 1 / |v| (a column
// whose new vector vanished under the projection reached an invariant
// subspace: beta_j = 0 and the column is marked converged by breakdown)
__global__ void ro_norm(ReorthArgs a) {
  const int c = threadIdx.x;
  if (c >= a.K) return;
  if (!a.mask[c] || a.done[c]) {
    a.scale[c] = 1.0;
    return;
  }
  double sum = 0.0;
  for (int b = 0; b < a.nupd; ++b) sum += a.npart[(size_t)b * a.K + c];
  const double nv = sqrt(sum);
  if (!(nv > 1e-10)) {
    a.Tb[c * a.ldT + a.j] = 0.0;
    a.done[c] = 2;
    a.scale[c] = 1.0;
    return;
  }
  a.Tb[c * a.ldT + a.j] *= nv;
  a.scale[c] = 1.0 / nv;
}

template <bool DF>
__global__ void __launch_bounds__(kRoBlock) ro_scale(ReorthArgs a) {
  const int K = a.K;
  for (size_t e = (size_t)blockIdx.x * kRoBlock + threadIdx.x; e < a.blk; e += (size_t)gridDim.x * kRoBlock) {
    const int c = (int)(e % (size_t)K);
    const double s = a.scale[c];
    if (s == 1.0) continue;
    if constexpr (DF) {
      float* vh = (float*)a.v;
      const df x = df_mul(df{vh[e], a.vlo[e]}, df_from_double(s));
      vh[e] = x.hi;
      a.vlo[e] = x.lo;
    } else {
      ((double*)a.v)[e] *= s;
    }
  }
}
#endif  // WL_REORTH_KERNELS

}  // namespace wl
