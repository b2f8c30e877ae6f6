// Outer Lanczos on the walk Laplacian for exp(-tau L) U0 (Sec. 4.1) in the
// refined form: the basis V_m, the inner-solve result Y = M^{-1} v_j and D_f
// are double-float vectors (two FP32 arrays each, see wl_df.cuh), so every
// element-wise operation of the outer recurrence is FP32 arithmetic while
// the basis keeps about 48 significant bits. The scalars (alpha_j, beta_j,
// the small tridiagonal problem) stay FP64.
//
// Basis block j: hi terms (n x K floats) followed by lo terms (n x K floats),
// i.e. the same 8 bytes per value as an FP64 block.
#pragma once
#include "wl_common.cuh"
#include "wl_df.cuh"
#include "wl_lanczos.cuh"

namespace wl {

struct DfLanczosArgs {
  const float* vjh;   // v_j (n x K)
  const float* vjl;
  const float* vmh;   // v_{j-1} (unused when j == 0)
  const float* vml;
  const float* yh;    // Y = M^{-1} v_j
  const float* yl;
  const float* dfh;   // D_f (n); NULL: zero (shift-and-invert: w = -a Y with Y = -R v_j)
  const float* dfl;
  df ascale;          // phi = a M^{-1}: w = D_f v_j - a Y
  float* wh;          // v_{j+1} out
  float* wl;
  double* Ta;         // K x ldT alphas
  double* Tb;         // K x ldT betas
  int* done;          // K flags (in/out)
  double* bn2;        // K: |v_{j+1}|^2 (1, or 0 for a finished column) for the next solve
  double* part;       // 2 G K
  GridBar* bar;
  int64_t n;
  int j;
  int ldT;
};

// per-thread double partials in the elementwise float layout -> CTA column sums
template <int K, int VW>
__device__ __forceinline__ void df_cta_sums(const double (&val)[VW], double* s_w, double* dst) {
  constexpr int G = K / VW, NW = kBlock / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double a[VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) a[v] = val[v];
#pragma unroll
  for (int off = G; off < 32; off <<= 1)
#pragma unroll
    for (int v = 0; v < VW; ++v) a[v] += __shfl_xor_sync(0xffffffffu, a[v], off);
  if (lane < G)
#pragma unroll
    for (int v = 0; v < VW; ++v) s_w[warp * K + lane * VW + v] = a[v];
  __syncthreads();
  if (tid < K) {
    double t = 0.0;
    for (int w = 0; w < NW; ++w) t += s_w[w * K + tid];
    dst[tid] = t;
  }
  __syncthreads();
}

// arguments of df_combine (U(tau) from the double-float basis)
struct DfCombineArgs {
  const float* basis;  // block j: hi at basis + 2 j n K, lo at basis + (2 j + 1) n K
  const float* yh;
  const float* yl;
  const int* mcol;
  const double* nrm;
  double* out;
  int64_t n, ld, tstride;
  int c0, ldT, ntau;
  const int32_t* perm;
};

#ifdef WL_EXPDF_KERNELS
// One step of K lockstep Lanczos recurrences, cooperative (three passes
// separated by two grid barriers):
//   w = D_f v_j - a Y ; alpha = (v_j, w)
//   w -= alpha v_j + beta_{j-1} v_{j-1} ; beta = |w|
//   v_{j+1} = w / beta
template <int K>
__global__ void __launch_bounds__(kBlock) df_lanczos_step(DfLanczosArgs a) {
  using C = Cfg<float, K>;
  constexpr int VW = C::VW, NW = kBlock / 32;
  __shared__ double s_tmp[kBlock];
  __shared__ double s_w[NW * K];
  __shared__ double s_red[K];
  __shared__ double s_alpha[K], s_bprev[K], s_inv[K];
  const int G = gridDim.x, cta = blockIdx.x, tid = threadIdx.x;
  const size_t nv = (size_t)a.n * K / VW;
  const int mycol = (tid % C::G) * VW;
  const bool first = (a.j == 0);
  const size_t stride = (size_t)G * kBlock;
  float S[VW], Cc[VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) S[v] = Cc[v] = 0.f;
  for (size_t e = (size_t)cta * kBlock + tid; e < nv; e += stride) {
    const size_t row = e * VW / K;
    const df d = a.dfh ? df{__ldg(a.dfh + row), __ldg(a.dfl + row)} : df{0.f, 0.f};
    const Pack<float, VW> vh = ldp<float, VW>(a.vjh + e * VW), vl = ldp<float, VW>(a.vjl + e * VW);
    const Pack<float, VW> yh = ldp<float, VW>(a.yh + e * VW), yl = ldp<float, VW>(a.yl + e * VW);
    Pack<float, VW> wh, wl;
#pragma unroll
    for (int v = 0; v < VW; ++v) {
      const df vv{vh.v[v], vl.v[v]};
      const df w = df_sub(df_mul(d, vv), df_mul(a.ascale, df{yh.v[v], yl.v[v]}));
      wh.v[v] = w.hi;
      wl.v[v] = w.lo;
      df_acc2(S[v], Cc[v], df_mul(vv, w));
    }
    stp<float, VW>(a.wh + e * VW, wh);
    stp<float, VW>(a.wl + e * VW, wl);
  }
  double acc[VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) acc[v] = (double)S[v] + (double)Cc[v];
  df_cta_sums<K, VW>(acc, s_w, a.part + (size_t)cta * K);
  if (!grid_sync(a.bar, G)) return;
  reduce_partials<K>(a.part, G, s_tmp, s_red);
  if (tid < K) {
    const int dn = a.done[tid];
    s_alpha[tid] = dn ? 0.0 : s_red[tid];
    s_bprev[tid] = (first || dn) ? 0.0 : a.Tb[tid * a.ldT + a.j - 1];
  }
  __syncthreads();
  df al[VW], bp[VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) {
    al[v] = df_from_double(s_alpha[mycol + v]);
    bp[v] = df_from_double(s_bprev[mycol + v]);
    S[v] = Cc[v] = 0.f;
  }
  for (size_t e = (size_t)cta * kBlock + tid; e < nv; e += stride) {
    Pack<float, VW> wh = ldp<float, VW>(a.wh + e * VW), wl = ldp<float, VW>(a.wl + e * VW);
    const Pack<float, VW> vh = ldp<float, VW>(a.vjh + e * VW), vl = ldp<float, VW>(a.vjl + e * VW);
    Pack<float, VW> mh, ml;
    if (!first) {
      mh = ldp<float, VW>(a.vmh + e * VW);
      ml = ldp<float, VW>(a.vml + e * VW);
    }
#pragma unroll
    for (int v = 0; v < VW; ++v) {
      df w = df_sub(df{wh.v[v], wl.v[v]}, df_mul(al[v], df{vh.v[v], vl.v[v]}));
      if (!first) w = df_sub(w, df_mul(bp[v], df{mh.v[v], ml.v[v]}));
      wh.v[v] = w.hi;
      wl.v[v] = w.lo;
      df_acc2(S[v], Cc[v], df_mul(w, w));
    }
    stp<float, VW>(a.wh + e * VW, wh);
    stp<float, VW>(a.wl + e * VW, wl);
  }
#pragma unroll
  for (int v = 0; v < VW; ++v) acc[v] = (double)S[v] + (double)Cc[v];
  df_cta_sums<K, VW>(acc, s_w, a.part + (size_t)G * K + (size_t)cta * K);
  if (!grid_sync(a.bar, G)) return;
  reduce_partials<K>(a.part + (size_t)G * K, G, s_tmp, s_red);
  if (tid < K) {
    const double b = sqrt(fmax(s_red[tid], 0.0));
    const int dn = a.done[tid];
    // invariant subspace reached (lucky breakdown): the column is exact
    const bool brk = dn || !(b > 1e-13 * (fabs(s_alpha[tid]) + s_bprev[tid] + 1e-300));
    s_inv[tid] = brk ? 0.0 : 1.0 / b;
    if (cta == 0) {
      a.Ta[tid * a.ldT + a.j] = s_alpha[tid];
      a.Tb[tid * a.ldT + a.j] = brk ? 0.0 : b;
      a.bn2[tid] = brk ? 0.0 : 1.0;
      if (brk && !dn) a.done[tid] = 2;  // 2: converged by breakdown at this step
    }
  }
  __syncthreads();
  df iv[VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) iv[v] = df_from_double(s_inv[mycol + v]);
  for (size_t e = (size_t)cta * kBlock + tid; e < nv; e += stride) {
    Pack<float, VW> wh = ldp<float, VW>(a.wh + e * VW), wl = ldp<float, VW>(a.wl + e * VW);
#pragma unroll
    for (int v = 0; v < VW; ++v) {
      const df w = df_mul(iv[v], df{wh.v[v], wl.v[v]});
      wh.v[v] = w.hi;
      wl.v[v] = w.lo;
    }
    stp<float, VW>(a.wh + e * VW, wh);
    stp<float, VW>(a.wl + e * VW, wl);
  }
}

// U(tau) = |u0| V_m y(tau) over a double-float basis, all tau from one read
// of the basis; y in double-float (yh, yl: K x ntau x ldT), output FP64.
// The coefficients of the CTA's columns are staged in shared memory (layout
// [j][tau][c]) when they fit; four basis blocks are read per round so that
// eight independent loads are in flight per thread.
constexpr int kCombSmemFloats = 10240;  // 40 KB of staged coefficients

template <int K>
__global__ void __launch_bounds__(kBlock) df_combine(DfCombineArgs a) {
  __shared__ float s_y[kCombSmemFloats];
  const size_t total = (size_t)a.n * K;
  int mmax = 0;
  for (int c = 0; c < K; ++c) mmax = max(mmax, a.mcol[c]);
  const bool staged = (size_t)mmax * a.ntau * K * 2 <= (size_t)kCombSmemFloats;
  if (staged) {
    const int cnt = mmax * a.ntau * K;
    for (int q = threadIdx.x; q < cnt; q += kBlock) {
      const int c = q % K, t = (q / K) % a.ntau, j = q / (K * a.ntau);
      const size_t src = ((size_t)c * a.ntau + t) * a.ldT + j;
      s_y[2 * q] = __ldg(a.yh + src);
      s_y[2 * q + 1] = __ldg(a.yl + src);
    }
  }
  __syncthreads();
  for (size_t e = (size_t)blockIdx.x * kBlock + threadIdx.x; e < total; e += (size_t)gridDim.x * kBlock) {
    const int c = (int)(e % K);
    const size_t i = e / K;
    const int m = a.mcol[c];
    float S[kMaxTau], Cc[kMaxTau];
#pragma unroll
    for (int t = 0; t < kMaxTau; ++t) S[t] = Cc[t] = 0.f;
    auto ycoef = [&](int j, int t) -> df {
      if (staged) {
        const int q = (j * a.ntau + t) * K + c;
        return df{s_y[2 * q], s_y[2 * q + 1]};
      }
      const size_t src = ((size_t)c * a.ntau + t) * a.ldT + j;
      return df{__ldg(a.yh + src), __ldg(a.yl + src)};
    };
    int j = 0;
    for (; j + 3 < m; j += 4) {
      df v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        v[u] = df{__ldcs(a.basis + (size_t)(2 * (j + u)) * total + e),
                  __ldcs(a.basis + (size_t)(2 * (j + u) + 1) * total + e)};
#pragma unroll
      for (int t = 0; t < kMaxTau; ++t)
        if (t < a.ntau) {
#pragma unroll
          for (int u = 0; u < 4; ++u) df_acc2(S[t], Cc[t], df_mul(v[u], ycoef(j + u, t)));
        }
    }
    for (; j < m; ++j) {
      const df v{__ldcs(a.basis + (size_t)(2 * j) * total + e), __ldcs(a.basis + (size_t)(2 * j + 1) * total + e)};
#pragma unroll
      for (int t = 0; t < kMaxTau; ++t)
        if (t < a.ntau) df_acc2(S[t], Cc[t], df_mul(v, ycoef(j, t)));
    }
    const double sc = a.nrm[c];
    const size_t io = a.perm ? (size_t)a.perm[i] : i;
    for (int t = 0; t < a.ntau; ++t)
      a.out[(size_t)t * a.tstride + io * a.ld + a.c0 + c] = sc * ((double)S[t] + (double)Cc[t]);
  }
}

// X (n x K FP64, contiguous; K a power of two <= 64) scaled per column by
// 1 / nrm[c] -> (hi, lo): one reciprocal per column and CTA, then a multiply
// per element
__global__ void __launch_bounds__(kBlock) df_scale_cols(const double* X, int64_t n, int K, const double* nrm,
                                                        float* hi, float* lo) {
  __shared__ double inv[64];
  if (threadIdx.x < K) inv[threadIdx.x] = nrm[threadIdx.x] > 0.0 ? 1.0 / nrm[threadIdx.x] : 0.0;
  __syncthreads();
  const size_t total = (size_t)n * K;
  for (size_t e = (size_t)blockIdx.x * kBlock + threadIdx.x; e < total; e += (size_t)gridDim.x * kBlock) {
    const double x = X[e] * inv[e & (size_t)(K - 1)];
    const float h = (float)x;
    hi[e] = h;
    lo[e] = (float)(x - (double)h);
  }
}

// FP64 vector -> (hi, lo)
__global__ void __launch_bounds__(kBlock) df_split(const double* x, size_t total, float* hi, float* lo) {
  for (size_t e = (size_t)blockIdx.x * kBlock + threadIdx.x; e < total; e += (size_t)gridDim.x * kBlock) {
    const float h = (float)x[e];
    hi[e] = h;
    lo[e] = (float)(x[e] - (double)h);
  }
}
#endif  // WL_EXPDF_KERNELS

}  // namespace wl
