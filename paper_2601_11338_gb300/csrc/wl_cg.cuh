// Lockstep conjugate gradients on M = ca I + cA A + cD D for K columns at once,
// as one persistent cooperative kernel (Sec. 4.2: each application of the
// resolvent walk Laplacian is one CG solve with the deformed Laplacian, which
// is positive definite for alpha < 1 / rho(Z), Prop. CGworks).
//
// Per iteration two phases, each ending in a bounded grid barrier:
//   U: r -= alpha q ; gamma' = (r, r)                      (own rows, coalesced)
//   S: s = M r (gather) ; x += alpha_prev p ; p = r + beta p ;
//      q = s + beta q ; delta = (p, q)                      (own rows, by class)
// so that q = M p is carried by the recurrence q_new = M r + beta q_old and
// the SpMM reads only r. The x update is deferred by one phase so it rides
// on the S pass that reads p anyway. Scalars are FP64 in shared memory and
// every CTA reduces the per-CTA partials in the same order, so all CTAs take
// identical decisions and reruns are bit-identical.
//
// Vector traffic per iteration: U reads r, q, writes r; S gathers r, reads
// x, p, q, writes x, p, q: 10 n K s bytes plus 4 nnz + 4 (n + 1) of graph.
#pragma once
#include "wl_common.cuh"

namespace wl {

enum ColStatus : int { kColActive = 0, kColDone = 1 };

#ifdef WL_PHASE_TIMING
// experiment builds only: per-CTA timestamps of the first iterations
constexpr int kStampIters = 8, kStampEv = 4, kStampCtas = 1024;
__device__ unsigned long long g_stamps[kStampCtas * kStampIters * kStampEv];
#define WL_STAMP(it, ev)                                                                         \
  if (threadIdx.x == 0 && blockIdx.x < kStampCtas && (it) < kStampIters)                          \
    g_stamps[(blockIdx.x * kStampIters + (it)) * kStampEv + (ev)] = globaltimer_ns();
#else
#define WL_STAMP(it, ev)
#endif

template <typename T>
struct CgArgs {
  Graph g;
  Part pt;
  T* x;
  T* r;
  T* p;
  T* q;
  double ca, cA, cD;      // operator coefficients
  const double* bnorm2;   // K: ||b_c||^2 (convergence reference); NULL: use ||r_0||^2
  const int* skip;        // K or NULL: columns marked nonzero are left untouched
  double* part;           // 2 * G * K partials (ping-pong)
  double* gamma_out;      // K: final ||r_c||^2 (recurrence)
  int* status;            // K: 0 ok, WL_ERR_* per column
  GridBar* bar;
  int max_iter;
  double tol2;            // relative tolerance squared
  int* iters_out;         // S phases executed
};

template <typename T, int K>
__global__ void __launch_bounds__(kBlock, kMinBlocks) cg_persistent(CgArgs<T> a) {
  using C = Cfg<T, K>;
  constexpr int VW = C::VW;
  constexpr int NW = kBlock / 32;
  __shared__ double s_tmp[kBlock];
  __shared__ double s_w[NW * K];
  __shared__ double s_red[K];
  __shared__ double s_alpha[K], s_beta[K], s_gamma[K], s_b2[K];
  __shared__ int s_done[K], s_stat[K], s_all;
  __shared__ __align__(16) T s_gath[kBlock * VW];

  const int G = gridDim.x, cta = blockIdx.x, tid = threadIdx.x;
  const int r0 = a.pt.rb[cta], r1 = a.pt.rb[cta + 1];
  const size_t v0 = (size_t)r0 * K / VW, v1 = (size_t)r1 * K / VW;  // vector range
  const int mycol = (tid % C::G) * VW;                                 // first column of this thread
  const T ca = (T)a.ca, cA = (T)a.cA, cD = (T)a.cD;
  const uint64_t keep = policy_keep(), strm = policy_stream();
  int buf = 0;
  int iters = 0;

  // ---- U0: gamma = (r, r)
  {
    T acc[VW];
#pragma unroll
    for (int v = 0; v < VW; ++v) acc[v] = T(0);
#pragma unroll 4
    for (size_t e = v0 + tid; e < v1; e += kBlock) {
      const Pack<T, VW> rr = ldp<T, VW>(a.r + e * VW);
#pragma unroll
      for (int v = 0; v < VW; ++v) acc[v] += rr.v[v] * rr.v[v];
    }
    cta_column_sums<T, K>(acc, s_w, a.part + (size_t)buf * G * K + (size_t)cta * K);
  }
  if (!grid_sync(a.bar, G)) return;
  reduce_partials<K>(a.part + (size_t)buf * G * K, G, s_tmp, s_red);
  buf ^= 1;
  if (tid < K) {
    const double g0 = s_red[tid], b2 = a.bnorm2 ? a.bnorm2[tid] : g0;
    s_gamma[tid] = g0;
    s_b2[tid] = b2;
    s_alpha[tid] = 0.0;
    s_beta[tid] = 0.0;
    s_stat[tid] = 0;
    int done = (b2 <= 0.0) || (g0 <= a.tol2 * b2) || (a.skip && a.skip[tid]);
    if (!isfinite(g0)) { done = 1; s_stat[tid] = WL_ERR_NONFINITE; }
    s_done[tid] = done;
  }
  __syncthreads();
  if (tid == 0) {
    int all = 1;
    for (int c = 0; c < K; ++c) all &= s_done[c];
    s_all = all;
  }
  __syncthreads();

  bool first = true;
  while (!s_all) {
    WL_STAMP(iters, 0);
    // ---- S: s = M r; x += alpha p; p = r + beta p; q = s + beta q; delta = (p, q)
    {
      T al[VW], be[VW], dacc[VW];
#pragma unroll
      for (int v = 0; v < VW; ++v) {
        al[v] = (T)s_alpha[mycol + v];
        be[v] = (T)s_beta[mycol + v];
        dacc[v] = T(0);
      }
      struct PreCG {
        Pack<T, VW> r, x, p, q;
      };
      auto pre = [&](int row, int lane_off) {
        PreCG v;
        const size_t o = (size_t)row * K + lane_off;
        v.r = ldh<T, VW>(a.r + o, keep);
        if (!first) {
          v.x = ldh<T, VW>(a.x + o, strm);
          v.p = ldh<T, VW>(a.p + o, strm);
          v.q = ldh<T, VW>(a.q + o, strm);
        }
        return v;
      };
      auto fin = [&](int row, int deg, int lane_off, const T (&nb)[VW], const PreCG& v) {
        const size_t o = (size_t)row * K + lane_off;
        Pack<T, VW> pp, qq;
        const T dg = (T)deg;
        if (first) {
#pragma unroll
          for (int u = 0; u < VW; ++u) {
            const T s = ca * v.r.v[u] + cA * nb[u] + cD * dg * v.r.v[u];
            pp.v[u] = v.r.v[u];
            qq.v[u] = s;
            dacc[u] += pp.v[u] * qq.v[u];
          }
        } else {
          Pack<T, VW> xx = v.x;
#pragma unroll
          for (int u = 0; u < VW; ++u) {
            const T s = ca * v.r.v[u] + cA * nb[u] + cD * dg * v.r.v[u];
            xx.v[u] += al[u] * v.p.v[u];
            pp.v[u] = v.r.v[u] + be[u] * v.p.v[u];
            qq.v[u] = s + be[u] * v.q.v[u];
            dacc[u] += pp.v[u] * qq.v[u];
          }
          sth<T, VW>(a.x + o, xx, strm);
        }
        sth<T, VW>(a.p + o, pp, strm);
        sth<T, VW>(a.q + o, qq, strm);
      };
      for_rows_gather<T, K>(a.g, a.pt, a.r, s_gath, pre, fin);
      cta_column_sums<T, K>(dacc, s_w, a.part + (size_t)buf * G * K + (size_t)cta * K);
    }
    WL_STAMP(iters, 1);
    ++iters;
    first = false;
    if (!grid_sync(a.bar, G)) return;
    reduce_partials<K>(a.part + (size_t)buf * G * K, G, s_tmp, s_red);
    buf ^= 1;
    if (tid < K) {
      const double delta = s_red[tid];
      if (!s_done[tid]) {
        if (!isfinite(delta)) {
          s_stat[tid] = WL_ERR_NONFINITE; s_done[tid] = 1; s_alpha[tid] = 0.0;
        } else if (delta <= 0.0) {
          s_stat[tid] = WL_ERR_NOT_SPD; s_done[tid] = 1; s_alpha[tid] = 0.0;
        } else {
          s_alpha[tid] = s_gamma[tid] / delta;
        }
      } else {
        s_alpha[tid] = 0.0;
      }
    }
    __syncthreads();

    WL_STAMP(iters - 1, 2);
    // ---- U: r -= alpha q; gamma' = (r, r)
    {
      T al[VW], acc[VW];
#pragma unroll
      for (int v = 0; v < VW; ++v) {
        al[v] = (T)s_alpha[mycol + v];
        acc[v] = T(0);
      }
#pragma unroll 4
      for (size_t e = v0 + tid; e < v1; e += kBlock) {
        Pack<T, VW> rr = ldh<T, VW>(a.r + e * VW, keep);
        const Pack<T, VW> qq = ldh<T, VW>(a.q + e * VW, strm);
#pragma unroll
        for (int v = 0; v < VW; ++v) {
          rr.v[v] -= al[v] * qq.v[v];
          acc[v] += rr.v[v] * rr.v[v];
        }
        sth<T, VW>(a.r + e * VW, rr, keep);
      }
      cta_column_sums<T, K>(acc, s_w, a.part + (size_t)buf * G * K + (size_t)cta * K);
    }
    WL_STAMP(iters - 1, 3);
    if (!grid_sync(a.bar, G)) return;
    reduce_partials<K>(a.part + (size_t)buf * G * K, G, s_tmp, s_red);
    buf ^= 1;
    if (tid < K) {
      const double gnew = s_red[tid];
      if (!s_done[tid]) {
        if (!isfinite(gnew)) {
          s_stat[tid] = WL_ERR_NONFINITE; s_done[tid] = 1; s_beta[tid] = 0.0;
        } else {
          s_beta[tid] = gnew / s_gamma[tid];
          s_gamma[tid] = gnew;
          if (gnew <= a.tol2 * s_b2[tid]) { s_done[tid] = 1; s_beta[tid] = 0.0; }
        }
      } else {
        s_beta[tid] = 0.0;
      }
    }
    __syncthreads();
    if (tid == 0) {
      int all = 1;
      for (int c = 0; c < K; ++c) all &= s_done[c];
      if (iters >= a.max_iter) all = 1;
      s_all = all;
    }
    __syncthreads();
  }

  // ---- F: x += alpha p (the deferred update of the last U phase)
  if (!first) {
    T al[VW];
#pragma unroll
    for (int v = 0; v < VW; ++v) al[v] = (T)s_alpha[mycol + v];
#pragma unroll 4
    for (size_t e = v0 + tid; e < v1; e += kBlock) {
      Pack<T, VW> xx = ldp<T, VW>(a.x + e * VW);
      const Pack<T, VW> pp = ldp<T, VW>(a.p + e * VW);
#pragma unroll
      for (int v = 0; v < VW; ++v) xx.v[v] += al[v] * pp.v[v];
      stp<T, VW>(a.x + e * VW, xx);
    }
  }
  if (cta == 0 && tid < K) {
    a.gamma_out[tid] = s_gamma[tid];
    int st = s_stat[tid];
    if (st == 0 && !s_done[tid]) st = WL_ERR_NO_CONVERGENCE;
    a.status[tid] = st;
    if (tid == 0) *a.iters_out = iters;
  }
}

// ------------------------------------------------------------------ FP64 residual for refinement
// x64 += d32 (skipped when `accumulate` is 0), grid barrier, then
// r64 = b64 - M x64 (gather of x64), r32 = (float) r64, d32 = 0, and the
// column norms ||r64||^2 written to rr_out (by CTA 0 after a second barrier).
struct ResArgs {
  Graph g;
  Part pt;
  double* x;        // FP64 iterate
  float* d;         // FP32 correction from the last inner solve (zeroed here)
  const double* b;  // FP64 right-hand side
  double* r;        // FP64 residual out
  float* r32;       // FP32 right-hand side of the next inner solve
  double ca, cA, cD;
  double* part;     // G * 2K
  double* rr_out;   // K: ||r64||^2
  double* bb_out;   // K: ||b||^2
  GridBar* bar;
  int accumulate;
};

template <int K>
__global__ void __launch_bounds__(kBlock, kMinBlocks) residual64(ResArgs a) {
  using C = Cfg<double, K>;
  using CF = Cfg<float, K>;
  constexpr int VW = C::VW;
  constexpr int NW = kBlock / 32;
  __shared__ double s_tmp[kBlock];
  __shared__ double s_w[NW * K];
  __shared__ double s_red[K];
  __shared__ __align__(16) double s_gath[kBlock * VW];
  const int G = gridDim.x, cta = blockIdx.x, tid = threadIdx.x;
  const int r0 = a.pt.rb[cta], r1 = a.pt.rb[cta + 1];
  const size_t e0 = (size_t)r0 * K, e1 = (size_t)r1 * K;
  double* part_r = a.part;
  double* part_b = a.part + (size_t)G * K;
  if (a.accumulate && a.d) {
    for (size_t e = e0 + tid; e < e1; e += kBlock) a.x[e] += (double)__ldcg(a.d + e);
    if (!grid_sync(a.bar, G)) return;
  }
  double acc[VW], bacc[VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) acc[v] = bacc[v] = 0.0;
  const double ca = a.ca, cA = a.cA, cD = a.cD;
  struct PreR {
    Pack<double, VW> x, b;
  };
  const uint64_t keep = policy_keep(), strm = policy_stream();
  auto pre = [&](int row, int lane_off) {
    PreR v;
    const size_t o = (size_t)row * K + lane_off;
    v.x = ldh<double, VW>(a.x + o, keep);
    v.b = ldh<double, VW>(a.b + o, strm);
    return v;
  };
  auto fin = [&](int row, int deg, int lane_off, const double (&nb)[VW], const PreR& v) {
    const size_t o = (size_t)row * K + lane_off;
    Pack<double, VW> rr;
#pragma unroll
    for (int u = 0; u < VW; ++u) {
      rr.v[u] = v.b.v[u] - (ca * v.x.v[u] + cA * nb[u] + cD * (double)deg * v.x.v[u]);
      acc[u] += rr.v[u] * rr.v[u];
      bacc[u] += v.b.v[u] * v.b.v[u];
      if (a.r32) a.r32[o + u] = (float)rr.v[u];
      if (a.d) a.d[o + u] = 0.0f;
    }
    sth<double, VW>(a.r + o, rr, strm);
  };
  for_rows_gather<double, K>(a.g, a.pt, a.x, s_gath, pre, fin);
  cta_column_sums<double, K>(acc, s_w, part_r + (size_t)cta * K);
  cta_column_sums<double, K>(bacc, s_w, part_b + (size_t)cta * K);
  if (!grid_sync(a.bar, G)) return;
  if (cta == 0) {
    reduce_partials<K>(part_r, G, s_tmp, s_red);
    if (tid < K) a.rr_out[tid] = s_red[tid];
    reduce_partials<K>(part_b, G, s_tmp, s_red);
    if (tid < K) a.bb_out[tid] = s_red[tid];
  }
  (void)CF::VW;
}

}  // namespace wl
