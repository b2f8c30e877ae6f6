// Lanczos for the extreme eigenvalues of Op = c0 I + cA A + cD D (k = 1, FP64)
// as high-occupancy phase kernels (Sec. 4.1; used for lambda_max(A) and the
// spectral-radius search of Z_mu, Prop. whe-we-converge).
//
// Step j (two kernels, no host synchronisation between steps):
//   S: v_j = w_{j-1} / beta_{j-1} (stored), w_j = Op v_j computed from the raw
//      w_{j-1} gathered and scaled once per row; alpha_j = (v_j, w_j)
//   U: w_j -= alpha_j v_j + beta_{j-1} v_{j-1}; beta_j = |w_j|
// The last CTA of each kernel reduces the partials in a fixed order and
// records alpha_j / beta_j; after m steps one CTA bisects T_m.
#pragma once
#include "wl_cg2.cuh"
#include "wl_lanczos.cuh"

namespace wl {

struct LzState {
  double alpha[512];
  double beta[512];  // beta[j] = |w_j|; beta_{-1} (start norm) in start_norm
  double start_norm;
  int m_eff;         // steps done before an (exact) breakdown, or m
  int stop;
  unsigned ticket;
  int brk;           // 1 after an (exact) breakdown: the run cannot be continued
  double out[8];     // theta_max(T_m), theta_max(T_{m-c}), theta_min(T_m), theta_min(T_{m-c}), m_eff
};

struct LzArgs {
  PhaseGraph g;
  double c0, cA, cD;
  double* V[2];  // normalised basis vectors (ping-pong)
  double* W[2];  // raw w vectors (ping-pong)
  double* part;
  LzState* st;
  int j;         // step index
  uint64_t seed;
};

#ifdef WL_LANCZOS2_KERNELS
__device__ inline double lz_start(int64_t i, uint64_t seed) {
  uint64_t z = (uint64_t)i * 0x9E3779B97F4A7C15ull + seed;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return 1.0 + 0.25 * ((double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5);
}

// start vector into W[1] (raw) and its norm; V[1] = 0 (v_{-1})
__global__ void __launch_bounds__(kPhaseBlock) lz_init(LzArgs a) {
  __shared__ double s_tmp[kPhaseBlock];
  __shared__ double s_out[1];
  double acc[1] = {0.0};
  for (int64_t i = (int64_t)blockIdx.x * kPhaseBlock + threadIdx.x; i < a.g.n; i += (int64_t)gridDim.x * kPhaseBlock) {
    const double x = lz_start(i, a.seed);
    a.W[1][i] = x;
    a.V[1][i] = 0.0;
    acc[0] += x * x;
  }
  if (!block_partials_last<double, 1>(acc, a.part, &a.st->ticket)) return;
  sum_partials<1>(a.part, gridDim.x, s_tmp, s_out);
  if (threadIdx.x == 0) {
    a.st->start_norm = sqrt(s_out[0]);
    a.st->stop = 0;
    a.st->brk = 0;
    a.st->m_eff = 0;
    a.st->ticket = 0;
  }
}

__global__ void __launch_bounds__(kPhaseBlock, kPhaseMinBlocks) lz_s(LzArgs a) {
  __shared__ double s_red[kPhaseBlock];
  __shared__ double s_tmp[kPhaseBlock];
  __shared__ double s_out[1];
  LzState* st = a.st;
  if (*(volatile int*)&st->stop) return;
  const int j = a.j, cur = j & 1, prv = cur ^ 1;
  const double bprev = (j == 0) ? st->start_norm : st->beta[j - 1];
  const double inv = 1.0 / bprev;
  const double* Wp = a.W[prv];
  double* Vc = a.V[cur];
  double* Wc = a.W[cur];
  const int tid = threadIdx.x;
  double acc[1] = {0.0};
  auto fin = [&](int64_t row, int deg, double nbsum) {
    const double vi = Wp[row] * inv;
    const double wi = a.c0 * vi + a.cA * (nbsum * inv) + a.cD * (double)deg * vi;
    Vc[row] = vi;
    Wc[row] = wi;
    acc[0] += vi * wi;
  };
  if ((int)blockIdx.x < a.g.nhub) {
    const int64_t row = a.g.hubs[blockIdx.x];
    const int beg = a.g.row_ptr[row], end = a.g.row_ptr[row + 1];
    double s = 0.0;
    for (int e = beg + tid; e < end; e += kPhaseBlock) s += Wp[__ldg(a.g.col + e)];
    s_red[tid] = s;
    __syncthreads();
    for (int w = kPhaseBlock / 2; w > 0; w >>= 1) {
      if (tid < w) s_red[tid] += s_red[tid + w];
      __syncthreads();
    }
    if (tid == 0) fin(row, end - beg, s_red[0]);
  } else {
    const int64_t nblk = (int64_t)gridDim.x - a.g.nhub;
    for (int64_t row = ((int64_t)blockIdx.x - a.g.nhub) * kPhaseBlock + tid; row < a.g.n; row += nblk * kPhaseBlock) {
      const int beg = a.g.row_ptr[row], end = a.g.row_ptr[row + 1];
      if (end - beg > kHubDeg) continue;
      double s = 0.0;
      int e = beg;
      for (; e + 3 < end; e += 4) {
        const int j0 = __ldg(a.g.col + e), j1 = __ldg(a.g.col + e + 1);
        const int j2 = __ldg(a.g.col + e + 2), j3 = __ldg(a.g.col + e + 3);
        s += (Wp[j0] + Wp[j1]) + (Wp[j2] + Wp[j3]);
      }
      for (; e < end; ++e) s += Wp[__ldg(a.g.col + e)];
      fin(row, end - beg, s);
    }
  }
  if (!block_partials_last<double, 1>(acc, a.part, &st->ticket)) return;
  sum_partials<1>(a.part, gridDim.x, s_tmp, s_out);
  if (tid == 0) {
    st->alpha[j] = s_out[0];
    st->ticket = 0;
  }
}

__global__ void __launch_bounds__(kPhaseBlock) lz_u(LzArgs a, int last) {
  __shared__ double s_tmp[kPhaseBlock];
  __shared__ double s_out[1];
  LzState* st = a.st;
  if (*(volatile int*)&st->stop) return;
  const int j = a.j, cur = j & 1, prv = cur ^ 1;
  const double al = st->alpha[j];
  const double bp = (j == 0) ? 0.0 : st->beta[j - 1];
  double* Wc = a.W[cur];
  const double* Vc = a.V[cur];
  const double* Vp = a.V[prv];
  double acc[1] = {0.0};
  for (int64_t i = (int64_t)blockIdx.x * kPhaseBlock + threadIdx.x; i < a.g.n; i += (int64_t)gridDim.x * kPhaseBlock) {
    const double w = Wc[i] - al * Vc[i] - bp * Vp[i];
    Wc[i] = w;
    acc[0] += w * w;
  }
  if (!block_partials_last<double, 1>(acc, a.part, &st->ticket)) return;
  sum_partials<1>(a.part, gridDim.x, s_tmp, s_out);
  if (threadIdx.x == 0) {
    const double b = sqrt(s_out[0]);
    st->beta[j] = b;
    st->m_eff = j + 1;
    // invariant subspace reached: T_{j+1} is exact
    if (!(b > 1e-13 * (fabs(al) + bp + 1e-300))) {
      st->brk = 1;
      st->stop = 1;
    } else if (last) {
      st->stop = 1;
    }
    st->ticket = 0;
  }
}

// re-open a run stopped at its last step (not after a breakdown) so that
// more steps can be appended
__global__ void lz_resume(LzState* st) {
  if (threadIdx.x == 0 && !st->brk) st->stop = 0;
}

// Extreme eigenvalues of T_m and T_{m - check} by multisection: four groups
// of kEigT threads, one group per eigenvalue. Each round evaluates kEigT
// Sturm counts spread across the group's bracket and keeps the sub-interval
// where the count passes the eigenvalue's index; 9 rounds shrink the
// Gershgorin bracket by 129^9 (below the FP64 spacing).
constexpr int kEigT = 128;
constexpr int kEigRounds = 9;

__global__ void __launch_bounds__(4 * kEigT) lz_eig(LzState* st, int check) {
  __shared__ double s_lo[4], s_hi[4];
  __shared__ int s_cnt[4][kEigT];
  const int m = st->m_eff;
  if (m <= 0) {
    if (threadIdx.x == 0) st->out[4] = 0.0;
    return;
  }
  const int grp = threadIdx.x / kEigT, t = threadIdx.x % kEigT;
  const int mm = (grp & 1) ? (m > check ? m - check : m) : m;
  const int idx = (grp < 2) ? mm - 1 : 0;
  if (t == 0) {
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < mm; ++i) {
      const double r = (i > 0 ? fabs(st->beta[i - 1]) : 0.0) + (i + 1 < mm ? fabs(st->beta[i]) : 0.0);
      lo = fmin(lo, st->alpha[i] - r);
      hi = fmax(hi, st->alpha[i] + r);
    }
    s_lo[grp] = lo;
    s_hi[grp] = hi;
  }
  __syncthreads();
  for (int round = 0; round < kEigRounds; ++round) {
    const double lo = s_lo[grp], w = s_hi[grp] - lo;
    s_cnt[grp][t] = sturm_count(st->alpha, st->beta, mm, lo + w * (double)(t + 1) / (double)(kEigT + 1));
    __syncthreads();
    if (t == 0) {
      int k = 0;
      while (k < kEigT && s_cnt[grp][k] <= idx) ++k;
      s_lo[grp] = lo + w * (double)k / (double)(kEigT + 1);
      s_hi[grp] = lo + w * (double)(k + 1) / (double)(kEigT + 1);
    }
    __syncthreads();
  }
  if (t == 0) st->out[grp] = 0.5 * (s_lo[grp] + s_hi[grp]);
  if (threadIdx.x == 0) st->out[4] = (double)m;
}
#endif  // WL_LANCZOS2_KERNELS

}  // namespace wl
