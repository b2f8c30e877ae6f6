// Spectral scale (Sec. 4.1 and Prop. whe-we-converge): the largest
// eigenpair of Op = c0 I + cA A + cD D (k = 1) by Lanczos, for lambda_max(A)
// and for the spectral-radius search of Z_mu.
//
// The basis is stored (double-float, one float2 per node: hi, lo), so a run
// can end with its Ritz vector, which then starts the next run (the search
// over lambda evaluates nearby operators; a warm start needs few steps).
// Every element operation is FP32 arithmetic on double-float values (GB300
// runs FP64 at 1/64 of the FP32 rate); the scalars are FP64.
//
// Step j (two kernels, no host synchronisation between steps):
//   S: v_j = w_{j-1} / beta_{j-1} (stored in V_j), w_j = Op v_j computed from
//      the raw w_{j-1} gathered and scaled once per row; alpha_j = (v_j, w_j)
//   U: w_j -= alpha_j v_j + beta_{j-1} v_{j-1}; beta_j = |w_j|
// Rows: more than kHubDeg entries -> one CTA each; kSpWarpDeg < deg <=
// kHubDeg -> one warp each (listed at build time); the rest one thread each.
// After every few steps one CTA finds the two largest eigenvalues of T_m
// (Sturm multisection), the top eigenvector y of T_m (inverse iteration) and
// the error bound min(r, r^2 / gap), r = beta_m |y_m|, and stops the run once
// the bound is below rtol |theta_1|.
#pragma once
#include "wl_cg2.cuh"
#include "wl_df.cuh"

namespace wl {

constexpr int kSpMax = 256;     // Lanczos steps held per run
constexpr int kSpWarpDeg = kMidDeg;  // rows with more entries (up to kHubDeg) get a warp each

struct SpState {
  double alpha[kSpMax];
  double beta[kSpMax];
  double y[kSpMax];     // top eigenvector of T_m (unit)
  double start_norm;    // |w_{-1}|: norm of the raw start vector
  double out[8];        // theta_1, theta_2, r = beta_m |y_m|, bound, m, |u|^2, u^T D u
  int m_eff;            // steps done (before a breakdown)
  int stop;             // the run is finished (converged, broken down or at its cap)
  int brk;              // exact breakdown: T_m holds exact eigenvalues
  unsigned ticket;
};

struct SpArgs {
  PhaseGraph g;
  const int32_t* mid;  // rows with kSpWarpDeg < deg <= kHubDeg
  int nmid;
  int nmid_blk;        // CTAs that walk the mid rows (after the hub CTAs)
  double c0, cA, cD;
  float2* V;           // basis, V_j at V + j n
  float2* W[2];        // raw w vectors (ping-pong): step j writes W[j & 1], gathers W[(j - 1) & 1]
  double* part;
  SpState* st;
  int j;
  uint64_t seed;
};

// One problem's share of a round of the batched searches (many graphs'
// Lanczos runs advanced together, each with its own operator, basis and
// state): an optional Ritz vector first, then the start of a run (or its
// continuation) and steps j0 .. j1 - 1.
struct SpJob {
  SpArgs a;        // a.j is not used: step s of the round is j0 + s
  double rtol;     // stopping bound of the run, relative to |theta_1|
  int j0, j1, cap;
  int mode;        // -1: no steps; 0: fresh seeded run; 1: new run from W[1]; 2: continue
  int ritz;        // 1: Ritz vector of the current run into W[1] first
  int gs, gu;      // CTAs of this problem in the S kernel and in the other row kernels
};

// A problem's state after a round (the fields of SpState the host reads)
struct SpOut {
  double start_norm;
  double out[8];
  int m_eff, stop, brk, pad;
};

#ifdef WL_SPEC_KERNELS
__device__ __forceinline__ df ld_df2(const float2* p) {
  const float2 v = *p;
  return df{v.x, v.y};
}

__device__ __forceinline__ void st_df2(float2* p, df v) { *p = make_float2(v.hi, v.lo); }

// CTA sums of NV per-thread values written to part[b NV + c] for CTA b of
// nb; the last of the nb CTAs to finish returns true (all partials visible
// to it). The same arithmetic as the phase kernels' reduction for one lane
// per row (butterfly over the warp, then the warps in order).
template <int NV>
__device__ __forceinline__ bool sp_partials_last(const double (&val)[NV], double* part, unsigned* ticket, int b,
                                                 int nb) {
  constexpr int NW = kPhaseBlock / 32;
  __shared__ double s_w[NW * NV];
  __shared__ int s_last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double a[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) a[v] = val[v];
#pragma unroll
  for (int off = 1; off < 32; off <<= 1)
#pragma unroll
    for (int v = 0; v < NV; ++v) a[v] += __shfl_xor_sync(0xffffffffu, a[v], off);
  if (lane == 0)
#pragma unroll
    for (int v = 0; v < NV; ++v) s_w[warp * NV + v] = a[v];
  __syncthreads();
  if (tid < NV) {
    double t = 0.0;
    for (int w = 0; w < NW; ++w) t += s_w[w * NV + tid];
    part[(size_t)b * NV + tid] = t;
    __threadfence();
  }
  __syncthreads();
  if (tid == 0) s_last = (atomicAdd(ticket, 1u) == (unsigned)nb - 1u) ? 1 : 0;
  __syncthreads();
  if (s_last) __threadfence();
  return s_last != 0;
}

__device__ inline double sp_start(int64_t i, uint64_t seed) {
  uint64_t z = (uint64_t)i * 0x9E3779B97F4A7C15ull + seed;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return 1.0 + 0.25 * ((double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5);
}

// The kernel bodies take their CTA index b and CTA count nb: the
// single-problem kernels pass blockIdx.x and gridDim.x, the batched ones the
// CTA's place within its problem's share of the grid.

// fresh run: seeded positive start vector into W[1], its norm, state reset
__device__ __forceinline__ void sp_init_body(const SpArgs& a, int b, int nb) {
  __shared__ double s_tmp[kPhaseBlock];
  __shared__ double s_out[1];
  double acc[1] = {0.0};
  float2* W = a.W[1];
  for (int64_t i = (int64_t)b * kPhaseBlock + threadIdx.x; i < a.g.n; i += (int64_t)nb * kPhaseBlock) {
    const float x = (float)sp_start(i, a.seed);  // any start vector will do: keep it exactly representable
    W[i] = make_float2(x, 0.f);
    acc[0] += (double)x * (double)x;
  }
  if (!sp_partials_last<1>(acc, a.part, &a.st->ticket, b, nb)) return;
  sum_partials<1>(a.part, nb, s_tmp, s_out);
  if (threadIdx.x == 0) {
    a.st->start_norm = sqrt(s_out[0]);
    a.st->stop = 0;
    a.st->brk = 0;
    a.st->m_eff = 0;
    a.st->ticket = 0;
  }
}

// resume = 0: a new run from the vector in W[1] (whose norm is start_norm);
// resume = 1: continue the current run (unless it broke down)
__device__ __forceinline__ void sp_restart_body(SpState* st, int resume) {
  if (threadIdx.x == 0) {
    if (resume) {
      if (!st->brk) st->stop = 0;
    } else {
      st->stop = 0;
      st->brk = 0;
      st->m_eff = 0;
      st->ticket = 0;
    }
  }
}

__device__ __forceinline__ void sp_s_body(const SpArgs& a, int j, int b, int nb) {
  __shared__ float s_red[3][kPhaseBlock];
  __shared__ double s_tmp[kPhaseBlock];
  __shared__ double s_out[1];
  SpState* st = a.st;
  if (*(volatile int*)&st->stop) return;
  const double bprev = (j == 0) ? st->start_norm : st->beta[j - 1];
  const df inv = df_from_double(1.0 / bprev);
  const df c0 = df_from_double(a.c0), cA = df_from_double(a.cA), cD = df_from_double(a.cD);
  // selects, not an indexed load: the arguments stay in registers
  const float2* __restrict__ Wp = (j & 1) ? a.W[0] : a.W[1];
  float2* Wc = (j & 1) ? a.W[1] : a.W[0];
  float2* Vj = a.V + (size_t)j * a.g.n;
  const int tid = threadIdx.x;
  float aS = 0.f, aC = 0.f;
  // neighbour sum (s, c, l) of the raw previous vector -> this row's v, w
  auto fin = [&](int64_t row, int deg, float s, float c, float l) {
    const df nb = df_mul(two_sum(s, c + l), inv);
    const df v = df_mul(ld_df2(Wp + row), inv);
    const df crow = df_add(c0, df_mul_f(cD, (float)deg));
    const df w = df_add(df_mul(crow, v), df_mul(cA, nb));
    st_df2(Vj + row, v);
    st_df2(Wc + row, w);
    df_acc2(aS, aC, df_mul(v, w));
  };
  auto gather = [&](int beg, int end, int step, float& s, float& c, float& l) {
    int e = beg;
    for (; e + 3 * step < end; e += 4 * step) {
      const int j0 = __ldg(a.g.col + e), j1 = __ldg(a.g.col + e + step);
      const int j2 = __ldg(a.g.col + e + 2 * step), j3 = __ldg(a.g.col + e + 3 * step);
      const float2 x0 = Wp[j0], x1 = Wp[j1], x2 = Wp[j2], x3 = Wp[j3];
      df_acc(s, c, x0.x);
      df_acc(s, c, x1.x);
      df_acc(s, c, x2.x);
      df_acc(s, c, x3.x);
      l += (x0.y + x1.y) + (x2.y + x3.y);
    }
    for (; e < end; e += step) {
      const float2 x0 = Wp[__ldg(a.g.col + e)];
      df_acc(s, c, x0.x);
      l += x0.y;
    }
  };
  if (b < a.g.nhub) {
    const int64_t row = a.g.hubs[b];
    const int beg = a.g.row_ptr[row], end = a.g.row_ptr[row + 1];
    float s = 0.f, c = 0.f, l = 0.f;
    gather(beg + tid, end, kPhaseBlock, s, c, l);
    s_red[0][tid] = s;
    s_red[1][tid] = c;
    s_red[2][tid] = l;
    __syncthreads();
    if (tid == 0) {
      for (int t = 1; t < kPhaseBlock; ++t) {
        const df u = two_sum(s, s_red[0][t]);
        s = u.hi;
        c += u.lo + s_red[1][t];
        l += s_red[2][t];
      }
      fin(row, end - beg, s, c, l);
    }
  } else if (b < a.g.nhub + a.nmid_blk) {
    const int lane = tid & 31;
    const int wg = (b - a.g.nhub) * (kPhaseBlock / 32) + (tid >> 5);
    for (int r = wg; r < a.nmid; r += a.nmid_blk * (kPhaseBlock / 32)) {
      const int64_t row = a.mid[r];
      const int beg = a.g.row_ptr[row], end = a.g.row_ptr[row + 1];
      float s = 0.f, c = 0.f, l = 0.f;
      for (int e = beg + lane; e < end; e += 32) {
        const float2 x = Wp[__ldg(a.g.col + e)];
        df_acc(s, c, x.x);
        l += x.y;
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const float so = __shfl_xor_sync(0xffffffffu, s, off);
        const float co = __shfl_xor_sync(0xffffffffu, c, off);
        const float lo = __shfl_xor_sync(0xffffffffu, l, off);
        const df u = two_sum(s, so);
        s = u.hi;
        c += u.lo + co;
        l += lo;
      }
      if (lane == 0) fin(row, end - beg, s, c, l);
    }
  } else {
    const int64_t nblk = (int64_t)nb - a.g.nhub - a.nmid_blk;
    const int bt = b - a.g.nhub - a.nmid_blk;
    const int lim = a.nmid_blk > 0 ? kSpWarpDeg : kHubDeg;
    for (int64_t row = (int64_t)bt * kPhaseBlock + tid; row < a.g.n; row += nblk * kPhaseBlock) {
      const int beg = a.g.row_ptr[row], end = a.g.row_ptr[row + 1];
      if (end - beg > lim) continue;
      float s = 0.f, c = 0.f, l = 0.f;
      gather(beg, end, 1, s, c, l);
      fin(row, end - beg, s, c, l);
    }
  }
  double acc[1] = {(double)aS + (double)aC};
  if (!sp_partials_last<1>(acc, a.part, &st->ticket, b, nb)) return;
  sum_partials<1>(a.part, nb, s_tmp, s_out);
  if (tid == 0) {
    st->alpha[j] = s_out[0];
    st->ticket = 0;
  }
}

__device__ __forceinline__ void sp_u_body(const SpArgs& a, int j, int last, int b, int nb) {
  __shared__ double s_tmp[kPhaseBlock];
  __shared__ double s_out[1];
  SpState* st = a.st;
  if (*(volatile int*)&st->stop) return;
  const double al = st->alpha[j];
  const double bp = (j == 0) ? 0.0 : st->beta[j - 1];
  const df dal = df_from_double(al), dbp = df_from_double(bp);
  float2* Wc = (j & 1) ? a.W[1] : a.W[0];
  const float2* Vj = a.V + (size_t)j * a.g.n;
  const float2* Vm = a.V + (size_t)(j > 0 ? j - 1 : 0) * a.g.n;
  float aS = 0.f, aC = 0.f;
  for (int64_t i = (int64_t)b * kPhaseBlock + threadIdx.x; i < a.g.n; i += (int64_t)nb * kPhaseBlock) {
    df w = df_sub(ld_df2(Wc + i), df_mul(dal, ld_df2(Vj + i)));
    if (j > 0) w = df_sub(w, df_mul(dbp, ld_df2(Vm + i)));
    st_df2(Wc + i, w);
    df_acc2(aS, aC, df_mul(w, w));
  }
  double acc[1] = {(double)aS + (double)aC};
  if (!sp_partials_last<1>(acc, a.part, &st->ticket, b, nb)) return;
  sum_partials<1>(a.part, nb, s_tmp, s_out);
  if (threadIdx.x == 0) {
    const double bj = sqrt(fmax(s_out[0], 0.0));
    st->beta[j] = bj;
    st->m_eff = j + 1;
    // invariant subspace reached: T_{j+1} is exact
    if (!(bj > 1e-13 * (fabs(al) + bp + 1e-300))) {
      st->brk = 1;
      st->stop = 1;
    } else if (last) {
      st->stop = 1;
    }
    st->ticket = 0;
  }
}

// Number of eigenvalues of T_m below x from the signs of the leading
// principal minors p_i(x) (Sturm sequence), with no division: p_{i+1} =
// (alpha_i - x) p_i - beta_{i-1}^2 p_{i-1}, rescaled by powers of two to
// stay in range; a zero minor takes the sign opposite to its predecessor.
// Sturm count (eigenvalues below x) of the tridiagonal with diagonal a and
// squared off-diagonal b2, by the scaled three-term determinant recurrence
__device__ inline int sturm_count_poly(const double* a, const double* b2, int m, double x) {
  double pm = 1.0, p = a[0] - x;
  int cnt = (p < 0.0) ? 1 : 0;
  double sprev = (p == 0.0) ? -1.0 : p;
  for (int i = 1; i < m; ++i) {
    const double pn = (a[i] - x) * p - b2[i - 1] * pm;
    pm = p;
    p = pn;
    const double ap = fabs(p);
    if (ap > 0x1p500) {
      p *= 0x1p-500;
      pm *= 0x1p-500;
    } else if (ap < 0x1p-500 && fabs(pm) < 0x1p-500) {
      p *= 0x1p500;
      pm *= 0x1p500;
    }
    const double sc = (p == 0.0) ? -sprev : p;
    if ((sc < 0.0) != (sprev < 0.0)) ++cnt;
    sprev = sc;
  }
  return cnt;
}

// Sturm count in FP32 by the pivot recurrence d_i = (a_i - x) - b_{i-1}^2 /
// d_{i-1} (the number of negative pivots of T - x I); a pivot of magnitude
// below `tiny` is replaced by -tiny. Used only to bracket eigenvalues
// coarsely: the bracket is widened and checked in FP64 before it is used.
__device__ inline int sturm_count_f32(const float* a, const float* b2, int m, float x) {
  constexpr float tiny = 1e-30f;
  float d = a[0] - x;
  if (fabsf(d) < tiny) d = -tiny;
  int cnt = (d < 0.f) ? 1 : 0;
  for (int i = 1; i < m; ++i) {
    d = (a[i] - x) - __fdividef(b2[i - 1], d);  // |d| >= tiny keeps the fast division in range
    if (fabsf(d) < tiny) d = -tiny;
    cnt += (d < 0.f) ? 1 : 0;
  }
  return cnt;
}

// Sturm count (eigenvalues below x) in double-float arithmetic: the scaled
// three-term determinant recurrence of sturm_count_poly on FP32 pairs. A
// dependent FP64 operation costs about a hundred cycles on this GPU, the
// FP32 operations of a double-float one a few each.
__device__ inline int sturm_count_df(const float* ah, const float* al, const float* bh, const float* bl, int m,
                                     df x) {
  df pm{1.f, 0.f};
  df p = df_sub(df{ah[0], al[0]}, x);
  int cnt = (p.hi < 0.f) ? 1 : 0;
  float sprev = (p.hi == 0.f) ? -1.f : p.hi;
  for (int i = 1; i < m; ++i) {
    const df pn = df_sub(df_mul(df_sub(df{ah[i], al[i]}, x), p), df_mul(df{bh[i - 1], bl[i - 1]}, pm));
    pm = p;
    p = pn;
    const float ap = fabsf(p.hi);
    if (ap > 0x1p64f) {
      p = df{p.hi * 0x1p-64f, p.lo * 0x1p-64f};
      pm = df{pm.hi * 0x1p-64f, pm.lo * 0x1p-64f};
    } else if (ap < 0x1p-64f && fabsf(pm.hi) < 0x1p-64f) {
      p = df{p.hi * 0x1p64f, p.lo * 0x1p64f};
      pm = df{pm.hi * 0x1p64f, pm.lo * 0x1p64f};
    }
    const float sc = (p.hi == 0.f) ? -sprev : p.hi;
    if ((sc < 0.f) != (sprev < 0.f)) ++cnt;
    sprev = sc;
  }
  return cnt;
}

// 1/a in double-float: an approximate FP32 reciprocal of a.hi and one
// correction step (|a.hi| between 2^-126 and 2^126)
__device__ __forceinline__ df df_rcp(df a) {
  const float r0 = __fdividef(1.f, a.hi);
  const df e = df_sub(df{1.f, 0.f}, df_mul_f(a, r0));
  return df_add(df{r0, 0.f}, df_mul_f(e, r0));
}

// Two largest eigenvalues of T_m (a group of kSpEigT threads per eigenvalue),
// then the top eigenvector by inverse iteration and the error bound; stops
// the run when the bound is below rtol |theta_1|. A dependent FP64 operation
// costs about a hundred cycles on this GPU (measured: a Sturm count over 256
// rows took 200k cycles in FP64), so the serial work runs in FP32 and
// double-float:
//   1. kSpEigCoarse rounds of FP32 multisection (kSpEigT points each) from
//      the Gershgorin interval bracket each eigenvalue to about 1e-6 ||T||;
//   2. the bracket, widened by kSpEigMargin ||T|| on both sides, is checked
//      by two double-float Sturm counts;
//   3. kSpEigFine rounds of double-float multisection narrow it to about
//      1e-14 ||T|| (the resolution of double-float counts; the searches
//      stop at 1e-10 to 1e-12 of theta_1);
//   4. inverse iteration in double-float gives the eigenvector.
// If a check fails (the FP32 counts were wrong, or T overflows FP32), that
// eigenvalue is found as before: kSpEigRounds rounds of FP64 multisection
// from the Gershgorin interval (129^7 > 1e14).
constexpr int kSpEigT = 128;
constexpr int kSpEigRounds = 7;
constexpr int kSpEigCoarse = 3;     // 129^3 > 2e6: the FP32 bracket is below 1e-6 of the interval
constexpr double kSpEigMargin = 1e-6;
constexpr int kSpEigFine = 4;       // 129^4 > 2.7e8: from 2.9e-6 ||T|| to 1.1e-14 ||T||
static_assert(kSpEigFine <= kSpEigRounds, "the narrow search ends within the full one");
static_assert(2 * kSpEigT == kSpMax, "one row per thread in the eigen step");

__device__ __forceinline__ void sp_eig_body(SpState* st, double rtol) {
  __shared__ double s_lo[2], s_hi[2];
  __shared__ int s_cnt[2][kSpEigT];
  __shared__ int s_ok[2];
  __shared__ double s_a[kSpMax], s_b[kSpMax], s_b2[kSpMax];
  __shared__ float s_af[kSpMax], s_b2f[kSpMax];
  __shared__ float s_ah[kSpMax], s_al[kSpMax], s_qh[kSpMax], s_ql[kSpMax];  // a and b^2 as pairs
  __shared__ float s_bh[kSpMax], s_bl[kSpMax];                              // b as pairs
  __shared__ float s_yh[kSpMax], s_yl[kSpMax], s_ch[kSpMax], s_cl[kSpMax];  // inverse iteration
  __shared__ double s_red[3][kSpEigT * 2 / 32];
  __shared__ double s_tn, s_glo, s_ghi, s_nn;
  const int m = st->m_eff;
  if (m <= 0 || m > kSpMax) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // one row per thread (m <= kSpMax = blockDim): staging and the Gershgorin
  // interval by a block reduction
  double glo = 1e300, ghi = -1e300, gtn = 0.0;
  if (tid < m) {
    const double a = st->alpha[tid], b = (tid + 1 < m) ? st->beta[tid] : 0.0;
    const double bp = (tid > 0) ? st->beta[tid - 1] : 0.0;
    s_a[tid] = a;
    s_b[tid] = b;
    s_b2[tid] = b * b;
    s_af[tid] = (float)a;
    s_b2f[tid] = (float)(b * b);
    const df ad = df_from_double(a), qd = df_from_double(b * b), bd = df_from_double(b);
    s_ah[tid] = ad.hi;
    s_al[tid] = ad.lo;
    s_qh[tid] = qd.hi;
    s_ql[tid] = qd.lo;
    s_bh[tid] = bd.hi;
    s_bl[tid] = bd.lo;
    const double r = fabs(bp) + fabs(b);
    glo = a - r;
    ghi = a + r;
    gtn = fabs(a) + r;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    glo = fmin(glo, __shfl_xor_sync(0xffffffffu, glo, off));
    ghi = fmax(ghi, __shfl_xor_sync(0xffffffffu, ghi, off));
    gtn = fmax(gtn, __shfl_xor_sync(0xffffffffu, gtn, off));
  }
  if (lane == 0) {
    s_red[0][warp] = glo;
    s_red[1][warp] = ghi;
    s_red[2][warp] = gtn;
  }
  __syncthreads();
  const int grp = tid / kSpEigT, t = tid % kSpEigT;
  const int idx = grp == 0 ? m - 1 : (m >= 2 ? m - 2 : m - 1);
  if (tid == 0) {
    double lo = 1e300, hi = -1e300, tn = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) {
      lo = fmin(lo, s_red[0][w]);
      hi = fmax(hi, s_red[1][w]);
      tn = fmax(tn, s_red[2][w]);
    }
    s_lo[0] = s_lo[1] = s_glo = lo;
    s_hi[0] = s_hi[1] = s_ghi = hi;
    s_tn = tn;
  }
  __syncthreads();
  // (1) FP32 multisection
  for (int round = 0; round < kSpEigCoarse; ++round) {
    const double lo = s_lo[grp], w = s_hi[grp] - lo;
    s_cnt[grp][t] = sturm_count_f32(s_af, s_b2f, m, (float)(lo + w * (double)(t + 1) / (double)(kSpEigT + 1)));
    __syncthreads();
    if (t == 0) {
      int k = 0;
      while (k < kSpEigT && s_cnt[grp][k] <= idx) ++k;
      s_lo[grp] = lo + w * (double)k / (double)(kSpEigT + 1);
      s_hi[grp] = lo + w * (double)(k + 1) / (double)(kSpEigT + 1);
    }
    __syncthreads();
  }
  // (2) widen by kSpEigMargin ||T|| and check with two double-float counts:
  // count(lo) <= idx < count(hi)
  const double mg = kSpEigMargin * s_tn;
  const double wlo = fmax(s_glo, s_lo[grp] - mg), whi = fmin(s_ghi, s_hi[grp] + mg);
  if (t < 2) s_cnt[grp][t] = sturm_count_df(s_ah, s_al, s_qh, s_ql, m, df_from_double(t == 0 ? wlo : whi));
  __syncthreads();
  if (t == 0) {
    const bool ok = whi > wlo && s_cnt[grp][0] <= idx && s_cnt[grp][1] > idx;
    s_ok[grp] = ok ? 1 : 0;
    s_lo[grp] = ok ? wlo : s_glo;
    s_hi[grp] = ok ? whi : s_ghi;
  }
  __syncthreads();
  // (3) multisection to the end: double-float counts from the checked
  // bracket, or FP64 counts from the Gershgorin interval where the check
  // failed (the loop is uniform over the block: every thread reaches its
  // barriers)
  const int rounds = (s_ok[0] && s_ok[1]) ? kSpEigFine : kSpEigRounds;
  for (int round = 0; round < rounds; ++round) {
    const bool nar = s_ok[grp] != 0;
    const bool act = nar ? round < kSpEigFine : true;
    const double lo = s_lo[grp], w = s_hi[grp] - lo;
    const double x = lo + w * (double)(t + 1) / (double)(kSpEigT + 1);
    if (act) s_cnt[grp][t] = nar ? sturm_count_df(s_ah, s_al, s_qh, s_ql, m, df_from_double(x))
                                 : sturm_count_poly(s_a, s_b2, m, x);
    __syncthreads();
    if (act && t == 0) {
      int k = 0;
      while (k < kSpEigT && s_cnt[grp][k] <= idx) ++k;
      s_lo[grp] = lo + w * (double)k / (double)(kSpEigT + 1);
      s_hi[grp] = lo + w * (double)(k + 1) / (double)(kSpEigT + 1);
    }
    __syncthreads();
  }
  const double th1 = 0.5 * (s_lo[0] + s_hi[0]);
  const double th2 = 0.5 * (s_lo[1] + s_hi[1]);
  // (4) top eigenvector: two steps of inverse iteration on T_m - sigma I,
  // sigma just above theta_1 (Thomas algorithm in double-float, tiny pivots
  // replaced, rescaled by a power of two after each step), then the FP64
  // norm by a block reduction
  if (tid == 0) {
    const double tn = s_tn;
    const df sig = df_from_double(th1 + 1e-13 * (tn + 1e-300));
    const float tiny = fmaxf(1e-30f, (float)(1e-15 * tn));
    for (int i = 0; i < m; ++i) {
      s_yh[i] = 1.f + 0.01f * (float)(i % 7);
      s_yl[i] = 0.f;
    }
    for (int it = 0; it < 2; ++it) {
      df cprev{0.f, 0.f}, yprev{0.f, 0.f}, bprev{0.f, 0.f};
      for (int i = 0; i < m; ++i) {
        df piv = df_sub(df{s_ah[i], s_al[i]}, sig);
        if (i > 0) piv = df_sub(piv, df_mul(bprev, cprev));
        if (fabsf(piv.hi) < tiny) piv = df{tiny, 0.f};
        const df rp = df_rcp(piv);
        const df bi{s_bh[i], s_bl[i]};
        cprev = df_mul(bi, rp);
        df yi{s_yh[i], s_yl[i]};
        if (i > 0) yi = df_sub(yi, df_mul(bprev, yprev));
        yprev = df_mul(yi, rp);
        s_ch[i] = cprev.hi;
        s_cl[i] = cprev.lo;
        s_yh[i] = yprev.hi;
        s_yl[i] = yprev.lo;
        bprev = bi;
      }
      df ynext{s_yh[m - 1], s_yl[m - 1]};
      float mx = fabsf(ynext.hi);
      for (int i = m - 2; i >= 0; --i) {
        ynext = df_sub(df{s_yh[i], s_yl[i]}, df_mul(df{s_ch[i], s_cl[i]}, ynext));
        s_yh[i] = ynext.hi;
        s_yl[i] = ynext.lo;
        mx = fmaxf(mx, fabsf(ynext.hi));
      }
      int ex = 0;
      frexpf(mx, &ex);
      const float sc = ldexpf(1.f, -ex);  // exact: the largest entry into [0.5, 1)
      for (int i = 0; i < m; ++i) {
        s_yh[i] *= sc;
        s_yl[i] *= sc;
      }
    }
  }
  __syncthreads();
  const double yv = (tid < m) ? (double)s_yh[tid] + (double)s_yl[tid] : 0.0;
  double nn = yv * yv;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, off);
  if (lane == 0) s_red[0][warp] = nn;
  __syncthreads();
  if (tid == 0) {
    double t2 = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) t2 += s_red[0][w];
    s_nn = t2;
  }
  __syncthreads();
  const double inv = 1.0 / sqrt(s_nn);
  if (tid < m) st->y[tid] = yv * inv;
  if (tid == m - 1) {
    const double r = fabs(st->beta[m - 1] * yv * inv);
    const double gap = th1 - th2;
    double bound = r;
    if (gap > 0.0) bound = fmin(r, r * r / gap);
    if (st->brk) bound = 0.0;
    st->out[0] = th1;
    st->out[1] = th2;
    st->out[2] = r;
    st->out[3] = bound;
    st->out[4] = (double)m;
    if (bound <= rtol * fabs(th1)) st->stop = 1;
  }
}

// Ritz vector u = V_m y into W[1] (the start of the next run), |u|^2 and
// u^T D u into out[5], out[6], start_norm = |u|
__device__ __forceinline__ void sp_ritz_body(const SpArgs& a, int b, int nb) {
  __shared__ double s_tmp[kPhaseBlock];
  __shared__ double s_out[2];
  __shared__ float s_y[2][kSpMax];
  SpState* st = a.st;
  const int m = min(max(st->m_eff, 0), kSpMax);
  for (int j = threadIdx.x; j < m; j += kPhaseBlock) {
    const df yy = df_from_double(st->y[j]);
    s_y[0][j] = yy.hi;
    s_y[1][j] = yy.lo;
  }
  __syncthreads();
  float nS = 0.f, nC = 0.f, dS = 0.f, dC = 0.f;
  float2* U = a.W[1];
  for (int64_t i = (int64_t)b * kPhaseBlock + threadIdx.x; i < a.g.n; i += (int64_t)nb * kPhaseBlock) {
    float s = 0.f, c = 0.f;
    for (int j = 0; j < m; ++j) df_acc2(s, c, df_mul(df{s_y[0][j], s_y[1][j]}, ld_df2(a.V + (size_t)j * a.g.n + i)));
    const df u = two_sum(s, c);
    st_df2(U + i, u);
    const df u2 = df_mul(u, u);
    df_acc2(nS, nC, u2);
    df_acc2(dS, dC, df_mul_f(u2, (float)(a.g.row_ptr[i + 1] - a.g.row_ptr[i])));
  }
  // two column sums through the K = 2 reduction (deterministic)
  double acc[2] = {(double)nS + (double)nC, (double)dS + (double)dC};
  if (!sp_partials_last<2>(acc, a.part, &st->ticket, b, nb)) return;
  sum_partials<2>(a.part, nb, s_tmp, s_out);
  if (threadIdx.x == 0) {
    st->out[5] = s_out[0];
    st->out[6] = s_out[1];
    st->start_norm = sqrt(s_out[0]);
    st->ticket = 0;
  }
}

// ---------------------------------------------------------------- one problem
__global__ void __launch_bounds__(kPhaseBlock) sp_init(SpArgs a) { sp_init_body(a, blockIdx.x, gridDim.x); }
__global__ void sp_restart(SpState* st, int resume) { sp_restart_body(st, resume); }
__global__ void __launch_bounds__(kPhaseBlock) sp_s(SpArgs a) { sp_s_body(a, a.j, blockIdx.x, gridDim.x); }
__global__ void __launch_bounds__(kPhaseBlock) sp_u(SpArgs a, int last) {
  sp_u_body(a, a.j, last, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(2 * kSpEigT) sp_eig(SpState* st, double rtol) { sp_eig_body(st, rtol); }
__global__ void __launch_bounds__(kPhaseBlock) sp_ritz(SpArgs a) { sp_ritz_body(a, blockIdx.x, gridDim.x); }

// ---------------------------------------------------------------- many problems
// The grid of a batched row kernel is the concatenation of the problems'
// shares: problem p owns CTAs off[p] .. off[p + 1] - 1 (off[np] = grid).
// Each CTA copies its problem's arguments into registers first: read in
// place, every field would be reloaded after each store (the stores could
// alias the job array).
__device__ __forceinline__ int sp_job_of(const int* __restrict__ off, int np, int b) {
  int lo = 0, hi = np;  // the p with off[p] <= b < off[p + 1]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(off + mid) <= b) lo = mid; else hi = mid;
  }
  return lo;
}

// Ritz vectors of the jobs that ask for one (CTAs by the gu offsets)
__global__ void __launch_bounds__(kPhaseBlock) sp_ritz_multi(const SpJob* __restrict__ jobs,
                                                             const int* __restrict__ off_u, int np) {
  const int p = sp_job_of(off_u, np, blockIdx.x);
  if (!jobs[p].ritz) return;
  const SpArgs a = jobs[p].a;
  sp_ritz_body(a, blockIdx.x - off_u[p], off_u[p + 1] - off_u[p]);
}

// Start of each job's run: one CTA per job. Mode 0 clears the whole state
// (tickets and flags start at zero, as the fresh run's init kernel needs).
__global__ void sp_prep_multi(const SpJob* __restrict__ jobs, int np) {
  const int p = blockIdx.x;
  if (p >= np) return;
  const SpJob& jb = jobs[p];
  if (jb.mode == 0) {
    uint32_t* w = (uint32_t*)jb.a.st;
    for (int i = threadIdx.x; i < (int)(sizeof(SpState) / 4); i += blockDim.x) w[i] = 0u;
  } else if (jb.mode == 1 || jb.mode == 2) {
    sp_restart_body(jb.a.st, jb.mode == 2 ? 1 : 0);
  }
}

__global__ void __launch_bounds__(kPhaseBlock) sp_init_multi(const SpJob* __restrict__ jobs,
                                                             const int* __restrict__ off_u, int np) {
  const int p = sp_job_of(off_u, np, blockIdx.x);
  if (jobs[p].mode != 0) return;
  const SpArgs a = jobs[p].a;
  sp_init_body(a, blockIdx.x - off_u[p], off_u[p + 1] - off_u[p]);
}

// step j0 + s of every job that has it
__global__ void __launch_bounds__(kPhaseBlock) sp_s_multi(const SpJob* __restrict__ jobs,
                                                          const int* __restrict__ off_s, int np, int s) {
  const int p = sp_job_of(off_s, np, blockIdx.x);
  const int j = jobs[p].j0 + s;
  if (jobs[p].mode < 0 || j >= jobs[p].j1) return;
  const SpArgs a = jobs[p].a;
  sp_s_body(a, j, blockIdx.x - off_s[p], off_s[p + 1] - off_s[p]);
}

__global__ void __launch_bounds__(kPhaseBlock) sp_u_multi(const SpJob* __restrict__ jobs,
                                                          const int* __restrict__ off_u, int np, int s) {
  const int p = sp_job_of(off_u, np, blockIdx.x);
  const int j = jobs[p].j0 + s;
  if (jobs[p].mode < 0 || j >= jobs[p].j1) return;
  const int last = (j == jobs[p].cap - 1) ? 1 : 0;
  const SpArgs a = jobs[p].a;
  sp_u_body(a, j, last, blockIdx.x - off_u[p], off_u[p + 1] - off_u[p]);
}

// the eigen step after step j0 + s of the jobs whose check falls there (every
// `check` steps and at the round's last step), one CTA per job
__global__ void __launch_bounds__(2 * kSpEigT) sp_eig_multi(const SpJob* __restrict__ jobs, int np, int s,
                                                            int check) {
  const int p = blockIdx.x;
  if (p >= np) return;
  const SpJob& jb = jobs[p];
  const int j = jb.j0 + s;
  if (jb.mode < 0 || j >= jb.j1) return;
  if ((j + 1) % check != 0 && j + 1 != jb.j1) return;
  sp_eig_body(jb.a.st, jb.rtol);
}

// the host's copy of every job's state
__global__ void sp_pack_multi(const SpJob* __restrict__ jobs, int np, SpOut* __restrict__ out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const SpState* st = jobs[p].a.st;
  SpOut o;
  o.start_norm = st->start_norm;
  for (int i = 0; i < 8; ++i) o.out[i] = st->out[i];
  o.m_eff = st->m_eff;
  o.stop = st->stop;
  o.brk = st->brk;
  o.pad = 0;
  out[p] = o;
}
#endif  // WL_SPEC_KERNELS

}  // namespace wl
