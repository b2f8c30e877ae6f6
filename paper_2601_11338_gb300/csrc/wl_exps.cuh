// The exponential walk function phi(A) V = sum_k c_k q_k V with c_k =
// beta^k / k! (Def. BDTW-Laplacian, Sec. 3.2.1) summed term by term: the
// walk counts of Eq. qrec act on the block V through
//   w_0 = V, w_1 = A w_0, w_2 = A w_1 - mu D w_0,
//   w_{k+1} = A w_k + mu (mu I - D) w_{k-1}   (k >= 2),
// one gather per term, and acc = sum_k c_k w_k. The kernels carry the terms
// s_k = c_k w_k themselves, not the counts: w_k grows like rho(Z_mu)^k and
// leaves the FP32 exponent range after about 17 terms when rho is near 160,
// while the terms of the convergent series stay bounded. With c_{k+1} / c_k =
// beta / (k+1) and c_{k+1} / c_{k-1} = beta^2 / (k (k+1)) the recurrence reads
//   s_{k+1} = (beta / (k+1)) A s_k + (beta^2 / (k (k+1))) mu (mu I - D) s_{k-1}
// (k = 1: the diagonal factor is -mu D), and acc = sum_k s_k. Every vector is
// a double-float pair (FP32 instructions only; GB300 runs FP64 at 1/64 of the
// FP32 rate).
//
// The last CTA of each term reduces |s_{k+1}|^2 and |acc|^2 per
// column; a column is finished after kExpQuiet consecutive terms below
// kExpRel |acc|, and the kernel of a finished series returns at once (the
// host launches terms in chunks and reads one flag between chunks).
#pragma once
#include "wl_cg2.cuh"
#include "wl_df.cuh"

namespace wl {

constexpr double kExpRel = 1e-17;  // a term this small (relative) adds nothing in double-float
constexpr int kExpQuiet = 3;       // consecutive small terms that end a column's series

struct ExpArgs {
  PhaseGraph g;
  const float* wh;  // s_k (gathered)
  const float* wl;
  const float* mh;  // s_{k-1} (own row; unused at k = 0)
  const float* ml;
  float* oh;        // s_{k+1} out
  float* ol;
  float* ah;        // acc += s_{k+1} (in place)
  float* al;
  df mu;
  df ak;            // beta / (k + 1): factor of A s_k
  df bk;            // beta^2 / (k (k + 1)) for k >= 1: factor of the diagonal term
  int k;
  int max_terms;
  double* part;     // 2 gridDim.x K partials
  CgState* st;      // done[c]: consecutive small terms; active; status
};

#ifdef WL_EXPS_KERNELS
template <int K, int VW>
__device__ __forceinline__ void exp_gather(const int32_t* __restrict__ col, int beg, int end, int step, const float* WH,
                                           const float* WL, int lane_off, float (&s)[VW], float (&c)[VW],
                                           float (&l)[VW]) {
  int e = beg;
  for (; e + step < end; e += 2 * step) {
    const int j0 = __ldg(col + e), j1 = __ldg(col + e + step);
    const Pack<float, VW> h0 = ld_plain<float, VW>(WH + (size_t)j0 * K + lane_off);
    const Pack<float, VW> h1 = ld_plain<float, VW>(WH + (size_t)j1 * K + lane_off);
    const Pack<float, VW> l0 = ld_plain<float, VW>(WL + (size_t)j0 * K + lane_off);
    const Pack<float, VW> l1 = ld_plain<float, VW>(WL + (size_t)j1 * K + lane_off);
#pragma unroll
    for (int v = 0; v < VW; ++v) {
      df_acc(s[v], c[v], h0.v[v]);
      df_acc(s[v], c[v], h1.v[v]);
      l[v] += l0.v[v] + l1.v[v];
    }
  }
  for (; e < end; e += step) {
    const int j0 = __ldg(col + e);
    const Pack<float, VW> h0 = ld_plain<float, VW>(WH + (size_t)j0 * K + lane_off);
    const Pack<float, VW> l0 = ld_plain<float, VW>(WL + (size_t)j0 * K + lane_off);
#pragma unroll
    for (int v = 0; v < VW; ++v) {
      df_acc(s[v], c[v], h0.v[v]);
      l[v] += l0.v[v];
    }
  }
}

template <int K>
__global__ void __launch_bounds__(kPhaseBlock, 4) exp_term(ExpArgs a) {
  using C = Cfg<float, K>;
  constexpr int VW = C::VW, G = C::G, RPB = kPhaseBlock / G;
  __shared__ __align__(16) float s_red[3][kPhaseBlock * VW];
  __shared__ double s_tmp[kPhaseBlock];
  __shared__ double s_out[2 * K];
  CgState* st = a.st;
  if (!*(volatile int*)&st->active) return;
  const int tid = threadIdx.x, sl = tid % G, lane_off = sl * VW;
  float tn[VW], an[VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) tn[v] = an[v] = 0.f;
  auto fin = [&](int64_t row, int deg, const float (&s)[VW], const float (&c)[VW], const float (&l)[VW]) {
    const size_t o = (size_t)row * K + lane_off;
    // diagonal coefficient of s_{k-1}: none at k = 0, bk (-mu d) at k = 1, bk mu (mu - d) after
    df corr{0.f, 0.f};
    if (a.k == 1) corr = df_mul(a.bk, df_mul_f(a.mu, -(float)deg));
    else if (a.k >= 2) corr = df_mul(a.bk, df_mul(a.mu, df_add_f(a.mu, -(float)deg)));
    Pack<float, VW> mh, ml;
    if (a.k >= 1) {
      mh = ld_plain<float, VW>(a.mh + o);
      ml = ld_plain<float, VW>(a.ml + o);
    }
    Pack<float, VW> ah = ld_plain<float, VW>(a.ah + o), al = ld_plain<float, VW>(a.al + o);
    Pack<float, VW> oh, ol;
#pragma unroll
    for (int v = 0; v < VW; ++v) {
      df w = df_mul(a.ak, two_sum(s[v], c[v] + l[v]));
      if (a.k >= 1) w = df_add(w, df_mul(corr, df{mh.v[v], ml.v[v]}));
      oh.v[v] = w.hi;
      ol.v[v] = w.lo;
      const df t = w;
      const df acc = df_add(df{ah.v[v], al.v[v]}, t);
      ah.v[v] = acc.hi;
      al.v[v] = acc.lo;
      tn[v] = __fmaf_rn(t.hi, t.hi, tn[v]);
      an[v] = __fmaf_rn(acc.hi, acc.hi, an[v]);
    }
    stp<float, VW>(a.oh + o, oh);
    stp<float, VW>(a.ol + o, ol);
    stp<float, VW>(a.ah + o, ah);
    stp<float, VW>(a.al + o, al);
  };
  if ((int)blockIdx.x < a.g.nhub) {
    const int64_t row = a.g.hubs[blockIdx.x];
    const int beg = a.g.row_ptr[row], end = a.g.row_ptr[row + 1];
    float s[VW], c[VW], l[VW];
#pragma unroll
    for (int v = 0; v < VW; ++v) s[v] = c[v] = l[v] = 0.f;
    exp_gather<K, VW>(a.g.col, beg + tid / G, end, RPB, a.wh, a.wl, lane_off, s, c, l);
#pragma unroll
    for (int v = 0; v < VW; ++v) {
      s_red[0][tid * VW + v] = s[v];
      s_red[1][tid * VW + v] = c[v];
      s_red[2][tid * VW + v] = l[v];
    }
    __syncthreads();
    if (tid < G) {
      for (int gr = 1; gr < RPB; ++gr)
#pragma unroll
        for (int v = 0; v < VW; ++v) {
          const int q = (gr * G + sl) * VW + v;
          const df t = two_sum(s[v], s_red[0][q]);
          s[v] = t.hi;
          c[v] += t.lo + s_red[1][q];
          l[v] += s_red[2][q];
        }
      fin(row, end - beg, s, c, l);
    }
  } else if ((int)blockIdx.x < a.g.nhub + a.g.nmid_blk) {
    const int lane = tid & 31;
    constexpr int WPB = kPhaseBlock / 32;
    for (int r = ((int)blockIdx.x - a.g.nhub) * WPB + (tid >> 5); r < a.g.nmid; r += a.g.nmid_blk * WPB) {
      const int64_t row = a.g.mids[r];
      const int beg = a.g.row_ptr[row], end = a.g.row_ptr[row + 1];
      float s[VW], c[VW], l[VW];
#pragma unroll
      for (int v = 0; v < VW; ++v) s[v] = c[v] = l[v] = 0.f;
      exp_gather<K, VW>(a.g.col, beg + lane / G, end, 32 / G, a.wh, a.wl, lane_off, s, c, l);
#pragma unroll
      for (int off = G; off < 32; off <<= 1)
#pragma unroll
        for (int v = 0; v < VW; ++v) {
          const float so = __shfl_xor_sync(0xffffffffu, s[v], off);
          const float co = __shfl_xor_sync(0xffffffffu, c[v], off);
          const float lo = __shfl_xor_sync(0xffffffffu, l[v], off);
          const df t = two_sum(s[v], so);
          s[v] = t.hi;
          c[v] += t.lo + co;
          l[v] += lo;
        }
      if (lane < G) fin(row, end - beg, s, c, l);
    }
  } else {
    const int nlist = a.g.nhub + a.g.nmid_blk;
    const int lim = a.g.nmid_blk > 0 ? kMidDeg : kHubDeg;
    const int64_t nblk = (int64_t)gridDim.x - nlist;
    for (int64_t row = ((int64_t)blockIdx.x - nlist) * RPB + tid / G; row < a.g.n; row += nblk * RPB) {
      const int beg = a.g.row_ptr[row], end = a.g.row_ptr[row + 1];
      if (end - beg > lim) continue;
      float s[VW], c[VW], l[VW];
#pragma unroll
      for (int v = 0; v < VW; ++v) s[v] = c[v] = l[v] = 0.f;
      exp_gather<K, VW>(a.g.col, beg, end, 1, a.wh, a.wl, lane_off, s, c, l);
      fin(row, end - beg, s, c, l);
    }
  }
  // |term|^2 in part[0 .. G K), |acc|^2 in part[G K .. 2 G K)
  double* part_a = a.part + (size_t)gridDim.x * K;
  {
    constexpr int NW = kPhaseBlock / 32;
    __shared__ double s_w[2 * NW * K];
    const int lane = tid & 31, warp = tid >> 5;
    double tp[VW], ap[VW];
#pragma unroll
    for (int v = 0; v < VW; ++v) {
      tp[v] = (double)tn[v];
      ap[v] = (double)an[v];
    }
#pragma unroll
    for (int off = G; off < 32; off <<= 1)
#pragma unroll
      for (int v = 0; v < VW; ++v) {
        tp[v] += __shfl_xor_sync(0xffffffffu, tp[v], off);
        ap[v] += __shfl_xor_sync(0xffffffffu, ap[v], off);
      }
    if (lane < G)
#pragma unroll
      for (int v = 0; v < VW; ++v) {
        s_w[warp * K + lane * VW + v] = tp[v];
        s_w[NW * K + warp * K + lane * VW + v] = ap[v];
      }
    __syncthreads();
    if (tid < K) {
      double t = 0.0, u = 0.0;
      for (int w = 0; w < NW; ++w) {
        t += s_w[w * K + tid];
        u += s_w[NW * K + w * K + tid];
      }
      a.part[(size_t)blockIdx.x * K + tid] = t;
      part_a[(size_t)blockIdx.x * K + tid] = u;
      __threadfence();
    }
    __syncthreads();
  }
  __shared__ int s_last;
  if (tid == 0) s_last = (atomicAdd(&st->ticket, 1u) == gridDim.x - 1) ? 1 : 0;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  sum_partials<K>(a.part, gridDim.x, s_tmp, s_out);
  sum_partials<K>(part_a, gridDim.x, s_tmp, s_out + K);
  if (tid < K) {
    const double t2 = s_out[tid], a2 = s_out[K + tid];
    if (!isfinite(t2) || !isfinite(a2)) {
      st->status[tid] = WL_ERR_NONFINITE;
      st->done[tid] = kExpQuiet;
    } else if (t2 <= kExpRel * kExpRel * a2) {
      st->done[tid] += 1;
    } else {
      st->done[tid] = 0;
    }
  }
  __syncthreads();
  if (tid == 0) {
    int any = 0;
    for (int c = 0; c < K; ++c) any |= (st->done[c] < kExpQuiet);
    st->iters = a.k + 1;
    st->active = (any && a.k + 1 < a.max_terms) ? 1 : 0;
    st->ticket = 0;
  }
}
#endif  // WL_EXPS_KERNELS

}  // namespace wl
