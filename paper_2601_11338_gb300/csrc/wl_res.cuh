// Residual of the iterative refinement (refined form, Sec. 4.2 solves) in
// double-float arithmetic: FP64-accurate, FP32 instructions only.
//
// The refined solve of M x = b keeps b, the residual r and the iterate x as
// double-float vectors (two FP32 arrays each) and corrects x with FP32 CG
// solves M d = fl32(r). The residual is updated, not recomputed:
//     r <- r - M d ,  x <- x + d
// which equals b - M x up to the double-float rounding of each step (about
// 2^-46 of |r| + |M d|), so the gathered operand is the 4-byte correction d
// instead of an 8-byte iterate. Only a warm start needs the full form
//     r = b - M x   (x = xh + xl gathered as two FP32 terms).
// M = ca I + cA A + cD D; the neighbour sum A y is accumulated with the
// error-free two-sum, M y and the subtraction in double-float.
//
// Each kernel ends in the deterministic last-CTA reduction of |r|^2 per
// column (from the FP32 leading terms: the convergence test needs a few
// digits of the norm, not all of them) into st->gamma.
#pragma once
#include "wl_cg2.cuh"
#include "wl_df.cuh"

namespace wl {

struct DfResArgs {
  PhaseGraph g;
  const float* yh;  // gathered operand: the correction d, or (FULL) the iterate's leading term
  const float* yl;  // FULL: the iterate's trailing term
  const float* bh;  // r_in: the previous residual, or (FULL) the right-hand side b
  const float* bl;
  float* rh;        // r_out (may alias r_in)
  float* rl;
  float* r32;       // copy of rh: right-hand side of the next FP32 inner solve (or NULL)
  float* xh;        // iterate, updated x += d in place (not FULL)
  float* xl;
  float* dnext;     // zeroed here (start of the next inner solve), or NULL
  df ca, cA, cD;
  double* part;     // gridDim.x * K partials
  CgState* st;      // st->gamma[c] = |r_out[:, c]|^2
  int x_zero;       // the iterate is zero on entry: x = d
  // optional per-row diagonal added to M as a double-float pair (shifted
  // solves); NULL: none. bh == NULL (FULL only): b = 0, r_out = -M x
  const float* dsh_h = nullptr;
  const float* dsh_l = nullptr;
};

// (s, c, l): neighbour sum of the leading terms with its rounding errors,
// and the plain sum of the trailing terms (FULL only)
template <int K, int VW, bool FULL>
__device__ __forceinline__ void df_row_gather(const int32_t* __restrict__ col, int beg, int end, int step,
                                              const float* YH, const float* YL, int lane_off, float (&s)[VW],
                                              float (&c)[VW], float (&l)[VW]) {
#if WL_GATHER_PRED
  constexpr int U = WL_GATHER_U;  // predicated batches, as in row_gather
  for (int e = beg; e < end; e += U * step) {
    int j[U];
#pragma unroll
    for (int u = 0; u < U; ++u) j[u] = (e + u * step < end) ? __ldg(col + e + u * step) : -1;
    Pack<float, VW> hh[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (j[u] >= 0) {
        hh[u] = ld_plain<float, VW>(YH + (size_t)j[u] * K + lane_off);
      } else {
#pragma unroll
        for (int v = 0; v < VW; ++v) hh[u].v[v] = 0.f;
      }
    }
    if constexpr (FULL) {
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (j[u] >= 0) {
          const Pack<float, VW> l0 = ld_plain<float, VW>(YL + (size_t)j[u] * K + lane_off);
#pragma unroll
          for (int v = 0; v < VW; ++v) l[v] += l0.v[v];
        }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int v = 0; v < VW; ++v) df_acc(s[v], c[v], hh[u].v[v]);
  }
  return;
#endif
  int e = beg;
  for (; e + 3 * step < end; e += 4 * step) {
    const int j0 = __ldg(col + e), j1 = __ldg(col + e + step);
    const int j2 = __ldg(col + e + 2 * step), j3 = __ldg(col + e + 3 * step);
    const Pack<float, VW> h0 = ld_plain<float, VW>(YH + (size_t)j0 * K + lane_off);
    const Pack<float, VW> h1 = ld_plain<float, VW>(YH + (size_t)j1 * K + lane_off);
    const Pack<float, VW> h2 = ld_plain<float, VW>(YH + (size_t)j2 * K + lane_off);
    const Pack<float, VW> h3 = ld_plain<float, VW>(YH + (size_t)j3 * K + lane_off);
    if constexpr (FULL) {
      const Pack<float, VW> l0 = ld_plain<float, VW>(YL + (size_t)j0 * K + lane_off);
      const Pack<float, VW> l1 = ld_plain<float, VW>(YL + (size_t)j1 * K + lane_off);
      const Pack<float, VW> l2 = ld_plain<float, VW>(YL + (size_t)j2 * K + lane_off);
      const Pack<float, VW> l3 = ld_plain<float, VW>(YL + (size_t)j3 * K + lane_off);
#pragma unroll
      for (int v = 0; v < VW; ++v) l[v] += (l0.v[v] + l1.v[v]) + (l2.v[v] + l3.v[v]);
    }
#pragma unroll
    for (int v = 0; v < VW; ++v) {
      df_acc(s[v], c[v], h0.v[v]);
      df_acc(s[v], c[v], h1.v[v]);
      df_acc(s[v], c[v], h2.v[v]);
      df_acc(s[v], c[v], h3.v[v]);
    }
  }
  for (; e < end; e += step) {
    const int j0 = __ldg(col + e);
    const Pack<float, VW> h0 = ld_plain<float, VW>(YH + (size_t)j0 * K + lane_off);
    if constexpr (FULL) {
      const Pack<float, VW> l0 = ld_plain<float, VW>(YL + (size_t)j0 * K + lane_off);
#pragma unroll
      for (int v = 0; v < VW; ++v) l[v] += l0.v[v];
    }
#pragma unroll
    for (int v = 0; v < VW; ++v) df_acc(s[v], c[v], h0.v[v]);
  }
}

// SH: the solve's M carries the per-row diagonal (dsh_h, dsh_l); a separate
// instance, so that the unshifted kernel carries no trace of it
template <int K, bool FULL, bool SH = false>
__global__ void __launch_bounds__(kPhaseBlock, 4) df_res(DfResArgs a) {
  using C = Cfg<float, K>;
  constexpr int VW = C::VW, G = C::G, RPB = kPhaseBlock / G;
  __shared__ __align__(16) float s_red[3][kPhaseBlock * VW];
  __shared__ double s_tmp[kPhaseBlock];
  __shared__ double s_out[K];
  const int tid = threadIdx.x, sl = tid % G, lane_off = sl * VW;
  float nacc[VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) nacc[v] = 0.f;

  auto fin = [&](int64_t row, int deg, const float (&s)[VW], const float (&c)[VW], const float (&l)[VW]) {
    const size_t o = (size_t)row * K + lane_off;
    df crow = df_add(a.ca, df_mul_f(a.cD, (float)deg));
    if constexpr (SH) crow = df_add(crow, df{a.dsh_h[row], a.dsh_l[row]});
    const Pack<float, VW> yh = ld_plain<float, VW>(a.yh + o);
    Pack<float, VW> yl;
    if constexpr (FULL) yl = ld_plain<float, VW>(a.yl + o);
    Pack<float, VW> bh, bl;
    if (!FULL || a.bh) {
      bh = ld_plain<float, VW>(a.bh + o);
      bl = ld_plain<float, VW>(a.bl + o);
    } else {
#pragma unroll
      for (int v = 0; v < VW; ++v) bh.v[v] = bl.v[v] = 0.f;
    }
    Pack<float, VW> xh, xl;
    if constexpr (!FULL) {
      if (!a.x_zero) {
        xh = ld_plain<float, VW>(a.xh + o);
        xl = ld_plain<float, VW>(a.xl + o);
      }
    }
    Pack<float, VW> rh, rl;
#pragma unroll
    for (int v = 0; v < VW; ++v) {
      const df nb = two_sum(s[v], c[v] + l[v]);
      const df y{yh.v[v], FULL ? yl.v[v] : 0.f};
      const df My = df_add(df_mul(crow, y), df_mul(a.cA, nb));
      const df r = df_sub(df{bh.v[v], bl.v[v]}, My);
      rh.v[v] = r.hi;
      rl.v[v] = r.lo;
      nacc[v] = __fmaf_rn(r.hi, r.hi, nacc[v]);
      if constexpr (!FULL) {
        if (a.x_zero) {
          xh.v[v] = yh.v[v];
          xl.v[v] = 0.f;
        } else {
          const df t = two_sum(xh.v[v], yh.v[v]);
          const df u = quick_two_sum(t.hi, t.lo + xl.v[v]);
          xh.v[v] = u.hi;
          xl.v[v] = u.lo;
        }
      }
    }
    stp<float, VW>(a.rh + o, rh);
    stp<float, VW>(a.rl + o, rl);
    if (a.r32) stp<float, VW>(a.r32 + o, rh);
    if constexpr (!FULL) {
      stp<float, VW>(a.xh + o, xh);
      stp<float, VW>(a.xl + o, xl);
      if (a.dnext) {
        Pack<float, VW> z;
#pragma unroll
        for (int v = 0; v < VW; ++v) z.v[v] = 0.f;
        stp<float, VW>(a.dnext + o, z);
      }
    }
  };

  if ((int)blockIdx.x < a.g.nhub) {
    // one hub row per CTA: RPB lane groups stride over the entries
    const int64_t row = a.g.hubs[blockIdx.x];
    const int beg = a.g.row_ptr[row], end = a.g.row_ptr[row + 1];
    float s[VW], c[VW], l[VW];
#pragma unroll
    for (int v = 0; v < VW; ++v) s[v] = c[v] = l[v] = 0.f;
    df_row_gather<K, VW, FULL>(a.g.col, beg + tid / G, end, RPB, a.yh, a.yl, lane_off, s, c, l);
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
          const int k = (gr * G + sl) * VW + v;
          const df t = two_sum(s[v], s_red[0][k]);
          s[v] = t.hi;
          c[v] += t.lo + s_red[1][k];
          l[v] += s_red[2][k];
        }
      fin(row, end - beg, s, c, l);
    }
  } else if ((int)blockIdx.x < a.g.nhub + a.g.nmid_blk) {
    // mid rows, one warp each (as in the CG S kernel)
    const int lane = tid & 31;
    constexpr int WPB = kPhaseBlock / 32;
    for (int r = ((int)blockIdx.x - a.g.nhub) * WPB + (tid >> 5); r < a.g.nmid; r += a.g.nmid_blk * WPB) {
      const int64_t row = a.g.mids[r];
      const int beg = a.g.row_ptr[row], end = a.g.row_ptr[row + 1];
      float s[VW], c[VW], l[VW];
#pragma unroll
      for (int v = 0; v < VW; ++v) s[v] = c[v] = l[v] = 0.f;
      df_row_gather<K, VW, FULL>(a.g.col, beg + lane / G, end, 32 / G, a.yh, a.yl, lane_off, s, c, l);
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
    const int lim = a.g.nmid_blk > 0 ? kMidDeg : kHubDeg;  // longer rows: hub CTAs or mid warps
    const int64_t nblk = (int64_t)gridDim.x - nlist;
    for (int64_t row = ((int64_t)blockIdx.x - nlist) * RPB + tid / G; row < a.g.n; row += nblk * RPB) {
      const int beg = a.g.row_ptr[row], end = a.g.row_ptr[row + 1];
      if (end - beg > lim) continue;
      float s[VW], c[VW], l[VW];
#pragma unroll
      for (int v = 0; v < VW; ++v) s[v] = c[v] = l[v] = 0.f;
      df_row_gather<K, VW, FULL>(a.g.col, beg, end, 1, a.yh, a.yl, lane_off, s, c, l);
      fin(row, end - beg, s, c, l);
    }
  }
  double dd[VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) dd[v] = (double)nacc[v];
  if (!block_partials_last<float, K>(dd, a.part, &a.st->ticket)) return;
  sum_partials<K>(a.part, gridDim.x, s_tmp, s_out);
  if (tid < K) a.st->gamma[tid] = s_out[tid];
  if (tid == 0) a.st->ticket = 0;
}

// b (n x K FP64, contiguous) * scale -> (bh, bl), r32 = bh, |b|^2 per column
// (from bh) -> b2[c]; the conversion is the one FP64 pass of a refined solve.
template <int K>
__global__ void __launch_bounds__(kPhaseBlock) df_from_f64(const double* b, double scale, int64_t n, float* bh,
                                                           float* bl, float* r32, double* part, CgState* st,
                                                           double* b2) {
  using C = Cfg<float, K>;
  constexpr int VW = C::VW;
  __shared__ double s_tmp[kPhaseBlock];
  __shared__ double s_out[K];
  const int tid = threadIdx.x;
  float acc[VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) acc[v] = 0.f;
  const size_t nv = (size_t)n * K / VW;
  for (size_t e = (size_t)blockIdx.x * kPhaseBlock + tid; e < nv; e += (size_t)gridDim.x * kPhaseBlock) {
    Pack<float, VW> hh, ll;
#pragma unroll
    for (int v = 0; v < VW; ++v) {
      const double x = b[e * VW + v] * scale;
      const float h = (float)x;
      hh.v[v] = h;
      ll.v[v] = (float)(x - (double)h);
      acc[v] = __fmaf_rn(h, h, acc[v]);
    }
    stp<float, VW>(bh + e * VW, hh);
    stp<float, VW>(bl + e * VW, ll);
    if (r32) stp<float, VW>(r32 + e * VW, hh);
  }
  double dd[VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) dd[v] = (double)acc[v];
  if (!block_partials_last<float, K>(dd, part, &st->ticket)) return;
  sum_partials<K>(part, gridDim.x, s_tmp, s_out);
  if (tid < K) b2[tid] = s_out[tid];
  if (tid == 0) st->ticket = 0;
}

}  // namespace wl
