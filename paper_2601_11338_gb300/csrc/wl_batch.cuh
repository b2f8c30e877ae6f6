// Batched walk-Laplacian solves: many graphs x many mu values in one set of
// launches (Sec. 4.2 applied to a collection of networks; the mu sweep of
// the backtrack-downweighted walks, Def. BDTW-Laplacian with theta = 1 - mu).
//
// Layout. The graphs are concatenated into one block-diagonal CSR. Its rows
// are cut into tiles that never cross a graph boundary; a row with more
// than kHubDeg entries gets a tile (and a CTA) of its own. Every vector is
// [slab][row][K] with one slab per mu value, so a launch covers all
// (mu, graph) problems: blockIdx.y is the slab, blockIdx.x the tile.
//
// Each problem (slab s, graph g) runs its own lockstep CG on
//   M_{s,g} = ca I + cA A + cD D  (per-problem coefficients)
// for K columns. Tiles write per-column partial sums; one CTA per problem
// then adds its tiles' partials in a fixed order (deterministic) and
// updates that problem's scalars. One iteration is
//   S: q = M r + beta q, p = r + beta p, delta partials
//   RS: alpha = gamma / delta
//   U: x += alpha p, r -= alpha q, gamma' partials
//   RU: beta = gamma' / gamma, convergence, problem and global activity
// A problem that has converged is skipped by every later launch.
#pragma once
#include "wl_cg2.cuh"
#include "wl_res.cuh"

namespace wl {

struct BTile {
  int32_t row_beg, row_end;  // global rows [row_beg, row_end)
  int32_t graph;             // graph index
  int32_t hub;               // 1: a single row with more than kHubDeg entries
};

struct BatchGraph {
  const int32_t* row_ptr;   // concatenated CSR (global rows and columns)
  const int32_t* col;
  const BTile* tiles;
  const int32_t* tile_beg;  // ngraph + 1: tiles of graph g are [tile_beg[g], tile_beg[g+1])
  const int32_t* goff;      // ngraph + 1: rows of graph g are [goff[g], goff[g+1])
  int ntile;
  int ngraph;
  int64_t n;                // total rows
};

// per-problem scalars; index (s * ngraph + g) * K + c for columns,
// s * ngraph + g for problems
struct BatchState {
  double* gamma;
  double* alpha;
  double* beta;
  double* b2;
  int* done;
  int* status;
  int* active;   // per problem
  int* iters;    // per problem: iterations of the current solve
  int* total;    // per problem: iterations summed over the refinement steps
  int* any;      // one flag: some problem still iterates
};

template <typename T>
struct BatchArgs {
  BatchGraph g;
  T* x;
  T* r;
  T* p;
  T* q;
  const double* ca;     // per problem
  const double* cA;
  const double* cD;
  const T* b;           // [n][K] right-hand side shared by all slabs, or NULL (then r holds it)
  const double* bscale; // per problem multiplier of b, or NULL
  const double* bnorm2; // per problem-column reference ||b||^2 for the tolerance, or NULL (||r_0||^2)
  const int* skip;      // per problem-column: 1 = do not iterate, or NULL
  double* part;         // [nslab][ntile][K]
  BatchState st;
  int max_iter;
  double tol2;
};

#ifdef WL_BATCH_KERNELS

// CTA column sums of per-thread values (thread t owns columns (t % G) VW + v),
// stored to out[0 .. K)
template <typename T, int K>
__device__ __forceinline__ void block_colsum_store(const double (&val)[Cfg<T, K>::VW], double* out) {
  using C = Cfg<T, K>;
  constexpr int VW = C::VW, G = C::G, NW = kPhaseBlock / 32;
  __shared__ double s_w[NW * K];
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
    out[tid] = t;
  }
}

// Sum over the tiles of one problem, fixed order: out[c] in shared memory
template <int K>
__device__ __forceinline__ void problem_sum(const double* part, int tb, int te, double* s_tmp, double* out) {
  constexpr int J = kPhaseBlock / K;
  const int tid = threadIdx.x, c = tid % K, j = tid / K;
  double s = 0.0;
  for (int t = tb + j; t < te; t += J) s += __ldcg(part + (size_t)t * K + c);
  s_tmp[tid] = s;
  __syncthreads();
  if (tid < K) {
    double u = 0.0;
    for (int jj = 0; jj < J; ++jj) u += s_tmp[jj * K + tid];
    out[tid] = u;
  }
  __syncthreads();
}

// rows of a tile that this kernel updates elementwise: a hub tile its one
// row, a plain tile its rows except hubs (those have their own tile)
__device__ __forceinline__ bool plain_row(const int32_t* row_ptr, int64_t row) {
  return row_ptr[row + 1] - row_ptr[row] <= kHubDeg;
}

// ---------------------------------------------------------------- init
// x = 0, r = bscale * b (or r as given), gamma_0 partials
template <typename T, int K>
__global__ void __launch_bounds__(kPhaseBlock) bcg_init(BatchArgs<T> a, const int* pmask) {
  using C = Cfg<T, K>;
  constexpr int VW = C::VW, G = C::G, RPB = kPhaseBlock / G;
  const BTile tl = a.g.tiles[blockIdx.x];
  const int s = blockIdx.y, pr = s * a.g.ngraph + tl.graph;
  if (pmask && !pmask[pr]) {  // problem not refining any more: zero partials only
    double z[Cfg<T, K>::VW];
#pragma unroll
    for (int v = 0; v < Cfg<T, K>::VW; ++v) z[v] = 0.0;
    block_colsum_store<T, K>(z, a.part + ((size_t)s * a.g.ntile + blockIdx.x) * K);
    return;
  }
  const int tid = threadIdx.x, lane_off = (tid % G) * VW;
  const size_t slab = (size_t)s * a.g.n * K;
  const T sc = a.bscale ? (T)a.bscale[pr] : T(1);
  double acc[VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) acc[v] = 0.0;
  for (int64_t row = tl.row_beg + tid / G; row < tl.row_end; row += RPB) {
    if (!tl.hub && !plain_row(a.g.row_ptr, row)) continue;
    const size_t o = slab + (size_t)row * K + lane_off;
    Pack<T, VW> rr;
    if (a.b) {
      const Pack<T, VW> bb = ld_plain<T, VW>(a.b + (size_t)row * K + lane_off);
#pragma unroll
      for (int v = 0; v < VW; ++v) rr.v[v] = sc * bb.v[v];
      stp<T, VW>(a.r + o, rr);
    } else {
      rr = ld_plain<T, VW>(a.r + o);
    }
    Pack<T, VW> z;
#pragma unroll
    for (int v = 0; v < VW; ++v) {
      z.v[v] = T(0);
      acc[v] += (double)rr.v[v] * (double)rr.v[v];
    }
    stp<T, VW>(a.x + o, z);
  }
  block_colsum_store<T, K>(acc, a.part + ((size_t)s * a.g.ntile + blockIdx.x) * K);
}

// gamma_0, reference norms, flags; grid (ngraph, nslab)
template <int K>
__global__ void __launch_bounds__(kPhaseBlock) bred_init(BatchGraph g, BatchState st, const double* part,
                                                          const double* bnorm2, const int* skip, const int* pmask,
                                                          double tol2) {
  __shared__ double s_tmp[kPhaseBlock];
  __shared__ double s_out[K];
  const int s = blockIdx.y, pr = s * g.ngraph + blockIdx.x;
  problem_sum<K>(part + (size_t)s * g.ntile * K, g.tile_beg[blockIdx.x], g.tile_beg[blockIdx.x + 1], s_tmp, s_out);
  const int tid = threadIdx.x;
  __shared__ int s_any;
  if (tid == 0) s_any = 0;
  __syncthreads();
  if (tid < K) {
    const int i = pr * K + tid;
    const double gn = s_out[tid];
    const double b2 = bnorm2 ? bnorm2[i] : gn;
    st.gamma[i] = gn;
    st.b2[i] = b2;
    st.alpha[i] = 0.0;
    st.beta[i] = 0.0;
    st.status[i] = 0;
    int done = (b2 <= 0.0) || (gn <= tol2 * b2) || (skip && skip[i]) || (pmask && !pmask[pr]);
    if (!isfinite(gn)) {
      done = 1;
      st.status[i] = WL_ERR_NONFINITE;
    }
    st.done[i] = done;
    if (!done) atomicOr(&s_any, 1);
  }
  __syncthreads();
  if (tid == 0) {
    st.iters[pr] = 0;
    st.active[pr] = s_any;
    if (s_any) atomicOr(st.any, 1);
  }
}

// ---------------------------------------------------------------- S
template <typename T, int K>
__global__ void __launch_bounds__(kPhaseBlock, kPhaseMinBlocks) bcg_s(BatchArgs<T> a) {
  using C = Cfg<T, K>;
  constexpr int VW = C::VW, G = C::G, RPB = kPhaseBlock / G;
  __shared__ __align__(16) T s_red[kPhaseBlock * VW];
  const BTile tl = a.g.tiles[blockIdx.x];
  const int s = blockIdx.y, pr = s * a.g.ngraph + tl.graph;
  if (!a.st.active[pr]) return;
  const int tid = threadIdx.x, sl = tid % G, lane_off = sl * VW;
  const bool first = a.st.iters[pr] == 0;
  const T ca = (T)a.ca[pr], cA = (T)a.cA[pr], cD = (T)a.cD[pr];
  T be[VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) be[v] = first ? T(0) : (T)a.st.beta[pr * K + lane_off + v];
  const size_t slab = (size_t)s * a.g.n * K;
  const T* __restrict__ R = a.r + slab;
  T* __restrict__ P = a.p + slab;
  T* __restrict__ Q = a.q + slab;
  T dacc[VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) dacc[v] = T(0);
  auto fin = [&](int64_t row, int deg, const T (&nb)[VW]) {
    const size_t o = (size_t)row * K + lane_off;
    const Pack<T, VW> rr = ld_plain<T, VW>(R + o);
    Pack<T, VW> pp, qq;
    if (first) {
#pragma unroll
      for (int v = 0; v < VW; ++v) {
        pp.v[v] = rr.v[v];
        qq.v[v] = ca * rr.v[v] + cA * nb[v] + cD * (T)deg * rr.v[v];
      }
    } else {
      const Pack<T, VW> po = ld_plain<T, VW>(P + o);
      const Pack<T, VW> qo = ld_plain<T, VW>(Q + o);
#pragma unroll
      for (int v = 0; v < VW; ++v) {
        pp.v[v] = rr.v[v] + be[v] * po.v[v];
        qq.v[v] = ca * rr.v[v] + cA * nb[v] + cD * (T)deg * rr.v[v] + be[v] * qo.v[v];
      }
    }
#pragma unroll
    for (int v = 0; v < VW; ++v) dacc[v] += pp.v[v] * qq.v[v];
    stp<T, VW>(P + o, pp);
    stp<T, VW>(Q + o, qq);
  };
  if (tl.hub) {
    const int64_t row = tl.row_beg;
    const int beg = a.g.row_ptr[row], end = a.g.row_ptr[row + 1];
    T acc[VW];
#pragma unroll
    for (int v = 0; v < VW; ++v) acc[v] = T(0);
    row_gather<T, K, VW>(a.g.col, beg + tid / G, end, RPB, R, lane_off, acc);
#pragma unroll
    for (int v = 0; v < VW; ++v) s_red[tid * VW + v] = acc[v];
    __syncthreads();
    if (tid < G) {
      for (int gr = 1; gr < RPB; ++gr)
#pragma unroll
        for (int v = 0; v < VW; ++v) acc[v] += s_red[(gr * G + sl) * VW + v];
      fin(row, end - beg, acc);
    }
  } else {
    for (int64_t row = tl.row_beg + tid / G; row < tl.row_end; row += RPB) {
      const int beg = a.g.row_ptr[row], end = a.g.row_ptr[row + 1];
      if (end - beg > kHubDeg) continue;
      T acc[VW];
#pragma unroll
      for (int v = 0; v < VW; ++v) acc[v] = T(0);
      row_gather<T, K, VW>(a.g.col, beg, end, 1, R, lane_off, acc);
      fin(row, end - beg, acc);
    }
  }
  double dd[VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) dd[v] = (double)dacc[v];
  block_colsum_store<T, K>(dd, a.part + ((size_t)s * a.g.ntile + blockIdx.x) * K);
}

// alpha = gamma / delta; grid (ngraph, nslab)
template <int K>
__global__ void __launch_bounds__(kPhaseBlock) bred_s(BatchGraph g, BatchState st, const double* part) {
  __shared__ double s_tmp[kPhaseBlock];
  __shared__ double s_out[K];
  const int s = blockIdx.y, pr = s * g.ngraph + blockIdx.x;
  if (!st.active[pr]) return;
  problem_sum<K>(part + (size_t)s * g.ntile * K, g.tile_beg[blockIdx.x], g.tile_beg[blockIdx.x + 1], s_tmp, s_out);
  const int tid = threadIdx.x;
  if (tid < K) {
    const int i = pr * K + tid;
    const double delta = s_out[tid];
    if (!st.done[i]) {
      if (!isfinite(delta)) {
        st.status[i] = WL_ERR_NONFINITE; st.done[i] = 1; st.alpha[i] = 0.0;
      } else if (delta <= 0.0) {
        st.status[i] = WL_ERR_NOT_SPD; st.done[i] = 1; st.alpha[i] = 0.0;
      } else {
        st.alpha[i] = st.gamma[i] / delta;
      }
    } else {
      st.alpha[i] = 0.0;
    }
  }
  if (tid == 0) {
    st.iters[pr] += 1;
    st.total[pr] += 1;
  }
}

// ---------------------------------------------------------------- U
template <typename T, int K>
__global__ void __launch_bounds__(kPhaseBlock) bcg_u(BatchArgs<T> a) {
  using C = Cfg<T, K>;
  constexpr int VW = C::VW, G = C::G, RPB = kPhaseBlock / G;
  const BTile tl = a.g.tiles[blockIdx.x];
  const int s = blockIdx.y, pr = s * a.g.ngraph + tl.graph;
  if (!a.st.active[pr]) return;
  const int tid = threadIdx.x, lane_off = (tid % G) * VW;
  T al[VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) al[v] = (T)a.st.alpha[pr * K + lane_off + v];
  const size_t slab = (size_t)s * a.g.n * K;
  double acc[VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) acc[v] = 0.0;
  for (int64_t row = tl.row_beg + tid / G; row < tl.row_end; row += RPB) {
    if (!tl.hub && !plain_row(a.g.row_ptr, row)) continue;
    const size_t o = slab + (size_t)row * K + lane_off;
    Pack<T, VW> xx = ld_plain<T, VW>(a.x + o);
    Pack<T, VW> rr = ld_plain<T, VW>(a.r + o);
    const Pack<T, VW> pp = ld_plain<T, VW>(a.p + o);
    const Pack<T, VW> qq = ld_plain<T, VW>(a.q + o);
#pragma unroll
    for (int v = 0; v < VW; ++v) {
      xx.v[v] += al[v] * pp.v[v];
      rr.v[v] -= al[v] * qq.v[v];
      acc[v] += (double)rr.v[v] * (double)rr.v[v];
    }
    stp<T, VW>(a.x + o, xx);
    stp<T, VW>(a.r + o, rr);
  }
  block_colsum_store<T, K>(acc, a.part + ((size_t)s * a.g.ntile + blockIdx.x) * K);
}

// beta, convergence, activity; grid (ngraph, nslab)
template <int K>
__global__ void __launch_bounds__(kPhaseBlock) bred_u(BatchGraph g, BatchState st, const double* part, double tol2,
                                                       int max_iter) {
  __shared__ double s_tmp[kPhaseBlock];
  __shared__ double s_out[K];
  __shared__ int s_any;
  const int s = blockIdx.y, pr = s * g.ngraph + blockIdx.x;
  if (!st.active[pr]) return;
  problem_sum<K>(part + (size_t)s * g.ntile * K, g.tile_beg[blockIdx.x], g.tile_beg[blockIdx.x + 1], s_tmp, s_out);
  const int tid = threadIdx.x;
  if (tid == 0) s_any = 0;
  __syncthreads();
  if (tid < K) {
    const int i = pr * K + tid;
    const double gn = s_out[tid];
    if (!st.done[i]) {
      if (!isfinite(gn)) {
        st.status[i] = WL_ERR_NONFINITE; st.done[i] = 1; st.beta[i] = 0.0;
      } else {
        st.beta[i] = gn / st.gamma[i];
        st.gamma[i] = gn;
        if (gn <= tol2 * st.b2[i]) { st.done[i] = 1; st.beta[i] = 0.0; }
      }
    } else {
      st.beta[i] = 0.0;
    }
    if (!st.done[i]) atomicOr(&s_any, 1);
  }
  __syncthreads();
  if (tid == 0) {
    const int act = (s_any && st.iters[pr] < max_iter) ? 1 : 0;
    st.active[pr] = act;
    if (act) atomicOr(st.any, 1);
  }
}

// ---------------------------------------------------------------- refined form
// Residual of the refinement in double-float arithmetic (FP32 instructions
// only), carried recursively as in the single-graph refined solve:
//   first pass (x = 0):  r = bscale b
//   later passes:        r <- r - M d,  x64 <- x64 + d
// with d the FP32 correction of the previous inner solve (gathered: 4 bytes
// per neighbour entry) and r = rh + rl a double-float vector. The neighbour
// sum A d is accumulated with the error-free two-sum, M d and the subtraction
// in double-float, so r stays equal to bscale b - M x64 up to about 2^-46 of
// |r| + |M d| per pass. r32 = rh is the next inner solve's right-hand side
// (the inner init zeroes d). Partials per column: (r, r) from the leading
// terms, and on the first pass (bscale b, bscale b).
struct BatchResArgs {
  BatchGraph g;
  const float* d32;     // [nslab][n][K] correction of the last inner solve
  const double* b;      // [n][K]
  const double* bscale; // per problem or NULL
  const double* ca;
  const double* cA;
  const double* cD;
  float* rh;            // [nslab][n][K] residual, leading term
  float* rl;            // [nslab][n][K] residual, trailing term
  float* r32;           // [nslab][n][K] inner right-hand side
  double* x64;          // [nslab][n][K] iterate
  double* part;         // [nslab][ntile][2K]
  const int* outer_active;  // per problem (NULL: all)
  const int* outer_iters;   // per problem: 0 means x64 = 0 and r = bscale b
};

template <int K>
__global__ void __launch_bounds__(kPhaseBlock, kPhaseMinBlocks) bres(BatchResArgs a) {
  using C = Cfg<float, K>;
  constexpr int VW = C::VW, G = C::G, RPB = kPhaseBlock / G;
  __shared__ __align__(16) float s_red[2][kPhaseBlock * VW];
  const BTile tl = a.g.tiles[blockIdx.x];
  const int s = blockIdx.y, pr = s * a.g.ngraph + tl.graph;
  if (a.outer_active && !a.outer_active[pr]) return;
  const bool first = a.outer_iters[pr] == 0;
  const int tid = threadIdx.x, sl = tid % G, lane_off = sl * VW;
  const size_t slab = (size_t)s * a.g.n * K;
  const df ca = df_from_double(a.ca[pr]), cA = df_from_double(a.cA[pr]), cD = df_from_double(a.cD[pr]);
  const double sc = a.bscale ? a.bscale[pr] : 1.0;
  const float* D = a.d32 + slab;
  float acc_r[VW], acc_b[VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) acc_r[v] = acc_b[v] = 0.f;
  auto fin = [&](int64_t row, int deg, const float (&sm)[VW], const float (&cm)[VW]) {
    const size_t o = (size_t)row * K + lane_off;
    Pack<float, VW> rh, rl;
    if (first) {
      const Pack<double, VW> bb = ld_plain<double, VW>(a.b + o);
#pragma unroll
      for (int v = 0; v < VW; ++v) {
        const df r = df_from_double(sc * bb.v[v]);
        rh.v[v] = r.hi;
        rl.v[v] = r.lo;
        acc_b[v] = __fmaf_rn(r.hi, r.hi, acc_b[v]);
      }
    } else {
      const df crow = df_add(ca, df_mul_f(cD, (float)deg));
      const Pack<float, VW> dd = ld_plain<float, VW>(D + o);
      const Pack<float, VW> ph = ld_plain<float, VW>(a.rh + slab + o);
      const Pack<float, VW> pl = ld_plain<float, VW>(a.rl + slab + o);
      Pack<double, VW> xx = ld_plain<double, VW>(a.x64 + slab + o);
#pragma unroll
      for (int v = 0; v < VW; ++v) {
        const df nb = two_sum(sm[v], cm[v]);
        const df Md = df_add(df_mul_f(crow, dd.v[v]), df_mul(cA, nb));
        const df r = df_sub(df{ph.v[v], pl.v[v]}, Md);
        rh.v[v] = r.hi;
        rl.v[v] = r.lo;
        xx.v[v] += (double)dd.v[v];
      }
      stp<double, VW>(a.x64 + slab + o, xx);
    }
#pragma unroll
    for (int v = 0; v < VW; ++v) acc_r[v] = __fmaf_rn(rh.v[v], rh.v[v], acc_r[v]);
    stp<float, VW>(a.rh + slab + o, rh);
    stp<float, VW>(a.rl + slab + o, rl);
    stp<float, VW>(a.r32 + slab + o, rh);
  };
  if (tl.hub) {
    const int64_t row = tl.row_beg;
    const int beg = a.g.row_ptr[row], end = a.g.row_ptr[row + 1];
    float sm[VW], cm[VW], lm[VW];
#pragma unroll
    for (int v = 0; v < VW; ++v) sm[v] = cm[v] = lm[v] = 0.f;
    if (!first) df_row_gather<K, VW, false>(a.g.col, beg + tid / G, end, RPB, D, nullptr, lane_off, sm, cm, lm);
#pragma unroll
    for (int v = 0; v < VW; ++v) {
      s_red[0][tid * VW + v] = sm[v];
      s_red[1][tid * VW + v] = cm[v];
    }
    __syncthreads();
    if (tid < G) {
      for (int gr = 1; gr < RPB; ++gr)
#pragma unroll
        for (int v = 0; v < VW; ++v) {
          const int k = (gr * G + sl) * VW + v;
          const df t = two_sum(sm[v], s_red[0][k]);
          sm[v] = t.hi;
          cm[v] += t.lo + s_red[1][k];
        }
      fin(row, end - beg, sm, cm);
    }
  } else {
    for (int64_t row = tl.row_beg + tid / G; row < tl.row_end; row += RPB) {
      const int beg = a.g.row_ptr[row], end = a.g.row_ptr[row + 1];
      if (end - beg > kHubDeg) continue;
      float sm[VW], cm[VW], lm[VW];
#pragma unroll
      for (int v = 0; v < VW; ++v) sm[v] = cm[v] = lm[v] = 0.f;
      if (!first) df_row_gather<K, VW, false>(a.g.col, beg, end, 1, D, nullptr, lane_off, sm, cm, lm);
      fin(row, end - beg, sm, cm);
    }
  }
  double pr_r[VW], pr_b[VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) {
    pr_r[v] = (double)acc_r[v];
    pr_b[v] = (double)acc_b[v];
  }
  double* out = a.part + ((size_t)s * a.g.ntile + blockIdx.x) * 2 * K;
  block_colsum_store<float, K>(pr_r, out);
  __syncthreads();
  block_colsum_store<float, K>(pr_b, out + K);
}

// outer (refinement) control per problem: the relative double-float residual
// decides convergence; the inner solve's reference norm is ||r||^2 and
// columns already converged are skipped. grid (ngraph, nslab)
struct BatchOuter {
  double* rn2;         // per problem-column ||r||^2 of the refinement residual (inner reference)
  double* bn2;         // per problem-column ||b||^2
  int* skip;           // per problem-column
  int* outer_active;   // per problem
  int* outer_iters;    // per problem
  int* status;         // per problem-column final status
  int* any;            // one flag
};

template <int K>
__global__ void __launch_bounds__(kPhaseBlock) bred_res(BatchGraph g, BatchOuter o, const double* part, double tol2,
                                                         int max_outer) {
  __shared__ double s_tmp[kPhaseBlock];
  __shared__ double s_out[2 * K];
  __shared__ int s_any;
  const int s = blockIdx.y, pr = s * g.ngraph + blockIdx.x;
  if (!o.outer_active[pr]) return;
  // 2K columns of partials: (r, r) then (b, b)
  {
    constexpr int K2 = 2 * K;
    constexpr int J = kPhaseBlock / K2 > 0 ? kPhaseBlock / K2 : 1;
    const int tid = threadIdx.x, c = tid % K2, j = tid / K2;
    double acc = 0.0;
    const double* pp = part + (size_t)s * g.ntile * K2;
    if (j < J)
      for (int t = g.tile_beg[blockIdx.x] + j; t < g.tile_beg[blockIdx.x + 1]; t += J)
        acc += __ldcg(pp + (size_t)t * K2 + c);
    s_tmp[tid] = (j < J) ? acc : 0.0;
    __syncthreads();
    if (tid < K2) {
      double u = 0.0;
      for (int jj = 0; jj < J; ++jj) u += s_tmp[jj * K2 + tid];
      s_out[tid] = u;
    }
    if (tid == 0) s_any = 0;
    __syncthreads();
  }
  const int tid = threadIdx.x;
  const int it = o.outer_iters[pr];
  if (tid < K) {
    const int i = pr * K + tid;
    const double rn = s_out[tid];
    const double bn = it == 0 ? s_out[K + tid] : o.bn2[i];  // ||bscale b||^2 from the first pass
    o.rn2[i] = rn;
    if (it == 0) o.bn2[i] = bn;
    int conv = (bn <= 0.0) || (rn <= tol2 * bn);
    if (!isfinite(rn)) {
      conv = 1;
      o.status[i] = WL_ERR_NONFINITE;
    } else {
      o.status[i] = conv ? 0 : WL_ERR_NO_CONVERGENCE;
    }
    o.skip[i] = conv;
    if (!conv) atomicOr(&s_any, 1);
  }
  __syncthreads();
  if (tid == 0) {
    const int act = (s_any && it < max_outer) ? 1 : 0;
    o.outer_active[pr] = act;
    o.outer_iters[pr] = it + 1;
    if (act) atomicOr(o.any, 1);
  }
}

// graph of a row: the last g with goff[g] <= row
__device__ __forceinline__ int graph_of(const BatchGraph& g, int64_t row) {
  int lo = 0, hi = g.ngraph - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (g.goff[mid] <= row) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------- outputs
// W[s] = Df[s] (.) V - phi_scale[s,g] X[s]   (phi V = (1 - mu^2 alpha^2) M^{-1} V)
template <typename T>
__global__ void __launch_bounds__(kPhaseBlock) bout(BatchGraph g, const double* Df, const double* V, const T* X,
                                                     const double* phi_scale, double* W, int K, int nslab) {
  const int64_t per = g.n * K;
  const int64_t total = per * nslab;
  for (int64_t e = (int64_t)blockIdx.x * kPhaseBlock + threadIdx.x; e < total; e += (int64_t)gridDim.x * kPhaseBlock) {
    const int s = (int)(e / per);
    const int64_t rem = e - (int64_t)s * per;
    const int64_t row = rem / K;
    W[e] = Df[(int64_t)s * g.n + row] * V[rem] - phi_scale[s * g.ngraph + graph_of(g, row)] * (double)X[e];
  }
}

#endif  // WL_BATCH_KERNELS

}  // namespace wl
