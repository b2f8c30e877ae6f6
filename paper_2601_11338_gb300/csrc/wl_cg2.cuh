// Lockstep conjugate gradients on M = ca I + cA A + cD D for K columns as
// high-occupancy phase kernels (Sec. 4.2: each application of the resolvent
// walk Laplacian is one CG solve with the deformed Laplacian, positive
// definite for alpha < 1 / rho(Z), Prop. CGworks).
//
// The gather of neighbour vectors is latency bound, so these kernels keep
// the SMs full of warps (G lanes per row, one 16-byte slice each, rows
// spread over a grid-stride loop) instead of persisting with few warps.
// Rows with more than kHubDeg entries are gathered by one CTA each; when the
// graph carries a list of mid rows (kMidDeg < deg <= kHubDeg), the S kernel
// spends a share of its CTAs (proportional to those rows' entries) on them,
// one warp per row, so that no lane group walks a long row alone, and the
// remaining CTAs take the short rows; the grid stays one wave.
//
// One iteration = two kernels:
//   S: s = M r ; x += alpha p ; p = r + beta p ; q = s + beta q ; delta = (p, q)
//   U: r -= alpha q ; gamma' = (r, r)
// Each kernel ends with a last-CTA reduction (fixed order, deterministic)
// that derives the next scalars and the per-column convergence on the
// device; a kernel finding the solve inactive returns at once, so the host
// launches iterations in chunks and reads one flag between chunks.
// Vector traffic per iteration: 10 n K s bytes + 4 nnz + 4 (n + 1).
#pragma once
#include "wl_common.cuh"

namespace wl {

constexpr int kHubDeg = 256;       // rows with more entries get a CTA each
constexpr int kMidDeg = 30;        // rows with more entries (up to kHubDeg) get a warp each in the S kernels
constexpr int kPhaseBlock = 256;   // threads per CTA of the phase kernels
#ifndef WL_PHASE_MINB
#define WL_PHASE_MINB 5
#endif
constexpr int kPhaseMinBlocks = WL_PHASE_MINB;  // CTAs per SM the S kernel's registers are sized for
// FP32 CG kernels: 5 CTAs per SM (48 registers) hold the eight predicated
// gathers per lane; measured 236 us per K = 16 iteration on the Chung-Lu 1e6
// graph (6 CTAs: 240 us; 4 CTAs: 248 us)
#ifndef WL_PHASE_MINB_F32
#define WL_PHASE_MINB_F32 5
#endif
constexpr int kPhaseMinBlocksF32 = WL_PHASE_MINB_F32;
template <typename T>
constexpr int phase_min_blocks() { return sizeof(T) == 4 ? kPhaseMinBlocksF32 : kPhaseMinBlocks; }


// Per-solve device state (written by the last CTA of each kernel).
struct CgState {
  double gamma[64], alpha[64], beta[64], b2[64];
  int done[64], status[64];
  int active;  // 1 while some column iterates and iters < max_iter
  int iters;   // S phases executed
  unsigned ticket;
  int pad;
};

struct PhaseGraph {
  const int32_t* row_ptr;
  const int32_t* col;
  int64_t n;
  const int32_t* hubs;  // rows with deg > kHubDeg
  int nhub;
  const int32_t* mids = nullptr;  // rows with kMidDeg < deg <= kHubDeg
  int nmid = 0;
  int nmid_blk = 0;               // CTAs (after the hub CTAs) that walk the mid rows; 0: no mid path
};

template <typename T>
struct PhaseArgs {
  PhaseGraph g;
  T* x;
  T* r;
  T* p;
  T* q;
  double ca, cA, cD;
  const double* bnorm2;  // K or NULL (then ||r_0||^2)
  const int* skip;       // K or NULL
  double* part;          // gridDim.x * K partials
  CgState* st;
  int max_iter;
  double tol2;
  // optional per-row diagonal added to M (the shifted solves of the
  // shift-and-invert Lanczos: M - a (D_f + sigma I)^{-1}); NULL: none
  const T* dshift = nullptr;
};

// ---------------------------------------------------------------- helpers
template <typename T, int VW>
__device__ __forceinline__ Pack<T, VW> ld_plain(const T* p) {
  return *reinterpret_cast<const Pack<T, VW>*>(p);
}

// Gathers per lane in flight in row_gather: predicated batches of 8 (1)
// measured 240 vs 252 us per K = 16 FP32 CG iteration against the unrolled
// loop with a serial tail (0), and 236 us with the FP32 kernels at 5 CTAs per
// SM (48 registers)
#ifndef WL_GATHER_PRED
#define WL_GATHER_PRED 1
#endif
#ifndef WL_GATHER_U
#define WL_GATHER_U 8
#endif
// the same choice for the FP64 kernels (the plain FP64 form), measured on its own
#ifndef WL_GATHER_PRED_F64
#define WL_GATHER_PRED_F64 0
#endif

// Sum of X over entries [beg, end) with stride `step`.
// WL_GATHER_PRED = 1: every batch of WL_GATHER_U entries, the last one too,
// issues its index loads and then its gathers together (predicated on the
// row end), so a short row costs one index latency and one gather latency
// per batch instead of a dependent pair per entry of its tail. (0: batches of
// four with the tail walked entry by entry.)
template <typename T, int K, int VW>
__device__ __forceinline__ void row_gather(const int32_t* __restrict__ col, int beg, int end, int step,
                                           const T* X, int lane_off, T (&acc)[VW]) {
  if constexpr (sizeof(T) == 4 ? WL_GATHER_PRED : WL_GATHER_PRED_F64) {
  constexpr int U = WL_GATHER_U;
  for (int e = beg; e < end; e += U * step) {
    int j[U];
#pragma unroll
    for (int u = 0; u < U; ++u) j[u] = (e + u * step < end) ? __ldg(col + e + u * step) : -1;
    Pack<T, VW> a[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (j[u] >= 0) {
        a[u] = ld_plain<T, VW>(X + (size_t)j[u] * K + lane_off);
      } else {
#pragma unroll
        for (int v = 0; v < VW; ++v) a[u].v[v] = T(0);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int v = 0; v < VW; ++v) acc[v] += a[u].v[v];
  }
  return;
  }
  int e = beg;
  for (; e + 3 * step < end; e += 4 * step) {
    const int j0 = __ldg(col + e), j1 = __ldg(col + e + step);
    const int j2 = __ldg(col + e + 2 * step), j3 = __ldg(col + e + 3 * step);
    const Pack<T, VW> a0 = ld_plain<T, VW>(X + (size_t)j0 * K + lane_off);
    const Pack<T, VW> a1 = ld_plain<T, VW>(X + (size_t)j1 * K + lane_off);
    const Pack<T, VW> a2 = ld_plain<T, VW>(X + (size_t)j2 * K + lane_off);
    const Pack<T, VW> a3 = ld_plain<T, VW>(X + (size_t)j3 * K + lane_off);
#pragma unroll
    for (int v = 0; v < VW; ++v) acc[v] += (a0.v[v] + a1.v[v]) + (a2.v[v] + a3.v[v]);
  }
  for (; e < end; e += step) {
    const Pack<T, VW> a0 = ld_plain<T, VW>(X + (size_t)__ldg(col + e) * K + lane_off);
#pragma unroll
    for (int v = 0; v < VW; ++v) acc[v] += a0.v[v];
  }
}

// CTA column sums of per-thread partials (thread t owns columns (t % G) VW + v)
// written to part[blockIdx.x * K + c]; then the last CTA to finish returns
// true (all partials visible to it).
template <typename T, int K>
__device__ __forceinline__ bool block_partials_last(const double (&val)[Cfg<T, K>::VW], double* part,
                                                    unsigned* ticket) {
  using C = Cfg<T, K>;
  constexpr int VW = C::VW, G = C::G, NW = kPhaseBlock / 32;
  __shared__ double s_w[NW * K];
  __shared__ int s_last;
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
    part[(size_t)blockIdx.x * K + tid] = t;
    __threadfence();
  }
  __syncthreads();
  if (tid == 0) s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1) ? 1 : 0;
  __syncthreads();
  if (s_last) __threadfence();
  return s_last != 0;
}

// Fixed-order sum over all CTAs' partials, by the last CTA: out[c] (shared).
template <int K>
__device__ __forceinline__ void sum_partials(const double* part, int nblk, double* s_tmp, double* out) {
  constexpr int J = kPhaseBlock / K;
  const int tid = threadIdx.x, c = tid % K, j = tid / K;
  double s = 0.0;
  int b = j;
  for (; b + 7 * J < nblk; b += 8 * J) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = __ldcg(part + (size_t)(b + u * J) * K + c);
#pragma unroll
    for (int u = 0; u < 8; ++u) s += v[u];
  }
  for (; b < nblk; b += J) s += __ldcg(part + (size_t)b * K + c);
  s_tmp[tid] = s;
  __syncthreads();
  if (tid < K) {
    double t = 0.0;
    for (int jj = 0; jj < J; ++jj) t += s_tmp[jj * K + tid];
    out[tid] = t;
  }
  __syncthreads();
}

// ---------------------------------------------------------------- S phase
// SH: the solve carries the per-row diagonal a.dshift (a separate instance,
// so that the unshifted kernel carries no trace of it)
template <typename T, int K, bool SH = false>
__global__ void __launch_bounds__(kPhaseBlock, phase_min_blocks<T>()) cg_s_phase(PhaseArgs<T> a) {
  using C = Cfg<T, K>;
  constexpr int VW = C::VW, G = C::G, RPB = kPhaseBlock / G;  // rows per CTA pass
  __shared__ __align__(16) T s_red[kPhaseBlock * VW];
  __shared__ double s_tmp[kPhaseBlock];
  __shared__ double s_out[K];
  CgState* st = a.st;
  if (!*(volatile int*)&st->active) return;
  const int tid = threadIdx.x, sl = tid % G, lane_off = sl * VW;
  const bool first = (st->iters == 0);
  const T ca = (T)a.ca, cA = (T)a.cA, cD = (T)a.cD;
  __shared__ T s_ab[2][K];
  if (tid < K) {
    s_ab[0][tid] = (T)st->alpha[tid];
    s_ab[1][tid] = (T)st->beta[tid];
  }
  __syncthreads();
  T dacc[VW];  // per-thread partials in the working precision (FP64 adds are scarce on this GPU)
#pragma unroll
  for (int v = 0; v < VW; ++v) dacc[v] = T(0);

  T* __restrict__ px = a.x;
  T* __restrict__ pp_ = a.p;
  T* __restrict__ pq = a.q;
  const T* __restrict__ pr = a.r;
  struct Own {
    Pack<T, VW> r, x, p, q;
  };
  // own-row r, loaded before the row's gathers so the two overlap
  auto own = [&](int64_t row) {
    Own o;
    const size_t off = (size_t)row * K + lane_off;
    o.r = ld_plain<T, VW>(pr + off);
    return o;
  };
  auto fin = [&](int64_t row, int deg, const T (&nb)[VW], const Own& w0) {
    const size_t o = (size_t)row * K + lane_off;
    Own w = w0;
    // the shift diagonal is loaded with x, p, q after the gathers: held
    // across them it costs the gather loop a register
    T dx = T(0);
    if constexpr (SH) dx = __ldg(a.dshift + row);
    if (!first) {
      w.x = ld_plain<T, VW>(px + o);
      w.p = ld_plain<T, VW>(pp_ + o);
      w.q = ld_plain<T, VW>(pq + o);
    }
    const Pack<T, VW>& rr = w.r;
    Pack<T, VW> pp, qq;
    const T dg = (T)deg;
    if (first) {
#pragma unroll
      for (int v = 0; v < VW; ++v) {
        pp.v[v] = rr.v[v];
        qq.v[v] = ca * rr.v[v] + cA * nb[v] + cD * dg * rr.v[v];
        if constexpr (SH) qq.v[v] += dx * rr.v[v];
      }
    } else {
      Pack<T, VW> xx = w.x;
#pragma unroll
      for (int v = 0; v < VW; ++v) {
        T s = ca * rr.v[v] + cA * nb[v] + cD * dg * rr.v[v];
        if constexpr (SH) s += dx * rr.v[v];
        const T al = s_ab[0][lane_off + v], be = s_ab[1][lane_off + v];
        xx.v[v] += al * w.p.v[v];
        pp.v[v] = rr.v[v] + be * w.p.v[v];
        qq.v[v] = s + be * w.q.v[v];
      }
      stp<T, VW>(px + o, xx);
    }
#pragma unroll
    for (int v = 0; v < VW; ++v) dacc[v] += pp.v[v] * qq.v[v];
    stp<T, VW>(pp_ + o, pp);
    stp<T, VW>(pq + o, qq);
  };

  if ((int)blockIdx.x < a.g.nhub) {
    // one hub row per CTA: RPB lane groups stride over the entries
    const int64_t row = a.g.hubs[blockIdx.x];
    const int beg = a.g.row_ptr[row], end = a.g.row_ptr[row + 1];
    T acc[VW];
#pragma unroll
    for (int v = 0; v < VW; ++v) acc[v] = T(0);
    row_gather<T, K, VW>(a.g.col, beg + tid / G, end, RPB, a.r, lane_off, acc);
#pragma unroll
    for (int v = 0; v < VW; ++v) s_red[tid * VW + v] = acc[v];
    __syncthreads();
    if (tid < G) {
      const Own w = own(row);
      for (int gr = 1; gr < RPB; ++gr)
#pragma unroll
        for (int v = 0; v < VW; ++v) acc[v] += s_red[(gr * G + sl) * VW + v];
      fin(row, end - beg, acc, w);
    }
  } else if ((int)blockIdx.x < a.g.nhub + a.g.nmid_blk) {
    // mid rows, one warp each: the 32 / G lane groups stride over the entries
    // and are combined by shuffles; lane group 0 finishes the row
    const int lane = tid & 31;
    constexpr int WPB = kPhaseBlock / 32;
    for (int r = ((int)blockIdx.x - a.g.nhub) * WPB + (tid >> 5); r < a.g.nmid; r += a.g.nmid_blk * WPB) {
      const int64_t row = a.g.mids[r];
      const int beg = a.g.row_ptr[row], end = a.g.row_ptr[row + 1];
      Own w;
      if (lane < G) w = own(row);
      T acc[VW];
#pragma unroll
      for (int v = 0; v < VW; ++v) acc[v] = T(0);
      row_gather<T, K, VW>(a.g.col, beg + lane / G, end, 32 / G, a.r, lane_off, acc);
#pragma unroll
      for (int off = G; off < 32; off <<= 1)
#pragma unroll
        for (int v = 0; v < VW; ++v) acc[v] += __shfl_xor_sync(0xffffffffu, acc[v], off);
      if (lane < G) fin(row, end - beg, acc, w);
    }
  } else {
    const int nlist = a.g.nhub + a.g.nmid_blk;
    const int lim = a.g.nmid_blk > 0 ? kMidDeg : kHubDeg;  // longer rows: hub CTAs or mid warps
    const int64_t nblk = (int64_t)gridDim.x - nlist;
    for (int64_t row = ((int64_t)blockIdx.x - nlist) * RPB + tid / G; row < a.g.n; row += nblk * RPB) {
      const int beg = a.g.row_ptr[row], end = a.g.row_ptr[row + 1];
      if (end - beg > lim) continue;
      const Own w = own(row);
      T acc[VW];
#pragma unroll
      for (int v = 0; v < VW; ++v) acc[v] = T(0);
      row_gather<T, K, VW>(a.g.col, beg, end, 1, a.r, lane_off, acc);
      fin(row, end - beg, acc, w);
    }
  }
  double dd[VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) dd[v] = (double)dacc[v];
  if (!block_partials_last<T, K>(dd, a.part, &st->ticket)) return;
  // last CTA: delta -> alpha, breakdown checks
  sum_partials<K>(a.part, gridDim.x, s_tmp, s_out);
  if (tid < K) {
    const double delta = s_out[tid];
    if (!st->done[tid]) {
      if (!isfinite(delta)) {
        st->status[tid] = WL_ERR_NONFINITE; st->done[tid] = 1; st->alpha[tid] = 0.0;
      } else if (delta <= 0.0) {
        st->status[tid] = WL_ERR_NOT_SPD; st->done[tid] = 1; st->alpha[tid] = 0.0;
      } else {
        st->alpha[tid] = st->gamma[tid] / delta;
      }
    } else {
      st->alpha[tid] = 0.0;
    }
  }
  if (tid == 0) {
    st->iters += 1;
    st->ticket = 0;
  }
}

// ---------------------------------------------------------------- U phase (and init)
// init = 1: gamma_0 = (r, r), convergence reference and flags, no update.
template <typename T, int K>
__global__ void __launch_bounds__(kPhaseBlock, phase_min_blocks<T>()) cg_u_phase(PhaseArgs<T> a, int init) {
  using C = Cfg<T, K>;
  constexpr int VW = C::VW, G = C::G;
  __shared__ double s_tmp[kPhaseBlock];
  __shared__ double s_out[K];
  CgState* st = a.st;
  if (!init && !*(volatile int*)&st->active) return;
  const int tid = threadIdx.x;
  const int mycol = (tid % G) * VW;  // kPhaseBlock * VW is a multiple of K
  T al[VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) al[v] = init ? T(0) : (T)st->alpha[mycol + v];
  T acc[VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) acc[v] = T(0);
  const size_t nv = (size_t)a.g.n * K / VW;
#pragma unroll 4
  for (size_t e = (size_t)blockIdx.x * kPhaseBlock + tid; e < nv; e += (size_t)gridDim.x * kPhaseBlock) {
    Pack<T, VW> rr = ld_plain<T, VW>(a.r + e * VW);
    if (!init) {
      const Pack<T, VW> qq = ld_plain<T, VW>(a.q + e * VW);
#pragma unroll
      for (int v = 0; v < VW; ++v) rr.v[v] -= al[v] * qq.v[v];
      stp<T, VW>(a.r + e * VW, rr);
    }
#pragma unroll
    for (int v = 0; v < VW; ++v) acc[v] += rr.v[v] * rr.v[v];
  }
  double dd[VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) dd[v] = (double)acc[v];
  if (!block_partials_last<T, K>(dd, a.part, &st->ticket)) return;
  sum_partials<K>(a.part, gridDim.x, s_tmp, s_out);
  if (tid < K) {
    const double gn = s_out[tid];
    if (init) {
      const double b2 = a.bnorm2 ? a.bnorm2[tid] : gn;
      st->gamma[tid] = gn;
      st->b2[tid] = b2;
      st->alpha[tid] = 0.0;
      st->beta[tid] = 0.0;
      st->status[tid] = 0;
      int done = (b2 <= 0.0) || (gn <= a.tol2 * b2) || (a.skip && a.skip[tid]);
      if (!isfinite(gn)) { done = 1; st->status[tid] = WL_ERR_NONFINITE; }
      st->done[tid] = done;
    } else if (!st->done[tid]) {
      if (!isfinite(gn)) {
        st->status[tid] = WL_ERR_NONFINITE; st->done[tid] = 1; st->beta[tid] = 0.0;
      } else {
        st->beta[tid] = gn / st->gamma[tid];
        st->gamma[tid] = gn;
        if (gn <= a.tol2 * st->b2[tid]) { st->done[tid] = 1; st->beta[tid] = 0.0; }
      }
    } else {
      st->beta[tid] = 0.0;
    }
  }
  __syncthreads();
  if (tid == 0) {
    if (init) st->iters = 0;
    int any = 0;
    for (int c = 0; c < K; ++c) any |= !st->done[c];
    st->active = (any && st->iters < a.max_iter) ? 1 : 0;
    st->ticket = 0;
  }
}

// x += alpha p: the deferred update of the last U phase
template <typename T, int K>
__global__ void __launch_bounds__(kPhaseBlock) cg_f_phase(PhaseArgs<T> a) {
  using C = Cfg<T, K>;
  constexpr int VW = C::VW, G = C::G;
  CgState* st = a.st;
  if (st->iters == 0) return;
  const int tid = threadIdx.x;
  const int mycol = (tid % G) * VW;
  T al[VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) al[v] = (T)st->alpha[mycol + v];
  const size_t nv = (size_t)a.g.n * K / VW;
  for (size_t e = (size_t)blockIdx.x * kPhaseBlock + tid; e < nv; e += (size_t)gridDim.x * kPhaseBlock) {
    Pack<T, VW> xx = ld_plain<T, VW>(a.x + e * VW);
    const Pack<T, VW> pp = ld_plain<T, VW>(a.p + e * VW);
#pragma unroll
    for (int v = 0; v < VW; ++v) xx.v[v] += al[v] * pp.v[v];
    stp<T, VW>(a.x + e * VW, xx);
  }
}

// ---------------------------------------------------------------- FP64 residual
// Start of an FP64-form solve from a warm start x: r = b - M x, column norms
// ||r||^2 -> st->gamma and ||b||^2 -> st->b2 (last CTA).
struct ResPhaseArgs {
  PhaseGraph g;
  const double* x;
  const double* b;  // NULL: b = 0 (then r = -M x)
  double* r;
  double ca, cA, cD;
  double* part;  // 2 * gridDim.x * K
  CgState* st;
};

template <int K>
__global__ void __launch_bounds__(kPhaseBlock, kPhaseMinBlocks) res_phase(ResPhaseArgs a) {
  using C = Cfg<double, K>;
  constexpr int VW = C::VW, G = C::G, RPB = kPhaseBlock / G;
  __shared__ __align__(16) double s_red[kPhaseBlock * VW];
  __shared__ double s_tmp[kPhaseBlock];
  __shared__ double s_out[K];
  const int tid = threadIdx.x, sl = tid % G, lane_off = sl * VW;
  const double ca = a.ca, cA = a.cA, cD = a.cD;
  double racc[2 * VW];  // (r, r) then (b, b)
#pragma unroll
  for (int v = 0; v < 2 * VW; ++v) racc[v] = 0.0;
  auto fin = [&](int64_t row, int deg, const double (&nb)[VW]) {
    const size_t o = (size_t)row * K + lane_off;
    const Pack<double, VW> xx = ld_plain<double, VW>(a.x + o);
    Pack<double, VW> bb;
    if (a.b) {
      bb = ld_plain<double, VW>(a.b + o);
    } else {
#pragma unroll
      for (int v = 0; v < VW; ++v) bb.v[v] = 0.0;
    }
    Pack<double, VW> rr;
#pragma unroll
    for (int v = 0; v < VW; ++v) {
      rr.v[v] = bb.v[v] - (ca * xx.v[v] + cA * nb[v] + cD * (double)deg * xx.v[v]);
      racc[v] += rr.v[v] * rr.v[v];
      racc[VW + v] += bb.v[v] * bb.v[v];
    }
    stp<double, VW>(a.r + o, rr);
  };
  if ((int)blockIdx.x < a.g.nhub) {
    const int64_t row = a.g.hubs[blockIdx.x];
    const int beg = a.g.row_ptr[row], end = a.g.row_ptr[row + 1];
    double acc[VW];
#pragma unroll
    for (int v = 0; v < VW; ++v) acc[v] = 0.0;
    row_gather<double, K, VW>(a.g.col, beg + tid / G, end, RPB, a.x, lane_off, acc);
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
    const int64_t nblk = (int64_t)gridDim.x - a.g.nhub;
    for (int64_t row = ((int64_t)blockIdx.x - a.g.nhub) * RPB + tid / G; row < a.g.n; row += nblk * RPB) {
      const int beg = a.g.row_ptr[row], end = a.g.row_ptr[row + 1];
      if (end - beg > kHubDeg) continue;
      double acc[VW];
#pragma unroll
      for (int v = 0; v < VW; ++v) acc[v] = 0.0;
      row_gather<double, K, VW>(a.g.col, beg, end, 1, a.x, lane_off, acc);
      fin(row, end - beg, acc);
    }
  }
  double rp[VW], bp[VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) {
    rp[v] = racc[v];
    bp[v] = racc[VW + v];
  }
  // two partial sets: (r, r) in part[0 .. G K), (b, b) in part[G K .. 2 G K)
  double* part_b = a.part + (size_t)gridDim.x * K;
  {
    using CC = Cfg<double, K>;
    constexpr int NW = kPhaseBlock / 32;
    __shared__ double s_w[2 * NW * K];
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int off = CC::G; off < 32; off <<= 1)
#pragma unroll
      for (int v = 0; v < VW; ++v) {
        rp[v] += __shfl_xor_sync(0xffffffffu, rp[v], off);
        bp[v] += __shfl_xor_sync(0xffffffffu, bp[v], off);
      }
    if (lane < CC::G)
#pragma unroll
      for (int v = 0; v < VW; ++v) {
        s_w[warp * K + lane * VW + v] = rp[v];
        s_w[NW * K + warp * K + lane * VW + v] = bp[v];
      }
    __syncthreads();
    if (tid < K) {
      double t = 0.0, u = 0.0;
      for (int w = 0; w < NW; ++w) {
        t += s_w[w * K + tid];
        u += s_w[NW * K + w * K + tid];
      }
      a.part[(size_t)blockIdx.x * K + tid] = t;
      part_b[(size_t)blockIdx.x * K + tid] = u;
      __threadfence();
    }
    __syncthreads();
  }
  __shared__ int s_last;
  if (tid == 0) s_last = (atomicAdd(&a.st->ticket, 1u) == gridDim.x - 1) ? 1 : 0;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  sum_partials<K>(a.part, gridDim.x, s_tmp, s_out);
  if (tid < K) a.st->gamma[tid] = s_out[tid];
  sum_partials<K>(part_b, gridDim.x, s_tmp, s_out);
  if (tid < K) a.st->b2[tid] = s_out[tid];
  if (tid == 0) a.st->ticket = 0;
}

}  // namespace wl
