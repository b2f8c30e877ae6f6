// Device-side building blocks shared by the walk-Laplacian kernels.
//
// Data layout: the graph is CSR with int32 row_ptr / col_idx and implicit
// unit values; vector blocks are row-major n x K with the K values of a
// node contiguous, so one gathered neighbour row is K * sizeof(T) contiguous
// bytes (64 B for K = 16 FP32) read with 16-byte vector loads.
//
// Work split: a persistent grid of G CTAs; CTA g owns the contiguous rows
// [rb[g], rb[g+1]) chosen so that deg + kRowCost per row is balanced. Inside
// its range the rows are listed by class (order[], built once per
// partition):
//   class C  deg > Tc          : the whole CTA gathers the row, reduced in smem
//   class W  Tw < deg <= Tc    : one warp per row, reduced by shuffles
//   class S  deg <= Tw         : one subgroup of G lanes per row, rows sorted
//                                by decreasing degree so a warp's rows are
//                                equally long
// Elementwise phases walk the contiguous range, fully coalesced.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "wl.h"

namespace wl {

constexpr int kBlock = 256;        // threads per CTA of the persistent kernels
#ifndef WL_MIN_BLOCKS
#define WL_MIN_BLOCKS 2
#endif
constexpr int kMinBlocks = WL_MIN_BLOCKS;  // CTAs per SM the register budget is sized for
#ifndef WL_BATCH_ENTRIES
#define WL_BATCH_ENTRIES 16  // neighbour entries per subgroup batch (gathers in flight per lane)
#endif
constexpr int kRowCost = 2;        // partition cost of a row beyond its entries
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // every device-side wait gives up after 2 s

// ------------------------------------------------------------------ grid barrier
// Sense counter + generation word in global memory. Used only by kernels
// launched cooperatively (all CTAs co-resident). Every wait is bounded:
// after kWaitLimitNs it records WL_ERR_TIMEOUT in `err` and returns false,
// and every caller then leaves the kernel.
struct GridBar {
  unsigned int count;
  unsigned int gen;
  int err;
  int pad;
};

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ bool grid_sync(GridBar* b, unsigned nblocks) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned g = ld_acquire(&b->gen);
    __threadfence();
    const unsigned prev = atomicAdd(&b->count, 1u);
    if (prev == nblocks - 1) {
      atomicExch(&b->count, 0u);
      __threadfence();
      st_release(&b->gen, g + 1u);
    } else {
      const uint64_t t0 = globaltimer_ns();
      while (ld_acquire(&b->gen) == g) {
        if (*(volatile int*)&b->err != 0) {  // another CTA gave up: leave too
          ok = 0;
          break;
        }
        if (globaltimer_ns() - t0 > kWaitLimitNs) {
          atomicExch(&b->err, WL_ERR_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    if (ok && *(volatile int*)&b->err != 0) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// ------------------------------------------------------------------ vector config
template <typename T, int K>
struct Cfg {
  static constexpr int VEC = 16 / (int)sizeof(T);  // elements in 16 bytes
  static constexpr int VW = K < VEC ? K : VEC;     // elements per lane
  static constexpr int G = K / VW;                 // lanes per row (subgroup)
  static constexpr int SUB = 32 / G;               // subgroups per warp
  static constexpr int NSUB = kBlock / G;          // subgroups per CTA
  // index loads per lane per batch; a batch covers E = G * BS entries and
  // every lane issues E independent gathers for it
  static constexpr int BS = (WL_BATCH_ENTRIES / G) > 8 ? 8 : ((WL_BATCH_ENTRIES / G) < 1 ? 1 : WL_BATCH_ENTRIES / G);
  static constexpr int E = G * BS;
  // rows with more than Tc entries are gathered by the whole CTA; all others
  // by one subgroup (chains of at most 32 batches)
  static constexpr int Tc = 32 * E;
  static constexpr int Tw = Tc;  // no warp-per-row class
  static_assert(G >= 1 && G <= 32, "subgroup size");
  static_assert(K % VW == 0, "K must be a multiple of the lane width");
};

template <typename T, int VW>
struct alignas(sizeof(T) * VW) Pack {
  T v[VW];
};

template <typename T, int VW>
struct VecOf;
template <>
struct VecOf<float, 4> { using type = float4; };
template <>
struct VecOf<float, 2> { using type = float2; };
template <>
struct VecOf<float, 1> { using type = float; };
template <>
struct VecOf<double, 2> { using type = double2; };
template <>
struct VecOf<double, 1> { using type = double; };

// Loads of vectors that the same kernel rewrites between grid barriers go
// through L2 (ld.global.cg): L1 is not coherent across SMs, and a load
// through a const __restrict__ pointer may otherwise become ld.global.nc.
template <typename T, int VW>
__device__ __forceinline__ Pack<T, VW> ldp(const T* p) {
  using V = typename VecOf<T, VW>::type;
  union {
    V v;
    Pack<T, VW> pk;
  } u;
  u.v = __ldcg(reinterpret_cast<const V*>(p));
  return u.pk;
}

template <typename T, int VW>
__device__ __forceinline__ void stp(T* p, const Pack<T, VW>& x) {
  *reinterpret_cast<Pack<T, VW>*>(p) = x;
}

// L2 eviction-priority policies (PTX createpolicy): vectors that later phases
// gather are kept (evict_last); streamed vectors are evicted first.
__device__ __forceinline__ uint64_t policy_keep() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_stream() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// Vector loads used inside the persistent kernels. WL_GATHER_LOAD selects the
// form: 0 = ld.global.cg (L2 only), 1 = default ld.global (L1 allocating;
// coherent across the grid barriers, whose gpu-scope acquire fence orders
// them after the other CTAs' writes), 2 = ld.global.cg with an L2
// eviction-priority policy.
#ifndef WL_GATHER_LOAD
#define WL_GATHER_LOAD 1
#endif

template <typename T, int VW>
__device__ __forceinline__ Pack<T, VW> ldh_asm(const T* p, uint64_t pol);

template <typename T, int VW>
__device__ __forceinline__ Pack<T, VW> ldh(const T* p, uint64_t pol) {
#if WL_GATHER_LOAD == 2
  return ldh_asm<T, VW>(p, pol);
#elif WL_GATHER_LOAD == 1
  (void)pol;
  return *reinterpret_cast<const Pack<T, VW>*>(p);
#else
  (void)pol;
  return ldp<T, VW>(p);
#endif
}

template <>
__device__ __forceinline__ Pack<float, 4> ldh_asm<float, 4>(const float* p, uint64_t pol) {
  Pack<float, 4> r;
  asm volatile("ld.global.cg.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
               : "=f"(r.v[0]), "=f"(r.v[1]), "=f"(r.v[2]), "=f"(r.v[3]) : "l"(p), "l"(pol));
  return r;
}
template <>
__device__ __forceinline__ Pack<float, 2> ldh_asm<float, 2>(const float* p, uint64_t pol) {
  Pack<float, 2> r;
  asm volatile("ld.global.cg.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(r.v[0]), "=f"(r.v[1]) : "l"(p), "l"(pol));
  return r;
}
template <>
__device__ __forceinline__ Pack<float, 1> ldh_asm<float, 1>(const float* p, uint64_t pol) {
  Pack<float, 1> r;
  asm volatile("ld.global.cg.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(r.v[0]) : "l"(p), "l"(pol));
  return r;
}
template <>
__device__ __forceinline__ Pack<double, 2> ldh_asm<double, 2>(const double* p, uint64_t pol) {
  Pack<double, 2> r;
  asm volatile("ld.global.cg.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;" : "=d"(r.v[0]), "=d"(r.v[1]) : "l"(p), "l"(pol));
  return r;
}
template <>
__device__ __forceinline__ Pack<double, 1> ldh_asm<double, 1>(const double* p, uint64_t pol) {
  Pack<double, 1> r;
  asm volatile("ld.global.cg.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(r.v[0]) : "l"(p), "l"(pol));
  return r;
}
template <typename T, int VW>
__device__ __forceinline__ void sth_asm(T* p, const Pack<T, VW>& x, uint64_t pol);

template <>
__device__ __forceinline__ void sth_asm<float, 4>(float* p, const Pack<float, 4>& x, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(x.v[0]), "f"(x.v[1]),
               "f"(x.v[2]), "f"(x.v[3]), "l"(pol) : "memory");
}
template <>
__device__ __forceinline__ void sth_asm<float, 2>(float* p, const Pack<float, 2>& x, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(p), "f"(x.v[0]), "f"(x.v[1]), "l"(pol)
               : "memory");
}
template <>
__device__ __forceinline__ void sth_asm<float, 1>(float* p, const Pack<float, 1>& x, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(x.v[0]), "l"(pol) : "memory");
}
template <>
__device__ __forceinline__ void sth_asm<double, 2>(double* p, const Pack<double, 2>& x, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v2.f64 [%0], {%1, %2}, %3;" ::"l"(p), "d"(x.v[0]), "d"(x.v[1]), "l"(pol)
               : "memory");
}
template <>
__device__ __forceinline__ void sth_asm<double, 1>(double* p, const Pack<double, 1>& x, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(p), "d"(x.v[0]), "l"(pol) : "memory");
}

template <typename T, int VW>
__device__ __forceinline__ void sth(T* p, const Pack<T, VW>& x, uint64_t pol) {
#if WL_GATHER_LOAD == 2
  sth_asm<T, VW>(p, x, pol);
#else
  (void)pol;
  stp<T, VW>(p, x);
#endif
}

// ------------------------------------------------------------------ partition view
struct Part {
  const int32_t* rb;     // G + 1 row boundaries
  const int32_t* seg;    // 4 G: [C start, W start, S start, end) offsets into order
  const int4* meta;      // n entries {row, row_ptr[row], row_ptr[row + 1], 0} in class order
};

struct Graph {
  const int32_t* row_ptr;
  const int32_t* col;
  int64_t n;
  int64_t nnz;
};

// ------------------------------------------------------------------ gathers
// Index loads of a batch are issued first (one per lane, coalesced when lanes
// read consecutive entries) and broadcast with shuffles, so every gather of
// the batch is an independent 16-byte load in flight. Gathered vectors use
// the keep (evict_last) L2 policy.
constexpr int kGatherInFlight = 8;  // vector gathers issued back to back per lane

template <typename T, int VW>
__device__ __forceinline__ void add_pack(T (&acc)[VW], const Pack<T, VW>& a) {
#pragma unroll
  for (int v = 0; v < VW; ++v) acc[v] += a.v[v];
}

template <int G, int BATCH>
__device__ __forceinline__ void load_idx(const int32_t* __restrict__ col, int e0, int end, int sl, int (&idx)[BATCH]) {
#pragma unroll
  for (int u = 0; u < BATCH; ++u) {
    const int p = e0 + u * G + sl;
    idx[u] = (p < end) ? __ldg(col + p) : -1;
  }
}

// Gathers for the G * BATCH entries whose indices the subgroup holds in idx.
template <typename T, int K, int VW, int G, int BATCH>
__device__ __forceinline__ void gather_idx_sub(const int (&idx)[BATCH], const T* X, int lane_off, unsigned sm,
                                               uint64_t pol, T (&acc)[VW]) {
  constexpr int CH = G < kGatherInFlight ? G : kGatherInFlight;
#pragma unroll
  for (int u = 0; u < BATCH; ++u) {
#pragma unroll
    for (int s0 = 0; s0 < G; s0 += CH) {
      Pack<T, VW> val[CH];
      int jj[CH];
#pragma unroll
      for (int s = 0; s < CH; ++s) {
        const int j = (G == 1) ? idx[u] : __shfl_sync(sm, idx[u], s0 + s, G);
        jj[s] = j;
        if (j >= 0) val[s] = ldh<T, VW>(X + (size_t)j * K + lane_off, pol);  // predicated: no load past the row
      }
#pragma unroll
      for (int s = 0; s < CH; ++s)
        if (jj[s] >= 0) add_pack<T, VW>(acc, val[s]);
    }
  }
}

// A whole warp sums entries of one row (32 indices per coalesced load);
// subgroup w = lane / G takes batch entries w, w + SUB, w + 2 SUB, ...
// Batches start at beg + 32 * first with stride 32 * step.
template <typename T, int K, int VW, int G>
__device__ __forceinline__ void gather_row_warp(const int32_t* __restrict__ col, int beg, int end, int first,
                                                int step, const T* X, int lane, int lane_off, uint64_t pol,
                                                T (&acc)[VW]) {
  constexpr int SUB = 32 / G;
  constexpr int CH = G < kGatherInFlight ? G : kGatherInFlight;
  const int w = lane / G;
  int e0 = beg + 32 * first;
  int idx = (e0 + lane < end) ? __ldg(col + e0 + lane) : -1;
  for (; e0 < end; e0 += 32 * step) {
    const int e1 = e0 + 32 * step;  // next batch's indices in flight during this batch's gathers
    const int idx_next = (e1 + lane < end) ? __ldg(col + e1 + lane) : -1;
#pragma unroll
    for (int t0 = 0; t0 < G; t0 += CH) {
      Pack<T, VW> val[CH];
      int jj[CH];
#pragma unroll
      for (int t = 0; t < CH; ++t) {
        const int j = __shfl_sync(0xffffffffu, idx, w + SUB * (t0 + t));
        jj[t] = j;
        if (j >= 0) val[t] = ldh<T, VW>(X + (size_t)j * K + lane_off, pol);
      }
#pragma unroll
      for (int t = 0; t < CH; ++t)
        if (jj[t] >= 0) add_pack<T, VW>(acc, val[t]);
    }
    idx = idx_next;
  }
}

// Visit every row of this CTA's partition. For each row exactly one subgroup
// (lanes sl = 0..G-1) runs pv = pre(row, lane_off) before the row's gathers
// (own-row loads overlap them) and fin(row, deg, lane_off, nbr_sum, pv)
// after, with nbr_sum[v] = sum over neighbours j of X[j, lane_off + v].
// Short rows (class S) are software-pipelined: metadata two rows ahead and
// indices one row ahead are in flight while a row is gathered. `red` holds
// kBlock * VW values of T in shared memory.
template <typename T, int K, class Pre, class Fin>
__device__ __forceinline__ void for_rows_gather(const Graph& g, const Part& pt, const T* X, T* red, Pre& pre,
                                                Fin& fin) {
  using C = Cfg<T, K>;
  using PV = decltype(pre(0, 0));
  constexpr int VW = C::VW;
  constexpr int G = C::G;
  constexpr int NW = kBlock / 32;
  constexpr int NSUB = C::NSUB;
  const int cta = blockIdx.x;
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int sub = tid / G;  // subgroup id in CTA
  const int sl = tid % G;   // lane in subgroup
  const int lane_off = sl * VW;
  const int c0 = pt.seg[4 * cta + 0], c1 = pt.seg[4 * cta + 1];
  const int c3 = pt.seg[4 * cta + 3];
  const uint64_t keep = policy_keep();

  // class C: whole CTA per row (warp w takes 32-entry batches w, w + NW, ...)
  for (int o = c0; o < c1; ++o) {
    const int4 m = pt.meta[o];
    PV pv;
    if (tid < G) pv = pre(m.x, lane_off);
    T acc[VW];
#pragma unroll
    for (int v = 0; v < VW; ++v) acc[v] = T(0);
    gather_row_warp<T, K, VW, G>(g.col, m.y, m.z, warp, NW, X, lane, lane_off, keep, acc);
#pragma unroll
    for (int off = G; off < 32; off <<= 1)
#pragma unroll
      for (int v = 0; v < VW; ++v) acc[v] += __shfl_xor_sync(0xffffffffu, acc[v], off);
    if (lane < G)
#pragma unroll
      for (int v = 0; v < VW; ++v) red[(warp * G + lane) * VW + v] = acc[v];
    __syncthreads();
    if (tid < G) {
      for (int w = 1; w < NW; ++w)
#pragma unroll
        for (int v = 0; v < VW; ++v) acc[v] += red[(w * G + sl) * VW + v];
      fin(m.x, m.z - m.y, lane_off, acc, pv);
    }
    __syncthreads();
  }
  // rows with at most Tc entries: one subgroup per row, rows in decreasing
  // degree order, as one flat loop over index batches of E entries; the next
  // batch's indices (same row or the next row's first) and the metadata of
  // the row after next are in flight while a batch is gathered.
  constexpr int BS = C::BS, E = C::E;
  const unsigned smask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
  const int4 none = make_int4(-1, 0, 0, 0);
  int o = c1 + sub;  // class W is empty: Tw == Tc
  int4 mc = (o < c3) ? pt.meta[o] : none;
  int4 mn = (o + NSUB < c3) ? pt.meta[o + NSUB] : none;
  int e = mc.y;
  int ic[BS];
  load_idx<G, BS>(g.col, e, mc.z, sl, ic);
  PV pv;
  if (o < c3) pv = pre(mc.x, lane_off);
  T acc[VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) acc[v] = T(0);
  while (o < c3) {
    const int e_next = e + E;
    const bool same = e_next < mc.z;
    int4 mnn = none;
    if (!same && o + 2 * NSUB < c3) mnn = pt.meta[o + 2 * NSUB];
    int in_[BS];
    if (same)
      load_idx<G, BS>(g.col, e_next, mc.z, sl, in_);
    else
      load_idx<G, BS>(g.col, mn.y, mn.z, sl, in_);
    gather_idx_sub<T, K, VW, G, BS>(ic, X, lane_off, smask, keep, acc);
    if (!same) {
      fin(mc.x, mc.z - mc.y, lane_off, acc, pv);
#pragma unroll
      for (int v = 0; v < VW; ++v) acc[v] = T(0);
      o += NSUB;
      mc = mn;
      mn = mnn;
      if (o < c3) pv = pre(mc.x, lane_off);
      e = mc.y;
    } else {
      e = e_next;
    }
#pragma unroll
    for (int u = 0; u < BS; ++u) ic[u] = in_[u];
  }
}

// Deterministic reduction of per-CTA partials part[g * K + c] (g < G) to
// out[c] (shared memory, double). Every CTA obtains bit-identical results.
template <int K>
__device__ __forceinline__ void reduce_partials(const double* __restrict__ part, int G, double* s_tmp,
                                                double* out) {
  constexpr int J = kBlock / K;  // chunks per column
  const int tid = threadIdx.x;
  const int c = tid % K, j = tid / K;
  double s = 0.0;
  int g = j;
  for (; g + 7 * J < G; g += 8 * J) {  // 8 independent loads, summed in a fixed order
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = __ldcg(part + (size_t)(g + u * J) * K + c);
#pragma unroll
    for (int u = 0; u < 8; ++u) s += v[u];
  }
  for (; g < G; g += J) s += __ldcg(part + (size_t)g * K + c);
  s_tmp[tid] = s;
  __syncthreads();
  if (tid < K) {
    double t = 0.0;
    for (int jj = 0; jj < J; ++jj) t += s_tmp[jj * K + tid];
    out[tid] = t;
  }
  __syncthreads();
}

// Per-thread column partials -> per-CTA column sums. Thread t owns columns
// (t % G) * VW + v, v < VW, in both the gather layout (subgroup lane sl =
// t % G) and the elementwise layout (vector index t + i * kBlock, since
// kBlock * VW is a multiple of K). Sums lanes of equal t % G by a fixed
// shuffle tree, then warps in order: deterministic. s_w holds
// (kBlock / 32) * K doubles; dst (K values, shared or global) is written by
// threads c < K.
template <typename T, int K>
__device__ __forceinline__ void cta_column_sums(const T (&val)[Cfg<T, K>::VW], double* s_w, double* dst) {
  using C = Cfg<T, K>;
  constexpr int VW = C::VW, G = C::G, NW = kBlock / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double a[VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) a[v] = (double)val[v];
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

}  // namespace wl
