// Graph preparation and small elementwise kernels of libwl.so:
// nnz-balanced row partition, per-CTA degree-class ordering, CSR validation
// (Sec. 2: simple graph = symmetric, loop-free 0/1 pattern), block packing
// and the apply epilogue W = D_f (.) V - phi V (Eq. weighted_laplacian).
#include "wl_host.h"

namespace wl {

// rb[g] = first row i with row_ptr[i] + kRowCost * i >= g * total / G
__global__ void k_partition_bounds(const int32_t* row_ptr, int64_t n, int G, int32_t* rb) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g > G) return;
  if (g == 0) { rb[0] = 0; return; }
  if (g == G) { rb[G] = (int32_t)n; return; }
  const double total = (double)row_ptr[n] + (double)kRowCost * (double)n;
  const double target = total * (double)g / (double)G;
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    const double c = (double)row_ptr[mid] + (double)kRowCost * (double)mid;
    if (c < target) lo = mid + 1; else hi = mid;
  }
  rb[g] = (int32_t)lo;
}

// One CTA per partition; one warp scatters the partition's rows into
// order[] by class C (deg > Tc), W (Tw < deg <= Tc), then S by decreasing
// degree. Stable (row id order within a bucket) and deterministic.
constexpr int kOrderBuckets = 1030;  // 0: C, 1: W, 2 + (Tw - deg): S, Tw <= 1027

__global__ void k_order(const int32_t* row_ptr, const int32_t* rb, int Tw, int Tc, int4* meta, int32_t* seg) {
  __shared__ int hist[kOrderBuckets];
  __shared__ int cur[kOrderBuckets];
  const int g = blockIdx.x, tid = threadIdx.x;
  const int r0 = rb[g], r1 = rb[g + 1];
  for (int i = tid; i < kOrderBuckets; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  auto bucket = [&](int row) {
    const int d = row_ptr[row + 1] - row_ptr[row];
    if (d > Tc) return 0;
    if (d > Tw) return 1;
    return 2 + (Tw - d);
  };
  for (int i = r0 + tid; i < r1; i += blockDim.x) atomicAdd(&hist[bucket(i)], 1);
  __syncthreads();
  if (tid == 0) {
    int run = r0;
    for (int b = 0; b < kOrderBuckets; ++b) {
      cur[b] = run;
      run += hist[b];
    }
    seg[4 * g + 0] = r0;
    seg[4 * g + 1] = r0 + hist[0];
    seg[4 * g + 2] = r0 + hist[0] + hist[1];
    seg[4 * g + 3] = r1;
  }
  __syncthreads();
  if (tid < 32) {
    const int lane = tid;
    for (int base = r0; base < r1; base += 32) {
      const int row = base + lane;
      const bool valid = row < r1;
      const int b = valid ? bucket(row) : -1;
      const unsigned act = __ballot_sync(0xffffffffu, valid);
      const unsigned peers = __match_any_sync(0xffffffffu, b) & act;
      const int rank = __popc(peers & ((1u << lane) - 1u));
      const int leader = __ffs(peers) - 1;
      int basepos = 0;
      if (valid && lane == leader) basepos = cur[b];
      basepos = __shfl_sync(0xffffffffu, basepos, valid ? leader : lane);
      if (valid) meta[basepos + rank] = make_int4(row, row_ptr[row], row_ptr[row + 1], 0);
      __syncwarp();
      if (valid && lane == leader) cur[b] += __popc(peers);
      __syncwarp();
    }
  }
}

cudaError_t launch_partition(const Graph& g, PartDev& p, cudaStream_t s) {
  if (p.Tw > kOrderBuckets - 3) return cudaErrorInvalidValue;
  k_partition_bounds<<<(p.G + 1 + 255) / 256, 256, 0, s>>>(g.row_ptr, g.n, p.G, p.rb);
  k_order<<<p.G, 256, 0, s>>>(g.row_ptr, p.rb, p.Tw, p.Tc, p.meta, p.seg);
  return cudaGetLastError();
}

// One warp per row: row_ptr monotone and within [0, nnz], columns strictly
// increasing in range, no self-loop, and (i, j) stored implies (j, i) stored
// (binary search in row j).
__global__ void k_validate(const int32_t* row_ptr, const int32_t* col, int64_t n, int64_t nnz, int* flags) {
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < n; i += nwarps) {
    const int64_t beg = row_ptr[i], end = row_ptr[i + 1];
    int f = 0;
    if (beg < 0 || end < beg || end > nnz) {
      if (lane == 0) atomicOr(flags, 1);
      continue;
    }
    for (int64_t e = beg + lane; e < end; e += 32) {
      const int32_t j = col[e];
      if (j < 0 || j >= n) { f |= 2; continue; }
      if (e > beg && col[e - 1] >= j) f |= 2;
      if (j == i) { f |= 4; continue; }
      int64_t lo = row_ptr[j], hi = row_ptr[j + 1] - 1;
      bool found = false;
      if (lo < 0 || hi >= nnz) { f |= 1; continue; }
      while (lo <= hi) {
        const int64_t mid = (lo + hi) >> 1;
        const int32_t v = col[mid];
        if (v == i) { found = true; break; }
        if (v < i) lo = mid + 1; else hi = mid - 1;
      }
      if (!found) f |= 8;
    }
    if (f) atomicOr(flags, f);
  }
}

__global__ void k_check_ends(const int32_t* row_ptr, int64_t n, int64_t nnz, int* flags) {
  if (row_ptr[0] != 0 || (int64_t)row_ptr[n] != nnz) atomicOr(flags, 1);
}

cudaError_t launch_validate(const Graph& g, int* flags, cudaStream_t s) {
  k_check_ends<<<1, 1, 0, s>>>(g.row_ptr, g.n, g.nnz, flags);
  if (g.n > 0) {
    const int64_t warps = g.n < 152 * 64 ? g.n : 152 * 64;
    k_validate<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(g.row_ptr, g.col, g.n, g.nnz, flags);
  }
  return cudaGetLastError();
}

template <typename T>
__global__ void k_pack(const double* src, int64_t ld, int c0, int kb, int64_t n, double scale, T* dst) {
  const int64_t total = n * kb;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / kb;
    const int c = (int)(e % kb);
    dst[e] = (T)(scale * src[i * ld + c0 + c]);
  }
}

static unsigned grid_for(int64_t total) {
  int64_t b = (total + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  if (b < 1) b = 1;
  return (unsigned)b;
}

cudaError_t launch_pack(const double* src, int64_t ld, int c0, int kb, int64_t n, double scale, void* dst,
                        bool to_f32, cudaStream_t s) {
  const unsigned gb = grid_for(n * kb);
  if (to_f32)
    k_pack<float><<<gb, 256, 0, s>>>(src, ld, c0, kb, n, scale, (float*)dst);
  else
    k_pack<double><<<gb, 256, 0, s>>>(src, ld, c0, kb, n, scale, (double*)dst);
  return cudaGetLastError();
}

__global__ void k_apply_out(const double* V, int64_t ldv, const double* X, const double* Df, int64_t n, int K, int c0,
                            double* W, int64_t ldw) {
  const int64_t total = n * K;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / K;
    const int c = (int)(e % K);
    W[i * ldw + c0 + c] = Df[i] * V[i * ldv + c0 + c] - X[e];
  }
}

cudaError_t launch_apply_out(const double* V, int64_t ldv, const double* X, const double* Df, int64_t n, int K,
                             int c0, double* W, int64_t ldw, cudaStream_t s) {
  k_apply_out<<<grid_for(n * K), 256, 0, s>>>(V, ldv, X, Df, n, K, c0, W, ldw);
  return cudaGetLastError();
}

__global__ void k_fill(double* dst, double v, int64_t count) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = v;
}

cudaError_t launch_fill(double* dst, double v, int64_t count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_fill<<<grid_for(count), 256, 0, s>>>(dst, v, count);
  return cudaGetLastError();
}

__global__ void k_degree_vector(const int32_t* row_ptr, int64_t n, double* out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (double)(row_ptr[i + 1] - row_ptr[i]);
}

cudaError_t launch_degree_vector(const Graph& g, double* out, cudaStream_t s) {
  if (g.n <= 0) return cudaSuccess;
  k_degree_vector<<<grid_for(g.n), 256, 0, s>>>(g.row_ptr, g.n, out);
  return cudaGetLastError();
}

// column norms of a contiguous n x K block: one CTA per column, fixed-order tree
__global__ void k_colnorms(const double* X, int64_t n, int K, double* out) {
  __shared__ double red[256];
  const int c = blockIdx.x;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += 256) {
    const double x = X[i * K + c];
    s += x * x;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = sqrt(red[0]);
}

cudaError_t launch_colnorms(const double* X, int64_t n, int K, double* out, cudaStream_t s) {
  k_colnorms<<<K, 256, 0, s>>>(X, n, K, out);
  return cudaGetLastError();
}

__global__ void k_scale_cols(const double* X, int64_t n, int K, const double* nrm, double* Y) {
  const int64_t total = n * K;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const double v = nrm[e % K];
    Y[e] = v > 0.0 ? X[e] / v : 0.0;
  }
}

cudaError_t launch_scale_cols(const double* X, int64_t n, int K, const double* nrm, double* Y, cudaStream_t s) {
  k_scale_cols<<<grid_for(n * K), 256, 0, s>>>(X, n, K, nrm, Y);
  return cudaGetLastError();
}

__global__ void k_f2d_acc(const float* src, double* dst, int64_t count) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] += (double)src[e];
}

cudaError_t launch_f2d_acc(const float* src, double* dst, int64_t count, cudaStream_t s) {
  k_f2d_acc<<<grid_for(count), 256, 0, s>>>(src, dst, count);
  return cudaGetLastError();
}

// W[:, c0:c0+K] = d (.) V - A V (identity function: L = D - A, Sec. 3.1)
template <int K>
__global__ void __launch_bounds__(kBlock) k_laplacian_apply(Graph g, Part pt, const double* Vp, int c0, double* W,
                                                            int64_t ldw) {
  using C = Cfg<double, K>;
  constexpr int VW = C::VW;
  __shared__ __align__(16) double s_gath[kBlock * VW];
  auto pre = [&](int row, int lane_off) { return ldp<double, VW>(Vp + (size_t)row * K + lane_off); };
  auto fin = [&](int row, int deg, int lane_off, const double (&nb)[VW], const Pack<double, VW>& vv) {
#pragma unroll
    for (int v = 0; v < VW; ++v) W[(size_t)row * ldw + c0 + lane_off + v] = (double)deg * vv.v[v] - nb[v];
  };
  for_rows_gather<double, K>(g, pt, Vp, s_gath, pre, fin);
}

cudaError_t launch_laplacian_apply(const Graph& g, const PartDev& p, const double* Vp, int K, int c0, double* W,
                                   int64_t ldw, cudaStream_t s) {
  const Part pt = p.view();
  switch (K) {
    case 1: k_laplacian_apply<1><<<p.G, kBlock, 0, s>>>(g, pt, Vp, c0, W, ldw); break;
    case 2: k_laplacian_apply<2><<<p.G, kBlock, 0, s>>>(g, pt, Vp, c0, W, ldw); break;
    case 4: k_laplacian_apply<4><<<p.G, kBlock, 0, s>>>(g, pt, Vp, c0, W, ldw); break;
    case 8: k_laplacian_apply<8><<<p.G, kBlock, 0, s>>>(g, pt, Vp, c0, W, ldw); break;
    case 16: k_laplacian_apply<16><<<p.G, kBlock, 0, s>>>(g, pt, Vp, c0, W, ldw); break;
    case 32: k_laplacian_apply<32><<<p.G, kBlock, 0, s>>>(g, pt, Vp, c0, W, ldw); break;
    case 64: k_laplacian_apply<64><<<p.G, kBlock, 0, s>>>(g, pt, Vp, c0, W, ldw); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace wl
