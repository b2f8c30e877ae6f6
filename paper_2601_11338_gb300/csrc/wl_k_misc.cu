// Graph preparation and small elementwise kernels of libwl.so:
// nnz-balanced row partition, per-CTA degree-class ordering, CSR validation
// (Sec. 2: simple graph = symmetric, loop-free 0/1 pattern), block packing
// and the apply epilogue W = D_f (.) V - phi V (Eq. weighted_laplacian).
#include <algorithm>

#include "wl_host.h"

namespace wl {

// One CTA in the bounded grid barrier, expecting `nblocks` CTAs
__global__ void k_selftest_wait(GridBar* bar, unsigned nblocks) { (void)grid_sync(bar, nblocks); }

cudaError_t launch_selftest_wait(GridBar* bar, unsigned nblocks, cudaStream_t s) {
  k_selftest_wait<<<1, 32, 0, s>>>(bar, nblocks);
  return cudaGetLastError();
}

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
// Column 2-norms of X (n x K FP64, row-major; K a power of two <= 64): each
// CTA sums its share of the rows with all threads reading consecutive
// elements (thread t meets column t % K only, the grid stride being a multiple
// of K), writes its K partial sums, and a second kernel adds the partials in
// a fixed order (the same result on every run).
constexpr int kColnormBlocks = 304;

__global__ void k_colnorms_part(const double* X, int64_t n, int K, double* part) {
  __shared__ double red[256];
  const int64_t total = n * K;
  double s = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < total; e += (int64_t)gridDim.x * 256) {
    const double x = X[e];
    s += x * x;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x < K) {
    double t = 0.0;
    for (int i = threadIdx.x; i < 256; i += K) t += red[i];
    part[(size_t)blockIdx.x * K + threadIdx.x] = t;
  }
}

__global__ void k_colnorms_sum(const double* part, int G, int K, double* out) {
  const int c = threadIdx.x;
  if (c >= K) return;
  double t = 0.0;
  for (int g = 0; g < G; ++g) t += part[(size_t)g * K + c];
  out[c] = sqrt(t);
}

cudaError_t launch_colnorms(const double* X, int64_t n, int K, double* out, double* scratch, cudaStream_t s) {
  if (K < 1 || K > 64 || (K & (K - 1)) != 0) return cudaErrorInvalidValue;
  const int G = (int)std::max<int64_t>(1, std::min<int64_t>(kColnormBlocks, (n * K + 255) / 256));
  k_colnorms_part<<<G, 256, 0, s>>>(X, n, K, scratch);
  k_colnorms_sum<<<1, 64, 0, s>>>(scratch, G, K, out);
  return cudaGetLastError();
}

// Y = X scaled per column by 1 / nrm[c] (0 where nrm[c] = 0): one reciprocal
// per column and CTA, then a multiply per element (an FP64 division per
// element cost this GPU 0.7 ms for 1.6e7 elements)
__global__ void k_scale_cols(const double* X, int64_t n, int K, const double* nrm, double* Y) {
  __shared__ double inv[64];
  if (threadIdx.x < K) inv[threadIdx.x] = nrm[threadIdx.x] > 0.0 ? 1.0 / nrm[threadIdx.x] : 0.0;
  __syncthreads();
  const int64_t total = n * K;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    Y[e] = X[e] * inv[(int)(e & (int64_t)(K - 1))];
}

cudaError_t launch_scale_cols(const double* X, int64_t n, int K, const double* nrm, double* Y, cudaStream_t s) {
  if (K < 1 || K > 64 || (K & (K - 1)) != 0) return cudaErrorInvalidValue;
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

// ---- discrete-time chain P = D_f^{-1} phi (Sec. 3.3, with D = diag(phi 1)):
// one step in column form is p <- phi (p / D_f)
__global__ void k_row_div(const double* X, const double* Df, int64_t n, int K, double* Y) {
  const int64_t total = n * K;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const double d = Df[e / K];
    Y[e] = d > 0.0 ? X[e] / d : 0.0;
  }
}

cudaError_t launch_row_div(const double* X, const double* Df, int64_t n, int K, double* Y, cudaStream_t s) {
  k_row_div<<<grid_for(n * K), 256, 0, s>>>(X, Df, n, K, Y);
  return cudaGetLastError();
}

// Y = A X for n x K blocks (FP64, one thread per row and column)
__global__ void k_adj_apply(const int32_t* row_ptr, const int32_t* col, const double* X, int64_t n, int K, double* Y) {
  const int64_t total = n * K;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / K;
    const int c = (int)(e % K);
    double acc = 0.0;
    for (int j = row_ptr[i]; j < row_ptr[i + 1]; ++j) acc += X[(int64_t)col[j] * K + c];
    Y[e] = acc;
  }
}

cudaError_t launch_adj_apply(const Graph& g, const double* X, int K, double* Y, cudaStream_t s) {
  k_adj_apply<<<grid_for(g.n * K), 256, 0, s>>>(g.row_ptr, g.col, X, g.n, K, Y);
  return cudaGetLastError();
}

// dst[row(i) * ld + c0 + c] = src[i * K + c], row(i) = perm[i] (perm NULL: i)
__global__ void k_unpack(const double* src, int64_t n, int K, int c0, const int32_t* perm, double* dst, int64_t ld) {
  const int64_t total = n * K;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / K;
    const int c = (int)(e % K);
    dst[(perm ? (int64_t)perm[i] : i) * ld + c0 + c] = src[e];
  }
}

cudaError_t launch_unpack(const double* src, int64_t n, int K, int c0, const int32_t* perm, double* dst, int64_t ld,
                          cudaStream_t s) {
  k_unpack<<<grid_for(n * K), 256, 0, s>>>(src, n, K, c0, perm, dst, ld);
  return cudaGetLastError();
}

// W[:, c0:c0+K] = d (.) V - A V (identity function: L = D - A, Sec. 3.1)
template <int K>
__global__ void __launch_bounds__(kBlock) k_laplacian_apply(Graph g, Part pt, const double* Vp, int c0,
                                                            const int32_t* perm, double* W, int64_t ldw) {
  using C = Cfg<double, K>;
  constexpr int VW = C::VW;
  __shared__ __align__(16) double s_gath[kBlock * VW];
  auto pre = [&](int row, int lane_off) { return ldp<double, VW>(Vp + (size_t)row * K + lane_off); };
  auto fin = [&](int row, int deg, int lane_off, const double (&nb)[VW], const Pack<double, VW>& vv) {
#pragma unroll
    for (int v = 0; v < VW; ++v)
      W[(size_t)(perm ? perm[row] : row) * ldw + c0 + lane_off + v] = (double)deg * vv.v[v] - nb[v];
  };
  for_rows_gather<double, K>(g, pt, Vp, s_gath, pre, fin);
}

cudaError_t launch_laplacian_apply(const Graph& g, const PartDev& p, const double* Vp, int K, int c0,
                                   const int32_t* perm, double* W, int64_t ldw, cudaStream_t s) {
  const Part pt = p.view();
  switch (K) {
    case 1: k_laplacian_apply<1><<<p.G, kBlock, 0, s>>>(g, pt, Vp, c0, perm, W, ldw); break;
    case 2: k_laplacian_apply<2><<<p.G, kBlock, 0, s>>>(g, pt, Vp, c0, perm, W, ldw); break;
    case 4: k_laplacian_apply<4><<<p.G, kBlock, 0, s>>>(g, pt, Vp, c0, perm, W, ldw); break;
    case 8: k_laplacian_apply<8><<<p.G, kBlock, 0, s>>>(g, pt, Vp, c0, perm, W, ldw); break;
    case 16: k_laplacian_apply<16><<<p.G, kBlock, 0, s>>>(g, pt, Vp, c0, perm, W, ldw); break;
    case 32: k_laplacian_apply<32><<<p.G, kBlock, 0, s>>>(g, pt, Vp, c0, perm, W, ldw); break;
    case 64: k_laplacian_apply<64><<<p.G, kBlock, 0, s>>>(g, pt, Vp, c0, perm, W, ldw); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace wl

// ======================================================================
// Node relabelling by decreasing degree (optional at build): nodes of
// similar degree become contiguous, so the most gathered rows (the hubs and
// their peers) share cache lines and stay in L2. The relabelled CSR keeps
// the pattern P A P^T; every vector crossing the C ABI is permuted on the
// way in and out, so callers never see the internal order.
// ======================================================================
namespace wl {

constexpr int kScanBlock = 1024;

// exclusive scan of in[0..n) (int64) into out[0..n] (out[n] = total);
// two levels: per-block sums, then a single-CTA scan of the block sums.
__global__ void k_scan_blocks(const int64_t* in, int64_t n, int64_t* out, int64_t* bsum) {
  __shared__ int64_t s[kScanBlock];
  const int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
  s[threadIdx.x] = (i < n) ? in[i] : 0;
  __syncthreads();
  for (int off = 1; off < kScanBlock; off <<= 1) {
    const int64_t v = threadIdx.x >= off ? s[threadIdx.x - off] : 0;
    __syncthreads();
    s[threadIdx.x] += v;
    __syncthreads();
  }
  if (i < n) out[i] = s[threadIdx.x] - ((i < n) ? in[i] : 0);
  if (threadIdx.x == kScanBlock - 1) bsum[blockIdx.x] = s[threadIdx.x];
}

__global__ void k_scan_sums(int64_t* bsum, int64_t nb) {
  // one CTA, sequential chunks of kScanBlock
  __shared__ int64_t s[kScanBlock];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < nb; base += kScanBlock) {
    const int64_t i = base + threadIdx.x;
    const int64_t x = (i < nb) ? bsum[i] : 0;
    s[threadIdx.x] = x;
    __syncthreads();
    for (int off = 1; off < kScanBlock; off <<= 1) {
      const int64_t v = threadIdx.x >= off ? s[threadIdx.x - off] : 0;
      __syncthreads();
      s[threadIdx.x] += v;
      __syncthreads();
    }
    if (i < nb) bsum[i] = carry + s[threadIdx.x] - x;  // exclusive
    __syncthreads();
    if (threadIdx.x == kScanBlock - 1) carry += s[threadIdx.x];
    __syncthreads();
  }
  if (threadIdx.x == 0) bsum[nb] = carry;
}

__global__ void k_scan_add(int64_t* out, int64_t n, const int64_t* bsum) {
  const int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
  if (i < n) out[i] += bsum[blockIdx.x];
  if (i == 0) out[n] = bsum[gridDim.x];
}

cudaError_t launch_scan(const int64_t* in, int64_t n, int64_t* out, int64_t* tmp, cudaStream_t s) {
  const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
  if (n == 0) return cudaMemsetAsync(out, 0, sizeof(int64_t), s);
  k_scan_blocks<<<(unsigned)nb, kScanBlock, 0, s>>>(in, n, out, tmp);
  k_scan_sums<<<1, kScanBlock, 0, s>>>(tmp, nb);
  k_scan_add<<<(unsigned)nb, kScanBlock, 0, s>>>(out, n, tmp);
  return cudaGetLastError();
}

// ---- stable counting sort of nodes by key = 31 - floor(log2(deg + 1)) (hubs first)
constexpr int kSortChunk = 4096;
constexpr int kKeys = 32;

__device__ __forceinline__ int degree_key(const int32_t* row_ptr, int64_t i) {
  const int d = row_ptr[i + 1] - row_ptr[i];
  return 31 - (31 - __clz(d + 1));  // = __clz(d + 1): larger degree -> smaller key
}

// hist[key * nchunks + chunk]
__global__ void k_key_hist(const int32_t* row_ptr, int64_t n, int64_t* hist, int nchunks) {
  __shared__ int h[kKeys];
  if (threadIdx.x < kKeys) h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t b = (int64_t)blockIdx.x * kSortChunk;
  for (int64_t i = b + threadIdx.x; i < b + kSortChunk && i < n; i += blockDim.x)
    atomicAdd(&h[degree_key(row_ptr, i)], 1);
  __syncthreads();
  if (threadIdx.x < kKeys) hist[(int64_t)threadIdx.x * nchunks + blockIdx.x] = h[threadIdx.x];
}

// one warp per chunk scatters in row order (stable): perm[new] = old
__global__ void k_key_scatter(const int32_t* row_ptr, int64_t n, const int64_t* off, int nchunks, int32_t* perm) {
  __shared__ int64_t cur[kKeys];
  const int lane = threadIdx.x;
  if (lane < kKeys) cur[lane] = off[(int64_t)lane * nchunks + blockIdx.x];
  __syncwarp();
  const int64_t b = (int64_t)blockIdx.x * kSortChunk;
  for (int64_t base = b; base < b + kSortChunk && base < n; base += 32) {
    const int64_t i = base + lane;
    const bool valid = i < n && i < b + kSortChunk;
    const int key = valid ? degree_key(row_ptr, i) : -1;
    const unsigned act = __ballot_sync(0xffffffffu, valid);
    const unsigned peers = __match_any_sync(0xffffffffu, key) & act;
    const int rank = __popc(peers & ((1u << lane) - 1u));
    const int leader = __ffs(peers) - 1;
    int64_t pos = 0;
    if (valid && lane == leader) pos = cur[key];
    pos = __shfl_sync(0xffffffffu, pos, valid ? leader : lane);
    if (valid) perm[pos + rank] = (int32_t)i;
    __syncwarp();
    if (valid && lane == leader) cur[key] += __popc(peers);
    __syncwarp();
  }
}

__global__ void k_inverse_perm(const int32_t* perm, int64_t n, int32_t* iperm) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    iperm[perm[i]] = (int32_t)i;
}

__global__ void k_perm_degrees(const int32_t* row_ptr, const int32_t* perm, int64_t n, int64_t* deg) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t o = perm[i];
    deg[i] = row_ptr[o + 1] - row_ptr[o];
  }
}

__global__ void k_i64_to_i32(const int64_t* in, int64_t n, int32_t* out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (int32_t)in[i];
}

// warp per new row: copy the old row's neighbours mapped to new labels
__global__ void k_perm_cols(const int32_t* row_ptr, const int32_t* col, const int32_t* perm, const int32_t* iperm,
                            const int32_t* new_rp, int64_t n, int32_t* new_col) {
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < n; r += nw) {
    const int32_t o = perm[r];
    const int beg = row_ptr[o], end = row_ptr[o + 1], dst = new_rp[r];
    for (int e = beg + lane; e < end; e += 32) new_col[dst + (e - beg)] = iperm[col[e]];
  }
}

cudaError_t launch_relabel(const Graph& g, int32_t* perm, int32_t* iperm, int32_t* new_rp, int32_t* new_col,
                           int64_t* tmp_i64 /* 2 (n + 1) + 2 * 32 * chunks + 2 */, cudaStream_t s) {
  const int64_t n = g.n;
  if (n == 0) return cudaMemsetAsync(new_rp, 0, sizeof(int32_t), s);
  const int nch = (int)((n + kSortChunk - 1) / kSortChunk);
  int64_t* hist = tmp_i64;                           // 32 * nch (+1)
  int64_t* off = hist + (int64_t)kKeys * nch + 1;    // 32 * nch + 1
  int64_t* sc = off + (int64_t)kKeys * nch + 1;      // scan scratch
  k_key_hist<<<nch, 256, 0, s>>>(g.row_ptr, n, hist, nch);
  cudaError_t e = launch_scan(hist, (int64_t)kKeys * nch, off, sc, s);
  if (e != cudaSuccess) return e;
  k_key_scatter<<<nch, 32, 0, s>>>(g.row_ptr, n, off, nch, perm);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_relabel_apply(g, perm, iperm, new_rp, new_col, sc + (n / kScanBlock + 2), s);
}

// the relabelled CSR for a given perm[new] = old: iperm, new row pointers
// (prefix sum of the permuted degrees) and new column labels
cudaError_t launch_relabel_apply(const Graph& g, const int32_t* perm, int32_t* iperm, int32_t* new_rp,
                                 int32_t* new_col, int64_t* tmp_i64 /* 2 (n + 1) + n / kScanBlock + 4 */,
                                 cudaStream_t s) {
  const int64_t n = g.n;
  if (n == 0) return cudaMemsetAsync(new_rp, 0, sizeof(int32_t), s);
  const unsigned gb = (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 32);
  k_inverse_perm<<<gb, 256, 0, s>>>(perm, n, iperm);
  int64_t* deg = tmp_i64;                     // n
  int64_t* rp64 = deg + n;                    // n + 1
  int64_t* sc2 = rp64 + n + 1;
  k_perm_degrees<<<gb, 256, 0, s>>>(g.row_ptr, perm, n, deg);
  cudaError_t e = launch_scan(deg, n, rp64, sc2, s);
  if (e != cudaSuccess) return e;
  k_i64_to_i32<<<gb, 256, 0, s>>>(rp64, n, new_rp);
  const int64_t warps = std::min<int64_t>(n, 152 * 64);
  k_perm_cols<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(g.row_ptr, g.col, perm, iperm, new_rp, n, new_col);
  return cudaGetLastError();
}

size_t relabel_tmp_i64(int64_t n) {
  const int64_t nch = (n + kSortChunk - 1) / kSortChunk;
  return (size_t)(2 * (kKeys * nch + 1) + (kKeys * nch) / kScanBlock + 2 + (n / kScanBlock + 2) + n + (n + 1) +
                  n / kScanBlock + 4);
}

// ---- cost-weighted partition, in bytes moved per CG iteration:
// cost(row) = row_bytes + deg * entry_bytes, with hub rows (deg > Tc,
// gathered by the whole CTA in a latency-bound chain) counted three times.
__global__ void k_row_cost(const int32_t* row_ptr, int64_t n, int Tc, int row_bytes, int entry_bytes,
                           int64_t* cost) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t d = row_ptr[i + 1] - row_ptr[i];
    cost[i] = (int64_t)row_bytes + (d > Tc ? 3 : 1) * d * (int64_t)entry_bytes;
  }
}

__global__ void k_partition_prefix(const int64_t* prefix, int64_t n, int G, int32_t* rb) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g > G) return;
  if (g == 0) { rb[0] = 0; return; }
  if (g == G) { rb[G] = (int32_t)n; return; }
  const double target = (double)prefix[n] * (double)g / (double)G;
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if ((double)prefix[mid] < target) lo = mid + 1; else hi = mid;
  }
  rb[g] = (int32_t)lo;
}

cudaError_t launch_partition_weighted(const Graph& g, PartDev& p, int64_t* tmp /* 2 (n + 1) + n / 1024 + 4 */,
                                      cudaStream_t s) {
  const int64_t n = g.n;
  if (p.Tw > kOrderBuckets - 3) return cudaErrorInvalidValue;
  int64_t* cost = tmp;
  int64_t* prefix = cost + n + 1;
  int64_t* sc = prefix + n + 1;
  const unsigned gb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 32));
  k_row_cost<<<gb, 256, 0, s>>>(g.row_ptr, n, p.Tc, p.row_bytes, p.entry_bytes, cost);
  cudaError_t e = launch_scan(cost, n, prefix, sc, s);
  if (e != cudaSuccess) return e;
  k_partition_prefix<<<(p.G + 1 + 255) / 256, 256, 0, s>>>(prefix, n, p.G, p.rb);
  k_order<<<p.G, 256, 0, s>>>(g.row_ptr, p.rb, p.Tw, p.Tc, p.meta, p.seg);
  return cudaGetLastError();
}

// ---- permuted copies across the API boundary
// dst[new * K + c] = scale * src[perm[new] * ld + c0 + c]
__global__ void k_pack_perm(const double* src, int64_t ld, int c0, int kb, int64_t n, double scale,
                            const int32_t* perm, double* dst) {
  const int64_t total = n * kb;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / kb;
    const int c = (int)(e % kb);
    dst[e] = scale * src[(int64_t)perm[i] * ld + c0 + c];
  }
}

// W[perm[i] * ldw + c0 + c] = Df[i] * Vp[i * K + c] - X[i * K + c]
__global__ void k_apply_out_perm(const double* Vp, const double* X, const double* Df, int64_t n, int K, int c0,
                                 const int32_t* perm, double* W, int64_t ldw) {
  const int64_t total = n * K;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / K;
    const int c = (int)(e % K);
    W[(int64_t)perm[i] * ldw + c0 + c] = Df[i] * Vp[e] - X[e];
  }
}

// out[perm[i]] = in[i] (scatter to caller order) or out[i] = in[perm[i]] (gather)
__global__ void k_permute_vec(const double* in, int64_t n, const int32_t* perm, int scatter, double* out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (scatter) out[perm[i]] = in[i]; else out[i] = in[perm[i]];
  }
}

cudaError_t launch_pack_perm(const double* src, int64_t ld, int c0, int kb, int64_t n, double scale,
                             const int32_t* perm, double* dst, cudaStream_t s) {
  k_pack_perm<<<grid_for(n * kb), 256, 0, s>>>(src, ld, c0, kb, n, scale, perm, dst);
  return cudaGetLastError();
}

cudaError_t launch_apply_out_perm(const double* Vp, const double* X, const double* Df, int64_t n, int K, int c0,
                                  const int32_t* perm, double* W, int64_t ldw, cudaStream_t s) {
  k_apply_out_perm<<<grid_for(n * K), 256, 0, s>>>(Vp, X, Df, n, K, c0, perm, W, ldw);
  return cudaGetLastError();
}

cudaError_t launch_permute_vec(const double* in, int64_t n, const int32_t* perm, bool scatter, double* out,
                               cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_permute_vec<<<grid_for(n), 256, 0, s>>>(in, n, perm, scatter ? 1 : 0, out);
  return cudaGetLastError();
}

}  // namespace wl
