// wl_degrees_noalloc: walk degrees D_f for callers that cannot allocate GPU
// memory.
//
// Some callers cannot call cudaMalloc at the point where they need walk
// degrees: code running inside a framework whose memory planner forbids
// allocation during its own execution step, real-time or embedded hosts
// that reserve all device memory up front, and plug-ins that only receive
// pre-allocated input and output buffers. This entry point takes the graph
// and the output buffer from the caller and keeps every intermediate vector
// in one fixed array compiled into the library, so it calls no cudaMalloc,
// no cudaFree and no allocating library routine.
//
// The array lives in device memory from the moment the library is loaded on
// a GPU until the process exits (every GPU that loads libwl.so holds it).
// Its host-side name is only a stand-in for the symbol, not a device
// address: the first call on each device resolves the address with
// cudaGetSymbolAddress while that device is current and caches it; later
// calls on that device reuse it.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>

#include "wl.h"
#include "wl_cg2.cuh"
#include "wl_host.h"

namespace wl {
namespace {

// Size limits of the fixed scratch array.
constexpr int64_t kNaMaxN = 1 << 18;          // nodes
constexpr int64_t kNaMaxGrid = 4096;          // CTAs of any one kernel (partials)
constexpr int kNaMaxDevices = 64;

// Layout (in doubles unless noted):
//   r, p, q    3 * kNaMaxN          CG vectors (x is the caller's output)
//   part       2 * (kNaMaxGrid + kNaMaxN)  per-CTA partial sums
//   state      CgState
//   hubs       kNaMaxN int32        rows with more than kHubDeg entries
//   misc       64 int32             flags and counters
constexpr size_t kNaVecBytes = 3 * kNaMaxN * sizeof(double);
constexpr size_t kNaPartBytes = 2 * (kNaMaxGrid + kNaMaxN) * sizeof(double);
constexpr size_t kNaStateBytes = ((sizeof(CgState) + 255) / 256) * 256;
constexpr size_t kNaHubBytes = kNaMaxN * sizeof(int32_t);
constexpr size_t kNaMiscBytes = 256;
constexpr size_t kNaBytes = kNaVecBytes + kNaPartBytes + kNaStateBytes + kNaHubBytes + kNaMiscBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

unsigned char* g_scratch_addr[kNaMaxDevices] = {nullptr};

// Resolve (once per device, with that device current) the device address of
// the scratch array.
int scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return WL_ERR_CUDA;
  if (dev < 0 || dev >= kNaMaxDevices) return WL_ERR_INVALID_ARG;
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      (void)cudaGetLastError();
      return WL_ERR_CUDA;
    }
    g_scratch_addr[dev] = (unsigned char*)p;
  }
  *out = g_scratch_addr[dev];
  return WL_OK;
}

// rows with more than kHubDeg entries, in increasing order, by one CTA
// (n <= kNaMaxN); count to misc[0]
__global__ void na_hub_list(const int32_t* row_ptr, int64_t n, int32_t* hubs, int* count) {
  __shared__ int s_base;
  __shared__ int s_warp[32];
  if (threadIdx.x == 0) s_base = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t b = 0; b < n; b += blockDim.x) {
    const int64_t i = b + threadIdx.x;
    const bool hub = i < n && (row_ptr[i + 1] - row_ptr[i] > kHubDeg);
    const unsigned m = __ballot_sync(0xffffffffu, hub);
    if (lane == 0) s_warp[warp] = __popc(m);
    __syncthreads();
    int before = s_base;
    for (int w = 0; w < warp; ++w) before += s_warp[w];
    if (hub) hubs[before + __popc(m & ((1u << lane) - 1u))] = (int32_t)i;
    __syncthreads();
    if (threadIdx.x == 0) {
      int t = 0;
      for (int w = 0; w < nw; ++w) t += s_warp[w];
      s_base += t;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *count = s_base;
}

__global__ void na_fill(double* v, double a, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = a;
}

int na_blocks() {
  int nb = 0, dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void*)cg_s_phase<double, 1>, kPhaseBlock, 0);
  const int g = (nb < 1 ? 1 : nb) * sms;
  return g > 2048 ? 2048 : g;
}

}  // namespace
}  // namespace wl

using namespace wl;

// Records the status in st (when given) and returns it: every exit of the
// entry point goes through here, so st->status always matches the return code.
static int na_done(wl_stats* st, int status) {
  if (st) st->status = status;
  return status;
}

#define NA_CU(call)                          \
  do {                                       \
    if ((call) != cudaSuccess) {             \
      (void)cudaGetLastError();              \
      return na_done(st, WL_ERR_CUDA);       \
    }                                        \
  } while (0)

extern "C" int wl_degrees_noalloc(const wl_csr* A, wl_variant v, double mu, double alpha, double tol, int max_iter,
                                  double* Df, void* stream, wl_stats* st) {
  if (st) memset(st, 0, sizeof(*st));
  if (!A || A->n < 0 || A->nnz < 0 || (A->n > 0 && (!A->row_ptr || !Df)) || (A->nnz > 0 && !A->col_idx))
    return na_done(st, WL_ERR_INVALID_ARG);
  if (A->n > kNaMaxN)  // the fixed scratch array holds vectors of at most kNaMaxN nodes
    return na_done(st, WL_ERR_INVALID_ARG);
  if (v != WL_ALLWALK && v != WL_NBT && v != WL_BTDW) return na_done(st, WL_ERR_INVALID_ARG);
  const double m = (v == WL_ALLWALK) ? 0.0 : (v == WL_NBT ? 1.0 : mu);
  if (!(m >= 0.0 && m <= 1.0) || !(alpha >= 0.0) || !std::isfinite(alpha)) return na_done(st, WL_ERR_INVALID_ARG);
  if (A->n == 0) return na_done(st, WL_OK);
  if (tol <= 0) tol = 1e-12;
  if (max_iter <= 0) max_iter = 2000;
  cudaStream_t s = (cudaStream_t)stream;

  unsigned char* base = nullptr;
  int rc = scratch_address(&base);
  if (rc != WL_OK) return na_done(st, rc);
  const int64_t n = A->n;
  double* r = (double*)base;
  double* p = r + kNaMaxN;
  double* q = p + kNaMaxN;
  double* part = (double*)(base + kNaVecBytes);
  CgState* state = (CgState*)(base + kNaVecBytes + kNaPartBytes);
  int32_t* hubs = (int32_t*)(base + kNaVecBytes + kNaPartBytes + kNaStateBytes);
  int* misc = (int*)(base + kNaVecBytes + kNaPartBytes + kNaStateBytes + kNaHubBytes);

  // the array keeps the previous call's contents: clear what must start at zero
  NA_CU(cudaMemsetAsync(misc, 0, kNaMiscBytes, s));
  NA_CU(cudaMemsetAsync(state, 0, sizeof(CgState), s));
  const Graph g{A->row_ptr, A->col_idx, n, A->nnz};
  NA_CU(launch_validate(g, misc, s));
  na_hub_list<<<1, 1024, 0, s>>>(A->row_ptr, n, hubs, misc + 1);
  NA_CU(cudaGetLastError());
  int hostv[2] = {0, 0};
  NA_CU(cudaMemcpyAsync(hostv, misc, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  NA_CU(cudaStreamSynchronize(s));
  if (hostv[0] & 3) return na_done(st, WL_ERR_UNSORTED);
  if (hostv[0] & 4) return na_done(st, WL_ERR_SELF_LOOP);
  if (hostv[0] & 8) return na_done(st, WL_ERR_NOT_SYMMETRIC);
  const int nhub = hostv[1];
  const int grid_u = na_blocks(), grid_s = grid_u + nhub;
  if (grid_s > kNaMaxGrid + kNaMaxN) return na_done(st, WL_ERR_INVALID_ARG);

  // M x = a 1, M = a I - alpha A + alpha^2 mu D (FP64 CG from x = 0)
  const double a = 1.0 - m * m * alpha * alpha;
  const PhaseGraph pg{A->row_ptr, A->col_idx, n, hubs, nhub};
  na_fill<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, s>>>(r, a, n);
  NA_CU(cudaGetLastError());
  NA_CU(cudaMemsetAsync(Df, 0, (size_t)n * sizeof(double), s));
  PhaseArgs<double> pa{pg, Df, r, p, q, a, -alpha, alpha * alpha * m, nullptr, nullptr, part, state, max_iter,
                       tol * tol};
  cg_u_phase<double, 1><<<grid_u, kPhaseBlock, 0, s>>>(pa, 1);
  NA_CU(cudaGetLastError());
  for (;;) {
    for (int i = 0; i < 8; ++i) {
      cg_s_phase<double, 1><<<grid_s, kPhaseBlock, 0, s>>>(pa);
      cg_u_phase<double, 1><<<grid_u, kPhaseBlock, 0, s>>>(pa, 0);
    }
    NA_CU(cudaGetLastError());
    int act[2] = {0, 0};
    NA_CU(cudaMemcpyAsync(act, &state->active, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    NA_CU(cudaStreamSynchronize(s));
    if (!act[0]) break;
  }
  cg_f_phase<double, 1><<<grid_u, kPhaseBlock, 0, s>>>(pa);
  NA_CU(cudaGetLastError());
  double gam = 0.0, b2 = 0.0;
  int iters = 0, status = 0, done = 0;
  NA_CU(cudaMemcpyAsync(&gam, &state->gamma[0], sizeof(double), cudaMemcpyDeviceToHost, s));
  NA_CU(cudaMemcpyAsync(&b2, &state->b2[0], sizeof(double), cudaMemcpyDeviceToHost, s));
  NA_CU(cudaMemcpyAsync(&iters, &state->iters, sizeof(int), cudaMemcpyDeviceToHost, s));
  NA_CU(cudaMemcpyAsync(&status, &state->status[0], sizeof(int), cudaMemcpyDeviceToHost, s));
  NA_CU(cudaMemcpyAsync(&done, &state->done[0], sizeof(int), cudaMemcpyDeviceToHost, s));
  NA_CU(cudaStreamSynchronize(s));
  if (status == 0 && !done) status = WL_ERR_NO_CONVERGENCE;
  if (st) {
    st->iters = iters;
    st->rel_res = b2 > 0 ? std::sqrt(gam / b2) : 0.0;
    st->alpha = alpha;
    st->mu = m;
    st->nnz_rhs_iters = (double)iters * (double)A->nnz;
  }
  return na_done(st, status);
}
