// FP64 instances of the CG phase kernels, the FP64 residual of a warm start
// and the FP64 <-> double-float split of an iterate, K = 1, 2, 4, ..., 64 columns.
#include "wl_cg2.cuh"
#include "wl_host.h"

namespace wl {

#define WL_FOR_K(X) X(1) X(2) X(4) X(8) X(16) X(32) X(64)

template <int K>
static cudaError_t run_cg64(const PhaseArgs<double>& a, int grid_s, int grid_u, int mode, int chunk,
                            cudaStream_t s) {
  if (mode == 0) {
    cg_u_phase<double, K><<<grid_u, kPhaseBlock, 0, s>>>(a, 1);
  } else if (mode == 1) {
    for (int i = 0; i < chunk; ++i) {
      if (a.dshift)
        cg_s_phase<double, K, true><<<grid_s, kPhaseBlock, 0, s>>>(a);
      else
        cg_s_phase<double, K><<<grid_s, kPhaseBlock, 0, s>>>(a);
      cg_u_phase<double, K><<<grid_u, kPhaseBlock, 0, s>>>(a, 0);
    }
  } else {
    cg_f_phase<double, K><<<grid_u, kPhaseBlock, 0, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_cg_phases_f64(int K, const PhaseArgs<double>& a, int grid_s, int grid_u, int mode, int chunk,
                                 cudaStream_t s) {
  switch (K) {
#define C64(k) \
  case k:      \
    return run_cg64<k>(a, grid_s, grid_u, mode, chunk, s);
    WL_FOR_K(C64)
#undef C64
  }
  return cudaErrorInvalidValue;
}

template <int K>
static cudaError_t run_res(const ResPhaseArgs& a, int grid, cudaStream_t s) {
  res_phase<K><<<grid, kPhaseBlock, 0, s>>>(a);
  return cudaGetLastError();
}

// FP64 iterate <-> double-float terms (xh, xl)
__global__ void __launch_bounds__(kPhaseBlock) split_x(const double* x, int64_t total, float* xh, float* xl) {
  for (int64_t e = (int64_t)blockIdx.x * kPhaseBlock + threadIdx.x; e < total; e += (int64_t)gridDim.x * kPhaseBlock) {
    const float h = (float)x[e];
    xh[e] = h;
    xl[e] = (float)(x[e] - (double)h);
  }
}

__global__ void __launch_bounds__(kPhaseBlock) join_x(const float* xh, const float* xl, int64_t total, double* x) {
  for (int64_t e = (int64_t)blockIdx.x * kPhaseBlock + threadIdx.x; e < total; e += (int64_t)gridDim.x * kPhaseBlock)
    x[e] = (double)xh[e] + (double)xl[e];
}

cudaError_t launch_split_x(const double* x, int64_t total, float* xh, float* xl, bool join, double* xout,
                           cudaStream_t s) {
  const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + kPhaseBlock - 1) / kPhaseBlock, 152 * 16));
  if (join)
    join_x<<<g, kPhaseBlock, 0, s>>>(xh, xl, total, xout);
  else
    split_x<<<g, kPhaseBlock, 0, s>>>(x, total, xh, xl);
  return cudaGetLastError();
}

cudaError_t launch_res_phases(int K, const ResPhaseArgs& a, int grid, cudaStream_t s) {
  switch (K) {
#define R64(k) \
  case k:      \
    return run_res<k>(a, grid, s);
    WL_FOR_K(R64)
#undef R64
  }
  return cudaErrorInvalidValue;
}

static int occ_blocks(const void* f) {
  int nb = 0, dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, kPhaseBlock, 0);
  return (nb < 1 ? 1 : nb) * sms;
}

int phase_blocks_f64(int K) {
  switch (K) {
#define F64(k) \
  case k:      \
    return occ_blocks((const void*)cg_s_phase<double, k>);
    WL_FOR_K(F64)
#undef F64
  }
  return 0;
}

int res_blocks(int K) {
  switch (K) {
#define RB(k) \
  case k:     \
    return occ_blocks((const void*)res_phase<k>);
    WL_FOR_K(RB)
#undef RB
  }
  return 0;
}

void thresholds_f64(int K, int* Tw, int* Tc) {
  switch (K) {
#define T64(k)                    \
  case k:                         \
    *Tw = Cfg<double, k>::Tw;     \
    *Tc = Cfg<double, k>::Tc;     \
    return;
    WL_FOR_K(T64)
#undef T64
  }
  *Tw = *Tc = 0;
}

// entries of the rows in a list (sum of their degrees)
__global__ void k_list_entries(const int32_t* row_ptr, const int32_t* rows, int64_t count, unsigned long long* out) {
  unsigned long long s = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    s += (unsigned long long)(row_ptr[rows[i] + 1] - row_ptr[rows[i]]);
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

cudaError_t launch_list_entries(const int32_t* row_ptr, const int32_t* rows, int64_t count, unsigned long long* out,
                                cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess || count <= 0) return e;
  const unsigned gb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((count + 255) / 256, 152 * 8));
  k_list_entries<<<gb, 256, 0, s>>>(row_ptr, rows, count, out);
  return cudaGetLastError();
}

// row lists: rows with lo < deg <= hi, in increasing row order
__global__ void k_row_flags(const int32_t* row_ptr, int64_t n, int lo, int hi, int64_t* flag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int d = row_ptr[i + 1] - row_ptr[i];
    flag[i] = (d > lo && d <= hi) ? 1 : 0;
  }
}

__global__ void k_row_scatter(const int64_t* flag, const int64_t* pos, int64_t n, int32_t* rows) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (flag[i]) rows[pos[i]] = (int32_t)i;
}

cudaError_t launch_row_list(const int32_t* row_ptr, int64_t n, int lo, int hi, int32_t* rows, int64_t* tmp,
                            int64_t* count, cudaStream_t s) {
  int64_t* flag = tmp;
  int64_t* pos = tmp + n + 1;
  int64_t* sc = pos + n + 1;
  const unsigned gb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 32));
  k_row_flags<<<gb, 256, 0, s>>>(row_ptr, n, lo, hi, flag);
  cudaError_t e = launch_scan(flag, n, pos, sc, s);
  if (e != cudaSuccess) return e;
  k_row_scatter<<<gb, 256, 0, s>>>(flag, pos, n, rows);
  e = cudaMemcpyAsync(count, pos + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace wl
