// XNysTrace kernels: Philox sketch, right-hand side, Gram, leave-one-out core.
#define WL_TRACE_KERNELS
#include <string.h>

#include "wl.h"
#include "wl_gram_tc.cuh"
#include "wl_host.h"
#include "wl_trace.cuh"

namespace wl {

static unsigned grid_cap(int64_t work, int64_t per, int cap) {
  int64_t b = (work + per - 1) / per;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (unsigned)b;
}

cudaError_t launch_philox_sketch(uint16_t* omega, int64_t n, int M, uint64_t seed, cudaStream_t s) {
  const int64_t total = n * M;
  philox_sketch<<<grid_cap((total + 3) / 4, 256, 152 * 32), 256, 0, s>>>(omega, total, seed);
  return cudaGetLastError();
}

__global__ void permute_rows_u16(const uint16_t* src, int64_t n, int M, const int32_t* perm, uint16_t* dst) {
  const int64_t total = n * M;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / M;
    dst[e] = src[(int64_t)perm[r] * M + (e % M)];
  }
}

cudaError_t launch_permute_rows_u16(const uint16_t* src, int64_t n, int M, const int32_t* perm, uint16_t* dst,
                                    cudaStream_t s) {
  permute_rows_u16<<<grid_cap(n * M, 256, 152 * 32), 256, 0, s>>>(src, n, M, perm, dst);
  return cudaGetLastError();
}

cudaError_t launch_sketch_rhs(const uint16_t* omega, int64_t n, int M, int K, double a, float* B, cudaStream_t s) {
  sketch_rhs<<<grid_cap(n * K, 256, 152 * 32), 256, 0, s>>>(omega, n, M, K, (float)a, B);
  return cudaGetLastError();
}

cudaError_t launch_sketch_block_f64(const uint16_t* omega, int64_t n, int M, int K, double* B, cudaStream_t s) {
  sketch_block_f64<<<grid_cap(n * K, 256, 152 * 32), 256, 0, s>>>(omega, n, M, K, B);
  return cudaGetLastError();
}

cudaError_t launch_to_f32(const double* X, int64_t total, float* Y, cudaStream_t s) {
  to_f32<<<grid_cap(total, 256, 152 * 32), 256, 0, s>>>(X, total, Y);
  return cudaGetLastError();
}

int gram_grid(int64_t n) {
  // about 4096 rows per chunk, at most 8 CTAs per SM worth of chunks
  int64_t g = (n + 4095) / 4096;
  if (g > 152 * 8) g = 152 * 8;
  if (g < 1) g = 1;
  return (int)g;
}

cudaError_t launch_gram(const uint16_t* omega, const float* Y, int64_t n, int M, int K, float* partial, int G,
                        double* out, bool tensor_cores, int* err, cudaStream_t s) {
  int64_t chunk = (n + G - 1) / G;
  // the tensor-core kernel's bulk copies need 16-byte aligned rows of Omega
  // and Y (stage offsets are then multiples of 16 bytes)
  if (tensor_cores && ((reinterpret_cast<uintptr_t>(omega) | reinterpret_cast<uintptr_t>(Y)) & 15u) != 0)
    tensor_cores = false;
  if (tensor_cores) {
    chunk = (chunk + kTcRows - 1) / kTcRows * kTcRows;  // each CTA's range starts at a stage boundary
    static bool attr = false;
    if (!attr) {
      cudaError_t e = cudaFuncSetAttribute(gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
      if (e != cudaSuccess) return e;
      attr = true;
    }
    gram_tc<<<G, kTcThreads, kTcSmem, s>>>(omega, Y, n, M, K, chunk, partial, err);
  } else {
    gram_cc<<<G, kGramThreads, 0, s>>>(omega, Y, n, M, K, chunk, partial);
  }
  gram_reduce<<<(2 * kMaxSketch * kMaxSketch + 255) / 256, 256, 0, s>>>(partial, G, out);
  return cudaGetLastError();
}

cudaError_t launch_gram_f64(const uint16_t* omega, const double* Y, int64_t n, int M, int K, double* partial, int G,
                            double* out, cudaStream_t s) {
  const int64_t chunk = (n + G - 1) / G;
  gram_f64<<<G, 256, 0, s>>>(omega, Y, n, M, K, chunk, partial);
  gram_reduce_f64<<<(2 * kMaxSketch * kMaxSketch + 255) / 256, 256, 0, s>>>(partial, G, out);
  return cudaGetLastError();
}

cudaError_t launch_nys_core(const double* gram, int M, double* out, cudaStream_t s) {
  const int smem = 4 * kMaxSketch * kMaxSketch * (int)sizeof(double);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(nys_core, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  nys_core<<<1, 256, smem, s>>>(gram, M, out);
  return cudaGetLastError();
}

}  // namespace wl

using namespace wl;

extern "C" int wl_sketch_gram(const uint16_t* omega, const float* Y, int64_t n, int M, int ldy, int tensor_cores,
                              double* out, void* stream) {
  if (!omega || !Y || !out || n < 0 || M < 1 || M > kMaxSketch || ldy < M) return WL_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int G = gram_grid(n);
  float* partial = nullptr;
  int* err = nullptr;
  cudaError_t e = cudaMalloc(&partial, sizeof(float) * (size_t)G * 2 * kMaxSketch * kMaxSketch);
  if (e == cudaSuccess) e = cudaMalloc(&err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (e == cudaSuccess) e = launch_gram(omega, Y, n, M, ldy, partial, G, out, tensor_cores != 0, err, s);
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(partial);
  cudaFree(err);
  if (e != cudaSuccess) return report_cuda_error(e, "wl_sketch_gram");
  return herr;
}

