// Learned warm start for the walk-degree solve (the paper has no learned
// part; this network only supplies the CG starting guess of D_f = phi 1).
//
// Node features (all from the graph alone, FP64, stored FP32):
//   f0 = log(1 + d_i), f1 = log(1 + (A d)_i), f2 = log(1 + t_i),
//   f3 = log(1 + (A d - d)_i)
// with t_i the triangles through i (degree-ordered intersection) and
// A d - d the nonbacktracking 2-walk count (p_2(A) 1 with p_2 = A^2 - D).
//
// The guess is x0 = x_an * exp(y): x_an = 1 + B 1 + B^2 1 is the two-term
// Neumann series of D_f = sum_k B^k 1, B = (alpha A - alpha^2 mu D) / a,
// a = 1 - mu^2 alpha^2 (Sec. 4.2, the resolvent's series), and y the output
// of a 4 -> 64 -> 64 -> 1 tanh perceptron on the standardised features,
// trained on log(D_f / x_an).
//
// Parameter vector (floats): mean[4], std[4], W1[64][4], b1[64],
// W2[64][64], b2[64], W3[64], b3 (4553 values).
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "wl.h"
#include "wl_host.h"

namespace wl {

constexpr int kH = 64;
constexpr int kIn = 4;
constexpr int kOffMean = 0, kOffStd = 4, kOffW1 = 8, kOffB1 = kOffW1 + kH * kIn, kOffW2 = kOffB1 + kH,
              kOffB2 = kOffW2 + kH * kH, kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH;
constexpr int kParams = kOffB3 + 1;        // 4553
constexpr int kTrain = kParams - kOffW1;   // 4545 trainable values (after the standardisation)
constexpr int kRowsCTA = 128;              // rows per CTA of the gradient kernel
constexpr int kPad = kH + 1;               // shared-memory row stride (bank-conflict free)

// ------------------------------------------------------------------ features
// one warp per row: d_i and (A d)_i; hub rows by a whole CTA each
__global__ void k_feat_ad(const int32_t* __restrict__ rp, const int32_t* __restrict__ col, int64_t n,
                          double* __restrict__ ad) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < n; i += nw) {
    const int beg = rp[i], end = rp[i + 1];
    double s = 0.0;
    for (int e = beg + lane; e < end; e += 32) {
      const int j = __ldg(col + e);
      s += (double)(rp[j + 1] - rp[j]);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) ad[i] = s;
  }
}

// rank order for the triangle orientation: (degree, index)
__device__ __forceinline__ bool ranks_above(int dj, int j, int di, int i) { return dj > di || (dj == di && j > i); }

// out-degree in the orientation (neighbours of higher rank)
__global__ void k_feat_outdeg(const int32_t* __restrict__ rp, const int32_t* __restrict__ col, int64_t n,
                              int64_t* __restrict__ outdeg) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < n; i += nw) {
    const int beg = rp[i], end = rp[i + 1], di = end - beg;
    int c = 0;
    for (int e = beg + lane; e < end; e += 32) {
      const int j = __ldg(col + e);
      c += ranks_above(rp[j + 1] - rp[j], j, di, (int)i) ? 1 : 0;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
    if (lane == 0) outdeg[i] = c;
  }
}

// oriented lists (ascending index order kept by an ordered warp compaction)
__global__ void k_feat_orient(const int32_t* __restrict__ rp, const int32_t* __restrict__ col, int64_t n,
                              const int64_t* __restrict__ orp, const int32_t* __restrict__ key,
                              int32_t* __restrict__ ocol, int32_t* __restrict__ okey) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < n; i += nw) {
    const int beg = rp[i], end = rp[i + 1], di = end - beg;
    int64_t o = orp[i];
    for (int e0 = beg; e0 < end; e0 += 32) {
      const int e = e0 + lane;
      bool keep = false;
      int j = 0;
      if (e < end) {
        j = __ldg(col + e);
        keep = ranks_above(rp[j + 1] - rp[j], j, di, (int)i);
      }
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      if (keep) {
        const int64_t q = o + __popc(m & ((1u << lane) - 1u));
        ocol[q] = j;
        okey[q] = key ? key[j] : j;
      }
      o += __popc(m);
    }
  }
}

// position in okey[lo, end) (ascending) holding k, or -1
__device__ __forceinline__ int64_t find_key(const int32_t* __restrict__ okey, int64_t lo, int64_t end, int k) {
  int64_t hi = end;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (okey[mid] < k) lo = mid + 1; else hi = mid;
  }
  return (lo < end && okey[lo] == k) ? lo : -1;
}

// Every triangle once: for i, each oriented neighbour j (one per lane) and
// each w in N+(i) and N+(j) adds one to t_i, t_j and t_w. The lists are
// ascending in key (the caller's node index, which is the column order of
// every row); two lists of similar length are merged, a much shorter one is
// looked up element by element in the longer one by binary search.
__global__ void k_feat_triangles(const int64_t* __restrict__ orp, const int32_t* __restrict__ ocol,
                                 const int32_t* __restrict__ okey, int64_t n, unsigned long long* __restrict__ t) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < n; i += nw) {
    const int64_t ib = orp[i], ie = orp[i + 1];
    unsigned long long ti = 0;
    for (int64_t e = ib + lane; e < ie; e += 32) {
      const int j = ocol[e];
      const int64_t jb = orp[j], je = orp[j + 1];
      const int64_t la = ie - ib, lb = je - jb;
      unsigned long long tj = 0;
      if (la > 16 * lb) {  // look up N+(j) in N+(i)
        for (int64_t b = jb; b < je; ++b) {
          const int64_t pos = find_key(okey, ib, ie, okey[b]);
          if (pos >= 0) {
            ++tj;
            atomicAdd(t + ocol[b], 1ull);
          }
        }
      } else if (lb > 16 * la) {  // look up N+(i) in N+(j)
        for (int64_t a = ib; a < ie; ++a) {
          const int64_t pos = find_key(okey, jb, je, okey[a]);
          if (pos >= 0) {
            ++tj;
            atomicAdd(t + ocol[a], 1ull);
          }
        }
      } else {
        int64_t a = ib, b = jb;
        while (a < ie && b < je) {
          const int kx = okey[a], ky = okey[b];
          if (kx == ky) {
            ++tj;
            atomicAdd(t + ocol[a], 1ull);
            ++a;
            ++b;
          } else if (kx < ky) {
            ++a;
          } else {
            ++b;
          }
        }
      }
      if (tj) atomicAdd(t + j, tj);
      ti += tj;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) ti += __shfl_xor_sync(0xffffffffu, ti, off);
    if (lane == 0 && ti) atomicAdd(t + i, ti);
  }
}

// features (FP32) and the analytic guess x_an (FP64), written at position
// perm[i] (perm == NULL: i)
__global__ void k_feat_out(const int32_t* __restrict__ rp, const double* __restrict__ ad,
                           const unsigned long long* __restrict__ t, int64_t n, double alpha, double mu,
                           const int32_t* __restrict__ perm, float* __restrict__ F, double* __restrict__ xan) {
  const double a = 1.0 - mu * mu * alpha * alpha;
  const double c1 = (alpha - alpha * alpha * mu) / a;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double d = (double)(rp[i + 1] - rp[i]);
    const double adi = ad[i];
    const int64_t o = perm ? (int64_t)perm[i] : i;
    if (F) {
      F[o * 4 + 0] = (float)log1p(d);
      F[o * 4 + 1] = (float)log1p(adi);
      F[o * 4 + 2] = (float)log1p((double)t[i]);
      F[o * 4 + 3] = (float)log1p(adi - d);
    }
    if (xan) xan[o] = 1.0 + c1 * d + c1 * (alpha * adi - alpha * alpha * mu * d * d) / a;
  }
}

// ------------------------------------------------------------------ network
__device__ __forceinline__ void load_params(const float* __restrict__ P, float* s) {
  for (int i = threadIdx.x; i < kParams; i += blockDim.x) s[i] = P[i];
  __syncthreads();
}

// y (per row) of the perceptron; x0 = exp(y) * xan (xan may be NULL: x0 = y)
__global__ void __launch_bounds__(128) k_mlp_predict(const float* __restrict__ P, const float* __restrict__ F,
                                                      int64_t rows, const double* __restrict__ xan,
                                                      double* __restrict__ out) {
  __shared__ float s[kParams];
  load_params(P, s);
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
    float x[kIn];
#pragma unroll
    for (int c = 0; c < kIn; ++c) x[c] = (F[r * 4 + c] - s[kOffMean + c]) / s[kOffStd + c];
    // z2 accumulated over the hidden units of layer 1, each computed once
    float z2[kH];
#pragma unroll
    for (int j = 0; j < kH; ++j) z2[j] = s[kOffB2 + j];
#pragma unroll 1
    for (int k = 0; k < kH; ++k) {
      float z = s[kOffB1 + k];
#pragma unroll
      for (int c = 0; c < kIn; ++c) z = fmaf(s[kOffW1 + k * kIn + c], x[c], z);
      const float h = tanhf(z);
#pragma unroll
      for (int j = 0; j < kH; ++j) z2[j] = fmaf(s[kOffW2 + j * kH + k], h, z2[j]);
    }
    float y = s[kOffB3];
#pragma unroll
    for (int j = 0; j < kH; ++j) y = fmaf(s[kOffW3 + j], tanhf(z2[j]), y);
    out[r] = xan ? xan[r] * exp((double)y) : (double)y;
  }
}

// Forward and backward over kRowsCTA rows of [row0, row0 + rows); writes the
// CTA's gradient partial (kTrain values, layout of the trainable parameters)
// and its sum of squared errors to part[blockIdx.x * (kTrain + 1) ...].
// Loss L = (1/B) sum (y - t)^2 over the B rows of the batch.
__global__ void __launch_bounds__(kRowsCTA) k_mlp_grad(const float* __restrict__ P, const float* __restrict__ F,
                                                        const float* __restrict__ T, int64_t row0, int64_t rows,
                                                        double inv_b, float* __restrict__ part) {
  extern __shared__ float sm[];
  float* s = sm;                            // parameters
  float* s_h1 = s + kParams + 3;            // [kRowsCTA][kPad]
  float* s_h2 = s_h1 + kRowsCTA * kPad;     // [kRowsCTA][kPad]
  float* s_g2 = s_h2 + kRowsCTA * kPad;     // dL/dz2
  float* s_g1 = s_g2 + kRowsCTA * kPad;     // dL/dz1
  float* s_x = s_g1 + kRowsCTA * kPad;      // [kRowsCTA][4] standardised inputs
  float* s_gy = s_x + kRowsCTA * kIn;       // [kRowsCTA]
  load_params(P, s);
  const int tid = threadIdx.x;
  const int64_t r = row0 + (int64_t)blockIdx.x * kRowsCTA + tid;
  const bool live = (int64_t)blockIdx.x * kRowsCTA + tid < rows;
  float* h1r = s_h1 + tid * kPad;
  float* h2r = s_h2 + tid * kPad;
  float* g2r = s_g2 + tid * kPad;
  float* g1r = s_g1 + tid * kPad;
  float gy = 0.f, sq = 0.f;
  if (live) {
    float x[kIn];
#pragma unroll
    for (int c = 0; c < kIn; ++c) {
      x[c] = (F[r * 4 + c] - s[kOffMean + c]) / s[kOffStd + c];
      s_x[tid * kIn + c] = x[c];
    }
#pragma unroll 8
    for (int k = 0; k < kH; ++k) {
      float z = s[kOffB1 + k];
#pragma unroll
      for (int c = 0; c < kIn; ++c) z = fmaf(s[kOffW1 + k * kIn + c], x[c], z);
      h1r[k] = tanhf(z);
    }
    float y = s[kOffB3];
    for (int j = 0; j < kH; ++j) {
      float z = s[kOffB2 + j];
      for (int k = 0; k < kH; ++k) z = fmaf(s[kOffW2 + j * kH + k], h1r[k], z);
      const float h = tanhf(z);
      h2r[j] = h;
      y = fmaf(s[kOffW3 + j], h, y);
    }
    const float e = y - T[r];
    sq = e * e;
    gy = (float)(2.0 * inv_b) * e;
    for (int j = 0; j < kH; ++j) g2r[j] = gy * s[kOffW3 + j] * (1.f - h2r[j] * h2r[j]);
    for (int k = 0; k < kH; ++k) {
      float gh = 0.f;
      for (int j = 0; j < kH; ++j) gh = fmaf(g2r[j], s[kOffW2 + j * kH + k], gh);
      g1r[k] = gh * (1.f - h1r[k] * h1r[k]);
    }
  } else {
    for (int k = 0; k < kH; ++k) {
      h1r[k] = h2r[k] = g2r[k] = g1r[k] = 0.f;
    }
#pragma unroll
    for (int c = 0; c < kIn; ++c) s_x[tid * kIn + c] = 0.f;
  }
  s_gy[tid] = gy;
  // squared error of the CTA (fixed order)
  __shared__ float s_sq[kRowsCTA];
  s_sq[tid] = sq;
  __syncthreads();
  float* out = part + (size_t)blockIdx.x * (kTrain + 1);
  const int nr = kRowsCTA;
  // W1 (256) and b1 (64): entries j*4 + c and j
  for (int q = tid; q < kH * kIn + kH; q += blockDim.x) {
    float acc = 0.f;
    if (q < kH * kIn) {
      const int j = q / kIn, c = q % kIn;
      for (int rr = 0; rr < nr; ++rr) acc = fmaf(s_g1[rr * kPad + j], s_x[rr * kIn + c], acc);
    } else {
      const int j = q - kH * kIn;
      for (int rr = 0; rr < nr; ++rr) acc += s_g1[rr * kPad + j];
    }
    out[q] = acc;
  }
  // W2 (4096): entry j*64 + k = sum_r g2[r][j] h1[r][k]
  for (int q = tid; q < kH * kH; q += blockDim.x) {
    const int j = q / kH, k = q % kH;
    float acc = 0.f;
    for (int rr = 0; rr < nr; ++rr) acc = fmaf(s_g2[rr * kPad + j], s_h1[rr * kPad + k], acc);
    out[kOffW2 - kOffW1 + q] = acc;
  }
  // b2, W3, b3
  for (int q = tid; q < 2 * kH + 1; q += blockDim.x) {
    float acc = 0.f;
    if (q < kH) {
      for (int rr = 0; rr < nr; ++rr) acc += s_g2[rr * kPad + q];
      out[kOffB2 - kOffW1 + q] = acc;
    } else if (q < 2 * kH) {
      const int j = q - kH;
      for (int rr = 0; rr < nr; ++rr) acc = fmaf(s_gy[rr], s_h2[rr * kPad + j], acc);
      out[kOffW3 - kOffW1 + j] = acc;
    } else {
      for (int rr = 0; rr < nr; ++rr) acc += s_gy[rr];
      out[kOffB3 - kOffW1] = acc;
    }
  }
  if (tid == 0) {
    float t = 0.f;
    for (int rr = 0; rr < nr; ++rr) t += s_sq[rr];
    out[kTrain] = t;
  }
}

// Sums the CTA partials in a fixed order (FP64). mode 0: write the gradient
// and loss; mode 1: Adam update of the trainable parameters (m, v state).
__global__ void k_mlp_reduce(const float* __restrict__ part, int nblk, double inv_b, float* __restrict__ P,
                             float* __restrict__ m, float* __restrict__ v, float lr, float b1, float b2, float eps,
                             double bc1, double bc2, int mode, float* __restrict__ grad, double* __restrict__ loss) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q > kTrain) return;
  double g = 0.0;
  for (int c = 0; c < nblk; ++c) g += (double)part[(size_t)c * (kTrain + 1) + q];
  if (q == kTrain) {
    if (loss) *loss = g * inv_b;
    return;
  }
  if (mode == 0) {
    grad[q] = (float)g;
    return;
  }
  const float gf = (float)g;
  const float mm = b1 * m[q] + (1.f - b1) * gf;
  const float vv = b2 * v[q] + (1.f - b2) * gf * gf;
  m[q] = mm;
  v[q] = vv;
  const double mh = (double)mm / bc1, vh = (double)vv / bc2;
  P[kOffW1 + q] = (float)((double)P[kOffW1 + q] - (double)lr * mh / (sqrt(vh) + (double)eps));
}

// feature means and standard deviations (FP64 partial sums per CTA)
__global__ void k_mlp_stats_part(const float* __restrict__ F, int64_t rows, double* __restrict__ part) {
  double s[2 * kIn] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
    for (int c = 0; c < kIn; ++c) {
      const double x = F[r * 4 + c];
      s[c] += x;
      s[kIn + c] += x * x;
    }
  __shared__ double sh[2 * kIn][256];
#pragma unroll
  for (int c = 0; c < 2 * kIn; ++c) sh[c][threadIdx.x] = s[c];
  __syncthreads();
  if (threadIdx.x < 2 * kIn) {
    double t = 0.0;
    for (int i = 0; i < (int)blockDim.x; ++i) t += sh[threadIdx.x][i];
    part[blockIdx.x * 2 * kIn + threadIdx.x] = t;
  }
}

__global__ void k_mlp_stats_fin(const double* __restrict__ part, int nblk, int64_t rows, float* __restrict__ P) {
  const int c = threadIdx.x;
  if (c >= kIn) return;
  double s = 0.0, s2 = 0.0;
  for (int b = 0; b < nblk; ++b) {
    s += part[b * 2 * kIn + c];
    s2 += part[b * 2 * kIn + kIn + c];
  }
  const double mean = s / (double)rows;
  const double var = fmax(s2 / (double)rows - mean * mean, 0.0);
  P[kOffMean + c] = (float)mean;
  P[kOffStd + c] = (float)fmax(sqrt(var), 1e-6);
}

// training target log(D_f / x_an)
__global__ void k_log_ratio(const double* __restrict__ Df, const double* __restrict__ xan, int64_t rows,
                            float* __restrict__ t) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x)
    t[r] = (float)log(Df[r] / xan[r]);
}

size_t grad_smem() { return sizeof(float) * (kParams + 3 + 4 * kRowsCTA * kPad + kRowsCTA * kIn + kRowsCTA); }

cudaError_t grad_setup() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)grad_smem());
  if (e == cudaSuccess) done = true;
  return e;
}

// ------------------------------------------------------------------ launchers (wl_host.h)
cudaError_t launch_features(const int32_t* rp, const int32_t* col, int64_t n, int64_t nnz, double alpha, double mu,
                            const int32_t* perm, const int32_t* perm_key, float* F, double* xan, void* tmp,
                            cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  // tmp: ad (n doubles), t (n u64), outdeg / orp (n + 1 int64 each), scan scratch, ocol (nnz / 2 + 1 int32)
  double* ad = (double*)tmp;
  unsigned long long* t = (unsigned long long*)(ad + n);
  int64_t* outdeg = (int64_t*)(t + n);
  int64_t* orp = outdeg + n + 1;
  int64_t* sc = orp + n + 1;
  int32_t* ocol = (int32_t*)(sc + n / 1024 + 64);
  int32_t* okey = ocol + nnz / 2 + 1;
  const unsigned gw = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n * 32 + 255) / 256, 152 * 64));
  const unsigned g1 = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 32));
  k_feat_ad<<<gw, 256, 0, s>>>(rp, col, n, ad);
  if (F) {  // triangles only for the network's inputs (x_an needs d and A d alone)
    cudaError_t e = cudaMemsetAsync(t, 0, sizeof(unsigned long long) * n, s);
    if (e != cudaSuccess) return e;
    k_feat_outdeg<<<gw, 256, 0, s>>>(rp, col, n, outdeg);
    e = launch_scan(outdeg, n, orp, sc, s);  // orp[0..n]: exclusive prefix, orp[n] = total
    if (e != cudaSuccess) return e;
    k_feat_orient<<<gw, 256, 0, s>>>(rp, col, n, orp, perm_key, ocol, okey);
    k_feat_triangles<<<gw, 256, 0, s>>>(orp, ocol, okey, n, t);
  }
  k_feat_out<<<g1, 256, 0, s>>>(rp, ad, t, n, alpha, mu, perm, F, xan);
  return cudaGetLastError();
}

size_t features_tmp_bytes(int64_t n, int64_t nnz) {
  return (size_t)n * 8 * 2 + (size_t)(n + 1) * 8 * 2 + (size_t)(n / 1024 + 64) * 8 + (size_t)(nnz / 2 + 1) * 8 + 256;
}

cudaError_t launch_mlp_predict(const float* P, const float* F, int64_t rows, const double* xan, double* out,
                               cudaStream_t s) {
  if (rows == 0) return cudaSuccess;
  const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((rows + 127) / 128, 152 * 16));
  k_mlp_predict<<<g, 128, 0, s>>>(P, F, rows, xan, out);
  return cudaGetLastError();
}

}  // namespace wl

using namespace wl;

namespace {

int mlp_err(cudaError_t e, const char* where) { return report_cuda_error(e, where); }

#define ML_CU(call)                                       \
  do {                                                    \
    cudaError_t e__ = (call);                             \
    if (e__ != cudaSuccess) return mlp_err(e__, #call);   \
  } while (0)

// staging and scratch of one synchronous call: released after the call's
// stream has been synchronised (or, on an early error, after a device sync)
struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) {
      cudaDeviceSynchronize();
      pool_free(p);
    }
  }
  cudaError_t alloc(size_t b) { return pool_malloc(&p, b ? b : 16); }
};

bool dev_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// device copy of a caller array (host or device); `own` keeps a copy alive
int stage(const void* src, size_t bytes, DevBuf& own, const void** dev, cudaStream_t s) {
  if (dev_ptr(src)) {
    *dev = src;
    return WL_OK;
  }
  ML_CU(own.alloc(bytes));
  ML_CU(cudaMemcpyAsync(own.p, src, bytes, cudaMemcpyHostToDevice, s));
  *dev = own.p;
  return WL_OK;
}

// gradient partials over rows [row0, row0 + rows)
int grad_pass(const float* P, const float* F, const float* T, int64_t row0, int64_t rows, float* part,
              cudaStream_t s) {
  ML_CU(grad_setup());
  const int nb = (int)((rows + kRowsCTA - 1) / kRowsCTA);
  k_mlp_grad<<<nb, kRowsCTA, grad_smem(), s>>>(P, F, T, row0, rows, 1.0 / (double)rows, part);
  ML_CU(cudaGetLastError());
  return WL_OK;
}

}  // namespace

extern "C" {

int wl_mlp_loss_grad(const float* params, const float* feats, const float* target, int64_t rows, double* loss,
                     float* grad, void* stream) {
  if (!params || !feats || !target || rows <= 0 || rows > (int64_t)1 << 30) return WL_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  DevBuf bp, bf, bt, bpart, bg, bl;
  const void *P, *F, *T;
  int rc;
  if ((rc = stage(params, sizeof(float) * kParams, bp, &P, s)) != WL_OK) return rc;
  if ((rc = stage(feats, sizeof(float) * 4 * rows, bf, &F, s)) != WL_OK) return rc;
  if ((rc = stage(target, sizeof(float) * rows, bt, &T, s)) != WL_OK) return rc;
  const int nb = (int)((rows + kRowsCTA - 1) / kRowsCTA);
  ML_CU(bpart.alloc(sizeof(float) * (size_t)nb * (kTrain + 1)));
  ML_CU(bg.alloc(sizeof(float) * kTrain));
  ML_CU(bl.alloc(sizeof(double)));
  if ((rc = grad_pass((const float*)P, (const float*)F, (const float*)T, 0, rows, (float*)bpart.p, s)) != WL_OK)
    return rc;
  k_mlp_reduce<<<(kTrain + 1 + 255) / 256, 256, 0, s>>>((const float*)bpart.p, nb, 1.0 / (double)rows, nullptr,
                                                       nullptr, nullptr, 0.f, 0.f, 0.f, 0.f, 1.0, 1.0, 0,
                                                       (float*)bg.p, (double*)bl.p);
  ML_CU(cudaGetLastError());
  // grad layout follows the parameter vector: zeros for the standardisation
  std::vector<float> gh(kParams, 0.f);
  ML_CU(cudaMemcpyAsync(gh.data() + kOffW1, bg.p, sizeof(float) * kTrain, cudaMemcpyDeviceToHost, s));
  double l = 0.0;
  ML_CU(cudaMemcpyAsync(&l, bl.p, sizeof(double), cudaMemcpyDeviceToHost, s));
  ML_CU(cudaStreamSynchronize(s));
  if (grad) ML_CU(cudaMemcpy(grad, gh.data(), sizeof(float) * kParams, cudaMemcpyDefault));
  if (loss) *loss = l;
  return WL_OK;
}

int wl_mlp_train(float* params, const float* feats, const float* target, int64_t rows, int steps, int64_t batch,
                 float lr, int standardize, double* final_loss, void* stream) {
  if (!params || !feats || !target || rows <= 0 || steps < 0 || rows > (int64_t)1 << 30) return WL_ERR_INVALID_ARG;
  if (batch <= 0 || batch > rows) batch = rows;
  cudaStream_t s = (cudaStream_t)stream;
  DevBuf bf, bt, bP, bpart, bm, bv, bl, bst;
  const void *F, *T;
  int rc;
  if ((rc = stage(feats, sizeof(float) * 4 * rows, bf, &F, s)) != WL_OK) return rc;
  if ((rc = stage(target, sizeof(float) * rows, bt, &T, s)) != WL_OK) return rc;
  ML_CU(bP.alloc(sizeof(float) * kParams));
  ML_CU(cudaMemcpyAsync(bP.p, params, sizeof(float) * kParams, cudaMemcpyDefault, s));
  float* P = (float*)bP.p;
  if (standardize) {
    const int sb = 152 * 4;
    ML_CU(bst.alloc(sizeof(double) * sb * 2 * kIn));
    k_mlp_stats_part<<<sb, 256, 0, s>>>((const float*)F, rows, (double*)bst.p);
    k_mlp_stats_fin<<<1, 32, 0, s>>>((const double*)bst.p, sb, rows, P);
    ML_CU(cudaGetLastError());
  }
  const int nb_max = (int)((batch + kRowsCTA - 1) / kRowsCTA);
  ML_CU(bpart.alloc(sizeof(float) * (size_t)std::max(nb_max, (int)((rows + kRowsCTA - 1) / kRowsCTA)) * (kTrain + 1)));
  ML_CU(bm.alloc(sizeof(float) * kTrain));
  ML_CU(bv.alloc(sizeof(float) * kTrain));
  ML_CU(bl.alloc(sizeof(double)));
  ML_CU(cudaMemsetAsync(bm.p, 0, sizeof(float) * kTrain, s));
  ML_CU(cudaMemsetAsync(bv.p, 0, sizeof(float) * kTrain, s));
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  int64_t off = 0;
  for (int it = 1; it <= steps; ++it) {
    if (off + batch > rows) off = 0;
    if ((rc = grad_pass(P, (const float*)F, (const float*)T, off, batch, (float*)bpart.p, s)) != WL_OK) return rc;
    const int nb = (int)((batch + kRowsCTA - 1) / kRowsCTA);
    k_mlp_reduce<<<(kTrain + 1 + 255) / 256, 256, 0, s>>>((const float*)bpart.p, nb, 1.0 / (double)batch, P,
                                                         (float*)bm.p, (float*)bv.p, lr, b1, b2, eps,
                                                         1.0 - std::pow((double)b1, it), 1.0 - std::pow((double)b2, it),
                                                         1, nullptr, (double*)bl.p);
    ML_CU(cudaGetLastError());
    off += batch;
  }
  // loss of the trained network over all rows
  if ((rc = grad_pass(P, (const float*)F, (const float*)T, 0, rows, (float*)bpart.p, s)) != WL_OK) return rc;
  k_mlp_reduce<<<(kTrain + 1 + 255) / 256, 256, 0, s>>>((const float*)bpart.p, (int)((rows + kRowsCTA - 1) / kRowsCTA),
                                                       1.0 / (double)rows, nullptr, nullptr, nullptr, 0.f, 0.f, 0.f,
                                                       0.f, 1.0, 1.0, 0, (float*)bm.p, (double*)bl.p);
  ML_CU(cudaGetLastError());
  double l = 0.0;
  ML_CU(cudaMemcpyAsync(&l, bl.p, sizeof(double), cudaMemcpyDeviceToHost, s));
  ML_CU(cudaMemcpyAsync(params, P, sizeof(float) * kParams, cudaMemcpyDefault, s));
  ML_CU(cudaStreamSynchronize(s));
  if (final_loss) *final_loss = l;
  return WL_OK;
}

int wl_mlp_predict(const float* params, const float* feats, int64_t rows, const double* xan, double* out,
                   void* stream) {
  if (!params || !feats || !out || rows < 0) return WL_ERR_INVALID_ARG;
  if (rows == 0) return WL_OK;
  cudaStream_t s = (cudaStream_t)stream;
  DevBuf bp, bf, bx, bo;
  const void *P, *F, *X = nullptr;
  int rc;
  if ((rc = stage(params, sizeof(float) * kParams, bp, &P, s)) != WL_OK) return rc;
  if ((rc = stage(feats, sizeof(float) * 4 * rows, bf, &F, s)) != WL_OK) return rc;
  if (xan && (rc = stage(xan, sizeof(double) * rows, bx, &X, s)) != WL_OK) return rc;
  double* o = out;
  const bool dev_out = dev_ptr(out);
  if (!dev_out) {
    ML_CU(bo.alloc(sizeof(double) * rows));
    o = (double*)bo.p;
  }
  ML_CU(launch_mlp_predict((const float*)P, (const float*)F, rows, (const double*)X, o, s));
  if (!dev_out) ML_CU(cudaMemcpyAsync(out, o, sizeof(double) * rows, cudaMemcpyDeviceToHost, s));
  ML_CU(cudaStreamSynchronize(s));
  return WL_OK;
}

int wl_mlp_param_count(void) { return kParams; }

// Checkpoint file of the network: a 32-byte header (magic "WLMLP001",
// uint32 inputs, hidden width, output width, parameter count, FNV-1a hash of
// the parameter bytes, uint32 zero) followed by the parameter vector as
// little-endian FP32 in the order of the parameter layout above.
namespace {
constexpr char kMlpMagic[8] = {'W', 'L', 'M', 'L', 'P', '0', '0', '1'};

uint32_t fnv1a(const unsigned char* p, size_t n) {
  uint32_t h = 2166136261u;
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 16777619u;
  }
  return h;
}

void put_u32(unsigned char* p, uint32_t v) {
  for (int i = 0; i < 4; ++i) p[i] = (unsigned char)(v >> (8 * i));
}

uint32_t get_u32(const unsigned char* p) {
  uint32_t v = 0;
  for (int i = 0; i < 4; ++i) v |= (uint32_t)p[i] << (8 * i);
  return v;
}
}  // namespace

int wl_mlp_save(const char* path, const float* params) {
  if (!path || !params) return WL_ERR_INVALID_ARG;
  std::vector<unsigned char> buf(32 + (size_t)kParams * 4);
  memcpy(buf.data(), kMlpMagic, 8);
  for (int i = 0; i < kParams; ++i) {
    uint32_t bits;
    memcpy(&bits, params + i, 4);
    put_u32(buf.data() + 32 + (size_t)i * 4, bits);
  }
  put_u32(buf.data() + 8, kIn);
  put_u32(buf.data() + 12, kH);
  put_u32(buf.data() + 16, 1);
  put_u32(buf.data() + 20, kParams);
  put_u32(buf.data() + 24, fnv1a(buf.data() + 32, (size_t)kParams * 4));
  put_u32(buf.data() + 28, 0);
  FILE* f = fopen(path, "wb");
  if (!f) return WL_ERR_INVALID_ARG;
  const size_t w = fwrite(buf.data(), 1, buf.size(), f);
  const int rc = fclose(f);
  return (w == buf.size() && rc == 0) ? WL_OK : WL_ERR_INVALID_ARG;
}

int wl_mlp_load(const char* path, float* params) {
  if (!path || !params) return WL_ERR_INVALID_ARG;
  FILE* f = fopen(path, "rb");
  if (!f) return WL_ERR_INVALID_ARG;
  std::vector<unsigned char> buf(32 + (size_t)kParams * 4);
  const size_t r = fread(buf.data(), 1, buf.size(), f);
  unsigned char extra;
  const bool trailing = fread(&extra, 1, 1, f) == 1;
  fclose(f);
  if (r != buf.size() || trailing || memcmp(buf.data(), kMlpMagic, 8) != 0) return WL_ERR_INVALID_ARG;
  if (get_u32(buf.data() + 8) != (uint32_t)kIn || get_u32(buf.data() + 12) != (uint32_t)kH ||
      get_u32(buf.data() + 16) != 1u || get_u32(buf.data() + 20) != (uint32_t)kParams)
    return WL_ERR_INVALID_ARG;
  if (get_u32(buf.data() + 24) != fnv1a(buf.data() + 32, (size_t)kParams * 4)) return WL_ERR_NONFINITE;
  for (int i = 0; i < kParams; ++i) {
    const uint32_t bits = get_u32(buf.data() + 32 + (size_t)i * 4);
    memcpy(params + i, &bits, 4);
  }
  return WL_OK;
}

int wl_mlp_targets(const double* Df, const double* xan, int64_t rows, float* target, void* stream) {
  if (!Df || !xan || !target || rows < 0) return WL_ERR_INVALID_ARG;
  if (rows == 0) return WL_OK;
  cudaStream_t s = (cudaStream_t)stream;
  DevBuf bd, bx, bt;
  const void *D, *X;
  int rc;
  if ((rc = stage(Df, sizeof(double) * rows, bd, &D, s)) != WL_OK) return rc;
  if ((rc = stage(xan, sizeof(double) * rows, bx, &X, s)) != WL_OK) return rc;
  float* T = target;
  const bool dev_out = dev_ptr(target);
  if (!dev_out) {
    ML_CU(bt.alloc(sizeof(float) * rows));
    T = (float*)bt.p;
  }
  const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((rows + 255) / 256, 152 * 16));
  k_log_ratio<<<g, 256, 0, s>>>((const double*)D, (const double*)X, rows, T);
  ML_CU(cudaGetLastError());
  if (!dev_out) ML_CU(cudaMemcpyAsync(target, T, sizeof(float) * rows, cudaMemcpyDeviceToHost, s));
  ML_CU(cudaStreamSynchronize(s));
  return WL_OK;
}

}  // extern "C"
