// Lanczos kernels (Sec. 4.1: f(A) v ~ |v| Q_k f(H_k) e_1 with the Lanczos
// process for symmetric operators), all FP64.
//
//  lanczos_step    : one step of K lockstep Lanczos recurrences on the walk
//                    Laplacian, w = D_f (.) v - X (X = phi v from a CG solve) or
//                    w = Op v; alpha, beta, and the next basis block.
//  tridiag_exp     : y = exp(-tau T_m) e_1 for one (column, tau) per CTA by the
//                    Chebyshev expansion of the exponential, whose coefficients
//                    are scaled modified Bessel functions e^{-z} I_k(z)
//                    (computed by Miller's backward recurrence).
//  combine         : U(tau) = |u0| V_m y(tau), one read of the basis for all tau.
#pragma once
#include "wl_common.cuh"

namespace wl {

// ------------------------------------------------------------------ one Lanczos step on L
struct LanczosStepArgs {
  Graph g;
  Part pt;
  const double* vj;     // n x K
  const double* vjm1;   // n x K (ignored when first)
  const double* X;      // n x K: phi v_j from the inner solve (mode 0)
  const double* Df;     // n walk degrees (mode 0; NULL: zero)
  double c0, cA, cD;    // mode 1: w = Op v_j
  double* vjp1;         // n x K out
  double* Ta;           // K x ldT alphas
  double* Tb;           // K x ldT betas
  int* done;            // K flags (in/out)
  double* part;         // 2 * G * K
  GridBar* bar;
  int j;                // step index (0-based); T entries written at [c * ldT + j]
  int ldT;
  int mode;             // 0: w = Df v - X ; 1: w = Op v (gather)
};

template <int K>
__global__ void __launch_bounds__(kBlock, kMinBlocks) lanczos_step(LanczosStepArgs a) {
  using C = Cfg<double, K>;
  constexpr int VW = C::VW;
  constexpr int NW = kBlock / 32;
  __shared__ double s_tmp[kBlock];
  __shared__ double s_w[NW * K];
  __shared__ double s_red[K];
  __shared__ double s_alpha[K], s_bprev[K];
  __shared__ __align__(16) double s_gath[kBlock * VW];
  const int G = gridDim.x, cta = blockIdx.x, tid = threadIdx.x;
  const int r0 = a.pt.rb[cta], r1 = a.pt.rb[cta + 1];
  const size_t v0 = (size_t)r0 * K / VW, v1 = (size_t)r1 * K / VW;
  const int mycol = (tid % C::G) * VW;
  const bool first = (a.j == 0);
  double acc[VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) acc[v] = 0.0;
  if (a.mode == 0) {
#pragma unroll 2
    for (size_t e = v0 + tid; e < v1; e += kBlock) {
      const size_t row = e * VW / K;
      const double d = a.Df ? __ldg(a.Df + row) : 0.0;  // NULL: w = -X (shift-and-invert: X = -R v_j)
      const Pack<double, VW> vv = ldp<double, VW>(a.vj + e * VW);
      const Pack<double, VW> xx = ldp<double, VW>(a.X + e * VW);
      Pack<double, VW> ww;
#pragma unroll
      for (int v = 0; v < VW; ++v) {
        ww.v[v] = d * vv.v[v] - xx.v[v];
        acc[v] += vv.v[v] * ww.v[v];
      }
      stp<double, VW>(a.vjp1 + e * VW, ww);
    }
  } else {
    auto pre = [&](int row, int lane_off) { return ldp<double, VW>(a.vj + (size_t)row * K + lane_off); };
    auto fin = [&](int row, int deg, int lane_off, const double (&nb)[VW], const Pack<double, VW>& vv) {
      const size_t o = (size_t)row * K + lane_off;
      Pack<double, VW> ww;
#pragma unroll
      for (int v = 0; v < VW; ++v) {
        ww.v[v] = a.c0 * vv.v[v] + a.cA * nb[v] + a.cD * (double)deg * vv.v[v];
        acc[v] += vv.v[v] * ww.v[v];
      }
      stp<double, VW>(a.vjp1 + o, ww);
    };
    for_rows_gather<double, K>(a.g, a.pt, a.vj, s_gath, pre, fin);
  }
  cta_column_sums<double, K>(acc, s_w, a.part + (size_t)cta * K);
  if (!grid_sync(a.bar, G)) return;
  reduce_partials<K>(a.part, G, s_tmp, s_red);
  if (tid < K) {
    const int dn = a.done[tid];
    s_alpha[tid] = dn ? 0.0 : s_red[tid];
    s_bprev[tid] = (first || dn) ? 0.0 : a.Tb[tid * a.ldT + a.j - 1];
  }
  __syncthreads();
  double al[VW], bp[VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) {
    al[v] = s_alpha[mycol + v];
    bp[v] = s_bprev[mycol + v];
    acc[v] = 0.0;
  }
#pragma unroll 2
  for (size_t e = v0 + tid; e < v1; e += kBlock) {
    Pack<double, VW> ww = ldp<double, VW>(a.vjp1 + e * VW);
    const Pack<double, VW> vv = ldp<double, VW>(a.vj + e * VW);
    Pack<double, VW> vm;
    if (!first) vm = ldp<double, VW>(a.vjm1 + e * VW);
#pragma unroll
    for (int v = 0; v < VW; ++v) {
      ww.v[v] -= al[v] * vv.v[v];
      if (!first) ww.v[v] -= bp[v] * vm.v[v];
      acc[v] += ww.v[v] * ww.v[v];
    }
    stp<double, VW>(a.vjp1 + e * VW, ww);
  }
  cta_column_sums<double, K>(acc, s_w, a.part + (size_t)G * K + (size_t)cta * K);
  if (!grid_sync(a.bar, G)) return;
  reduce_partials<K>(a.part + (size_t)G * K, G, s_tmp, s_red);
  __shared__ double s_inv[K];
  if (tid < K) {
    const double b = sqrt(s_red[tid]);
    const int dn = a.done[tid];
    // invariant subspace reached (lucky breakdown): the column is exact
    const bool brk = dn || !(b > 1e-13 * (fabs(s_alpha[tid]) + s_bprev[tid] + 1e-300));
    s_inv[tid] = brk ? 0.0 : 1.0 / b;
    if (cta == 0) {
      a.Ta[tid * a.ldT + a.j] = s_alpha[tid];
      a.Tb[tid * a.ldT + a.j] = brk ? 0.0 : b;
      if (brk && !dn) a.done[tid] = 2;  // 2: converged by breakdown at this step
    }
  }
  __syncthreads();
  double iv[VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) iv[v] = s_inv[mycol + v];
  for (size_t e = v0 + tid; e < v1; e += kBlock) {
    Pack<double, VW> ww = ldp<double, VW>(a.vjp1 + e * VW);
#pragma unroll
    for (int v = 0; v < VW; ++v) ww.v[v] *= iv[v];
    stp<double, VW>(a.vjp1 + e * VW, ww);
  }
}

// ------------------------------------------------------------------ exp of the tridiagonal
struct TridiagArgs {
  const double* Ta;   // K x ldT
  const double* Tb;   // K x ldT
  const int* mcol;    // K: steps available per column
  const double* taus; // ntau
  double* y;          // K x ntau x ldT (out)
  double* yprev;      // K x ntau x ldT (previous result, updated in place after err)
  const int* mprev;   // K: length of yprev (0: none)
  double* err;        // K x ntau: |y - [yprev; 0]|_2 / |y|_2, or kErrVanished when y = 0
  int ldT;
  int ntau;
  int psd;            // 1: operator is PSD, use 0 as lower spectral bound
  int max_terms;      // cap of the expansion length
};

constexpr int kTridiagMax = 1024;   // max Lanczos steps handled per column
// err of a (column, tau) whose y underflowed to zero: the Krylov space does
// not yet reach the slow modes (exp(-tau L) conserves the mass 1^T u0, so the
// exact result of a start vector with mass never vanishes); never converged
constexpr double kErrVanished = 1e300;
constexpr int kChebMax = 2048;      // max Chebyshev terms (|tau| (hi - lo) / 2 up to ~4e4)
// dynamic shared memory of tridiag_exp: T (2 vectors), 3 recurrence vectors, coefficients
constexpr int kTridiagSmem = (5 * kTridiagMax + kChebMax) * (int)sizeof(double);

#ifdef WL_LANCZOS_KERNELS
__global__ void __launch_bounds__(kBlock) tridiag_exp(TridiagArgs a) {
  extern __shared__ __align__(16) double s_tri[];  // kTridiagSmem bytes
  double* const s_a = s_tri;                      // diagonal
  double* const s_b = s_tri + kTridiagMax;        // off-diagonal
  double* const s_v = s_tri + 2 * kTridiagMax;    // three Chebyshev vectors
  double* const s_c = s_tri + 5 * kTridiagMax;    // Chebyshev coefficients
  __shared__ double s_lohi[2];
  __shared__ int s_N;
  const int c = blockIdx.x, t = blockIdx.y, tid = threadIdx.x;
  const int m = a.mcol[c];
  const double tau = a.taus[t];
  for (int i = tid; i < m; i += kBlock) {
    s_a[i] = a.Ta[c * a.ldT + i];
    s_b[i] = (i + 1 < m) ? a.Tb[c * a.ldT + i] : 0.0;
  }
  __syncthreads();
  if (tid == 0) {
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < m; ++i) {
      const double r = (i > 0 ? fabs(s_b[i - 1]) : 0.0) + fabs(s_b[i]);
      lo = fmin(lo, s_a[i] - r);
      hi = fmax(hi, s_a[i] + r);
    }
    if (a.psd) lo = fmax(lo, 0.0);
    if (hi < lo) hi = lo;
    s_lohi[0] = lo;
    s_lohi[1] = hi;
    // coefficients of exp(-tau x) on [lo, hi] in Chebyshev polynomials of
    // t = (x - mid) / half: exp(-tau x) = exp(-tau mid) exp(-z t), z = tau half,
    // exp(-z t) = I_0(|z|) + 2 sum_k s^k I_k(|z|) T_k(t), s = -sign(z).
    const double half = 0.5 * (hi - lo);
    const double zz = fabs(tau) * half;
    int N = (int)ceil(sqrt(90.0 * zz) + 30.0);
    if (N > a.max_terms - 1) N = a.max_terms - 1;
    if (N > kChebMax - 1) N = kChebMax - 1;
    if (zz < 1e-30) {  // exp(-z t) = 1 + O(1e-30) on [-1, 1]
      s_c[0] = 1.0;
      N = 0;
    } else {
      // Miller: backward recurrence I_{k-1} = (2k / z) I_k + I_{k+1}, normalised
      // by I_0 + 2 sum I_k = e^z (so the stored values are e^{-z} I_k).
      const int M0 = 2 * N + 60;
      double ikp1 = 0.0, ik = 1e-280;
      for (int k = M0; k >= 1; --k) {
        const double ikm1 = (2.0 * k / zz) * ik + ikp1;
        ikp1 = ik;
        ik = ikm1;
        if (k - 1 <= N) s_c[k - 1] = ik;
        if (fabs(ik) > 1e250) {
          ik *= 1e-250;
          ikp1 *= 1e-250;
          for (int q = k - 1; q <= N; ++q) s_c[q] *= 1e-250;
        }
      }
      // ik now holds I_0 (scaled); complete the normalisation sum with the
      // tail k > N from the stored values only (the tail beyond N is < 1e-18).
      double S = s_c[0];
      for (int k = 1; k <= N; ++k) S += 2.0 * s_c[k];
      const double sgn = (tau >= 0.0) ? -1.0 : 1.0;
      double sk = 1.0;
      for (int k = 0; k <= N; ++k) {
        s_c[k] = (k == 0 ? 1.0 : 2.0) * sk * (s_c[k] / S);
        sk *= sgn;
      }
    }
    s_N = N;
  }
  __syncthreads();
  const double lo = s_lohi[0], hi = s_lohi[1];
  const double half = 0.5 * (hi - lo), mid = 0.5 * (hi + lo);
  const double zz = fabs(tau) * half;
  const double pref = exp(-tau * mid + zz);
  const int N = s_N;
  const double ih = (half > 0.0) ? 1.0 / half : 0.0;
  // Chebyshev three-term recurrence on vectors: v0 = e1, v1 = T~ e1,
  // v_{k+1} = 2 T~ v_k - v_{k-1}, T~ = (T - mid I) / half
  constexpr int RPT = kTridiagMax / kBlock;  // rows per thread
  double yacc[RPT];
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int i = tid + q * kBlock;
    yacc[q] = 0.0;
    if (i < m) {
      s_v[i] = (i == 0) ? 1.0 : 0.0;
      yacc[q] = s_c[0] * s_v[i];
    }
  }
  __syncthreads();
  int pv = 0, cv = 0, nv = 1;
  if (N >= 1) {
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      const int i = tid + q * kBlock;
      if (i < m) {
        double s = (s_a[i] - mid) * s_v[i];
        if (i > 0) s += s_b[i - 1] * s_v[i - 1];
        if (i + 1 < m) s += s_b[i] * s_v[i + 1];
        s_v[kTridiagMax + i] = s * ih;
        yacc[q] += s_c[1] * s_v[kTridiagMax + i];
      }
    }
    __syncthreads();
    pv = 0; cv = 1; nv = 2;
    for (int k = 2; k <= N; ++k) {
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        const int i = tid + q * kBlock;
        if (i < m) {
          double s = (s_a[i] - mid) * s_v[cv * kTridiagMax + i];
          if (i > 0) s += s_b[i - 1] * s_v[cv * kTridiagMax + i - 1];
          if (i + 1 < m) s += s_b[i] * s_v[cv * kTridiagMax + i + 1];
          const double nxt = 2.0 * s * ih - s_v[pv * kTridiagMax + i];
          s_v[nv * kTridiagMax + i] = nxt;
          yacc[q] += s_c[k] * nxt;
        }
      }
      __syncthreads();
      const int tmp = pv; pv = cv; cv = nv; nv = tmp;
    }
  }
  // write y and the change against the previous result
  double* yo = a.y + ((size_t)c * a.ntau + t) * a.ldT;
  double* yp = a.yprev + ((size_t)c * a.ntau + t) * a.ldT;
  const int mp = a.mprev[c];
  double e2 = 0.0, y2 = 0.0;
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int i = tid + q * kBlock;
    if (i < m) {
      const double yi = pref * yacc[q];
      yo[i] = yi;
      const double d = yi - (i < mp ? yp[i] : 0.0);
      e2 += d * d;
      y2 += yi * yi;
    }
  }
  s_v[tid] = e2;  // reuse (m may be < kBlock, slots are free after the loop)
  s_v[kBlock + tid] = y2;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0, sy = 0.0;
    for (int i = 0; i < kBlock; ++i) {
      s += s_v[i];
      sy += s_v[kBlock + i];
    }
    a.err[c * a.ntau + t] = sy > 0.0 ? sqrt(s / sy) : kErrVanished;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int i = tid + q * kBlock;
    if (i < m) yp[i] = yo[i];
  }
}

// One warp per (column, tau), for m <= kWarpRows: the same Chebyshev
// expansion summed by Clenshaw's backward recurrence, which runs in the same
// direction as Miller's recurrence for the Bessel coefficients, so neither
// the coefficients nor a block barrier is needed: every lane carries the
// scalar recurrence and kRowsPerLane consecutive rows of the vectors, and
// the tridiagonal product takes its two off-lane neighbours by shuffles.
// With B_{N+1} = B_{N+2} = 0 and B_k = c_k e_1 + 2 X B_{k+1} - B_{k+2}
// (X = (T - mid) / half), sum_{k<=N} c_k T_k(X) e_1 = c_0 e_1 + X B_1 - B_2.
constexpr int kRowsPerLane = 4;
constexpr int kWarpRows = 32 * kRowsPerLane;

__global__ void __launch_bounds__(128) tridiag_exp_warp(TridiagArgs a, int K) {
  const int lane = threadIdx.x & 31;
  const int pair = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int c = pair / a.ntau, t = pair % a.ntau;
  if (c >= K) return;  // whole warp
  const int m = a.mcol[c];
  const double tau = a.taus[t];
  const double* Ta = a.Ta + (size_t)c * a.ldT;
  const double* Tb = a.Tb + (size_t)c * a.ldT;
  // rows i = lane * R + q of this lane
  constexpr int R = kRowsPerLane;
  double al[R], bl[R], bm;  // diagonal, coupling to row i+1, coupling of the lane's first row to row i-1
  double lo = 1e300, hi = -1e300;
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int i = lane * R + q;
    al[q] = (i < m) ? Ta[i] : 0.0;
    bl[q] = (i + 1 < m) ? Tb[i] : 0.0;
  }
  bm = (lane * R > 0 && lane * R < m) ? Tb[lane * R - 1] : 0.0;
  // Gershgorin bounds
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int i = lane * R + q;
    if (i < m) {
      const double left = (q == 0) ? fabs(bm) : fabs(bl[q - 1]);
      const double r = left + fabs(bl[q]);
      lo = fmin(lo, al[q] - r);
      hi = fmax(hi, al[q] + r);
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, off));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, off));
  }
  if (a.psd) lo = fmax(lo, 0.0);
  if (hi < lo) hi = lo;
  const double half = 0.5 * (hi - lo), mid = 0.5 * (hi + lo);
  const double zz = fabs(tau) * half;
  const double pref = exp(-tau * mid + zz);
  const double ih = (half > 0.0) ? 1.0 / half : 0.0;
  int N = (int)ceil(sqrt(90.0 * zz) + 30.0);
  if (N > a.max_terms - 1) N = a.max_terms - 1;
  if (N > kChebMax - 1) N = kChebMax - 1;
  double yv[R];
  if (zz < 1e-30) {  // exp(-z x) = 1 + O(1e-30) on [-1, 1]
#pragma unroll
    for (int q = 0; q < R; ++q) yv[q] = (lane * R + q == 0) ? pref : 0.0;
  } else {
    // X v for the lane's rows (shuffles for the neighbours across lanes)
    auto xmul = [&](const double (&v)[R], double (&out)[R]) {
      const double prev = __shfl_up_sync(0xffffffffu, v[R - 1], 1);
      const double next = __shfl_down_sync(0xffffffffu, v[0], 1);
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const double vm = (q == 0) ? (lane > 0 ? prev : 0.0) : v[q - 1];
        const double vp = (q == R - 1) ? (lane < 31 ? next : 0.0) : v[q + 1];
        const double bmq = (q == 0) ? bm : bl[q - 1];
        out[q] = ((al[q] - mid) * v[q] + bmq * vm + bl[q] * vp) * ih;
      }
    };
    const double sgn = (tau >= 0.0) ? -1.0 : 1.0;
    const int M0 = 2 * N + 60;
    const double tz = 2.0 / zz;
    double ikp1 = 0.0, ik = 1e-280;  // Miller: I_{k-1} = (2k / z) I_k + I_{k+1}
    double b1[R], b2[R];             // B_{k+1}, B_{k+2}
#pragma unroll
    for (int q = 0; q < R; ++q) b1[q] = b2[q] = 0.0;
    double S = 0.0;                  // I_0 + 2 sum_{k=1}^{N} I_k (unnormalised)
    double c0 = 0.0;
    for (int k = M0; k >= 1; --k) {
      const double ikm1 = (tz * k) * ik + ikp1;
      ikp1 = ik;
      ik = ikm1;  // I_{k-1}
      const int kk = k - 1;
      if (kk <= N) {
        const double ck = (kk == 0 ? 1.0 : 2.0) * ((kk & 1) ? sgn : 1.0) * ik;
        S += (kk == 0 ? 1.0 : 2.0) * ik;
        if (kk >= 1) {
          double xb[R];
          xmul(b1, xb);
#pragma unroll
          for (int q = 0; q < R; ++q) {
            const double bk = ((lane * R + q == 0) ? ck : 0.0) + 2.0 * xb[q] - b2[q];
            b2[q] = b1[q];
            b1[q] = bk;
          }
        } else {
          c0 = ck;
        }
      }
      if (fabs(ik) > 1e250) {  // rescale everything linear in the I_k
        ik *= 1e-250;
        ikp1 *= 1e-250;
        S *= 1e-250;
        c0 *= 1e-250;
#pragma unroll
        for (int q = 0; q < R; ++q) {
          b1[q] *= 1e-250;
          b2[q] *= 1e-250;
        }
      }
    }
    // sum = c0 e_1 + X B_1 - B_2, normalised by S
    double xb[R];
    xmul(b1, xb);
    const double sc = pref / S;
#pragma unroll
    for (int q = 0; q < R; ++q) yv[q] = sc * (((lane * R + q == 0) ? c0 : 0.0) + xb[q] - b2[q]);
  }
  // write y and the change against the previous result
  double* yo = a.y + ((size_t)c * a.ntau + t) * a.ldT;
  double* yp = a.yprev + ((size_t)c * a.ntau + t) * a.ldT;
  const int mp = a.mprev[c];
  double e2 = 0.0, y2 = 0.0;
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int i = lane * R + q;
    if (i < m) {
      yo[i] = yv[q];
      const double d = yv[q] - (i < mp ? yp[i] : 0.0);
      e2 += d * d;
      y2 += yv[q] * yv[q];
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    e2 += __shfl_xor_sync(0xffffffffu, e2, off);
    y2 += __shfl_xor_sync(0xffffffffu, y2, off);
  }
  if (lane == 0) a.err[c * a.ntau + t] = y2 > 0.0 ? sqrt(e2 / y2) : kErrVanished;
  __syncwarp();
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int i = lane * R + q;
    if (i < m) yp[i] = yv[q];
  }
}

#endif  // WL_LANCZOS_KERNELS

// ------------------------------------------------------------------ U = |u0| V y
struct CombineArgs {
  const double* basis;  // m blocks of n x K (block j at basis + j n K)
  const double* y;      // K x ntau x ldT
  const int* mcol;      // K: steps per column
  const double* nrm;    // K: |u0_c|
  double* out;          // ntau blocks, element (t, i, c) at out[t * tstride + i * ld + c0 + c]
  int64_t n;
  int64_t ld;
  int64_t tstride;
  int c0;
  int ldT;
  int ntau;
  const int32_t* perm;  // internal row i goes to caller row perm[i] (NULL: identity)
};

constexpr int kMaxTau = 8;

template <int K>
__global__ void __launch_bounds__(kBlock) combine(CombineArgs a) {
  const size_t total = (size_t)a.n * K;
  for (size_t e = (size_t)blockIdx.x * kBlock + threadIdx.x; e < total; e += (size_t)gridDim.x * kBlock) {
    const int c = (int)(e % K);
    const size_t i = e / K;
    const int m = a.mcol[c];
    double acc[kMaxTau];
#pragma unroll
    for (int t = 0; t < kMaxTau; ++t) acc[t] = 0.0;
    const double* yc = a.y + (size_t)c * a.ntau * a.ldT;
    for (int j = 0; j < m; ++j) {
      const double vij = __ldcs(a.basis + (size_t)j * total + e);
#pragma unroll
      for (int t = 0; t < kMaxTau; ++t)
        if (t < a.ntau) acc[t] += vij * __ldg(yc + (size_t)t * a.ldT + j);
    }
    const double s = a.nrm[c];
    const size_t io = a.perm ? (size_t)a.perm[i] : i;
    for (int t = 0; t < a.ntau; ++t) a.out[(size_t)t * a.tstride + io * a.ld + a.c0 + c] = s * acc[t];
  }
}

}  // namespace wl
