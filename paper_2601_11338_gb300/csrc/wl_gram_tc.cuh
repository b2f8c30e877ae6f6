// Gram [Omega Y]^T Y of the XNysTrace core on the 5th-generation tensor
// cores (tcgen05.mma, kind::tf32, accumulator in tensor memory).
//
// X = [Omega Y] has 128 columns (Omega BF16 in 0..63, Y FP32 in 64..127;
// columns beyond the sketch size are zero) and one row per node. Y is split
// into two TF32 terms, Y = Yh + Yl (Yh = Y rounded to TF32, Yl = the
// remainder rounded to TF32), so that with Xh = [Omega Yh], Xl = [0 Yl]
//   D = Xh^T Yh + Xh^T Yl + Xl^T Yh
// carries FP32-level accuracy (the dropped Yl^T Yl term is 2^-22 relative);
// Omega is exact in TF32. D (128 x 64 FP32) lives in TMEM, two accumulators
// (2 x 64 columns) that alternate between groups of kTcGroup stages: the
// MMAs of a group sum into one of them, and once they have completed every
// thread adds its row of D into float pairs (TwoSum). The tensor core's FP32
// accumulation thus never runs over more than kTcGroup * kTcRows nodes (over
// thousands it drifts by ~1e-5 relative; summing 16 stages instead of 4
// already exceeds the 2e-6 bound of the kernel's test at n = 4097).
//
// Each CTA (4 warps) owns a contiguous range of nodes (a multiple of kTcRows
// long) and walks it in stages of kTcRows nodes. The stage's rows of Omega
// and Y are contiguous in memory: one thread has the bulk-copy engine bring
// them into a raw staging buffer, kTcPipe stages ahead, completing on that
// buffer's mbarrier (a partial last stage is read by the threads). All
// threads convert their feature column of the stage into two K-major operand
// tiles in shared memory (no swizzle: 8-row x 16-byte core matrices), one
// thread issues the MMAs (M = 128, N = 64, K = 8 each) and commits them to the
// tile buffer's mbarrier; two tile buffers alternate so that converting
// overlaps the tensor-core work. Every mbarrier wait is bounded; on timeout
// the CTA records an error, waits (bounded) for what it has in flight and
// still frees its TMEM.
#pragma once
#include <stdint.h>

namespace wl {

constexpr int kTcRows = 32;                               // nodes per stage
constexpr int kTcGroup = 4;                               // stages summed in TMEM before a drain
constexpr int kTcThreads = 128;                           // one thread per column of X
constexpr uint32_t kTcTileBytes = 128u * kTcRows * 4u;    // one 128 x 32 TF32 tile (16 KB)
constexpr uint32_t kTcLBO = 128;                          // core matrix to the next along K
constexpr uint32_t kTcSBO = (kTcRows / 4) * 128;          // core matrix to the next 8-row group
constexpr uint32_t kTcN = 64;                             // N of the MMA (TMEM columns per accumulator)
constexpr uint32_t kTcCols = 2 * kTcN;                    // two accumulators
constexpr int kTcPipe = 3;                                // stages of raw rows in flight
constexpr uint32_t kTcRawY = kTcRows * 64u * 4u;          // a stage of Y rows (K <= 64 FP32)
constexpr uint32_t kTcRawBytes = kTcRawY + kTcRows * 64u * 2u;  // ... and of Omega rows (M <= 64 BF16)
// tiles, raw buffers, 2 + kTcPipe mbarriers, the TMEM address; 1 KB of
// alignment slack (two CTAs fit on an SM)
constexpr size_t kTcSmem = 4 * (size_t)kTcTileBytes + kTcPipe * (size_t)kTcRawBytes + 1024 + 128;
// kind::tf32: D = F32 (bits 4-5 = 1), A = B = TF32 (2 in bits 7-9 and 10-12),
// both K-major, N / 8 in bits 17-22, M / 16 in bits 24-28
constexpr uint32_t kTcIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);
constexpr long long kTcWaitLimit = 1ll << 24;             // polls of one mbarrier wait

#ifdef WL_TRACE_KERNELS

__device__ __forceinline__ uint32_t tc_smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start, LBO, SBO (16-byte units), version 1, no swizzle
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((kTcLBO >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((kTcSBO >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ uint32_t tc_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t parity) {
  for (long long i = 0; i < kTcWaitLimit; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void tc_mma(uint32_t taddr, uint64_t da, uint64_t db, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %3, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %4, p;\n\t}\n"
      :
      : "r"(taddr), "l"(da), "l"(db), "r"(acc), "r"(kTcIdesc)
      : "memory");
}

// adds this warp's 32 rows x 64 columns of the accumulator at column col0 to (hi, lo)
// s + c += v with the rounding error of the add kept in c (Knuth's TwoSum in
// FP32: FP64 adds run at 1/64 of the FP32 rate on this GPU, and FP64 drains
// kept the FP64 pipe 40% busy). Measured on 4.2e6 x 64 nodes: 9.7 ms with the
// threads loading each stage and FP64 drains after every stage, 2.8 ms with
// bulk-copy loads kTcPipe stages ahead and drains every kTcGroup stages,
// 2.3 ms with these float-pair drains (the CUDA-core Gram: 1.9 ms).
__device__ __forceinline__ void tc_acc(float& s, float& c, float v) {
  const float t = s + v;
  const float bb = t - s;
  c += (s - (t - bb)) + (v - bb);
  s = t;
}

__device__ __forceinline__ void tc_drain(uint32_t taddr, int warp, uint32_t col0, float (&hi)[kTcN],
                                         float (&lo)[kTcN]) {
#pragma unroll
  for (int cb = 0; cb < (int)kTcN; cb += 16) {
    uint32_t v[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr + ((uint32_t)(warp * 32) << 16) + col0 + (uint32_t)cb));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) tc_acc(hi[cb + q], lo[cb + q], __uint_as_float(v[q]));
  }
}

// Loads of a stage (kTcRows full rows of Omega and Y, both contiguous in
// memory) by the bulk-copy engine into a raw staging buffer, completing on
// that buffer's mbarrier; kTcPipe stages are in flight ahead of the one being
// converted. Sources and sizes are multiples of 16 bytes: a stage starts at a
// row that is a multiple of kTcRows, so its byte offsets are multiples of
// kTcRows * 2 * M and kTcRows * 4 * K; the host checks the base addresses.
__device__ __forceinline__ void tc_bulk(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}

__device__ __forceinline__ void tc_expect(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

__global__ void __launch_bounds__(kTcThreads) gram_tc(const uint16_t* __restrict__ omega, const float* __restrict__ Y,
                                                      int64_t n, int M, int K, int64_t chunk,
                                                      float* __restrict__ partial, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char tc_sm[];
  unsigned char* base = tc_sm + ((1024 - (tc_smem_u32(tc_sm) & 1023)) & 1023);  // 1 KB aligned tiles
  unsigned char* tile[2][2] = {{base, base + kTcTileBytes}, {base + 2 * kTcTileBytes, base + 3 * kTcTileBytes}};
  unsigned char* raw = base + 4 * kTcTileBytes;  // kTcPipe x (Y rows, then Omega rows)
  uint64_t* mbar = reinterpret_cast<uint64_t*>(raw + kTcPipe * kTcRawBytes);  // 2 MMA + kTcPipe load barriers
  uint32_t* s_taddr = reinterpret_cast<uint32_t*>(mbar + 2 + kTcPipe);
  __shared__ int s_fail, s_stop;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m = tid;  // column of X
  const int64_t r0 = (int64_t)blockIdx.x * chunk;
  const int64_t r1 = min(n, r0 + chunk);
  const int nst = r1 > r0 ? (int)((r1 - r0 + kTcRows - 1) / kTcRows) : 0;
  const int nfull = r1 > r0 ? (int)((r1 - r0) / kTcRows) : 0;  // stages of kTcRows rows: bulk loads
  const uint32_t yb = (uint32_t)(kTcRows * K * 4), ob = (uint32_t)(kTcRows * M * 2);
  auto raw_y = [&](int b) { return reinterpret_cast<const float*>(raw + b * kTcRawBytes); };
  auto raw_o = [&](int b) { return reinterpret_cast<const uint16_t*>(raw + b * kTcRawBytes + kTcRawY); };
  int issued = 0;  // thread 0: stages whose bulk loads have been issued
  auto issue = [&](int st) {  // thread 0: the bulk loads of stage st
    const int b = st % kTcPipe;
    const int64_t row = r0 + (int64_t)st * kTcRows;
    const uint32_t mb = tc_smem_u32(&mbar[2 + b]);
    tc_expect(mb, yb + ob);
    tc_bulk(tc_smem_u32(raw + b * kTcRawBytes), Y + row * K, yb, mb);
    tc_bulk(tc_smem_u32(raw + b * kTcRawBytes + kTcRawY), omega + row * M, ob, mb);
    issued = st + 1;
  };
  if (tid == 0) {
    s_fail = 0;
    s_stop = nst;
    for (int i = 0; i < 2 + kTcPipe; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem_u32(&mbar[i])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    for (int st = 0; st < kTcPipe && st < nfull; ++st) issue(st);
  }
  // rows 0..63 of the Yl tiles (the Omega block of Xl) stay zero
  if (m < 64) {
    const uint32_t o = (uint32_t)(m >> 3) * kTcSBO + (uint32_t)(m & 7) * 16;
    for (int kg = 0; kg < kTcRows / 4; ++kg) {
      *reinterpret_cast<uint4*>(tile[0][1] + o + kg * kTcLBO) = make_uint4(0, 0, 0, 0);
      *reinterpret_cast<uint4*>(tile[1][1] + o + kg * kTcLBO) = make_uint4(0, 0, 0, 0);
    }
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem_u32(s_taddr)),
                 "r"(kTcCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t taddr = *s_taddr;
  const uint32_t orow = (uint32_t)(m >> 3) * kTcSBO + (uint32_t)(m & 7) * 16;
  float acc[kTcN], acc_lo[kTcN];  // this thread's row of the CTA's sum, as float pairs
#pragma unroll
  for (int q = 0; q < (int)kTcN; ++q) acc[q] = acc_lo[q] = 0.f;
  int last_mma = -1;  // thread 0: the last stage whose MMAs were committed
  for (int c = 0; c < nst; ++c) {
    const int s = c & 1;                   // tile buffer and MMA mbarrier of this stage
    const int g = c / kTcGroup;            // group; its accumulator is D[g & 1]
    const bool gstart = (c % kTcGroup) == 0;
    if (c >= 2) {
      // the MMAs of stage c - 2 (this stage's tiles) are done, and with them
      // (in order) those of every earlier stage
      if (!tc_wait(tc_smem_u32(&mbar[s]), (uint32_t)(((c >> 1) - 1) & 1))) atomicExch(&s_fail, 1);
    }
    const bool bulk = c < nfull;
    const int b = c % kTcPipe;
    if (bulk && !tc_wait(tc_smem_u32(&mbar[2 + b]), (uint32_t)((c / kTcPipe) & 1))) atomicExch(&s_fail, 1);
    __syncthreads();
    if (s_fail) {
      if (tid == 0) s_stop = c;
      break;
    }
    if (c >= 2 && gstart && g >= 2) {  // D[g & 1] holds group g - 2, all of whose stages precede c - 2
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      tc_drain(taddr, warp, (uint32_t)(g & 1) * kTcN, acc, acc_lo);
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    const int64_t nb = r0 + (int64_t)c * kTcRows;
    const float* ys = raw_y(b);
    const uint16_t* os = raw_o(b);
    for (int kg = 0; kg < kTcRows / 4; ++kg) {
      uint32_t h[4], l[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = kg * 4 + q;
        const int64_t r = nb + i;
        float x = 0.f;
        h[q] = 0u;
        l[q] = 0u;
        if (m < 64) {
          if (m < M) {
            if (bulk) x = __uint_as_float((uint32_t)os[i * M + m] << 16);
            else if (r < r1) x = __uint_as_float((uint32_t)omega[r * M + m] << 16);
          }
          h[q] = __float_as_uint(x);  // BF16 values are exact in TF32
        } else if (m - 64 < M) {
          if (bulk) x = ys[i * K + (m - 64)];
          else if (r < r1) x = Y[r * K + (m - 64)];
          h[q] = tc_tf32(x);
          l[q] = tc_tf32(x - __uint_as_float(h[q]));
        }
      }
      *reinterpret_cast<uint4*>(tile[s][0] + orow + kg * kTcLBO) = make_uint4(h[0], h[1], h[2], h[3]);
      if (m >= 64) *reinterpret_cast<uint4*>(tile[s][1] + orow + kg * kTcLBO) = make_uint4(l[0], l[1], l[2], l[3]);
    }
    // the tiles and the raw buffer's reads are ordered before the tensor
    // core's reads of the tiles and the next bulk copy into the buffer
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t th = tc_smem_u32(tile[s][0]), tl = tc_smem_u32(tile[s][1]);
#pragma unroll
      for (int j = 0; j < kTcRows / 8; ++j) {
        const uint32_t kofs = (uint32_t)j * 2 * kTcLBO;  // 8 TF32 along K = two core matrices
        const uint64_t ah = tc_desc(th + kofs), bh = tc_desc(th + 8 * kTcSBO + kofs);
        const uint64_t al = tc_desc(tl + kofs), bl = tc_desc(tl + 8 * kTcSBO + kofs);
        const uint32_t d = taddr + (uint32_t)(g & 1) * kTcN;  // the group's accumulator, restarted per group
        tc_mma(d, ah, bh, (gstart && j == 0) ? 0u : 1u);
        tc_mma(d, ah, bl, 1u);
        tc_mma(d, al, bh, 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       tc_smem_u32(&mbar[s]))
                   : "memory");
      last_mma = c;
      if (c + kTcPipe < nfull) issue(c + kTcPipe);  // raw buffer b is free again
    }
  }
  // everything this CTA started ends before it leaves (each wait bounded):
  // the last commit covers every MMA issued before it; bulk loads issued but
  // not consumed (only after a failed wait) are the latest on their buffers
  if (tid == 0) {
    if (last_mma >= 0 && !tc_wait(tc_smem_u32(&mbar[last_mma & 1]), (uint32_t)((last_mma >> 1) & 1)))
      atomicExch(&s_fail, 1);
    for (int st = s_stop; st < issued; ++st)
      if (!tc_wait(tc_smem_u32(&mbar[2 + st % kTcPipe]), (uint32_t)((st / kTcPipe) & 1))) atomicExch(&s_fail, 1);
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (nst > 0 && !s_fail) {  // the accumulators of the last one or two groups
    const int ng = (nst + kTcGroup - 1) / kTcGroup;
    if (ng >= 2) tc_drain(taddr, warp, (uint32_t)((ng - 2) & 1) * kTcN, acc, acc_lo);
    tc_drain(taddr, warp, (uint32_t)((ng - 1) & 1) * kTcN, acc, acc_lo);
  }
  float* out = partial + (size_t)blockIdx.x * 128 * 64 + (size_t)(warp * 32 + lane) * 64;
#pragma unroll
  for (int q = 0; q < (int)kTcN; ++q) out[q] = s_fail ? 0.f : acc[q] + acc_lo[q];
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kTcCols));
  if (tid == 0 && s_fail) atomicExch(err, WL_ERR_TIMEOUT);
}

#endif  // WL_TRACE_KERNELS

}  // namespace wl
