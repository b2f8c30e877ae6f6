// Batched executor: many graphs x many mu values, walk degrees and walk
// Laplacian applies for all of them from one CUDA graph launch.
//
// Build: the graphs are validated and their spectral scales found
// (lambda_max(A), rho(Z_mu) per graph and mu, Sec. 4.1; alpha = alpha_rel /
// rho(Z_mu) per problem), then concatenated into one block-diagonal CSR on
// the device and cut into tiles (wl_batch.cuh).
//
// Run: one CUDA graph holds the D_f solve (K = 1, right-hand side
// (1 - mu^2 alpha^2) 1, so x = phi 1 = D_f), the solve M X = V for the
// caller's K columns, and W = D_f (.) V - (1 - mu^2 alpha^2) X for every
// problem. Each solve's iteration loop is a conditional while node whose
// condition the last kernel of the body sets on the device, so the host
// issues one launch and no synchronisation inside the solve; the refined
// form nests the FP32 CG loop inside the FP64 refinement loop. Every loop
// is bounded on the device (per-problem iteration caps and a hard cap on
// body executions), so the graph always ends.
//
// The rows per plain tile are tuned once per (K, form) by timing the S
// kernel on the batch itself for a few tile heights.
#define WL_BATCH_KERNELS
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "wl.h"
#include "wl_batch.cuh"
#include "wl_host.h"

using namespace wl;

namespace {

// spectral scales of the batch: lambda_max(A) and rho(Z_mu) to 1e-10
// relative (alpha = alpha_rel / rho needs no more); up to 128 graphs'
// searches in flight together
constexpr double kSpecRtol = 1e-10;
constexpr int kSpecThreads = 128;

constexpr int kLoopHardCap = 1 << 20;  // body executions of one while node, whatever the flags say

struct DBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

// growth and release happen only between runs (every run ends synchronised)
cudaError_t dalloc(DBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return cudaSuccess;
  pool_free(b.p);
  b.p = nullptr;
  b.bytes = 0;
  cudaError_t e = pool_malloc(&b.p, bytes);
  if (e == cudaSuccess) b.bytes = bytes;
  return e;
}

void dfree(DBuf& b) {
  pool_free(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

int cuerr(cudaError_t e, const char* where) { return report_cuda_error(e, where); }

#define BT_CU(call)                                        \
  do {                                                     \
    cudaError_t e__ = (call);                              \
    if (e__ != cudaSuccess) return cuerr(e__, #call);      \
  } while (0)
#define BT_TRY(call)              \
  do {                            \
    int s__ = (call);             \
    if (s__ != WL_OK) return s__; \
  } while (0)

bool valid_k(int k) { return k == 1 || k == 2 || k == 4 || k == 8 || k == 16 || k == 32 || k == 64; }

struct TileSet {
  int R = 0;  // rows per plain tile
  int ntile = 0;
  DBuf tiles, tile_beg;
};

// device buffers of one solve width K
struct SolveBufs {
  int K = 0;
  DBuf x, r, p, q;      // FP64 form: doubles; refined: x = d32, r/p/q FP32
  DBuf x64;             // refined form: FP64 iterate
  DBuf rdf;             // refined form: double-float residual (rh then rl, FP32 each)
  DBuf part;            // [nslab][ntile][2K] doubles
  DBuf colstate;        // gamma, alpha, beta, b2, rn2, bn2 (doubles) per problem-column
  DBuf colint;          // done, status, skip, ostatus (ints) per problem-column
  DBuf probint;         // active, iters, outer_active, outer_iters, total iters (ints) per problem
  DBuf flags;           // any_inner, any_outer, host copy, loop counters (ints)
};

struct Exec {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

}  // namespace

struct wl_batch {
  int ngraph = 0, nslab = 0;
  int64_t n = 0, nnz = 0;
  wl_params prm;
  cudaStream_t stream = nullptr;
  cudaStream_t cap[3] = {nullptr, nullptr, nullptr};
  std::vector<int32_t> goff_h;
  std::vector<int32_t> rp_h;  // concatenated row_ptr (host copy, for tiling)
  DBuf rp, col, goff;
  std::vector<TileSet> tilesets;       // candidate tile heights
  std::map<int, int> tuned;            // K * 2 + refined -> tileset index
  std::vector<double> mu, lmax, rho, alpha, phi;  // per graph / per problem
  DBuf ca, cA, cD, phis;                           // per problem (device)
  DBuf ones;                                       // n doubles = 1
  DBuf Vin, Df, W;                                 // staged input and outputs
  SolveBufs sb1, sbk;
  std::map<int, Exec> execs;                       // K * 2 + refined -> graph
  // per-problem results of the last run
  std::vector<int> iters_df, iters_v, outer_df, outer_v, status_p;
  std::vector<double> relres_df, relres_v;
  int* h_pin = nullptr;
};

namespace {

int nprob(const wl_batch* b) { return b->ngraph * b->nslab; }

BatchGraph bgraph(const wl_batch* b, const TileSet& t) {
  return BatchGraph{(const int32_t*)b->rp.p, (const int32_t*)b->col.p, (const BTile*)t.tiles.p,
                    (const int32_t*)t.tile_beg.p, (const int32_t*)b->goff.p, t.ntile, b->ngraph, b->n};
}

// tiles of R rows within each graph; one extra tile per hub row
int make_tiles(wl_batch* b, int R, TileSet& t) {
  std::vector<BTile> tl;
  std::vector<int32_t> tb(b->ngraph + 1, 0);
  for (int g = 0; g < b->ngraph; ++g) {
    tb[g] = (int32_t)tl.size();
    const int32_t r0 = b->goff_h[g], r1 = b->goff_h[g + 1];
    for (int32_t r = r0; r < r1; r += R) tl.push_back(BTile{r, std::min(r1, r + R), g, 0});
    for (int32_t r = r0; r < r1; ++r)
      if (b->rp_h[r + 1] - b->rp_h[r] > kHubDeg) tl.push_back(BTile{r, r + 1, g, 1});
  }
  tb[b->ngraph] = (int32_t)tl.size();
  t.R = R;
  t.ntile = (int)tl.size();
  if (t.ntile > 0x7fffffff / 2) return WL_ERR_INVALID_ARG;
  BT_CU(dalloc(t.tiles, sizeof(BTile) * std::max<size_t>(tl.size(), 1)));
  BT_CU(dalloc(t.tile_beg, sizeof(int32_t) * tb.size()));
  if (!tl.empty()) BT_CU(cudaMemcpy(t.tiles.p, tl.data(), sizeof(BTile) * tl.size(), cudaMemcpyHostToDevice));
  BT_CU(cudaMemcpy(t.tile_beg.p, tb.data(), sizeof(int32_t) * tb.size(), cudaMemcpyHostToDevice));
  return WL_OK;
}

int max_tiles(const wl_batch* b) {
  int m = 0;
  for (const auto& t : b->tilesets) m = std::max(m, t.ntile);
  return m;
}

int alloc_solve(wl_batch* b, SolveBufs& s, int K) {
  s.K = K;
  const size_t elems = (size_t)b->nslab * b->n * K;
  const size_t np = nprob(b), nc = np * K;
  BT_CU(dalloc(s.x, elems * 8));
  BT_CU(dalloc(s.r, elems * 8));
  BT_CU(dalloc(s.p, elems * 8));
  BT_CU(dalloc(s.q, elems * 8));
  BT_CU(dalloc(s.x64, elems * 8));
  if (b->prm.prec == WL_REFINED) BT_CU(dalloc(s.rdf, elems * 8));
  BT_CU(dalloc(s.part, (size_t)b->nslab * std::max(max_tiles(b), 1) * 2 * K * 8));
  BT_CU(dalloc(s.colstate, nc * 6 * 8));
  BT_CU(dalloc(s.colint, nc * 4 * 4));
  BT_CU(dalloc(s.probint, np * 5 * 4));
  BT_CU(dalloc(s.flags, 64 * 4));
  return WL_OK;
}

// state views
BatchState bstate(const wl_batch* b, SolveBufs& s) {
  const size_t nc = (size_t)nprob(b) * s.K, np = nprob(b);
  double* cs = (double*)s.colstate.p;
  int* ci = (int*)s.colint.p;
  int* pi = (int*)s.probint.p;
  int* fl = (int*)s.flags.p;
  return BatchState{cs, cs + nc, cs + 2 * nc, cs + 3 * nc, ci, ci + nc, pi, pi + np, pi + 4 * np, fl + 0};
}

BatchOuter bouter(const wl_batch* b, SolveBufs& s) {
  const size_t nc = (size_t)nprob(b) * s.K, np = nprob(b);
  double* cs = (double*)s.colstate.p;
  int* ci = (int*)s.colint.p;
  int* pi = (int*)s.probint.p;
  int* fl = (int*)s.flags.p;
  return BatchOuter{cs + 4 * nc, cs + 5 * nc, ci + 2 * nc, pi + 2 * np, pi + 3 * np, ci + 3 * nc, fl + 1};
}

int* host_copy_flag(SolveBufs& s) { return (int*)s.flags.p + 2; }
int* loop_counter(SolveBufs& s, int depth) { return (int*)s.flags.p + 4 + depth; }

__global__ void bfill_int(int* p, int n, int v) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = v;
}

// Reads and clears `any`, bounds the number of body executions, and sets
// the while node's condition (graph mode) or a device copy (stepped mode).
__global__ void bloop_cond(int* any, int* host_copy, int* counter, int cap, unsigned long long handle, int graph_mode) {
  int v = *(volatile int*)any;
  *any = 0;
  const int c = *counter + 1;
  *counter = c;
  if (c > cap) v = 0;
  if (host_copy) *host_copy = v;
  if (graph_mode) cudaGraphSetConditional((cudaGraphConditionalHandle)handle, v ? 1u : 0u);
}

// Emits a sequence of launches either into a CUDA graph under construction
// (while nodes for loops) or directly on a stream (loops driven by the host,
// one flag read per iteration: the stepped mode used to check the graph).
struct Emitter {
  bool graph;
  cudaStream_t st[3];
  int depth = 0;
  int* host_pin = nullptr;
  cudaStream_t s() const { return st[depth]; }

  template <class Body>
  int loop(SolveBufs& sb, int* any, int cap, Body body) {
    int* counter = loop_counter(sb, depth);
    cap = std::min(cap, kLoopHardCap);
    if (!graph) {
      BT_CU(cudaMemsetAsync(counter, 0, sizeof(int), s()));
      if (depth + 1 >= 3) return WL_ERR_INVALID_ARG;
      int rc = WL_OK;
      for (int guard = 0; guard <= cap + 1 && rc == WL_OK; ++guard) {
        bloop_cond<<<1, 1, 0, s()>>>(any, host_copy_flag(sb), counter, cap, 0ull, 0);
        BT_CU(cudaGetLastError());
        BT_CU(cudaMemcpyAsync(host_pin, host_copy_flag(sb), sizeof(int), cudaMemcpyDeviceToHost, s()));
        BT_CU(cudaStreamSynchronize(s()));
        if (!*host_pin) break;
        ++depth;  // nested loops keep their own body counters, as in the graph
        rc = body();
        --depth;
      }
      return rc;
    }
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    BT_CU(cudaMemsetAsync(counter, 0, sizeof(int), s()));
    BT_CU(cudaStreamGetCaptureInfo(s(), &cs, nullptr, &g, nullptr, nullptr, nullptr));
    cudaGraphConditionalHandle h;
    BT_CU(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
    bloop_cond<<<1, 1, 0, s()>>>(any, nullptr, counter, cap, (unsigned long long)h, 1);  // entry condition
    BT_CU(cudaGetLastError());
    BT_CU(cudaStreamGetCaptureInfo(s(), &cs, nullptr, &g, &deps, nullptr, &nd));
    alignas(cudaGraphNodeParams) unsigned char np_raw[sizeof(cudaGraphNodeParams)];
    memset(np_raw, 0, sizeof(np_raw));
    cudaGraphNodeParams& np = *reinterpret_cast<cudaGraphNodeParams*>(np_raw);
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    BT_CU(cudaGraphAddNode(&node, g, deps, nullptr, nd, &np));
    cudaGraph_t body_graph = np.conditional.phGraph_out[0];
    BT_CU(cudaStreamUpdateCaptureDependencies(s(), &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    if (depth + 1 >= 3) return WL_ERR_INVALID_ARG;
    ++depth;
    cudaError_t e = cudaStreamBeginCaptureToGraph(s(), body_graph, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
      --depth;
      return cuerr(e, "cudaStreamBeginCaptureToGraph");
    }
    int rc = body();
    if (rc == WL_OK) {
      bloop_cond<<<1, 1, 0, s()>>>(any, nullptr, counter, cap, (unsigned long long)h, 1);
      if (cudaGetLastError() != cudaSuccess) rc = WL_ERR_CUDA;
    }
    cudaGraph_t out = nullptr;
    e = cudaStreamEndCapture(s(), &out);
    --depth;
    if (rc != WL_OK) return rc;
    if (e != cudaSuccess) return cuerr(e, "cudaStreamEndCapture (loop body)");
    return WL_OK;
  }
};

unsigned grid1(int64_t work) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((work + kPhaseBlock - 1) / kPhaseBlock, 152 * 16));
}

// ---- per-K launch dispatch
#define BT_FOR_K(X) X(1) X(2) X(4) X(8) X(16) X(32) X(64)

template <typename T>
int emit_init(int K, const BatchArgs<T>& a, const int* pmask, int nslab, cudaStream_t s) {
  const dim3 grid(a.g.ntile, nslab);
  switch (K) {
#define C(k) case k: bcg_init<T, k><<<grid, kPhaseBlock, 0, s>>>(a, pmask); break;
    BT_FOR_K(C)
#undef C
    default: return WL_ERR_INVALID_ARG;
  }
  BT_CU(cudaGetLastError());
  return WL_OK;
}

int emit_red_init(int K, const BatchGraph& g, const BatchState& st, const double* part, const double* bn2,
                  const int* skip, const int* pmask, double tol2, int nslab, cudaStream_t s) {
  const dim3 grid(g.ngraph, nslab);
  switch (K) {
#define C(k) case k: bred_init<k><<<grid, kPhaseBlock, 0, s>>>(g, st, part, bn2, skip, pmask, tol2); break;
    BT_FOR_K(C)
#undef C
    default: return WL_ERR_INVALID_ARG;
  }
  BT_CU(cudaGetLastError());
  return WL_OK;
}

template <typename T>
int emit_iteration(int K, const BatchArgs<T>& a, int nslab, cudaStream_t s) {
  const dim3 gt(a.g.ntile, nslab), gp(a.g.ngraph, nslab);
  switch (K) {
#define C(k)                                                                      \
  case k:                                                                         \
    bcg_s<T, k><<<gt, kPhaseBlock, 0, s>>>(a);                                    \
    bred_s<k><<<gp, kPhaseBlock, 0, s>>>(a.g, a.st, a.part);                       \
    bcg_u<T, k><<<gt, kPhaseBlock, 0, s>>>(a);                                    \
    bred_u<k><<<gp, kPhaseBlock, 0, s>>>(a.g, a.st, a.part, a.tol2, a.max_iter);   \
    break;
    BT_FOR_K(C)
#undef C
    default: return WL_ERR_INVALID_ARG;
  }
  BT_CU(cudaGetLastError());
  return WL_OK;
}

int emit_res(int K, const BatchResArgs& a, int nslab, cudaStream_t s) {
  const dim3 gt(a.g.ntile, nslab);
  switch (K) {
#define C(k) case k: bres<k><<<gt, kPhaseBlock, 0, s>>>(a); break;
    BT_FOR_K(C)
#undef C
    default: return WL_ERR_INVALID_ARG;
  }
  BT_CU(cudaGetLastError());
  return WL_OK;
}

int emit_red_res(int K, const BatchGraph& g, const BatchOuter& o, const double* part, double tol2, int max_outer,
                 int nslab, cudaStream_t s) {
  const dim3 gp(g.ngraph, nslab);
  switch (K) {
#define C(k) case k: bred_res<k><<<gp, kPhaseBlock, 0, s>>>(g, o, part, tol2, max_outer); break;
    BT_FOR_K(C)
#undef C
    default: return WL_ERR_INVALID_ARG;
  }
  BT_CU(cudaGetLastError());
  return WL_OK;
}

// one batched solve M_{s,g} X = bscale b for all problems: X ends in
// sb.x (FP64 form) or sb.x64 (refined form)
int emit_solve(wl_batch* b, Emitter& em, SolveBufs& sb, const TileSet& ts, const double* rhs, const double* bscale) {
  const int K = sb.K, nslab = b->nslab, np = nprob(b);
  const BatchGraph g = bgraph(b, ts);
  const BatchState st = bstate(b, sb);
  const double tol2 = b->prm.tol * b->prm.tol;
  cudaStream_t s = em.s();
  BT_CU(cudaMemsetAsync(sb.flags.p, 0, sb.flags.bytes, s));
  BT_CU(cudaMemsetAsync(st.total, 0, sizeof(int) * np, s));
  if (b->prm.prec == WL_FP64) {
    BatchArgs<double> a{g, (double*)sb.x.p, (double*)sb.r.p, (double*)sb.p.p, (double*)sb.q.p,
                        (const double*)b->ca.p, (const double*)b->cA.p, (const double*)b->cD.p, rhs, bscale,
                        nullptr, nullptr, (double*)sb.part.p, st, b->prm.max_iter, tol2};
    BT_TRY(emit_init<double>(K, a, nullptr, nslab, s));
    BT_TRY(emit_red_init(K, g, st, a.part, nullptr, nullptr, nullptr, tol2, nslab, s));
    return em.loop(sb, st.any, b->prm.max_iter + 2, [&]() { return emit_iteration<double>(K, a, nslab, em.s()); });
  }
  // refined: double-float residual / FP64 iterate around an FP32 CG whose
  // target is the inner tolerance relative to the current residual
  const BatchOuter o = bouter(b, sb);
  const double tin = std::min(1e-3, std::max(4e-6, 0.5 * std::sqrt(b->prm.tol)));
  BT_CU(cudaMemsetAsync(sb.x64.p, 0, (size_t)nslab * b->n * K * 8, s));
  bfill_int<<<grid1(np), kPhaseBlock, 0, s>>>(o.outer_active, np, 1);
  BT_CU(cudaGetLastError());
  BT_CU(cudaMemsetAsync(o.outer_iters, 0, sizeof(int) * np, s));
  bfill_int<<<1, 1, 0, s>>>(o.any, 1, 1);
  BT_CU(cudaGetLastError());
  const size_t elems = (size_t)nslab * b->n * K;
  BatchResArgs ra{g, (const float*)sb.x.p, rhs, bscale, (const double*)b->ca.p, (const double*)b->cA.p,
                  (const double*)b->cD.p, (float*)sb.rdf.p, (float*)sb.rdf.p + elems, (float*)sb.r.p,
                  (double*)sb.x64.p, (double*)sb.part.p, o.outer_active, o.outer_iters};
  BatchArgs<float> ia{g, (float*)sb.x.p, (float*)sb.r.p, (float*)sb.p.p, (float*)sb.q.p, (const double*)b->ca.p,
                      (const double*)b->cA.p, (const double*)b->cD.p, nullptr, nullptr, o.rn2, o.skip,
                      (double*)sb.part.p, st, b->prm.max_iter, tin * tin};
  return em.loop(sb, o.any, b->prm.max_outer + 2, [&]() -> int {
    cudaStream_t so = em.s();
    BT_TRY(emit_res(K, ra, nslab, so));
    BT_TRY(emit_red_res(K, g, o, ra.part, tol2, b->prm.max_outer, nslab, so));
    BT_TRY(emit_init<float>(K, ia, o.outer_active, nslab, so));
    BT_TRY(emit_red_init(K, g, st, ia.part, o.rn2, o.skip, o.outer_active, tin * tin, nslab, so));
    // the correction d ends in sb.x; the next residual pass adds it to x64
    return em.loop(sb, st.any, b->prm.max_iter + 2, [&]() { return emit_iteration<float>(K, ia, nslab, em.s()); });
  });
}

// the whole run: D_f solve, V solve, outputs
int emit_run(wl_batch* b, Emitter& em, int K, const TileSet& ts) {
  BT_TRY(emit_solve(b, em, b->sb1, ts, (const double*)b->ones.p, (const double*)b->phis.p));
  const bool refined = b->prm.prec == WL_REFINED;
  const double* Dsrc = refined ? (const double*)b->sb1.x64.p : (const double*)b->sb1.x.p;
  BT_CU(cudaMemcpyAsync(b->Df.p, Dsrc, (size_t)b->nslab * b->n * 8, cudaMemcpyDeviceToDevice, em.s()));
  BT_TRY(emit_solve(b, em, b->sbk, ts, (const double*)b->Vin.p, nullptr));
  const double* X = refined ? (const double*)b->sbk.x64.p : (const double*)b->sbk.x.p;
  const BatchGraph g = bgraph(b, ts);
  bout<double><<<grid1((int64_t)b->n * K * b->nslab), kPhaseBlock, 0, em.s()>>>(
      g, (const double*)b->Df.p, (const double*)b->Vin.p, X, (const double*)b->phis.p, (double*)b->W.p, K, b->nslab);
  BT_CU(cudaGetLastError());
  return WL_OK;
}

// S-kernel time (ms) of one tile height for K columns on the batch itself
int time_tiles(wl_batch* b, const TileSet& ts, int K, float* ms) {
  SolveBufs& sb = (K == 1) ? b->sb1 : b->sbk;
  cudaStream_t s = b->stream;
  const BatchGraph g = bgraph(b, ts);
  const BatchState st = bstate(b, sb);
  const int np = nprob(b);
  // r = 1, active problems, first iteration
  bfill_int<<<grid1(np), kPhaseBlock, 0, s>>>(st.active, np, 1);
  BT_CU(cudaMemsetAsync(st.iters, 0, sizeof(int) * np, s));
  BT_CU(cudaMemsetAsync(sb.r.p, 0, (size_t)b->nslab * b->n * K * 4, s));
  cudaEvent_t e0, e1;
  BT_CU(cudaEventCreate(&e0));
  BT_CU(cudaEventCreate(&e1));
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    BT_CU(cudaEventRecord(e0, s));
    BatchArgs<float> a{g, (float*)sb.x.p, (float*)sb.r.p, (float*)sb.p.p, (float*)sb.q.p, (const double*)b->ca.p,
                       (const double*)b->cA.p, (const double*)b->cD.p, nullptr, nullptr, nullptr, nullptr,
                       (double*)sb.part.p, st, 1, 0.0};
    switch (K) {
#define C(k) case k: bcg_s<float, k><<<dim3(g.ntile, b->nslab), kPhaseBlock, 0, s>>>(a); break;
      BT_FOR_K(C)
#undef C
    }
    BT_CU(cudaGetLastError());
    BT_CU(cudaEventRecord(e1, s));
    BT_CU(cudaEventSynchronize(e1));
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    if (rep > 0) best = std::min(best, t);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = best;
  return WL_OK;
}

int tune(wl_batch* b, int K, int* which) {
  const int key = K * 2 + (b->prm.prec == WL_REFINED);
  auto it = b->tuned.find(key);
  if (it != b->tuned.end()) {
    *which = it->second;
    return WL_OK;
  }
  int best = 0;
  float best_ms = 1e30f;
  for (int i = 0; i < (int)b->tilesets.size(); ++i) {
    float ms = 0.f;
    BT_TRY(time_tiles(b, b->tilesets[i], K, &ms));
    if (ms < best_ms) {
      best_ms = ms;
      best = i;
    }
  }
  b->tuned[key] = best;
  *which = best;
  return WL_OK;
}

void free_exec(Exec& x) {
  if (x.exec) cudaGraphExecDestroy(x.exec);
  if (x.graph) cudaGraphDestroy(x.graph);
  x.exec = nullptr;
  x.graph = nullptr;
}

void free_batch(wl_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  (void)cudaGetLastError();
  for (auto& kv : b->execs) free_exec(kv.second);
  for (auto& t : b->tilesets) {
    dfree(t.tiles);
    dfree(t.tile_beg);
  }
  SolveBufs* sbs[] = {&b->sb1, &b->sbk};
  for (SolveBufs* s : sbs) {
    DBuf* bufs[] = {&s->x, &s->r, &s->p, &s->q, &s->x64, &s->rdf, &s->part, &s->colstate, &s->colint, &s->probint, &s->flags};
    for (DBuf* d : bufs) dfree(*d);
  }
  DBuf* bufs[] = {&b->rp, &b->col, &b->goff, &b->ca, &b->cA, &b->cD, &b->phis, &b->ones, &b->Vin, &b->Df, &b->W};
  for (DBuf* d : bufs) dfree(*d);
  for (cudaStream_t& c : b->cap)
    if (c) cudaStreamDestroy(c);
  if (b->h_pin) pool_free_host(b->h_pin);
  delete b;
}

bool is_dev(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

int wl_batch_build(const wl_csr* graphs, int ngraph, const double* mus, int nmu, const wl_params* p, wl_batch** out,
                   wl_stats* st) {
  NvtxRange nvtx__("wl_batch_build");
  if (st) memset(st, 0, sizeof(*st));
  if (!out) return WL_ERR_INVALID_ARG;
  *out = nullptr;
  if (!graphs || ngraph <= 0 || !mus || nmu <= 0 || !p) return WL_ERR_INVALID_ARG;
  if (p->f != WL_F_RESOLVENT) return WL_ERR_UNSUPPORTED;
  if (p->prec != WL_FP64 && p->prec != WL_REFINED) return WL_ERR_INVALID_ARG;
  for (int j = 0; j < nmu; ++j)
    if (!(mus[j] >= 0.0 && mus[j] <= 1.0)) return WL_ERR_INVALID_ARG;
  int64_t n = 0, nnz = 0;
  for (int g = 0; g < ngraph; ++g) {
    const wl_csr& A = graphs[g];
    if (A.n < 0 || A.nnz < 0 || (A.n > 0 && !A.row_ptr) || (A.nnz > 0 && !A.col_idx)) return WL_ERR_INVALID_ARG;
    n += A.n;
    nnz += A.nnz;
  }
  if (n >= (int64_t)INT32_MAX || nnz >= (int64_t)INT32_MAX) return WL_ERR_INVALID_ARG;
  wl_batch* b = new wl_batch();
  auto fail = [&](int rc) {
    free_batch(b);
    if (st) st->status = rc;
    return rc;
  };
  b->ngraph = ngraph;
  b->nslab = nmu;
  b->n = n;
  b->nnz = nnz;
  b->prm = *p;
  if (b->prm.tol <= 0) b->prm.tol = 1e-12;
  if (b->prm.max_iter <= 0) b->prm.max_iter = 2000;
  if (b->prm.max_outer <= 0) b->prm.max_outer = 400;
  if (b->prm.max_outer > 500) b->prm.max_outer = 500;
  b->stream = (cudaStream_t)p->stream;
  b->mu.assign(mus, mus + nmu);
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  cudaEventRecord(t0, b->stream);

  // spectral scales: graphs spread over host threads, each on its own stream
  int sp_rounds = 0;
  b->lmax.assign(ngraph, 0.0);
  b->rho.assign((size_t)ngraph * nmu, 0.0);
  {
    std::atomic<int> next(0);
    std::atomic<int> err(WL_OK);
    std::mutex mtx;
    std::string msg;
    int dev = 0;
    cudaGetDevice(&dev);
    // One host thread per graph (up to kSpecThreads at a time), each with its
    // own stream for its validation and lists; their Lanczos rounds meet in
    // one SpBatch and run as shared launches over all graphs in flight.
    const int nth = std::min(ngraph, kSpecThreads);
    SpBatch* spb = sp_batch_new(nth);
    if (!spb) return fail(report_cuda_error(cudaGetLastError(), "cudaStreamCreate"));
    std::vector<std::thread> th;
    for (int t = 0; t < nth; ++t)
      th.emplace_back([&]() {
        struct Leave {  // however the thread ends, the others stop waiting for it
          SpBatch* b;
          ~Leave() {
            sp_batch_bind(nullptr);
            sp_batch_leave(b);
          }
        } leave{spb};
        cudaSetDevice(dev);
        sp_batch_bind(spb);
        cudaStream_t s = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
          err = WL_ERR_CUDA;
          return;
        }
        std::vector<double> r(nmu);
        for (int g; (g = next++) < ngraph && err == WL_OK;) {
          double lm = 0.0;
          const int rc = graph_spectral(&graphs[g], mus, nmu, s, &lm, r.data(), kSpecRtol);
          if (rc != WL_OK) {
            std::lock_guard<std::mutex> lk(mtx);
            if (err == WL_OK) {
              err = rc;
              msg = "graph " + std::to_string(g) + ": " + last_error_copy();
            }
            break;
          }
          b->lmax[g] = lm;
          for (int j = 0; j < nmu; ++j) b->rho[(size_t)j * ngraph + g] = r[j];
        }
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
      });
    for (auto& x : th) x.join();
    sp_rounds = sp_batch_rounds(spb);
    sp_batch_free(spb);
    if (err != WL_OK) {
      report_error(msg);
      return fail(err);
    }
  }
  // per-problem coefficients of M = (1 - mu^2 a^2) I - a A + a^2 mu D
  const int np = ngraph * nmu;
  b->alpha.assign(np, 0.0);
  b->phi.assign(np, 1.0);
  std::vector<double> ca(np), cA(np), cD(np);
  for (int j = 0; j < nmu; ++j)
    for (int g = 0; g < ngraph; ++g) {
      const int pr = j * ngraph + g;
      const double rho = b->rho[pr], m = mus[j];
      double a = p->alpha;
      if (p->alpha_rel > 0) a = rho > 0 ? p->alpha_rel / rho : 0.0;
      if (!(a >= 0.0) || !std::isfinite(a) || a * rho >= 1.0) return fail(WL_ERR_ALPHA_RANGE);
      b->alpha[pr] = a;
      b->phi[pr] = 1.0 - m * m * a * a;
      ca[pr] = b->phi[pr];
      cA[pr] = -a;
      cD[pr] = a * a * m;
    }
  // concatenated CSR (host copy for tiling, device copy for the kernels)
  b->goff_h.assign(ngraph + 1, 0);
  b->rp_h.assign(n + 1, 0);
  std::vector<int32_t> col_h(std::max<int64_t>(nnz, 1));
  {
    int64_t ro = 0, eo = 0;
    std::vector<int32_t> rp;
    for (int g = 0; g < ngraph; ++g) {
      const wl_csr& A = graphs[g];
      b->goff_h[g] = (int32_t)ro;
      rp.resize(A.n + 1);
      cudaError_t e = cudaMemcpy(rp.data(), A.row_ptr, sizeof(int32_t) * (A.n + 1), cudaMemcpyDefault);
      if (e == cudaSuccess && A.nnz > 0)
        e = cudaMemcpy(col_h.data() + eo, A.col_idx, sizeof(int32_t) * A.nnz, cudaMemcpyDefault);
      if (e != cudaSuccess) return fail(cuerr(e, "copy graph"));
      for (int64_t i = 0; i < A.n; ++i) b->rp_h[ro + i] = (int32_t)(eo + rp[i]);
      for (int64_t e2 = 0; e2 < A.nnz; ++e2) col_h[eo + e2] += (int32_t)ro;
      ro += A.n;
      eo += A.nnz;
    }
    b->goff_h[ngraph] = (int32_t)ro;
    b->rp_h[n] = (int32_t)eo;
  }
  cudaError_t e = dalloc(b->rp, sizeof(int32_t) * (n + 1));
  if (e == cudaSuccess) e = dalloc(b->col, sizeof(int32_t) * col_h.size());
  if (e == cudaSuccess) e = dalloc(b->goff, sizeof(int32_t) * (ngraph + 1));
  if (e == cudaSuccess) e = cudaMemcpy(b->rp.p, b->rp_h.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->col.p, col_h.data(), sizeof(int32_t) * col_h.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->goff.p, b->goff_h.data(), sizeof(int32_t) * (ngraph + 1), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = dalloc(b->ca, 8 * np);
  if (e == cudaSuccess) e = dalloc(b->cA, 8 * np);
  if (e == cudaSuccess) e = dalloc(b->cD, 8 * np);
  if (e == cudaSuccess) e = dalloc(b->phis, 8 * np);
  if (e == cudaSuccess) e = cudaMemcpy(b->ca.p, ca.data(), 8 * np, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->cA.p, cA.data(), 8 * np, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->cD.p, cD.data(), 8 * np, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->phis.p, b->phi.data(), 8 * np, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = dalloc(b->ones, 8 * std::max<int64_t>(n, 1));
  if (e != cudaSuccess) return fail(cuerr(e, "batch device buffers"));
  if (launch_fill((double*)b->ones.p, 1.0, n, b->stream) != cudaSuccess)
    return fail(cuerr(cudaGetLastError(), "fill"));
  // candidate tile heights
  for (int R : {64, 128, 256, 512}) {
    b->tilesets.emplace_back();
    int rc = make_tiles(b, R, b->tilesets.back());
    if (rc != WL_OK) return fail(rc);
  }
  int rc = alloc_solve(b, b->sb1, 1);
  if (rc != WL_OK) return fail(rc);
  for (int i = 0; i < 3; ++i)
    if (cudaStreamCreateWithFlags(&b->cap[i], cudaStreamNonBlocking) != cudaSuccess)
      return fail(cuerr(cudaGetLastError(), "cudaStreamCreate"));
  if (pool_malloc_host((void**)&b->h_pin, 64 * sizeof(int)) != cudaSuccess)
    return fail(cuerr(cudaGetLastError(), "cudaMallocHost"));
  cudaEventRecord(t1, b->stream);
  cudaEventSynchronize(t1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, t0, t1);
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  if (st) {
    st->time_ms = ms;
    st->outer_iters = sp_rounds;
    st->status = WL_OK;
  }
  *out = b;
  return WL_OK;
}

int wl_batch_run(wl_batch* b, const double* V, int k, double* Df, double* W, int stepped, wl_stats* st) {
  NvtxRange nvtx__("wl_batch_run");
  if (st) memset(st, 0, sizeof(*st));
  if (!b || !V || !Df || !W || !valid_k(k)) return WL_ERR_INVALID_ARG;
  const int nslab = b->nslab, np = nprob(b);
  cudaStream_t s = b->stream;
  cudaError_t e = cudaSuccess;
  if (b->sbk.K != k) {
    for (auto& kv : b->execs) free_exec(kv.second);
    b->execs.clear();
    SolveBufs fresh;
    std::swap(b->sbk, fresh);
    DBuf* bufs[] = {&fresh.x, &fresh.r, &fresh.p, &fresh.q, &fresh.x64, &fresh.rdf, &fresh.part, &fresh.colstate, &fresh.colint,
                    &fresh.probint, &fresh.flags};
    for (DBuf* d : bufs) dfree(*d);
    BT_TRY(alloc_solve(b, b->sbk, k));
    e = dalloc(b->Vin, (size_t)b->n * k * 8);
    if (e == cudaSuccess) e = dalloc(b->Df, (size_t)nslab * b->n * 8);
    if (e == cudaSuccess) e = dalloc(b->W, (size_t)nslab * b->n * k * 8);
    if (e != cudaSuccess) return cuerr(e, "batch run buffers");
  }
  cudaEvent_t t0, t1;
  BT_CU(cudaEventCreate(&t0));
  BT_CU(cudaEventCreate(&t1));
  BT_CU(cudaEventRecord(t0, s));
  BT_CU(cudaMemcpyAsync(b->Vin.p, V, (size_t)b->n * k * 8, cudaMemcpyDefault, s));
  int which = 0;
  BT_TRY(tune(b, k, &which));
  const TileSet& ts = b->tilesets[which];
  const int key = k * 2 + (b->prm.prec == WL_REFINED);
  int launches = 0;
  if (stepped) {
    Emitter em{false, {s, s, s}};
    em.host_pin = b->h_pin;
    BT_TRY(emit_run(b, em, k, ts));
  } else {
    Exec& x = b->execs[key];
    if (!x.exec) {
      // capture on a private stream ordered after the caller's stream
      BT_CU(cudaStreamSynchronize(s));
      Emitter em{true, {b->cap[0], b->cap[1], b->cap[2]}};
      BT_CU(cudaGraphCreate(&x.graph, 0));
      BT_CU(cudaStreamBeginCaptureToGraph(b->cap[0], x.graph, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
      int rc = emit_run(b, em, k, ts);
      cudaGraph_t outg = nullptr;
      cudaError_t ee = cudaStreamEndCapture(b->cap[0], &outg);
      if (rc != WL_OK || ee != cudaSuccess) {
        free_exec(x);
        b->execs.erase(key);
        return rc != WL_OK ? rc : cuerr(ee, "cudaStreamEndCapture");
      }
      ee = cudaGraphInstantiate(&x.exec, x.graph, 0);
      if (ee != cudaSuccess) {
        free_exec(x);
        b->execs.erase(key);
        return cuerr(ee, "cudaGraphInstantiate");
      }
    }
    BT_CU(cudaGraphLaunch(x.exec, s));
    launches = 1;
  }
  BT_CU(cudaMemcpyAsync(Df, b->Df.p, (size_t)nslab * b->n * 8, cudaMemcpyDefault, s));
  BT_CU(cudaMemcpyAsync(W, b->W.p, (size_t)nslab * b->n * k * 8, cudaMemcpyDefault, s));
  BT_CU(cudaEventRecord(t1, s));
  BT_CU(cudaEventSynchronize(t1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, t0, t1);
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  // per-problem results
  b->iters_df.assign(np, 0);
  b->iters_v.assign(np, 0);
  b->outer_df.assign(np, 0);
  b->outer_v.assign(np, 0);
  b->status_p.assign(np, 0);
  b->relres_df.assign(np, 0.0);
  b->relres_v.assign(np, 0.0);
  const bool refined = b->prm.prec == WL_REFINED;
  int worst = WL_OK;
  double max_rel = 0.0, units = 0.0;
  for (int which_solve = 0; which_solve < 2; ++which_solve) {
    SolveBufs& sb = which_solve == 0 ? b->sb1 : b->sbk;
    const int K = sb.K;
    const size_t nc = (size_t)np * K;
    std::vector<int> pi(np * 5), ci(nc * 4);
    std::vector<double> cs(nc * 6);
    BT_CU(cudaMemcpy(pi.data(), sb.probint.p, sizeof(int) * pi.size(), cudaMemcpyDeviceToHost));
    BT_CU(cudaMemcpy(ci.data(), sb.colint.p, sizeof(int) * ci.size(), cudaMemcpyDeviceToHost));
    BT_CU(cudaMemcpy(cs.data(), sb.colstate.p, sizeof(double) * cs.size(), cudaMemcpyDeviceToHost));
    for (int pr = 0; pr < np; ++pr) {
      const int g = pr % b->ngraph;
      const int64_t gn = b->goff_h[g + 1] - b->goff_h[g];
      const int64_t gnnz = b->rp_h[b->goff_h[g + 1]] - b->rp_h[b->goff_h[g]];
      int it = pi[4 * np + pr], outer = refined ? pi[3 * np + pr] : 0;
      double rel = 0.0;
      int stat = WL_OK;
      for (int c = 0; c < K; ++c) {
        const size_t i = (size_t)pr * K + c;
        int sc;
        if (refined) {
          sc = ci[3 * nc + i];
          const double rn = cs[4 * nc + i], bn = cs[5 * nc + i];
          rel = std::max(rel, bn > 0 ? std::sqrt(rn / bn) : 0.0);
        } else {
          sc = ci[nc + i];
          if (sc == WL_OK && !ci[i]) sc = WL_ERR_NO_CONVERGENCE;
          const double gm = cs[i], b2 = cs[3 * nc + i];
          rel = std::max(rel, b2 > 0 ? std::sqrt(gm / b2) : 0.0);
        }
        if (sc != WL_OK && stat == WL_OK) stat = sc;
      }
      (void)gn;
      units += (double)it * (double)gnnz * K;
      if (which_solve == 0) {
        b->iters_df[pr] = it;
        b->outer_df[pr] = outer;
        b->relres_df[pr] = rel;
      } else {
        b->iters_v[pr] = it;
        b->outer_v[pr] = outer;
        b->relres_v[pr] = rel;
      }
      if (stat != WL_OK && b->status_p[pr] == WL_OK) b->status_p[pr] = stat;
      if (stat != WL_OK && worst == WL_OK) worst = stat;
      max_rel = std::max(max_rel, rel);
    }
  }
  if (st) {
    st->status = worst;
    st->time_ms = ms;
    st->rel_res = max_rel;
    st->nnz_rhs_iters = units;
    st->launches = launches;
  }
  return worst;
}

int wl_batch_info(const wl_batch* b, int graph, int mu_index, double* alpha, double* rho, double* lambda_max,
                  int* iters_df, int* iters_v, int* status) {
  if (!b || graph < 0 || graph >= b->ngraph || mu_index < 0 || mu_index >= b->nslab) return WL_ERR_INVALID_ARG;
  const int pr = mu_index * b->ngraph + graph;
  if (alpha) *alpha = b->alpha[pr];
  if (rho) *rho = b->rho[pr];
  if (lambda_max) *lambda_max = b->lmax[graph];
  if (iters_df) *iters_df = pr < (int)b->iters_df.size() ? b->iters_df[pr] : 0;
  if (iters_v) *iters_v = pr < (int)b->iters_v.size() ? b->iters_v[pr] : 0;
  if (status) *status = pr < (int)b->status_p.size() ? b->status_p[pr] : 0;
  return WL_OK;
}

int wl_batch_tile_rows(const wl_batch* b, int k) {
  if (!b) return 0;
  auto it = b->tuned.find(k * 2 + (b->prm.prec == WL_REFINED));
  return it == b->tuned.end() ? 0 : b->tilesets[it->second].R;
}

void wl_batch_destroy(wl_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  free_batch(b);
}

}  // extern "C"
