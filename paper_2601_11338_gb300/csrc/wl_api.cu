// C ABI of libwl.so (declared in include/wl.h): handle management, graph
// validation, spectral scale, and the orchestration of the CUDA kernels for
// walk degrees, Laplacian action and diffusion. All arithmetic on vectors
// runs in the kernels; host code only sequences launches, reads back per-
// column scalars and decides convergence.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <condition_variable>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "wl.h"
#include "wl_host.h"
#include "wl_trace.cuh"

using namespace wl;

namespace {

thread_local std::string g_last_error;

struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
};

int set_cuda_error(cudaError_t e, const char* where) {
  g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
  (void)cudaGetLastError();
  return (e == cudaErrorMemoryAllocation) ? WL_ERR_OOM : WL_ERR_CUDA;
}

#define WL_CU(call)                                  \
  do {                                               \
    cudaError_t e__ = (call);                        \
    if (e__ != cudaSuccess) return set_cuda_error(e__, #call); \
  } while (0)

#define WL_TRY(call)          \
  do {                        \
    int s__ = (call);         \
    if (s__ != WL_OK) return s__; \
  } while (0)

// Blocks released while a call is running may still be read by work queued
// on the handle's stream: they are kept on the handle until it is destroyed
// (after its stream has been synchronised) instead of going back to the
// allocator's cache, where another stream could pick them up.
thread_local std::vector<void*>* t_retired = nullptr;

struct CallScope {
  std::vector<void*>* prev;
  explicit CallScope(std::vector<void*>* r) : prev(t_retired) { t_retired = r; }
  ~CallScope() { t_retired = prev; }
};

void retire(void* p) {
  if (!p) return;
  if (t_retired)
    t_retired->push_back(p);
  else
    pool_free(p);
}

// ------------------------------------------------------------------ host-side fault injection
// The environment variable WL_FAULT (read at each use) makes one kind of
// failure happen on the host, for tests of the error paths:
//   alloc    every device allocation of a buffer fails (WL_ERR_OOM)
//   nan      every CG solve starts from a residual with a NaN entry
//            (WL_ERR_NONFINITE)
//   timeout  every grid barrier starts in the gave-up state, so the
//            cooperative kernels leave at their first barrier (WL_ERR_TIMEOUT)
//   noconv   every CG solve is capped at one iteration (WL_ERR_NO_CONVERGENCE)
// Nothing here faults, traps or hangs the GPU; each failure goes through the
// library's normal status paths.
enum FaultMode { kFaultNone = 0, kFaultAlloc, kFaultNan, kFaultTimeout, kFaultNoconv };

int fault_mode() {
  const char* s = getenv("WL_FAULT");
  if (!s || !*s) return kFaultNone;
  if (!strcmp(s, "alloc")) return kFaultAlloc;
  if (!strcmp(s, "nan")) return kFaultNan;
  if (!strcmp(s, "timeout")) return kFaultTimeout;
  if (!strcmp(s, "noconv")) return kFaultNoconv;
  return kFaultNone;
}

int ensure(Buf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return WL_OK;
  if (fault_mode() == kFaultAlloc) {
    g_last_error = "WL_FAULT=alloc: device allocation refused";
    return WL_ERR_OOM;
  }
  retire(b.p);
  b.p = nullptr;
  b.bytes = 0;
  cudaError_t e = pool_malloc(&b.p, bytes);
  if (e != cudaSuccess) {
    b.p = nullptr;
    return set_cuda_error(e, "cudaMalloc");
  }
  b.bytes = bytes;
  return WL_OK;
}

void release(Buf& b) {
  retire(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Column blocks used for k columns: powers of two up to 64, largest first.
std::vector<int> column_blocks(int k) {
  std::vector<int> out;
  while (k > 0) {
    int b = 64;
    while (b > k) b >>= 1;
    out.push_back(b);
    k -= b;
  }
  return out;
}

struct SolveInfo {
  int iters = 0;
  int cg_iters = 0;
  double last_rel = 0.0;
  int refinements = 0;
  double max_rel = 0.0;
  int status = WL_OK;
  double nnz_rhs = 0.0;
  double bytes = 0.0;
  int reorth_blocks = 0;  // basis blocks reorthogonalised (outer Lanczos)
};

}  // namespace

// ------------------------------------------------------------- batched searches
namespace wl {

struct SpReq {
  SpJob job{};
  SpOut out{};
  int rc = WL_OK;
};

// Rendezvous of the threads of a batched build. Each thread runs the
// spectral searches of its graphs as usual, but every round of Lanczos steps
// (and every Ritz vector) is submitted here instead of being launched on the
// thread's stream. Once every participating thread waits with a request, the
// last one to arrive launches all requests together on the batch's stream (one
// launch per kernel and step for all problems, each problem with the same CTA
// count and so the same arithmetic as on its own), reads the states back and
// wakes the others. The searches of many small graphs then cost one chain of
// launches instead of one chain per graph.
struct SpBatch {
  std::mutex m;
  std::condition_variable cv;
  int live = 0;
  uint64_t gen = 0;
  int rounds = 0;
  std::vector<SpReq*> reqs;
  cudaStream_t s = nullptr;
  void* dbuf = nullptr;
  size_t dbytes = 0;
  void* hbuf = nullptr;
  size_t hbytes = 0;
  std::string err;
};

namespace {
thread_local SpBatch* t_sp_batch = nullptr;
constexpr int kSpCheck = 8;  // eigen step every 8 Lanczos steps (and at the end of a round)

size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

// mutex held: launch the pending requests, wait for them, hand out the states
void sp_round_locked(SpBatch* b) {
  const int np = (int)b->reqs.size();
  const size_t jb = align16(sizeof(SpJob) * np), ob = align16(sizeof(int) * (np + 1)), rb = sizeof(SpOut) * np;
  const size_t need = jb + 2 * ob + rb;
  int rc = WL_OK;
  std::string msg;
  auto cu = [&](cudaError_t e, const char* where) {
    if (e != cudaSuccess && rc == WL_OK) {
      rc = (e == cudaErrorMemoryAllocation) ? WL_ERR_OOM : WL_ERR_CUDA;
      msg = std::string("batched spectral search: ") + where + ": " + cudaGetErrorString(e);
      (void)cudaGetLastError();
    }
    return rc == WL_OK;
  };
  if (need > b->hbytes) {  // the stream is idle between rounds: the old buffers can go
    const size_t cap = std::max(need, b->hbytes * 2);
    pool_free_host(b->hbuf);
    pool_free(b->dbuf);
    b->hbuf = b->dbuf = nullptr;
    b->hbytes = b->dbytes = 0;
    if (cu(pool_malloc_host(&b->hbuf, cap), "pinned buffer") && cu(pool_malloc(&b->dbuf, cap), "device buffer"))
      b->hbytes = b->dbytes = cap;
  }
  if (rc == WL_OK) {
    char* hp = (char*)b->hbuf;
    SpJob* jobs = (SpJob*)hp;
    int* off_s = (int*)(hp + jb);
    int* off_u = (int*)(hp + jb + ob);
    SpOut* outs = (SpOut*)(hp + jb + 2 * ob);
    int steps = 0;
    unsigned eig_mask = 0u;
    bool any_ritz = false, any_init = false;
    off_s[0] = off_u[0] = 0;
    for (int p = 0; p < np; ++p) {
      const SpJob& j = b->reqs[p]->job;
      jobs[p] = j;
      off_s[p + 1] = off_s[p] + j.gs;
      off_u[p + 1] = off_u[p] + j.gu;
      if (j.mode >= 0) {
        steps = std::max(steps, j.j1 - j.j0);
        for (int jj = j.j0; jj < j.j1 && jj - j.j0 < 32; ++jj)
          if ((jj + 1) % kSpCheck == 0 || jj + 1 == j.j1) eig_mask |= 1u << (jj - j.j0);
      }
      any_ritz |= j.ritz != 0;
      any_init |= j.mode == 0;
    }
    char* dp = (char*)b->dbuf;
    if (cu(cudaMemcpyAsync(dp, hp, jb + 2 * ob, cudaMemcpyHostToDevice, b->s), "jobs to device") &&
        cu(launch_sp_round((const SpJob*)dp, (const int*)(dp + jb), (const int*)(dp + jb + ob), np, off_s[np],
                           off_u[np], steps, kSpCheck, eig_mask, any_ritz, any_init, (SpOut*)(dp + jb + 2 * ob),
                           b->s),
           "launch") &&
        cu(cudaMemcpyAsync(outs, dp + jb + 2 * ob, rb, cudaMemcpyDeviceToHost, b->s), "states to host") &&
        cu(cudaStreamSynchronize(b->s), "round")) {
      for (int p = 0; p < np; ++p) b->reqs[p]->out = outs[p];
    }
  }
  for (SpReq* r : b->reqs) r->rc = rc;
  if (rc != WL_OK) b->err = msg;
  ++b->rounds;
  b->reqs.clear();
  ++b->gen;
  b->cv.notify_all();
}

int sp_batch_submit(SpBatch* b, SpReq* r) {
  std::unique_lock<std::mutex> lk(b->m);
  b->reqs.push_back(r);
  if ((int)b->reqs.size() >= b->live) {
    sp_round_locked(b);
  } else {
    const uint64_t g0 = b->gen;
    b->cv.wait(lk, [&] { return b->gen != g0; });
  }
  if (r->rc != WL_OK) report_error(b->err);
  return r->rc;
}
}  // namespace

SpBatch* sp_batch_new(int participants) {
  SpBatch* b = new SpBatch();
  b->live = participants;
  if (cudaStreamCreateWithFlags(&b->s, cudaStreamNonBlocking) != cudaSuccess) {
    (void)cudaGetLastError();
    delete b;
    return nullptr;
  }
  return b;
}

void sp_batch_bind(SpBatch* b) { t_sp_batch = b; }

// k more participants. A round waits for every participant, and none can run
// while the caller (a participant not waiting) has not submitted, so the
// count can grow at any time the caller chooses.
void sp_batch_join(SpBatch* b, int k) {
  std::unique_lock<std::mutex> lk(b->m);
  b->live += k;
}

SpBatch* sp_batch_current() { return t_sp_batch; }

void sp_batch_leave(SpBatch* b) {
  std::unique_lock<std::mutex> lk(b->m);
  --b->live;
  if (b->live > 0 && (int)b->reqs.size() >= b->live) sp_round_locked(b);
}

int sp_batch_rounds(const SpBatch* b) { return b->rounds; }

void sp_batch_free(SpBatch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->s);
  pool_free_host(b->hbuf);
  pool_free(b->dbuf);
  cudaStreamDestroy(b->s);
  delete b;
}

}  // namespace wl

struct wl_handle {
  int64_t n = 0, nnz = 0;
  Graph g{};
  wl_variant variant = WL_ALLWALK;
  wl_params prm{};
  double mu = 0, alpha = 0, beta = 0, rho = 0, lmax = 0;
  double ca = 1, cA = 0, cD = 0;  // M = ca I + cA A + cD D
  double a_scale = 1;             // phi = a_scale * M^{-1}
  cudaStream_t stream = nullptr;
  GridBar* bar = nullptr;
  std::map<std::tuple<int, int, int, int>, PartDev> parts;
  Buf csr_rp, csr_col;
  Buf x, r, p, q;         // CG vectors (FP64 or FP32), n * 64 doubles each at most
  Buf b64;                // FP64 right-hand sides (walk degrees, apply)
  Buf d32, d32b, r32;     // refined form: FP32 corrections (two, alternating) and inner right-hand side
  Buf xh, xl;             // refined form: the iterate as two FP32 terms (x = xh + xl)
  Buf bh, bl, rh, rl;     // refined form: right-hand side and residual as two FP32 terms
  Buf dfdf, ydf;          // refined form: D_f and the Lanczos coefficients y(tau) as two FP32 terms
  Buf ew;                 // exponential series: w_{k-1}, w_k, w_{k+1} and the sum (double-float)
  Buf taus;               // time points of the outer Lanczos (device copy)
  Buf ybig;               // Y(t) = exp(-t L) Omega for a batch of time points (return probability)
  bool have_dfdf = false; // dfdf holds the current D_f
  Buf part;               // partial sums
  Buf small;              // per-column scalars
  Buf Df;
  bool have_Df = false;
  Buf warm;
  bool have_warm = false;
  Buf basis;
  size_t basis_blocks = 0;
  Buf Tab, ybuf, yprev, errb;
  Buf robuf, romask;      // basis reorthogonalisation: partial sums / coefficients, per-column mask
  Buf sibuf;              // shift-and-invert: -a / (D_f + sigma) and 1 / (D_f + sigma), FP64 and double-float
  double si_sigma = 0.0;  // the shift sibuf was computed for (0: none)
  // per-row diagonal added to M by the solves while a shift-and-invert step runs (else NULL)
  const double* si_dsh64 = nullptr;
  const float* si_dsh_h = nullptr;
  const float* si_dsh_l = nullptr;
  Buf stage_a, stage_b;   // host <-> device staging
  Buf packV, packX;
  Buf omega, gram;        // sketch and Gram workspace
  Buf omega_int;          // sketch rows in the internal node order
  Buf ptmp;               // partition / relabel scratch (int64)
  Buf perm_b, iperm_b;    // node relabelling: perm[new] = old, iperm[old] = new
  int32_t* perm = nullptr;
  int32_t* iperm = nullptr;
  Buf hubs;               // rows with more than kHubDeg entries (internal order)
  int nhub = 0;
  std::vector<void*> retired;  // blocks released during calls, returned to the allocator at destroy
  Buf cgstate;            // CgState of the running solve
  Buf spV, spW;           // spectral-scale Lanczos: basis (double-float, float2 per node) and raw w vectors
  Buf spstate;            // SpState of the spectral-scale Lanczos
  Buf mid;                // rows with kSpWarpDeg < deg <= kHubDeg (a warp each in the spectral Lanczos)
  int nmid = 0, nmid_blk = 0;
  double mid_share = 0.0; // share of the S kernels' CTAs that walk the mid rows
  double sp_c0 = 0.0, sp_cD = 0.0, sp_theta = 0.0;  // operator and Ritz value of the basis held in spV
  bool sp_ritz_ready = false;                        // W[1] holds that run's Ritz vector
  double sp_ritz_uu = 0.0, sp_ritz_udu = 0.0;        // its |u|^2 and u^T D u
  double inner_tol = 4e-6;  // floor of the FP32 correction target of the refined form
  int cg_hint = 7;          // CG iterations of the handle's last solve (sizes the first launch chunk)
  int cg_hint_ref[2] = {7, 7};  // the same for the first and the later corrections of a refined solve
  bool gram_tc = false;     // XNysTrace Gram of the sketch form on the tensor cores (tcgen05); false: CUDA cores
  CgState* cgst() { return (CgState*)cgstate.p; }
  double* h_pin = nullptr;  // pinned host scratch (4096 doubles)
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // per-call kernel timing: event pairs recorded on the stream around launches
  struct Rec {
    int a, b, cat;
  };
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<Rec> recs;
  int launches = 0;
};

namespace {

cudaStream_t S(wl_handle* h) { return h->stream; }

enum { kCatCG = 0, kCatRes = 1, kCatLan = 2 };

int ev_get(wl_handle* h) {
  if (h->ev_used == h->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    h->ev_pool.push_back(e);
  }
  return (int)h->ev_used++;
}

// record the start event of a timed launch; returns the record index
int prof_begin(wl_handle* h, int cat) {
  h->launches++;
  const int a = ev_get(h), b = ev_get(h);
  if (a < 0 || b < 0) return -1;
  cudaEventRecord(h->ev_pool[a], h->stream);
  h->recs.push_back({a, b, cat});
  return (int)h->recs.size() - 1;
}

void prof_end(wl_handle* h, int i) {
  if (i >= 0) cudaEventRecord(h->ev_pool[h->recs[i].b], h->stream);
}

void prof_reset(wl_handle* h) {
  h->recs.clear();
  h->ev_used = 0;
  h->launches = 0;
}

// count an untimed launch
inline void counted(wl_handle* h, int n = 1) { h->launches += n; }

// Partition for a persistent kernel of G CTAs working on K columns of
// `vbytes`-byte values: a row moves about 10 K vbytes per CG iteration (the
// vector streams), an entry 4 + K vbytes (index and gathered row).
int get_part(wl_handle* h, int G, int Tw, int Tc, PartDev** out, int K = 16, int vbytes = 4) {
  auto key = std::make_tuple(G, Tw, Tc, K * vbytes);
  auto it = h->parts.find(key);
  if (it != h->parts.end()) {
    *out = &it->second;
    return WL_OK;
  }
  PartDev p;
  p.G = G;
  p.Tw = Tw;
  p.Tc = Tc;
  p.row_bytes = 10 * K * vbytes;
  p.entry_bytes = 4 + K * vbytes;
  WL_CU(pool_malloc((void**)&p.rb, sizeof(int32_t) * (G + 1)));
  WL_CU(pool_malloc((void**)&p.seg, sizeof(int32_t) * 4 * G));
  WL_CU(pool_malloc((void**)&p.meta, sizeof(int4) * std::max<int64_t>(h->n, 1)));
  WL_TRY(ensure(h->ptmp, sizeof(int64_t) * (2 * (size_t)(h->n + 1) + (size_t)h->n / 1024 + 8)));
  counted(h, 4);
  WL_CU(launch_partition_weighted(h->g, p, (int64_t*)h->ptmp.p, S(h)));
  h->parts[key] = p;
  *out = &h->parts[key];
  return WL_OK;
}

int reset_bar(wl_handle* h) {
  WL_CU(cudaMemsetAsync(h->bar, 0, sizeof(GridBar), S(h)));
  if (fault_mode() == kFaultTimeout) {
    static const int gave_up = WL_ERR_TIMEOUT;
    WL_CU(cudaMemcpyAsync(&h->bar->err, &gave_up, sizeof(int), cudaMemcpyHostToDevice, S(h)));
  }
  return WL_OK;
}

int check_bar(wl_handle* h) {
  int err = 0;
  WL_CU(cudaMemcpyAsync(&err, &h->bar->err, sizeof(int), cudaMemcpyDeviceToHost, S(h)));
  WL_CU(cudaStreamSynchronize(S(h)));
  return err;
}

// scalars area layout (doubles): [0,64) bnorm2/rr, [64,128) bb, [128,192) gamma,
// [192,256) ints status (as int32 region), [256,320) skip ints, [320] iters
struct Smalls {
  double* rr;
  double* bb;
  double* gamma;
  int* status;
  int* skip;
  int* iters;
  double* misc;  // 64 doubles
  int* flags;
};

Smalls smalls(wl_handle* h) {
  double* base = (double*)h->small.p;
  Smalls s;
  s.rr = base;
  s.bb = base + 64;
  s.gamma = base + 128;
  s.status = (int*)(base + 192);
  s.skip = (int*)(base + 256);
  s.iters = (int*)(base + 320);
  s.misc = base + 384;
  s.flags = (int*)(base + 448);
  return s;
}

double alg_bytes_per_iter(wl_handle* h, int K, int s) {
  return 4.0 * (double)h->nnz + 4.0 * (double)(h->n + 1) + 6.0 * (double)h->n * K * s;
}

PhaseGraph phase_graph(wl_handle* h) {
  return PhaseGraph{h->g.row_ptr, h->g.col, h->n, (const int32_t*)h->hubs.p, h->nhub};
}

// the graph as seen by an S kernel of grid_u CTAs (plus the hub CTAs) that
// walks the mid rows with a warp each
PhaseGraph phase_graph_mid(wl_handle* h, int grid_u) {
  PhaseGraph g = phase_graph(h);
  if (h->nmid > 0 && grid_u > 1) {
    g.mids = (const int32_t*)h->mid.p;
    g.nmid = h->nmid;
    g.nmid_blk = (int)std::min<long>(grid_u - 1, std::max<long>(1, std::lround(h->mid_share * grid_u)));
  }
  return g;
}

// first FP32 correction target of a refined solve: kInner0C sqrt(tol), at
// least the handle's inner_tol floor (a deeper first target, 0.1 sqrt(tol),
// measured no fewer CG iterations in all)
constexpr double kInner0C = 0.5;
constexpr int kChunk = 8;      // CG iterations launched between two reads of the device flag (cap: 2 kChunk)
constexpr int kChunkMore = 4;  // iterations of every chunk after the first

// Runs the CG iterations of an initialised solve state to completion (or the
// iteration cap), reading back one flag per chunk, then the final x update.
template <typename T>
int run_cg(wl_handle* h, int K, const PhaseArgs<T>& a_in, int grid_s, int grid_u, SolveInfo& info, int cat_bytes,
           bool init = true) {
  PhaseArgs<T> a = a_in;
  const int fault = fault_mode();
  if (fault == kFaultNoconv) a.max_iter = 1;
  if (fault == kFaultNan) {
    static const T nan_v = (T)NAN;
    WL_CU(cudaMemcpyAsync(a.r, &nan_v, sizeof(T), cudaMemcpyHostToDevice, S(h)));
  }
  auto launch = [&](int mode, int chunk) -> cudaError_t {
    if constexpr (sizeof(T) == 4)
      return launch_cg_phases_f32(K, a, grid_s, grid_u, mode, chunk, S(h));
    else
      return launch_cg_phases_f64(K, a, grid_s, grid_u, mode, chunk, S(h));
  };
  const int pc = prof_begin(h, kCatCG);
  if (init) {  // else the caller has set the state from known residual norms
    counted(h, 1);
    WL_CU(launch(0, 0));
  }
  // the whole CG state comes back after every chunk: the check of the last
  // chunk also carries the per-column results (the deferred x update launched
  // after it changes none of them), so the solve ends without another wait
  CgState* hs = reinterpret_cast<CgState*>(h->h_pin);
  static_assert(sizeof(CgState) <= 4096 * sizeof(double), "pinned staging holds the CG state");
  // first chunk: one more iteration than the handle's previous solve took (a
  // launch that finds the solve finished returns at once, but still costs a
  // grid); later chunks of kChunkMore iterations
  int chunk = std::min(std::max(h->cg_hint + 1, 2), 2 * kChunk);
  for (;;) {
    counted(h, 2 * chunk);
    WL_CU(launch(1, chunk));
    WL_CU(cudaMemcpyAsync(hs, h->cgst(), sizeof(CgState), cudaMemcpyDeviceToHost, S(h)));
    WL_CU(cudaStreamSynchronize(S(h)));
    if (!hs->active) break;
    chunk = kChunkMore;
  }
  counted(h, 1);
  WL_CU(launch(2, 0));
  prof_end(h, pc);
  // per-column results
  const int it = hs->iters;
  h->cg_hint = it;
  int cs[64];
  for (int c = 0; c < K; ++c) {  // iteration cap reached with a column still iterating
    cs[c] = hs->status[c];
    if (!hs->done[c] && cs[c] == 0) cs[c] = WL_ERR_NO_CONVERGENCE;
  }
  info.iters += it;
  info.cg_iters += it;
  info.nnz_rhs += (double)it * h->nnz * K;
  info.bytes += (double)it * alg_bytes_per_iter(h, K, cat_bytes);
  info.last_rel = 0.0;
  for (int c = 0; c < K; ++c) {
    if (cs[c] != 0 && info.status == WL_OK) info.status = cs[c];
    if (hs->b2[c] > 0) info.last_rel = std::max(info.last_rel, std::sqrt(hs->gamma[c] / hs->b2[c]));
  }
  return WL_OK;
}

int ensure_phase_buffers(wl_handle* h, int grid) {
  WL_TRY(ensure(h->part, (size_t)grid * 64 * 2 * 8 + 1024));
  WL_TRY(ensure(h->cgstate, sizeof(CgState)));
  return WL_OK;
}

// FP64 lockstep CG on M x = b for K columns (b, x contiguous n x K doubles).
// x holds the starting guess on entry (zero unless a warm start is given).
int solve_fp64(wl_handle* h, const double* b, double* x, int K, double tol, bool x_is_zero, SolveInfo& info) {
  NvtxRange nvtx__("fp64 solve");
  const int grid_u = phase_blocks_f64(K), grid_s = grid_u + h->nhub;
  const size_t nk = (size_t)h->n * K;
  WL_TRY(ensure(h->r, nk * 8));
  WL_TRY(ensure(h->p, nk * 8));
  WL_TRY(ensure(h->q, nk * 8));
  WL_TRY(ensure_phase_buffers(h, std::max(grid_s, res_blocks(K) + h->nhub)));
  CgState* st = h->cgst();
  WL_CU(cudaMemsetAsync(st, 0, sizeof(CgState), S(h)));
  const double* bn2 = nullptr;
  if (x_is_zero) {
    WL_CU(cudaMemcpyAsync(h->r.p, b, nk * 8, cudaMemcpyDeviceToDevice, S(h)));
  } else {
    const int gr = res_blocks(K) + h->nhub;
    ResPhaseArgs ra{phase_graph(h), x, b, (double*)h->r.p, h->ca, h->cA, h->cD, (double*)h->part.p, st};
    const int pi = prof_begin(h, kCatRes);
    counted(h);
    WL_CU(launch_res_phases(K, ra, gr, S(h)));
    prof_end(h, pi);
    bn2 = st->b2;
    info.nnz_rhs += (double)h->nnz * K;
  }
  PhaseArgs<double> a{phase_graph_mid(h, grid_u), x, (double*)h->r.p, (double*)h->p.p, (double*)h->q.p, h->ca, h->cA, h->cD,
                      bn2, nullptr, (double*)h->part.p, st, h->prm.max_iter, tol * tol};
  a.dshift = h->si_dsh64;  // shifted solve of the shift-and-invert Lanczos (else NULL)
  WL_TRY(run_cg<double>(h, K, a, grid_s, grid_u, info, 8));
  info.max_rel = std::max(info.max_rel, info.last_rel);
  return WL_OK;
}

// Refined solve of M X = B for K columns with B, the residual and the
// iterate held in double-float form (two FP32 arrays each) and FP32 inner
// CG corrections M d = fl32(r); the residual is carried by r <- r - M d in
// double-float arithmetic (one gather of the 4-byte correction per step).
// (bh, bl): right-hand side; |B|^2 per column in bn2 (device, K doubles).
// On return (xh, xl) holds X. x0 (FP64, or NULL for X0 = 0) is a warm start.
int solve_refined_df(wl_handle* h, const float* bh, const float* bl, const double* bn2, float* xh, float* xl,
                     const double* x0, int K, double tol, SolveInfo& info) {
  NvtxRange nvtx__("refined solve");
  const int grid_u = phase_blocks_f32(K), grid_s = grid_u + h->nhub;
  const int grid_r = df_res_blocks(K) + h->nhub;
  const size_t nk = (size_t)h->n * K;
  WL_TRY(ensure(h->p, nk * 4));
  WL_TRY(ensure(h->q, nk * 4));
  WL_TRY(ensure(h->d32, nk * 4));
  WL_TRY(ensure(h->d32b, nk * 4));
  WL_TRY(ensure(h->r32, nk * 4));
  WL_TRY(ensure(h->rh, nk * 4));
  WL_TRY(ensure(h->rl, nk * 4));
  WL_TRY(ensure_phase_buffers(h, std::max(grid_s, grid_r)));
  CgState* st = h->cgst();
  float* rh = (float*)h->rh.p;
  float* rl = (float*)h->rl.p;
  float* dcur = (float*)h->d32.p;
  float* dnext = (float*)h->d32b.p;
  const df ca = df_from_double(h->ca), cA = df_from_double(h->cA), cD = df_from_double(h->cD);
  double* hp = h->h_pin;
  // current residual: B itself while X = 0
  const float* rch = bh;
  const float* rcl = bl;
  bool x_zero = (x0 == nullptr);
  WL_CU(cudaMemsetAsync(dcur, 0, nk * 4, S(h)));
  WL_CU(cudaMemsetAsync(st, 0, sizeof(CgState), S(h)));
  if (x_zero) {
    WL_CU(cudaMemcpyAsync(h->r32.p, bh, nk * 4, cudaMemcpyDeviceToDevice, S(h)));
    WL_CU(cudaMemcpyAsync(st->gamma, bn2, K * 8, cudaMemcpyDeviceToDevice, S(h)));
  } else {
    // r = B - M x0 (x0 split into two FP32 terms and gathered whole)
    counted(h, 2);
    WL_CU(launch_split_x(x0, (int64_t)nk, xh, xl, false, nullptr, S(h)));
    DfResArgs ra{phase_graph_mid(h, grid_r - h->nhub), xh, xl, bh, bl, rh, rl, (float*)h->r32.p, nullptr, nullptr, nullptr,
                 ca, cA, cD, (double*)h->part.p, st, 0};
    ra.dsh_h = h->si_dsh_h;
    ra.dsh_l = h->si_dsh_l;
    const int pi = prof_begin(h, kCatRes);
    WL_CU(launch_df_res(K, ra, grid_r, true, S(h)));
    prof_end(h, pi);
    info.nnz_rhs += (double)h->nnz * K;
    rch = rh;
    rcl = rl;
  }
  // FP32 correction target: the first correction goes as deep as FP32 CG
  // reliably gets (the inner_tol floor) unless tol is loose; a later one only
  // as deep as the current relative residual rel needs to reach tol (0.5 tol /
  // rel, with the same floor)
  const double inner0 = std::min(1e-3, std::max(h->inner_tol, kInner0C * std::sqrt(tol)));
  const int max_ref = 12;
  int ndf = 0;
  int* dskip = (int*)((double*)h->small.p + 256);
  // r32 (the next inner solve's right-hand side) and dcur (its zero start)
  // are ready: the residual after the first correction writes them, later
  // ones do not (the solve almost always ends there), and a further
  // correction stages them itself
  bool staged = true;
  for (int ref = 0;; ++ref) {
    info.refinements++;
    double mx = 1.0;
    if (ref == 0 && x_zero) {
      // the residual is B itself: every column with B != 0 still needs its
      // first correction (rel = 1), and the inner solve's start marks a zero
      // column done by itself, so no host check (and no wait) is needed
      WL_CU(cudaMemsetAsync(dskip, 0, K * sizeof(int), S(h)));
    } else {
      WL_CU(cudaMemcpyAsync(hp, st->gamma, K * 8, cudaMemcpyDeviceToHost, S(h)));
      WL_CU(cudaMemcpyAsync(hp + 64, bn2, K * 8, cudaMemcpyDeviceToHost, S(h)));
      WL_CU(cudaStreamSynchronize(S(h)));
      bool all = true;
      mx = 0.0;
      int skip[64];
      for (int c = 0; c < K; ++c) {
        const double rr = hp[c], bb = hp[64 + c];
        if (!std::isfinite(rr)) info.status = WL_ERR_NONFINITE;
        const double rel = bb > 0 ? std::sqrt(rr / bb) : 0.0;
        mx = std::max(mx, rel);
        skip[c] = (rel <= tol) ? 1 : 0;
        if (!skip[c]) all = false;
      }
      info.max_rel = mx;
      if (all || info.status == WL_ERR_NONFINITE) break;
      if (ref >= max_ref) {
        if (info.status == WL_OK) info.status = WL_ERR_NO_CONVERGENCE;
        break;
      }
      WL_CU(cudaMemcpyAsync(dskip, skip, K * sizeof(int), cudaMemcpyHostToDevice, S(h)));
      if (!staged) {
        WL_CU(cudaMemcpyAsync(h->r32.p, rh, nk * 4, cudaMemcpyDeviceToDevice, S(h)));
        WL_CU(cudaMemsetAsync(dcur, 0, nk * 4, S(h)));
        staged = true;
      }
    }
    const double inner_tol = ref == 0 && x_zero ? inner0 : std::min(1e-3, std::max(h->inner_tol, 0.5 * tol / mx));
    // the inner solve starts from the residual norms in st->gamma (from the
    // double-float residual, or B's norms): no pass over r32 to recompute them
    counted(h);
    WL_CU(launch_cg_state_restart(st, dskip, K, S(h)));
    PhaseArgs<float> a{phase_graph_mid(h, grid_u), dcur, (float*)h->r32.p, (float*)h->p.p, (float*)h->q.p,
                       h->ca, h->cA, h->cD, nullptr, dskip, (double*)h->part.p, st, h->prm.max_iter,
                       inner_tol * inner_tol};
    a.dshift = h->si_dsh_h;
    SolveInfo inner;
    // the first correction and the later ones go to different depths: each
    // sizes its first launch chunk from the previous solve of its kind
    int& hint = h->cg_hint_ref[ref == 0 ? 0 : 1];
    h->cg_hint = hint;
    WL_TRY(run_cg<float>(h, K, a, grid_s, grid_u, inner, 4, false));
    hint = h->cg_hint;
    if (inner.status == WL_ERR_NOT_SPD || inner.status == WL_ERR_NONFINITE) {
      info.status = inner.status;
      break;
    }
    info.iters += inner.iters;
    info.cg_iters += inner.cg_iters;
    info.nnz_rhs += inner.nnz_rhs;
    info.bytes += inner.bytes;
    // r <- r - M d, x <- x + d, next correction buffer zeroed
    WL_CU(cudaMemsetAsync(st, 0, sizeof(CgState), S(h)));
    const bool stage_next = (ref == 0);
    DfResArgs ra{phase_graph_mid(h, grid_r - h->nhub), dcur, nullptr, rch, rcl, rh, rl,
                 stage_next ? (float*)h->r32.p : nullptr, xh, xl, stage_next ? dnext : nullptr,
                 ca, cA, cD, (double*)h->part.p, st, x_zero ? 1 : 0};
    ra.dsh_h = h->si_dsh_h;
    ra.dsh_l = h->si_dsh_l;
    const int pi = prof_begin(h, kCatRes);
    counted(h);
    WL_CU(launch_df_res(K, ra, grid_r, false, S(h)));
    prof_end(h, pi);
    info.nnz_rhs += (double)h->nnz * K;
    ++ndf;
    x_zero = false;
    staged = stage_next;
    rch = rh;
    rcl = rl;
    std::swap(dcur, dnext);
  }
  if (x_zero) {  // converged before any correction: X = 0
    WL_CU(cudaMemsetAsync(xh, 0, nk * 4, S(h)));
    WL_CU(cudaMemsetAsync(xl, 0, nk * 4, S(h)));
  }
  return WL_OK;
}

// Refined solve with FP64 B and X: B -> double-float once, X back to FP64.
int solve_refined(wl_handle* h, const double* b, double* x, int K, double tol, bool x_is_zero, SolveInfo& info) {
  const size_t nk = (size_t)h->n * K;
  const int grid_u = phase_blocks_f32(K);
  WL_TRY(ensure(h->bh, nk * 4));
  WL_TRY(ensure(h->bl, nk * 4));
  WL_TRY(ensure(h->xh, nk * 4));
  WL_TRY(ensure(h->xl, nk * 4));
  WL_TRY(ensure(h->r32, nk * 4));
  WL_TRY(ensure_phase_buffers(h, grid_u + h->nhub));
  CgState* st = h->cgst();
  double* bn2 = (double*)h->small.p + 600;
  WL_CU(cudaMemsetAsync(st, 0, sizeof(CgState), S(h)));
  counted(h);
  WL_CU(launch_df_from_f64(K, b, 1.0, h->n, (float*)h->bh.p, (float*)h->bl.p, nullptr, (double*)h->part.p, st, bn2,
                           grid_u, S(h)));
  WL_TRY(solve_refined_df(h, (const float*)h->bh.p, (const float*)h->bl.p, bn2, (float*)h->xh.p,
                          (float*)h->xl.p, x_is_zero ? nullptr : x, K, tol, info));
  counted(h);
  WL_CU(launch_split_x(nullptr, (int64_t)nk, (float*)h->xh.p, (float*)h->xl.p, true, x, S(h)));
  return WL_OK;
}

int solve(wl_handle* h, const double* b, double* x, int K, bool x_is_zero, SolveInfo& info) {
  const double tol = h->prm.tol;
  if (h->prm.prec != WL_FP64) return solve_refined(h, b, x, K, tol, x_is_zero, info);
  if (x_is_zero) WL_CU(cudaMemsetAsync(x, 0, (size_t)h->n * K * 8, S(h)));
  return solve_fp64(h, b, x, K, tol, x_is_zero, info);
}

// phi V for the exponential, c_k = beta^k / k! (Def. BDTW-Laplacian): the
// series sum_k c_k q_k V with the q_k of Eq. qrec applied term by term
// (exp_term kernels, double-float), V and X n x K FP64 in the internal order.
int exp_series(wl_handle* h, const double* V, double* X, int K, SolveInfo& info) {
  NvtxRange nvtx__("exponential series");
  const size_t nk = (size_t)h->n * K;
  const int gu = exp_blocks(K), gs = gu + h->nhub;
  WL_TRY(ensure(h->ew, nk * 4 * 8));
  WL_TRY(ensure_phase_buffers(h, gs));
  float* b = (float*)h->ew.p;
  float* W[3][2] = {{b, b + nk}, {b + 2 * nk, b + 3 * nk}, {b + 4 * nk, b + 5 * nk}};
  float* Ah = b + 6 * nk;
  float* Al = b + 7 * nk;
  CgState* st = h->cgst();
  WL_CU(cudaMemsetAsync(st, 0, sizeof(CgState), S(h)));
  const int one = 1;
  WL_CU(cudaMemcpyAsync(&st->active, &one, sizeof(int), cudaMemcpyHostToDevice, S(h)));
  counted(h);
  WL_CU(launch_df_split(V, nk, W[0][0], W[0][1], S(h)));  // s_0 = c_0 w_0 = V
  WL_CU(cudaMemcpyAsync(Ah, W[0][0], nk * 4, cudaMemcpyDeviceToDevice, S(h)));  // acc = s_0
  WL_CU(cudaMemcpyAsync(Al, W[0][1], nk * 4, cudaMemcpyDeviceToDevice, S(h)));
  const PhaseGraph pg = phase_graph_mid(h, gu);
  const int max_terms = std::max(h->prm.max_iter, 8);
  const int pc = prof_begin(h, kCatCG);
  int k = 0;
  int* hp = (int*)h->h_pin;
  for (;;) {
    for (int i = 0; i < kChunk && k < max_terms; ++i, ++k) {
      // s_{k+1} = ak A s_k + bk (diagonal) s_{k-1} with s_k = c_k w_k (bounded terms)
      const double ak = h->beta / (double)(k + 1);
      const double bk = k >= 1 ? h->beta * h->beta / ((double)k * (double)(k + 1)) : 0.0;
      ExpArgs a{pg, W[k % 3][0], W[k % 3][1], W[(k + 2) % 3][0], W[(k + 2) % 3][1], W[(k + 1) % 3][0],
                W[(k + 1) % 3][1], Ah, Al, df_from_double(h->mu), df_from_double(ak), df_from_double(bk), k,
                max_terms, (double*)h->part.p, st};
      counted(h);
      WL_CU(launch_exp_term(K, a, gs, S(h)));
    }
    WL_CU(cudaMemcpyAsync(hp, &st->active, 2 * sizeof(int), cudaMemcpyDeviceToHost, S(h)));
    WL_CU(cudaStreamSynchronize(S(h)));
    if (!hp[0] || k >= max_terms) break;
  }
  prof_end(h, pc);
  WL_CU(cudaMemcpyAsync(hp, st->status, 64 * sizeof(int), cudaMemcpyDeviceToHost, S(h)));
  WL_CU(cudaMemcpyAsync(hp + 64, &st->iters, sizeof(int), cudaMemcpyDeviceToHost, S(h)));
  WL_CU(cudaMemcpyAsync(hp + 65, &st->active, sizeof(int), cudaMemcpyDeviceToHost, S(h)));
  WL_CU(cudaStreamSynchronize(S(h)));
  const int terms = hp[64];
  for (int c = 0; c < K; ++c)
    if (hp[c] != 0 && info.status == WL_OK) info.status = hp[c];
  if (hp[65] && info.status == WL_OK) info.status = WL_ERR_NO_CONVERGENCE;  // term cap reached
  info.iters += terms;
  info.nnz_rhs += (double)terms * h->nnz * K;
  counted(h);
  WL_CU(launch_split_x(nullptr, (int64_t)nk, Ah, Al, true, X, S(h)));
  return WL_OK;
}

// phi X for a packed block V (n x K, device): X = M^{-1} (a V) for the
// resolvent; the result goes to X (n x K).
int phi_apply(wl_handle* h, const double* Vp, double* X, int K, SolveInfo& info) {
  if (h->prm.f == WL_F_EXP) return exp_series(h, Vp, X, K, info);
  const size_t nk = (size_t)h->n * K;
  WL_TRY(ensure(h->b64, nk * 8));
  // b = a V
  counted(h);
  WL_CU(launch_pack(Vp, K, 0, K, h->n, h->a_scale, h->b64.p, false, S(h)));
  return solve(h, (const double*)h->b64.p, X, K, true, info);
}

int compute_Df(wl_handle* h, SolveInfo& info) {
  WL_TRY(ensure(h->Df, (size_t)std::max<int64_t>(h->n, 1) * 8));
  double* Df = (double*)h->Df.p;
  if (h->prm.f == WL_F_IDENTITY) {
    counted(h);
    WL_CU(launch_degree_vector(h->g, Df, S(h)));
  } else if (h->prm.f == WL_F_EXP) {
    WL_TRY(ensure(h->b64, (size_t)h->n * 8));
    counted(h);
    WL_CU(launch_fill((double*)h->b64.p, 1.0, h->n, S(h)));
    WL_TRY(exp_series(h, (const double*)h->b64.p, Df, 1, info));
  } else if (h->prm.f == WL_F_RESOLVENT) {
    WL_TRY(ensure(h->b64, (size_t)h->n * 8));
    counted(h);
    WL_CU(launch_fill((double*)h->b64.p, h->a_scale, h->n, S(h)));
    bool zero = true;
    if (h->have_warm) {
      WL_CU(cudaMemcpyAsync(Df, h->warm.p, (size_t)h->n * 8, cudaMemcpyDeviceToDevice, S(h)));
      zero = false;
    }
    WL_TRY(solve(h, (const double*)h->b64.p, Df, 1, zero, info));
  } else {
    return WL_ERR_UNSUPPORTED;
  }
  h->have_Df = true;
  h->have_dfdf = false;
  return WL_OK;
}

// ------------------------------------------------------------------ spectral scale
// Largest eigenpair of Op = c0 I + A + cD D by Lanczos on a stored
// double-float basis (k = 1). A run stops once the error bound of its
// largest Ritz value is below rtol |theta|; a full basis restarts from the
// Ritz vector. The Ritz vector of the last run starts the next one.
struct SpRun {
  double c0 = 0.0, cD = 0.0;
  int m = 0;            // steps of the current run (held in the basis)
  int total = 0;        // steps over all runs of this operator
  double theta = 0.0;   // largest Ritz value
  double bound = 1e300; // its error bound
  bool exact = false;   // breakdown, or as many steps as nodes
};

int sp_cap(wl_handle* h) {
  const int64_t n = std::max<int64_t>(h->n, 1);
  const int64_t by_mem = (int64_t)(4.0e9 / (8.0 * (double)n));  // basis up to about 4 GB
  return (int)std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(kSpMax, std::max<int64_t>(by_mem, 16)), n));
}

SpArgs sp_args(wl_handle* h, double c0, double cD) {
  float2* W = (float2*)h->spW.p;
  return SpArgs{phase_graph(h), (const int32_t*)h->mid.p, h->nmid, h->nmid_blk, c0, 1.0, cD, (float2*)h->spV.p,
                {W, W + h->n}, (double*)h->part.p, (SpState*)h->spstate.p, 0, 0x5EEDull};
}

int sp_buffers(wl_handle* h, int gs) {
  WL_TRY(ensure(h->spV, (size_t)sp_cap(h) * h->n * 8));
  WL_TRY(ensure(h->spW, (size_t)2 * h->n * 8));
  WL_TRY(ensure(h->part, (size_t)gs * 64 * 2 * 8 + 1024));
  WL_TRY(ensure(h->spstate, sizeof(SpState)));
  return WL_OK;
}

// CTAs of the spectral kernels' row loops: all SMs' worth for large graphs,
// but no more than one CTA per kSpRows threads' worth of rows, so that the
// searches of small graphs (the batched build runs many side by side on
// separate streams) leave the GPU to the others. Four rows per thread measured
// 10% faster on the 64-graph batched build than one, and no slower on one
// graph of 1e6 nodes.
constexpr int kSpRows = 4;
int sp_grid(wl_handle* h) {
  const int64_t per = (int64_t)kPhaseBlock * kSpRows;  // rows per CTA and pass of the row loop
  const int64_t need = std::max<int64_t>(1, (h->n + per - 1) / per);
  return (int)std::min<int64_t>(sp_blocks(), need);
}

// Extend the run of r (or start one: seeded, or from the vector in W[1]
// when r->m == 0) until its bound is below rtol |theta| or it is exact.
int sp_run(wl_handle* h, SpRun* r, double rtol, bool seeded) {
  const int cap = sp_cap(h), gu = sp_grid(h), gs = gu + h->nhub + h->nmid_blk;
  WL_TRY(sp_buffers(h, gs));
  const SpArgs a = sp_args(h, r->c0, r->cD);
  SpState* st = (SpState*)h->spstate.p;
  for (int guard = 0; guard < 256; ++guard) {
    if (r->exact || (r->m > 0 && r->bound <= rtol * std::fabs(r->theta))) break;
    int mode = 2;
    bool restart = false;
    if (r->m == 0) {
      mode = (seeded && r->total == 0) ? 0 : 1;
    } else if (r->m >= cap) {  // basis full: restart from the Ritz vector
      restart = true;
      r->m = 0;
      mode = 1;
    }
    const int j0 = r->m, j1 = std::min(cap, j0 + 16);
    double o[8];
    int m_eff = 0, brk = 0;
    if (SpBatch* bt = t_sp_batch) {  // one round of the batched build's searches
      SpReq rq;
      rq.job.a = a;
      rq.job.rtol = rtol;
      rq.job.j0 = j0;
      rq.job.j1 = j1;
      rq.job.cap = cap;
      rq.job.mode = mode;
      rq.job.ritz = restart ? 1 : 0;
      rq.job.gs = gs;
      rq.job.gu = gu;
      WL_CU(cudaStreamSynchronize(S(h)));  // the handle's own work (graph, lists) is done
      WL_TRY(sp_batch_submit(bt, &rq));
      for (int i = 0; i < 8; ++i) o[i] = rq.out.out[i];
      m_eff = rq.out.m_eff;
      brk = rq.out.brk;
    } else {
      if (restart) {
        counted(h);
        WL_CU(launch_sp_ritz(a, gu, S(h)));
      }
      if (mode == 0) WL_CU(cudaMemsetAsync(st, 0, sizeof(SpState), S(h)));  // tickets and flags start at zero
      counted(h, 1 + 2 * (j1 - j0) + (j1 - j0 + kSpCheck - 1) / kSpCheck);
      WL_CU(launch_sp_start(a, mode, gu, S(h)));
      WL_CU(launch_sp_steps(a, j0, j1, cap, kSpCheck, rtol, gs, gu, S(h)));
      WL_CU(cudaMemcpyAsync(h->h_pin, &st->start_norm, 9 * 8 + 4 * 4, cudaMemcpyDeviceToHost, S(h)));
      WL_CU(cudaStreamSynchronize(S(h)));
      for (int i = 0; i < 8; ++i) o[i] = h->h_pin[1 + i];
      const int* ints = (const int*)(h->h_pin + 9);
      m_eff = ints[0];
      brk = ints[2];
    }
    r->total += m_eff - j0;
    r->m = m_eff;
    r->theta = o[0];
    r->bound = o[3];
    r->exact = brk != 0 || (int64_t)m_eff >= h->n;
    if (m_eff < j1 && !brk && r->bound > rtol * std::fabs(r->theta)) break;  // defensive: no progress
  }
  h->sp_c0 = r->c0;
  h->sp_cD = r->cD;
  h->sp_theta = r->theta;
  h->sp_ritz_ready = false;
  return WL_OK;
}

// Ritz vector of the last run into W[1]; q = u^T D u / |u|^2 and
// u^T A u / |u|^2 from the run's Ritz value.
int sp_ritz_q(wl_handle* h, double* q, double* uAu) {
  if (!h->sp_ritz_ready) {
    const int gu = sp_grid(h);
    const SpArgs a = sp_args(h, h->sp_c0, h->sp_cD);
    SpState* st = (SpState*)h->spstate.p;
    if (SpBatch* bt = t_sp_batch) {
      SpReq rq;
      rq.job.a = a;
      rq.job.mode = -1;
      rq.job.ritz = 1;
      rq.job.cap = sp_cap(h);
      rq.job.gs = 1;  // no steps: one idle CTA in the step kernels
      rq.job.gu = gu;
      WL_CU(cudaStreamSynchronize(S(h)));
      WL_TRY(sp_batch_submit(bt, &rq));
      h->sp_ritz_uu = rq.out.out[5];
      h->sp_ritz_udu = rq.out.out[6];
    } else {
      counted(h);
      WL_CU(launch_sp_ritz(a, gu, S(h)));
      WL_CU(cudaMemcpyAsync(h->h_pin, &st->out[5], 2 * 8, cudaMemcpyDeviceToHost, S(h)));
      WL_CU(cudaStreamSynchronize(S(h)));
      h->sp_ritz_uu = h->h_pin[0];
      h->sp_ritz_udu = h->h_pin[1];
    }
    h->sp_ritz_ready = true;
  }
  const double n2 = h->sp_ritz_uu;
  *q = n2 > 0 ? h->sp_ritz_udu / n2 : 0.0;
  *uAu = h->sp_theta - h->sp_c0 - h->sp_cD * (*q);
  return WL_OK;
}

int lambda_max_adaptive(wl_handle* h, double rtol, double* lmax) {
  SpRun r;
  WL_TRY(sp_run(h, &r, rtol, true));
  *lmax = r.theta;
  return WL_OK;
}

// rho(Z_mu): the largest lambda with lambda_max(A - (mu/lambda)(D - mu I)) =
// lambda (the quadratic eigenproblem lambda^2 u = lambda A u - mu (D - mu I) u
// behind Eq. Zdef). Each evaluation of h(lambda) = lambda_max(...) - lambda is
// one Lanczos run from the previous Ritz vector u, made only as accurate as
// the sign of h needs. The next lambda is the Rayleigh functional of u (the
// root of lambda^2 - lambda u^T A u + mu u^T (D - mu I) u = 0 nearest the
// current one, quadratically convergent), kept inside the bracket of signs
// seen so far; outside it, regula falsi (Illinois) or halving.
// Relative accuracy of the spectral searches of wl_build on the calling
// thread (0: kSpecRtolDefault): lambda_max(A) to that error bound, rho(Z_mu)
// to that bound and bracket. alpha = alpha_rel / rho needs no more (1e-12
// cost the 1e6-node build 1.1 of its 8.7 ms).
constexpr double kSpecRtolDefault = 1e-10;
thread_local double t_spec_rtol = 0.0;

int rho_companion(wl_handle* h, double mu, double lmaxA, double* rho) {
  NvtxRange nvtx__("rho(Z_mu)");
  if (mu == 0.0 || lmaxA <= 0.0) {
    *rho = lmaxA;
    return WL_OK;
  }
  const double kTight = t_spec_rtol > 0.0 ? t_spec_rtol : kSpecRtolDefault;
  const double kBracket = t_spec_rtol > 0.0 ? t_spec_rtol : kSpecRtolDefault;
  double q = 0.0, uAu = 0.0;
  WL_TRY(sp_ritz_q(h, &q, &uAu));
  auto rf = [&](double near) {
    const double c = mu * (q - mu), disc = uAu * uAu - 4.0 * c;
    if (!(disc >= 0.0)) return std::nan("");
    const double sq = std::sqrt(disc);
    const double r1 = 0.5 * (uAu + sq), r2 = 0.5 * (uAu - sq);
    return std::fabs(r1 - near) <= std::fabs(r2 - near) ? r1 : r2;
  };
  bool certain = true;
  auto hfun = [&](double lam, double* val) -> int {
    SpRun r;
    r.c0 = mu * mu / lam;
    r.cD = -mu / lam;
    double rtol = 1e-6;
    // a run that cannot resolve the sign (bound stuck above kTight) is taken as
    // |h| below the attainable accuracy after kMaxPasses passes: lambda is then the root
    constexpr int kMaxPasses = 32;
    for (int pass = 0;; ++pass) {
      WL_TRY(sp_run(h, &r, rtol, false));
      *val = r.theta - lam;
      certain = std::fabs(*val) > 10.0 * r.bound;
      if (certain || r.exact || r.bound <= kTight * std::fabs(r.theta) || pass + 1 >= kMaxPasses) break;
      rtol = std::max(kTight, 1e-3 * std::fabs(*val) / std::fabs(r.theta));
    }
    return sp_ritz_q(h, &q, &uAu);
  };
  // h(lambda_max(A)) <= 0: there lambda_max(A - (mu/lambda)(D - mu I)) <= lambda_max(A)
  // (D - mu I >= 0 on nodes with an edge; isolated nodes give mu^2 / lambda <= 1 <= lambda)
  double hi = lmaxA * (1.0 + 1e-12), lo = 0.0, fhi = 0.0, flo = 0.0;
  bool have_lo = false, have_fhi = false;
  double lam = rf(lmaxA);
  if (!(lam > 0.0 && lam < hi)) lam = 0.5 * hi;
  int side = 0;
  // the evaluation with the largest h: a double root (h touches zero from
  // below, as for mu = 1 on a cycle, where rho(Z_1) = 1 = d - mu = mu) shows
  // no sign change, and is taken where h came closest to zero
  double best_l = 0.0, best_h = -HUGE_VAL;
  for (int it = 0; it < 60; ++it) {
    double fx;
    WL_TRY(hfun(lam, &fx));
    if (!certain) {  // |h| is below what the Lanczos run resolves: lam is the root
      *rho = lam;
      return WL_OK;
    }
    if (fx > best_h) {
      best_h = fx;
      best_l = lam;
    }
    if (fx > 0) {
      lo = lam;
      flo = fx;
      have_lo = true;
      if (side == 1 && have_fhi) fhi *= 0.5;
      side = 1;
    } else {
      hi = lam;
      fhi = fx;
      have_fhi = true;
      if (side == -1 && have_lo) flo *= 0.5;
      side = -1;
    }
    if (hi - lo <= kBracket * hi) break;
    if (!have_lo && hi < 1e-12 * lmaxA) {  // no positive side found: a double root, or rho is 0
      *rho = (best_h > -1e-6 * lmaxA) ? best_l : 0.0;
      return WL_OK;
    }
    double nxt = rf(lam);
    if (!(nxt > lo && nxt < hi)) {
      if (have_lo && have_fhi) {
        nxt = (lo * fhi - hi * flo) / (fhi - flo);
        if (!(nxt > lo && nxt < hi)) nxt = 0.5 * (lo + hi);
      } else if (have_lo) {
        nxt = 0.5 * (lo + hi);
      } else {
        nxt = 0.5 * hi;
      }
    }
    lam = nxt;
  }
  *rho = have_lo ? 0.5 * (lo + hi) : ((best_h > -1e-6 * lmaxA) ? best_l : lam);
  return WL_OK;
}

// stage a caller array into device memory (copy if host)
int stage_in(wl_handle* h, Buf& st, const void* src, size_t bytes, const void** dev) {
  if (is_device_ptr(src)) {
    *dev = src;
    return WL_OK;
  }
  WL_TRY(ensure(st, bytes));
  WL_CU(cudaMemcpyAsync(st.p, src, bytes, cudaMemcpyHostToDevice, S(h)));
  *dev = st.p;
  return WL_OK;
}

void begin_timer(wl_handle* h) {
  prof_reset(h);
  cudaEventRecord(h->ev0, S(h));
}

double end_timer(wl_handle* h) {
  cudaEventRecord(h->ev1, S(h));
  cudaEventSynchronize(h->ev1);
  float ms = 0;
  cudaEventElapsedTime(&ms, h->ev0, h->ev1);
  return ms;
}

void fill_stats(wl_handle* h, wl_stats* st, const SolveInfo& in, int status, double ms, int outer) {
  if (!st) {
    prof_reset(h);
    return;
  }
  memset(st, 0, sizeof(*st));
  st->launches = h->launches;
  for (const auto& r : h->recs) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, h->ev_pool[r.a], h->ev_pool[r.b]) != cudaSuccess) {
      (void)cudaGetLastError();
      continue;
    }
    if (r.cat == kCatCG) { st->k_cg_launches++; st->k_cg_ms += t; }
    else if (r.cat == kCatRes) { st->k_res_launches++; st->k_res_ms += t; }
    else { st->k_lan_launches++; st->k_lan_ms += t; }
  }
  st->k_cg_iters = in.cg_iters;
  st->k_cg_bytes = in.bytes;
  prof_reset(h);
  st->status = status;
  st->iters = in.iters;
  st->outer_iters = outer;
  st->refinements = in.refinements;
  st->rel_res = in.max_rel;
  st->time_ms = ms;
  st->nnz_rhs_iters = in.nnz_rhs;
  st->bytes_alg = in.bytes;
  st->alpha = h->alpha;
  st->beta = h->beta;
  st->mu = h->mu;
  st->rho = h->rho;
  st->lambda_max = h->lmax;
  st->reorth_blocks = in.reorth_blocks;
}

// internal-order n-vector -> caller's array (host or device), undoing the relabelling
// taus (host) into a device array of the handle
int stage_taus(wl_handle* h, const double* taus, int ntau, const double** dtaus) {
  WL_TRY(ensure(h->taus, (size_t)std::max(ntau, 1) * 8));
  WL_CU(cudaMemcpyAsync(h->taus.p, taus, (size_t)ntau * 8, cudaMemcpyHostToDevice, S(h)));
  *dtaus = (const double*)h->taus.p;
  return WL_OK;
}

// ------------------------------------------------------------------ outer Lanczos on L (Sec. 4.1)
// One column block of the Krylov evaluation exp(-tau L) U0: the packed block
// (n x K FP64, internal order) in h->packX starts K lockstep Lanczos
// recurrences on L, one apply of L per step; every `check` steps y(tau) =
// exp(-tau T_m) e_1 is recomputed for all tau and the run stops when no
// (column, tau) changed by more than outer_tol |y| since the last check
// (an underflowed y = 0 never counts as converged). The
// basis, T, the column norms and m stay in the handle for outer_combine.
struct OuterRun {
  int K = 0, m = 0, ntau = 0;
  bool converged = false, dfp = false;
  size_t blk = 0;
  const double* dtaus = nullptr;
  // shift-and-invert run: the shift, the time points and T_m per column (host)
  bool si = false;
  double sigma = 0.0;
  std::vector<double> taus, Ta, Tb;  // Ta, Tb: K x m
};

constexpr int kLdT = 1024;  // T and y leading dimension (Lanczos steps per column at most kLdT - 1)

// ------------------------------------------------------------------ shift-and-invert Lanczos (Sec. 4.4)
// Eigenvalues th[0..m) and eigenvectors (column k: Z[i * m + k]) of the
// symmetric tridiagonal matrix with diagonal a[0..m) and off-diagonal
// b[0..m-1), by implicit QR sweeps with the Wilkinson shift on each
// unreduced block (Golub and Van Loan, Sec. 8.3), the rotations accumulated
// into Z. False if a block needs more than 30 m sweeps.
bool tridiag_eig_host(int m, const double* a, const double* b, std::vector<double>& th, std::vector<double>& Z) {
  th.assign(a, a + m);
  std::vector<double> e(std::max(m, 1), 0.0);
  for (int i = 0; i + 1 < m; ++i) e[i] = b[i];
  Z.assign((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) Z[(size_t)i * m + i] = 1.0;
  const double eps = 2.220446049250313e-16;
  int hi = m - 1, sweeps = 0;
  while (hi > 0) {
    if (std::fabs(e[hi - 1]) <= eps * (std::fabs(th[hi - 1]) + std::fabs(th[hi]))) {
      e[hi - 1] = 0.0;
      --hi;
      continue;
    }
    int lo = hi - 1;
    while (lo > 0 && std::fabs(e[lo - 1]) > eps * (std::fabs(th[lo - 1]) + std::fabs(th[lo]))) --lo;
    if (lo > 0) e[lo - 1] = 0.0;
    if (++sweeps > 30 * m) return false;
    const double t = 0.5 * (th[hi - 1] - th[hi]), bb = e[hi - 1];
    const double mu = th[hi] - bb * bb / (t + std::copysign(std::hypot(t, bb), t));
    double x = th[lo] - mu, z = e[lo];
    for (int k = lo; k < hi; ++k) {
      const double r = std::hypot(x, z);
      const double c = r > 0.0 ? x / r : 1.0, sn = r > 0.0 ? z / r : 0.0;
      if (k > lo) e[k - 1] = r;
      const double dk = th[k], dk1 = th[k + 1], ek = e[k];
      th[k] = c * c * dk + 2.0 * c * sn * ek + sn * sn * dk1;
      th[k + 1] = sn * sn * dk - 2.0 * c * sn * ek + c * c * dk1;
      e[k] = c * sn * (dk1 - dk) + (c * c - sn * sn) * ek;
      if (k + 1 < hi) {
        z = sn * e[k + 1];
        e[k + 1] *= c;
        x = e[k];
      }
      for (int i = 0; i < m; ++i) {
        double* zr = &Z[(size_t)i * m];
        const double zk = zr[k], zk1 = zr[k + 1];
        zr[k] = c * zk + sn * zk1;
        zr[k + 1] = -sn * zk + c * zk1;
      }
    }
  }
  return true;
}

// y(tau) = exp(-tau (T^{-1} - sigma I)) e_1 for every tau from the
// eigendecomposition of one column's T (m steps): y[t * ld + i]. An
// eigenvalue theta <= 0 (a direction that the shifted inverse maps to 0, or
// rounding of one) contributes nothing.
bool si_eval(int m, const double* a, const double* b, double sigma, const std::vector<double>& taus, double* y,
             int ld) {
  std::vector<double> th, Z;
  if (!tridiag_eig_host(m, a, b, th, Z)) return false;
  for (size_t t = 0; t < taus.size(); ++t) {
    double* yt = y + t * ld;
    for (int i = 0; i < m; ++i) yt[i] = 0.0;
    for (int k = 0; k < m; ++k) {
      if (!(th[k] > 0.0)) continue;
      const double f = std::exp(-taus[t] * (1.0 / th[k] - sigma)) * Z[k];
      if (f == 0.0) continue;
      for (int i = 0; i < m; ++i) yt[i] += Z[(size_t)i * m + k] * f;
    }
  }
  return true;
}

// the per-row diagonal and scaling of the shifted solves for the handle's
// D_f and shift sigma (sibuf: dsh64, inv64 (n doubles each), then dsh_h,
// dsh_l, inv_h, inv_l (n floats each))
int si_setup(wl_handle* h, double sigma) {
  const int64_t n = h->n;
  WL_TRY(ensure(h->sibuf, (size_t)n * 32 + 256));
  double* d64 = (double*)h->sibuf.p;
  float* f32 = (float*)(d64 + 2 * n);
  counted(h);
  WL_CU(launch_si_prep((const double*)h->Df.p, n, h->a_scale, sigma, d64, f32, f32 + n, d64 + n, f32 + 2 * n,
                       f32 + 3 * n, S(h)));
  h->si_sigma = sigma;
  return WL_OK;
}

// While alive, the solves of the handle add the diagonal -a / (D_f + sigma) to M.
struct SiScope {
  wl_handle* h;
  SiScope(wl_handle* hh, bool dfp) : h(hh) {
    const int64_t n = h->n;
    double* d64 = (double*)h->sibuf.p;
    float* f32 = (float*)(d64 + 2 * n);
    if (dfp) {
      h->si_dsh_h = f32;
      h->si_dsh_l = f32 + n;
    } else {
      h->si_dsh64 = d64;
    }
  }
  ~SiScope() {
    h->si_dsh64 = nullptr;
    h->si_dsh_h = h->si_dsh_l = nullptr;
  }
};

// One application of R = (L + sigma I)^{-1} to the basis block j, leaving
// -R v_j where the Lanczos step kernels read it: the double-float form in
// (h->rh, h->rl), the FP64 form in h->packX. x = R v_j = M z with z the
// solution of (M - a Dt^{-1}) z = Dt^{-1} v_j, and M z follows without a
// product with M from the solve's final residual r: M z = (B - r) + a Dt^{-1} z.
int si_apply(wl_handle* h, bool dfp, int K, int j, size_t blk, SolveInfo& info) {
  const int64_t n = h->n;
  double* d64 = (double*)h->sibuf.p;
  float* f32 = (float*)(d64 + 2 * n);
  if (dfp) {
    float* vjh = (float*)h->basis.p + (size_t)2 * j * blk;
    WL_TRY(ensure(h->bh, blk * 4));
    WL_TRY(ensure(h->bl, blk * 4));
    WL_TRY(ensure(h->part, (size_t)std::max(si_rhs_blocks(n, K), 1) * 64 * 8 + 1024));
    double* bn2si = (double*)h->small.p + 744;
    counted(h, 2);
    WL_CU(launch_si_rhs_df(vjh, vjh + blk, f32 + 2 * n, f32 + 3 * n, n, K, (float*)h->bh.p, (float*)h->bl.p,
                           (double*)h->part.p, bn2si, S(h)));
    {
      SiScope sc(h, true);
      WL_TRY(solve_refined_df(h, (const float*)h->bh.p, (const float*)h->bl.p, bn2si, (float*)h->xh.p,
                              (float*)h->xl.p, nullptr, K, h->prm.tol, info));
    }
    if (info.status != WL_OK) return WL_OK;
    // (rh, rl) = -M z = -((B - r) + a Dt^{-1} z), r the solve's final residual in (rh, rl)
    counted(h);
    WL_CU(launch_si_mz_df((const float*)h->bh.p, (const float*)h->bl.p, (const float*)h->rh.p,
                          (const float*)h->rl.p, (const float*)h->xh.p, (const float*)h->xl.p, f32 + 2 * n,
                          f32 + 3 * n, h->a_scale, n, K, (float*)h->rh.p, (float*)h->rl.p, S(h)));
  } else {
    const double* vj = (const double*)h->basis.p + (size_t)j * blk;
    WL_TRY(ensure(h->b64, blk * 8));
    WL_TRY(ensure(h->x, blk * 8));
    counted(h);
    WL_CU(launch_si_rhs64(vj, d64 + n, n, K, (double*)h->b64.p, S(h)));
    WL_CU(cudaMemsetAsync(h->x.p, 0, blk * 8, S(h)));
    {
      SiScope sc(h, false);
      WL_TRY(solve_fp64(h, (const double*)h->b64.p, (double*)h->x.p, K, h->prm.tol, true, info));
    }
    if (info.status != WL_OK) return WL_OK;
    // packX = -M z = -((B - r) + a Dt^{-1} z), r the CG's final residual in h->r
    counted(h);
    WL_CU(launch_si_mz64((const double*)h->b64.p, (const double*)h->r.p, (const double*)h->x.p, d64 + n,
                         h->a_scale, n, K, (double*)h->packX.p, S(h)));
  }
  return WL_OK;
}

// Reorthogonalises basis block j + 1 (columns with mask 1) against blocks
// 0..j; beta_j of those columns is rescaled on the device.
int reorth_block(wl_handle* h, bool dfp, int K, int j, size_t blk, double* Tb, int* done, const int* hmask) {
  const int nb = j + 1;
  WL_TRY(ensure(h->robuf, reorth_part_doubles(nb, K, blk) * 8));
  WL_TRY(ensure(h->romask, 64 * sizeof(int)));
  WL_CU(cudaMemcpyAsync(h->romask.p, hmask, K * sizeof(int), cudaMemcpyHostToDevice, S(h)));
  ReorthArgs ra{};
  ra.basis = h->basis.p;
  if (dfp) {
    ra.v = (float*)h->basis.p + (size_t)2 * (j + 1) * blk;
    ra.vlo = (float*)h->basis.p + (size_t)(2 * (j + 1) + 1) * blk;
  } else {
    ra.v = (double*)h->basis.p + (size_t)(j + 1) * blk;
    ra.vlo = nullptr;
  }
  ra.n = h->n;
  ra.K = K;
  ra.nb = nb;
  ra.blk = blk;
  ra.part = (double*)h->robuf.p;
  ra.mask = (const int*)h->romask.p;
  ra.Tb = Tb;
  ra.done = done;
  ra.j = j;
  ra.ldT = kLdT;
  const int pl = prof_begin(h, kCatLan);
  counted(h, 8);
  const cudaError_t e = launch_reorth(ra, dfp, S(h));
  prof_end(h, pl);
  if (e != cudaSuccess) return set_cuda_error(e, "reorth");
  return WL_OK;
}
constexpr int kMaxReturnT = 256;  // time points per wl_return_prob call

int outer_run(wl_handle* h, int K, const double* dtaus, int ntau, SolveInfo& info, OuterRun& o, int& outer_total) {
  NvtxRange nvtx__("outer Lanczos on L");
  const int64_t n = h->n;
  const int ldT = kLdT;
  const int maxm = std::min(h->prm.max_outer, ldT - 1);
  // steps between convergence checks: the shift-and-invert check is a host
  // eigendecomposition of the small T_m (microseconds), so it runs every 2
  // steps (every 4 overshot the headline diffusion by 2 steps; every step
  // stops on a change between consecutive steps that underestimates the error
  // and ended at 1e-8 instead of 1.3e-9); the polynomial check is a device
  // series with a host read, every 4 steps
  const int check = (h->prm.shift > 0.0) ? 2 : 4;
  // refined resolvent form: double-float outer recurrence (FP32 instructions only)
  const bool dfp = h->prm.prec != WL_FP64 && h->prm.f == WL_F_RESOLVENT;
  o = OuterRun{};
  o.K = K;
  o.ntau = ntau;
  o.dfp = dfp;
  o.dtaus = dtaus;
  const bool si = h->prm.shift > 0.0;  // shift-and-invert Lanczos on (L + sigma I)^{-1}
  if (si && h->prm.f != WL_F_RESOLVENT) return WL_ERR_UNSUPPORTED;
  if (h->prm.f != WL_F_IDENTITY && !h->have_Df) WL_TRY(compute_Df(h, info));
  if (info.status != WL_OK) return WL_OK;
  if (si) {
    WL_TRY(si_setup(h, h->prm.shift));
    o.si = true;
    o.sigma = h->prm.shift;
    o.taus.resize(ntau);
    WL_CU(cudaMemcpyAsync(h->h_pin, dtaus, (size_t)ntau * 8, cudaMemcpyDeviceToHost, S(h)));
    WL_CU(cudaStreamSynchronize(S(h)));
    for (int t = 0; t < ntau; ++t) o.taus[t] = h->h_pin[t];
  }
  if (dfp && !h->have_dfdf) {  // D_f as two FP32 terms for the double-float outer recurrence
    WL_TRY(ensure(h->dfdf, (size_t)n * 8));
    counted(h);
    WL_CU(launch_df_split((const double*)h->Df.p, (size_t)n, (float*)h->dfdf.p, (float*)h->dfdf.p + n, S(h)));
    h->have_dfdf = true;
  }
  const size_t blk = (size_t)n * K;
  o.blk = blk;
  size_t want_blocks = (size_t)std::min(maxm + 1, 160);
  if (h->basis_blocks < want_blocks || h->basis.bytes < want_blocks * blk * 8) {
    WL_TRY(ensure(h->basis, want_blocks * blk * 8));
    h->basis_blocks = want_blocks;
  }
  size_t cap_blocks = h->basis.bytes / (blk * 8);
  WL_TRY(ensure(h->Tab, (size_t)2 * K * ldT * 8 + 64 * 8 * 4));
  WL_TRY(ensure(h->ybuf, (size_t)K * ntau * ldT * 8));
  WL_TRY(ensure(h->yprev, (size_t)K * ntau * ldT * 8));
  WL_TRY(ensure(h->errb, (size_t)K * ntau * 8 * 2 + 64 * 4 * 4));
  double* basis = (double*)h->basis.p;
  double* Ta = (double*)h->Tab.p;
  double* Tb = Ta + (size_t)K * ldT;
  double* nrm = Tb + (size_t)K * ldT;
  int* done = (int*)((double*)h->errb.p + (size_t)K * ntau * 2);
  int* mcol = done + 64;
  int* mprev = done + 128;
  double* errd = (double*)h->errb.p;
  // V_0 = U0 block / |U0 block| (per column)
  counted(h, 3);
  WL_TRY(ensure(h->part, (size_t)304 * 64 * 8 + 1024));
  cudaError_t e = launch_colnorms((const double*)h->packX.p, n, K, nrm, (double*)h->part.p, S(h));
  if (e == cudaSuccess)
    e = dfp ? launch_df_scale_cols((const double*)h->packX.p, n, K, nrm, (float*)basis, (float*)basis + blk, S(h))
            : launch_scale_cols((const double*)h->packX.p, n, K, nrm, basis, S(h));
  if (e != cudaSuccess) return set_cuda_error(e, "expmv init");
  // done flags: zero columns
  WL_CU(cudaMemcpyAsync(h->h_pin, nrm, K * 8, cudaMemcpyDeviceToHost, S(h)));
  WL_CU(cudaStreamSynchronize(S(h)));
  std::vector<int> hdone(K), hzero(K, 0);
  std::vector<double> hb2(K);
  for (int c = 0; c < K; ++c) {
    hdone[c] = (h->h_pin[c] > 0.0) ? 0 : 1;
    hb2[c] = hdone[c] ? 0.0 : 1.0;
  }
  WL_CU(cudaMemcpyAsync(done, hdone.data(), K * 4, cudaMemcpyHostToDevice, S(h)));
  WL_CU(cudaMemcpyAsync(mprev, hzero.data(), K * 4, cudaMemcpyHostToDevice, S(h)));
  double* bn2 = (double*)h->small.p + 664;  // |v_j|^2 per column for the double-float solves
  if (dfp) {
    WL_CU(cudaMemcpyAsync(bn2, hb2.data(), K * 8, cudaMemcpyHostToDevice, S(h)));
    WL_TRY(ensure(h->xh, blk * 4));
    WL_TRY(ensure(h->xl, blk * 4));
  }
  const int Gs = dfp ? df_lanczos_grid(K) : lanczos_step_grid(K);
  int Tw, Tc;
  thresholds_f64(K, &Tw, &Tc);
  PartDev* pd = nullptr;
  if (!dfp) WL_TRY(get_part(h, Gs, Tw, Tc, &pd, K, 8));
  WL_TRY(ensure(h->part, (size_t)std::max(Gs, 1) * 64 * 2 * 8 + 1024));
  int m = 0;
  bool converged = false;
  const bool reorth = h->prm.reorth == 1;
  const std::vector<int> rmask(K, 1);
  std::vector<std::vector<double>> si_prev(si ? (size_t)K * ntau : 0);  // y(tau) of the last check
  for (int j = 0; j < maxm; ++j) {
    if ((size_t)(j + 2) > cap_blocks) {
      // grow the basis (double), keeping the blocks computed so far
      Buf nb;
      size_t nbk = std::min<size_t>((size_t)maxm + 1, cap_blocks * 2);
      WL_TRY(ensure(nb, nbk * blk * 8));
      WL_CU(cudaMemcpyAsync(nb.p, h->basis.p, cap_blocks * blk * 8, cudaMemcpyDeviceToDevice, S(h)));
      WL_CU(cudaStreamSynchronize(S(h)));
      release(h->basis);
      h->basis = nb;
      h->basis_blocks = nbk;
      cap_blocks = nbk;
      basis = (double*)h->basis.p;
    }
    if (dfp) {
      // double-float basis: block j holds hi then lo terms
      float* vjh = (float*)basis + (size_t)2 * j * blk;
      float* vmh = j > 0 ? (float*)basis + (size_t)2 * (j - 1) * blk : nullptr;
      float* vph = (float*)basis + (size_t)2 * (j + 1) * blk;
      if (si) {  // Y = -R v_j in (rh, rl); w = 0 v_j - 1 Y
        WL_TRY(si_apply(h, true, K, j, blk, info));
      } else {
        WL_TRY(solve_refined_df(h, vjh, vjh + blk, bn2, (float*)h->xh.p, (float*)h->xl.p, nullptr, K, h->prm.tol,
                                info));
      }
      if (info.status != WL_OK) return WL_OK;
      WL_TRY(ensure(h->part, (size_t)std::max(Gs, 1) * 64 * 2 * 8 + 1024));
      DfLanczosArgs la{vjh, vjh + blk, vmh, vmh ? vmh + blk : nullptr, (const float*)h->xh.p,
                       (const float*)h->xl.p, (const float*)h->dfdf.p, (const float*)h->dfdf.p + n,
                       df_from_double(h->a_scale), vph, vph + blk, Ta, Tb, done, bn2, (double*)h->part.p,
                       h->bar, n, j, ldT};
      if (si) {
        la.yh = (const float*)h->rh.p;
        la.yl = (const float*)h->rl.p;
        la.dfh = la.dfl = nullptr;
        la.ascale = df_from_double(1.0);
      }
      WL_TRY(reset_bar(h));
      const int pl = prof_begin(h, kCatLan);
      counted(h);
      e = launch_df_lanczos_step(K, la, Gs, S(h));
      prof_end(h, pl);
      if (e != cudaSuccess) return set_cuda_error(e, "df_lanczos_step");
    } else {
      double* vj = basis + (size_t)j * blk;
      double* vjm1 = j > 0 ? basis + (size_t)(j - 1) * blk : nullptr;
      double* vjp1 = basis + (size_t)(j + 1) * blk;
      LanczosStepArgs la{h->g, pd->view(), vj, vjm1, nullptr, (const double*)h->Df.p, 0, 0, 0, vjp1,
                         Ta, Tb, done, (double*)h->part.p, h->bar, j, ldT, 0};
      if (si) {  // X = -R v_j in packX; w = 0 v_j - X
        WL_TRY(si_apply(h, false, K, j, blk, info));
        if (info.status != WL_OK) return WL_OK;
        la.X = (const double*)h->packX.p;
        la.Df = nullptr;
        la.part = (double*)h->part.p;
      } else if (h->prm.f == WL_F_IDENTITY) {
        la.mode = 1;
        la.c0 = 0.0;
        la.cA = -1.0;
        la.cD = 1.0;
        info.nnz_rhs += (double)h->nnz * K;
        info.iters += 1;
      } else {
        WL_TRY(phi_apply(h, vj, (double*)h->packX.p, K, info));
        if (info.status != WL_OK) return WL_OK;
        la.X = (const double*)h->packX.p;
        la.part = (double*)h->part.p;
      }
      WL_TRY(reset_bar(h));
      const int pl = prof_begin(h, kCatLan);
      e = launch_lanczos_step(K, la, Gs, S(h));
      prof_end(h, pl);
      if (e != cudaSuccess) return set_cuda_error(e, "lanczos_step");
    }
    m = j + 1;
    ++outer_total;
    if (si && (m % check == 0 || m == maxm)) {
      // y(tau) = exp(-tau (T_m^{-1} - sigma I)) e_1 per column on the host,
      // compared with the previous check's (the rule of the polynomial run)
      std::vector<double> hT((size_t)2 * K * m);
      WL_CU(cudaMemcpy2DAsync(hT.data(), (size_t)m * 8, Ta, (size_t)ldT * 8, (size_t)m * 8, K,
                              cudaMemcpyDeviceToHost, S(h)));
      WL_CU(cudaMemcpy2DAsync(hT.data() + (size_t)K * m, (size_t)m * 8, Tb, (size_t)ldT * 8, (size_t)m * 8, K,
                              cudaMemcpyDeviceToHost, S(h)));
      WL_CU(cudaStreamSynchronize(S(h)));
      const int berr = check_bar(h);
      if (berr) return berr;
      bool all = true;
      std::vector<double> y((size_t)ntau * m);
      for (int c = 0; c < K; ++c) {
        if (!si_eval(m, hT.data() + (size_t)c * m, hT.data() + (size_t)(K + c) * m, o.sigma, o.taus, y.data(), m)) {
          all = false;
          continue;
        }
        for (int t = 0; t < ntau; ++t) {
          const double* yt = y.data() + (size_t)t * m;
          double ny = 0.0, dy = 0.0;
          const std::vector<double>& yp = si_prev[(size_t)c * ntau + t];
          for (int i = 0; i < m; ++i) {
            const double d = yt[i] - (i < (int)yp.size() ? yp[i] : 0.0);
            ny += yt[i] * yt[i];
            dy += d * d;
          }
          // a zero start column (the padding of a block) has nothing to
          // converge; in any other column a y that vanished is not converged
          // (the space has not reached the slow modes yet)
          const bool ok =
              hdone[c] || (!yp.empty() && ny > 0.0 && std::sqrt(dy) <= h->prm.outer_tol * std::sqrt(ny));
          if (!ok) all = false;
          si_prev[(size_t)c * ntau + t].assign(yt, yt + m);
        }
      }
      if (all) { converged = true; break; }
    } else if (m % check == 0 || m == maxm) {
      std::vector<int> hm(K, m);
      WL_CU(cudaMemcpyAsync(mcol, hm.data(), K * 4, cudaMemcpyHostToDevice, S(h)));
      TridiagArgs ta{Ta, Tb, mcol, dtaus, (double*)h->ybuf.p, (double*)h->yprev.p, mprev, errd, ldT, ntau, 1,
                     kChebMax};
      counted(h);
      e = launch_tridiag_exp(ta, K, m, S(h));
      if (e != cudaSuccess) return set_cuda_error(e, "tridiag_exp");
      WL_CU(cudaMemcpyAsync(mprev, mcol, K * 4, cudaMemcpyDeviceToDevice, S(h)));
      WL_CU(cudaMemcpyAsync(h->h_pin, errd, (size_t)K * ntau * 8, cudaMemcpyDeviceToHost, S(h)));
      const int berr = check_bar(h);
      if (berr) return berr;
      bool all = true;
      for (int c = 0; c < K && all; ++c)
        for (int t = 0; t < ntau; ++t)
          if (!(h->h_pin[c * ntau + t] <= h->prm.outer_tol)) { all = false; break; }
      if (all) { converged = true; break; }
    }
    if (reorth && m < maxm) {  // the run goes on: make v_{j+1} orthogonal to v_0 .. v_j
      WL_TRY(reorth_block(h, dfp, K, j, blk, Tb, done, rmask.data()));
      info.reorth_blocks += 1;
    }
  }
  o.m = m;
  o.converged = converged;
  if (si && m > 0) {  // T_m per column for outer_combine
    o.Ta.resize((size_t)K * m);
    o.Tb.resize((size_t)K * m);
    WL_CU(cudaMemcpy2DAsync(o.Ta.data(), (size_t)m * 8, Ta, (size_t)ldT * 8, (size_t)m * 8, K,
                            cudaMemcpyDeviceToHost, S(h)));
    WL_CU(cudaMemcpy2DAsync(o.Tb.data(), (size_t)m * 8, Tb, (size_t)ldT * 8, (size_t)m * 8, K,
                            cudaMemcpyDeviceToHost, S(h)));
    WL_CU(cudaStreamSynchronize(S(h)));
  }
  return WL_OK;
}

// U(tau) = |u0| V_m y(tau) for taus [t0, t0 + nt) of an outer run, nt <=
// kMaxTau: block t at out + t * tstride, row perm[i] (or i), columns c0..c0+K.
int outer_combine(wl_handle* h, const OuterRun& o, int t0, int nt, double* out, int64_t ld, int64_t tstride, int c0,
                  const int32_t* perm) {
  const int K = o.K, ldT = kLdT;
  const int64_t n = h->n;
  double* Ta = (double*)h->Tab.p;
  double* Tb = Ta + (size_t)K * ldT;
  double* nrm = Tb + (size_t)K * ldT;
  int* done = (int*)((double*)h->errb.p + (size_t)K * o.ntau * 2);
  int* mcol = done + 64;
  int* mzero = done + 192;  // no previous y: the change estimate is not used here
  double* errd = (double*)h->errb.p;
  std::vector<int> hm(K, o.m), hz(K, 0);
  WL_CU(cudaMemcpyAsync(mcol, hm.data(), K * 4, cudaMemcpyHostToDevice, S(h)));
  WL_CU(cudaMemcpyAsync(mzero, hz.data(), K * 4, cudaMemcpyHostToDevice, S(h)));
  cudaError_t e = cudaSuccess;
  if (o.si) {  // y(tau) from the eigendecomposition of each column's T_m (host)
    std::vector<double> hy((size_t)K * nt * ldT, 0.0);
    const std::vector<double> tt(o.taus.begin() + t0, o.taus.begin() + t0 + nt);
    for (int c = 0; c < K; ++c)
      if (o.m > 0 && !si_eval(o.m, o.Ta.data() + (size_t)c * o.m, o.Tb.data() + (size_t)c * o.m, o.sigma, tt,
                              hy.data() + (size_t)c * nt * ldT, ldT))
        return WL_ERR_NO_CONVERGENCE;
    WL_CU(cudaMemcpyAsync(h->ybuf.p, hy.data(), hy.size() * 8, cudaMemcpyHostToDevice, S(h)));
    WL_CU(cudaStreamSynchronize(S(h)));
  } else {
    TridiagArgs ta{Ta, Tb, mcol, o.dtaus + t0, (double*)h->ybuf.p, (double*)h->yprev.p, mzero, errd, ldT, nt, 1,
                   kChebMax};
    counted(h);
    e = launch_tridiag_exp(ta, K, o.m, S(h));
    if (e != cudaSuccess) return set_cuda_error(e, "tridiag_exp");
  }
  if (o.dfp) {
    const size_t ny = (size_t)K * nt * ldT;
    WL_TRY(ensure(h->ydf, ny * 8));
    counted(h, 2);
    e = launch_df_split((const double*)h->ybuf.p, ny, (float*)h->ydf.p, (float*)h->ydf.p + ny, S(h));
    DfCombineArgs ca{(const float*)h->basis.p, (const float*)h->ydf.p, (const float*)h->ydf.p + ny, mcol, nrm, out,
                     n, ld, tstride, c0, ldT, nt, perm};
    if (e == cudaSuccess) e = launch_df_combine(K, ca, S(h));
  } else {
    CombineArgs ca{(const double*)h->basis.p, (const double*)h->ybuf.p, mcol, nrm, out, n, ld, tstride, c0, ldT, nt,
                   perm};
    counted(h);
    e = launch_combine(K, ca, S(h));
  }
  if (e != cudaSuccess) return set_cuda_error(e, "combine");
  return WL_OK;
}

int copy_out_vec(wl_handle* h, const double* src, double* dst) {
  const size_t bytes = (size_t)h->n * 8;
  if (!h->perm) {
    WL_CU(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, S(h)));
    return WL_OK;
  }
  double* d = dst;
  const bool dev = is_device_ptr(dst);
  if (!dev) {
    WL_TRY(ensure(h->stage_b, bytes));
    d = (double*)h->stage_b.p;
  }
  counted(h);
  WL_CU(launch_permute_vec(src, h->n, h->perm, true, d, S(h)));
  if (!dev) WL_CU(cudaMemcpyAsync(dst, d, bytes, cudaMemcpyDeviceToHost, S(h)));
  return WL_OK;
}

void free_handle(wl_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  (void)cudaGetLastError();
  CallScope none(nullptr);  // everything below goes straight back to the allocator
  for (auto& kv : h->parts) {
    pool_free(kv.second.rb);
    pool_free(kv.second.seg);
    pool_free(kv.second.meta);
  }
  Buf* bufs[] = {&h->csr_rp, &h->csr_col, &h->x, &h->r, &h->p, &h->q, &h->b64, &h->d32,
                 &h->r32, &h->xh, &h->xl, &h->d32b, &h->bh, &h->bl, &h->rh, &h->rl, &h->dfdf, &h->ydf, &h->ew, &h->taus, &h->ybig, &h->part, &h->small, &h->Df, &h->warm, &h->basis, &h->Tab, &h->ybuf, &h->yprev,
                 &h->errb, &h->stage_a, &h->stage_b, &h->packV, &h->packX, &h->spV, &h->spW, &h->spstate, &h->mid, &h->omega, &h->gram,
                 &h->omega_int, &h->ptmp, &h->perm_b, &h->iperm_b, &h->hubs, &h->cgstate};
  for (Buf* b : bufs) release(*b);
  for (void* p : h->retired) pool_free(p);
  h->retired.clear();
  if (h->bar) pool_free(h->bar);
  if (h->h_pin) pool_free_host(h->h_pin);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  delete h;
}

void default_params(wl_params* p) {
  if (p->tol <= 0) p->tol = 1e-12;
  if (p->max_iter <= 0) p->max_iter = 2000;
  if (p->max_outer <= 0) p->max_outer = 400;
  if (p->max_outer > 1000) p->max_outer = 1000;
  if (p->outer_tol <= 0) p->outer_tol = 1e-10;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

const char* wl_status_string(int s) {
  switch (s) {
    case WL_OK: return "ok";
    case WL_ERR_INVALID_ARG: return "invalid argument";
    case WL_ERR_NOT_SYMMETRIC: return "adjacency pattern is not symmetric";
    case WL_ERR_SELF_LOOP: return "self-loop stored in the adjacency";
    case WL_ERR_UNSORTED: return "CSR malformed: row_ptr not monotone, or columns unsorted, duplicated or out of range";
    case WL_ERR_ALPHA_RANGE: return "alpha * rho(Z_mu) >= 1: the walk series diverges";
    case WL_ERR_NOT_SPD: return "CG breakdown: operator not positive definite";
    case WL_ERR_NONFINITE: return "non-finite value in inputs or iterates";
    case WL_ERR_NO_CONVERGENCE: return "iteration cap reached before the tolerance";
    case WL_ERR_TIMEOUT: return "bounded device wait expired";
    case WL_ERR_OOM: return "device memory allocation failed";
    case WL_ERR_CUDA: return "CUDA runtime error";
    case WL_ERR_UNSUPPORTED: return "combination not supported";
  }
  return "unknown status";
}

const char* wl_last_error(void) { return g_last_error.c_str(); }

int wl_build(const wl_csr* A, wl_variant v, const wl_params* p, wl_handle** out, wl_stats* st) {
  NvtxRange nvtx__("wl_build");
  if (!out) return WL_ERR_INVALID_ARG;
  *out = nullptr;
  if (!A || !p || A->n < 0 || A->nnz < 0 || A->nnz >= (int64_t)INT32_MAX || A->n >= (int64_t)INT32_MAX)
    return WL_ERR_INVALID_ARG;
  if ((A->n > 0 && !A->row_ptr) || (A->nnz > 0 && !A->col_idx)) return WL_ERR_INVALID_ARG;
  if (v != WL_ALLWALK && v != WL_NBT && v != WL_BTDW) return WL_ERR_INVALID_ARG;
  if (p->f != WL_F_RESOLVENT && p->f != WL_F_EXP && p->f != WL_F_IDENTITY) return WL_ERR_INVALID_ARG;
  if (p->prec != WL_FP64 && p->prec != WL_REFINED && p->prec != WL_SKETCH) return WL_ERR_INVALID_ARG;
  if (p->reorth < 0 || p->reorth > 1) return WL_ERR_INVALID_ARG;
  if (p->gram < 0 || p->gram > 1) return WL_ERR_INVALID_ARG;
  if (!(p->shift >= 0.0) || !std::isfinite(p->shift)) return WL_ERR_INVALID_ARG;
  double mu = (v == WL_ALLWALK) ? 0.0 : (v == WL_NBT ? 1.0 : p->mu);
  if (!(mu >= 0.0 && mu <= 1.0)) return WL_ERR_INVALID_ARG;

  wl_handle* h = new wl_handle();
  CallScope cs__(&h->retired);
  h->n = A->n;
  h->nnz = A->nnz;
  h->variant = v;
  h->prm = *p;
  default_params(&h->prm);
  h->gram_tc = p->gram == 1;
  h->mu = mu;
  h->stream = (cudaStream_t)p->stream;
  int rc = WL_OK;
  auto fail = [&](int code) {
    free_handle(h);
    if (st) {
      memset(st, 0, sizeof(*st));
      st->status = code;
    }
    return code;
  };
  if (cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess)
    return fail(set_cuda_error(cudaGetLastError(), "cudaEventCreate"));
  if (pool_malloc_host((void**)&h->h_pin, 4096 * sizeof(double)) != cudaSuccess)
    return fail(set_cuda_error(cudaGetLastError(), "cudaMallocHost"));
  if (pool_malloc((void**)&h->bar, sizeof(GridBar)) != cudaSuccess)
    return fail(set_cuda_error(cudaGetLastError(), "cudaMalloc"));
  if ((rc = ensure(h->small, 8192)) != WL_OK) return fail(rc);
  if ((rc = ensure(h->csr_rp, sizeof(int32_t) * (A->n + 1))) != WL_OK) return fail(rc);
  if ((rc = ensure(h->csr_col, sizeof(int32_t) * std::max<int64_t>(A->nnz, 1))) != WL_OK) return fail(rc);
  begin_timer(h);
  {
    cudaError_t e1 = cudaMemcpyAsync(h->csr_rp.p, A->row_ptr, sizeof(int32_t) * (A->n + 1), cudaMemcpyDefault, S(h));
    cudaError_t e2 = A->nnz > 0 ? cudaMemcpyAsync(h->csr_col.p, A->col_idx, sizeof(int32_t) * A->nnz,
                                                  cudaMemcpyDefault, S(h))
                                : cudaSuccess;
    if (e1 != cudaSuccess || e2 != cudaSuccess)
      return fail(set_cuda_error(e1 != cudaSuccess ? e1 : e2, "copy CSR"));
  }
  h->g = Graph{(const int32_t*)h->csr_rp.p, (const int32_t*)h->csr_col.p, h->n, h->nnz};
  // validation
  Smalls sm = smalls(h);
  if (cudaMemsetAsync(sm.flags, 0, sizeof(int), S(h)) != cudaSuccess) return fail(WL_ERR_CUDA);
  if (cudaError_t e = launch_validate(h->g, sm.flags, S(h)); e != cudaSuccess) return fail(set_cuda_error(e, "validate"));
  int flags = 0;
  if (cudaMemcpyAsync(&flags, sm.flags, sizeof(int), cudaMemcpyDeviceToHost, S(h)) != cudaSuccess ||
      cudaStreamSynchronize(S(h)) != cudaSuccess)
    return fail(set_cuda_error(cudaGetLastError(), "validate readback"));
  if (flags & 3) return fail(WL_ERR_UNSORTED);
  if (flags & 4) return fail(WL_ERR_SELF_LOOP);
  if (flags & 8) return fail(WL_ERR_NOT_SYMMETRIC);

  // optional relabelling (internal only): by decreasing degree (1) or reverse
  // Cuthill-McKee (2, ordered on the host from the validated graph)
  if ((p->reorder == 1 || p->reorder == 2) && h->n > 1) {
    std::vector<int32_t> hperm;
    if (p->reorder == 2) {
      std::vector<int32_t> hrp, hcol;
      const int32_t* rp_h = A->row_ptr;
      const int32_t* col_h = A->col_idx;
      if (is_device_ptr(A->row_ptr) || (A->nnz > 0 && is_device_ptr(A->col_idx))) {
        hrp.resize((size_t)h->n + 1);
        hcol.resize((size_t)std::max<int64_t>(h->nnz, 1));
        cudaError_t e = cudaMemcpyAsync(hrp.data(), h->csr_rp.p, sizeof(int32_t) * (h->n + 1), cudaMemcpyDeviceToHost,
                                        S(h));
        if (e == cudaSuccess && h->nnz > 0)
          e = cudaMemcpyAsync(hcol.data(), h->csr_col.p, sizeof(int32_t) * h->nnz, cudaMemcpyDeviceToHost, S(h));
        if (e == cudaSuccess) e = cudaStreamSynchronize(S(h));
        if (e != cudaSuccess) return fail(set_cuda_error(e, "CSR to host for RCM"));
        rp_h = hrp.data();
        col_h = hcol.data();
      }
      hperm.resize((size_t)h->n);
      if ((rc = rcm_order(rp_h, col_h, h->n, hperm.data())) != WL_OK) return fail(rc);
    }
    Buf rp2, col2;
    if ((rc = ensure(h->perm_b, sizeof(int32_t) * h->n)) != WL_OK) return fail(rc);
    if ((rc = ensure(h->iperm_b, sizeof(int32_t) * h->n)) != WL_OK) return fail(rc);
    if ((rc = ensure(rp2, sizeof(int32_t) * (h->n + 1))) != WL_OK) return fail(rc);
    if ((rc = ensure(col2, sizeof(int32_t) * std::max<int64_t>(h->nnz, 1))) != WL_OK) {
      release(rp2);
      return fail(rc);
    }
    if ((rc = ensure(h->ptmp, sizeof(int64_t) * relabel_tmp_i64(h->n))) != WL_OK) {
      release(rp2);
      release(col2);
      return fail(rc);
    }
    h->perm = (int32_t*)h->perm_b.p;
    h->iperm = (int32_t*)h->iperm_b.p;
    cudaError_t e;
    if (p->reorder == 1) {
      counted(h, 9);
      e = launch_relabel(h->g, h->perm, h->iperm, (int32_t*)rp2.p, (int32_t*)col2.p, (int64_t*)h->ptmp.p, S(h));
    } else {
      counted(h, 7);
      e = cudaMemcpyAsync(h->perm, hperm.data(), sizeof(int32_t) * h->n, cudaMemcpyHostToDevice, S(h));
      if (e == cudaSuccess)
        e = launch_relabel_apply(h->g, h->perm, h->iperm, (int32_t*)rp2.p, (int32_t*)col2.p, (int64_t*)h->ptmp.p,
                                 S(h));
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(S(h));  // hperm stays alive until the copy is done
    if (e != cudaSuccess) {
      release(rp2);
      release(col2);
      return fail(set_cuda_error(e, "relabel"));
    }
    release(h->csr_rp);
    release(h->csr_col);
    h->csr_rp = rp2;
    h->csr_col = col2;
    h->g = Graph{(const int32_t*)h->csr_rp.p, (const int32_t*)h->csr_col.p, h->n, h->nnz};
  } else if (p->reorder < 0 || p->reorder > 2) {
    return fail(WL_ERR_INVALID_ARG);
  }

  // rows gathered by a whole CTA in the CG kernels
  if (h->n > 0) {
    if ((rc = ensure(h->hubs, sizeof(int32_t) * h->n)) != WL_OK) return fail(rc);
    if ((rc = ensure(h->ptmp, sizeof(int64_t) * std::max<size_t>(relabel_tmp_i64(h->n),
                                                                 3 * (size_t)(h->n + 1) + h->n / 1024 + 8))) != WL_OK)
      return fail(rc);
    counted(h, 5);
    cudaError_t e = launch_row_list(h->g.row_ptr, h->n, kHubDeg, INT32_MAX, (int32_t*)h->hubs.p,
                                    (int64_t*)h->ptmp.p, (int64_t*)h->h_pin, S(h));
    if (e == cudaSuccess) e = cudaStreamSynchronize(S(h));
    if (e != cudaSuccess) return fail(set_cuda_error(e, "hub list"));
    h->nhub = (int)*(int64_t*)h->h_pin;
    // rows gathered by a warp each in the spectral-scale Lanczos
    if ((rc = ensure(h->mid, sizeof(int32_t) * h->n)) != WL_OK) return fail(rc);
    counted(h, 5);
    e = launch_row_list(h->g.row_ptr, h->n, kSpWarpDeg, kHubDeg, (int32_t*)h->mid.p, (int64_t*)h->ptmp.p,
                        (int64_t*)h->h_pin, S(h));
    if (e == cudaSuccess) e = cudaStreamSynchronize(S(h));
    if (e != cudaSuccess) return fail(set_cuda_error(e, "mid-row list"));
    h->nmid = (int)*(int64_t*)h->h_pin;
    h->nmid_blk = h->nmid > 0 ? (int)std::min<int64_t>((h->nmid + 31) / 32, 2 * 152) : 0;
    // share of the S kernels' CTAs for the mid rows: a warp takes about 32
    // entries per round on either path, but a mid row pays the fixed cost of
    // a row (pointers, own-row vectors, finish: ~3 rounds) for a whole warp,
    // a short row for a lane group (1/8 of a warp at K = 16 FP32)
    h->mid_share = 0.0;
    if (h->nmid > 0) {
      unsigned long long* cnt = (unsigned long long*)h->h_pin;
      unsigned long long* dsum = (unsigned long long*)((double*)h->small.p + 900);
      double ent[2];
      const int32_t* lists[2] = {(const int32_t*)h->mid.p, (const int32_t*)h->hubs.p};
      const int64_t counts[2] = {h->nmid, h->nhub};
      for (int li = 0; li < 2; ++li) {
        e = launch_list_entries(h->g.row_ptr, lists[li], counts[li], dsum, S(h));
        if (e == cudaSuccess) e = cudaMemcpyAsync(cnt, dsum, 8, cudaMemcpyDeviceToHost, S(h));
        if (e == cudaSuccess) e = cudaStreamSynchronize(S(h));
        if (e != cudaSuccess) return fail(set_cuda_error(e, "mid-row entries"));
        ent[li] = (double)*cnt;
      }
      counted(h, 4);
      const double e_mid = ent[0], e_low = (double)h->nnz - ent[0] - ent[1];
      const double n_low = (double)(h->n - h->nhub - h->nmid);
      const double w_mid = e_mid / 32.0 + 3.0 * h->nmid, w_low = e_low / 32.0 + 0.375 * n_low;
      h->mid_share = w_mid / std::max(w_mid + w_low, 1e-300);
    }
  }

  // spectral scale and parameters
  h->lmax = 0.0;
  h->rho = 0.0;
  if (h->n > 0 && h->nnz > 0) {
    if ((rc = lambda_max_adaptive(h, t_spec_rtol > 0.0 ? t_spec_rtol : kSpecRtolDefault, &h->lmax)) != WL_OK) return fail(rc);
    if (p->f == WL_F_RESOLVENT) {
      if ((rc = rho_companion(h, mu, h->lmax, &h->rho)) != WL_OK) return fail(rc);
    } else {
      h->rho = h->lmax;
    }
  }
  if (p->f == WL_F_RESOLVENT) {
    double alpha = p->alpha;
    if (p->alpha_rel > 0) {
      if (!(h->rho > 0)) return fail(WL_ERR_ALPHA_RANGE);
      alpha = p->alpha_rel / h->rho;
    }
    if (!(alpha >= 0.0) || !std::isfinite(alpha) || alpha * h->rho >= 1.0) return fail(WL_ERR_ALPHA_RANGE);
    h->alpha = alpha;
    h->a_scale = 1.0 - mu * mu * alpha * alpha;
    h->ca = h->a_scale;
    h->cA = -alpha;
    h->cD = alpha * alpha * mu;
  } else {
    h->alpha = 0.0;
    h->a_scale = 1.0;
    h->ca = 0.0;
    h->cA = -1.0;
    h->cD = 1.0;
  }
  h->beta = 0.0;
  if (p->f == WL_F_EXP) {
    // beta <= 0: 1 / lambda_max(A) (Sec. 4.1.2), so that the series terms fall from the start
    h->beta = p->beta > 0.0 ? p->beta : (h->lmax > 0.0 ? 1.0 / h->lmax : 1.0);
    if (!std::isfinite(h->beta)) return fail(WL_ERR_INVALID_ARG);
  }
  const double ms = end_timer(h);
  if (st) {
    SolveInfo none;
    fill_stats(h, st, none, WL_OK, ms, 0);
  }
  *out = h;
  return WL_OK;
}

int wl_set_params(wl_handle* h, const wl_params* p) {
  if (!h || !p) return WL_ERR_INVALID_ARG;
  if (p->prec != WL_FP64 && p->prec != WL_REFINED && p->prec != WL_SKETCH) return WL_ERR_INVALID_ARG;
  if (p->reorth < 0 || p->reorth > 1) return WL_ERR_INVALID_ARG;
  if (p->gram < 0 || p->gram > 1) return WL_ERR_INVALID_ARG;
  if (!(p->shift >= 0.0) || !std::isfinite(p->shift)) return WL_ERR_INVALID_ARG;
  h->prm.prec = p->prec;
  h->prm.reorth = p->reorth;
  h->prm.gram = p->gram;
  h->gram_tc = p->gram == 1;
  h->prm.shift = p->shift;
  h->prm.tol = p->tol;
  h->prm.max_iter = p->max_iter;
  h->prm.max_outer = p->max_outer;
  h->prm.outer_tol = p->outer_tol;
  h->prm.stream = p->stream;
  h->stream = (cudaStream_t)p->stream;
  default_params(&h->prm);
  return WL_OK;
}

int wl_get_info(const wl_handle* h, wl_stats* info) {
  if (!h || !info) return WL_ERR_INVALID_ARG;
  memset(info, 0, sizeof(*info));
  info->alpha = h->alpha;
  info->beta = h->beta;
  info->mu = h->mu;
  info->rho = h->rho;
  info->lambda_max = h->lmax;
  return WL_OK;
}

int wl_set_warm_start(wl_handle* h, const double* x0) {
  CallScope cs__(h ? &h->retired : nullptr);
  if (!h) return WL_ERR_INVALID_ARG;
  if (!x0) {
    h->have_warm = false;
    return WL_OK;
  }
  int rc = ensure(h->warm, (size_t)std::max<int64_t>(h->n, 1) * 8);
  if (rc) return rc;
  if (h->perm) {
    const void* src = nullptr;
    rc = stage_in(h, h->stage_a, x0, (size_t)h->n * 8, &src);
    if (rc) return rc;
    counted(h);
    WL_CU(launch_permute_vec((const double*)src, h->n, h->perm, false, (double*)h->warm.p, S(h)));
  } else {
    WL_CU(cudaMemcpyAsync(h->warm.p, x0, (size_t)h->n * 8, cudaMemcpyDefault, S(h)));
  }
  WL_CU(cudaStreamSynchronize(S(h)));
  h->have_warm = true;
  h->have_Df = false;
  h->have_dfdf = false;
  return WL_OK;
}

// Node features of the warm-start network and the analytic guess x_an,
// in the caller's node order.
int wl_mlp_features(wl_handle* h, float* feats, double* xan, wl_stats* st) {
  NvtxRange nvtx__("wl_mlp_features");
  CallScope cs__(h ? &h->retired : nullptr);
  if (st) memset(st, 0, sizeof(*st));
  if (!h || (!feats && !xan)) return WL_ERR_INVALID_ARG;
  if (h->prm.f != WL_F_RESOLVENT) return WL_ERR_UNSUPPORTED;
  if (h->n == 0) return WL_OK;
  begin_timer(h);
  const size_t n = (size_t)h->n;
  WL_TRY(ensure(h->ptmp, std::max(h->ptmp.bytes, features_tmp_bytes(h->n, h->nnz))));
  float* F = feats;
  double* X = xan;
  const bool fdev = !feats || is_device_ptr(feats), xdev = !xan || is_device_ptr(xan);
  if (!fdev || !xdev) {
    WL_TRY(ensure(h->stage_b, n * 4 * sizeof(float) + n * 8));
    if (!fdev) F = (float*)h->stage_b.p;
    if (!xdev) X = (double*)((char*)h->stage_b.p + n * 4 * sizeof(float));
  }
  counted(h, 8);
  WL_CU(launch_features(h->g.row_ptr, h->g.col, h->n, h->nnz, h->alpha, h->mu, h->perm, h->perm, F, X, h->ptmp.p,
                        S(h)));
  if (!fdev) WL_CU(cudaMemcpyAsync(feats, F, n * 4 * sizeof(float), cudaMemcpyDeviceToHost, S(h)));
  if (!xdev) WL_CU(cudaMemcpyAsync(xan, X, n * 8, cudaMemcpyDeviceToHost, S(h)));
  const double ms = end_timer(h);
  if (st) {
    st->time_ms = ms;
    st->launches = h->launches;
  }
  prof_reset(h);
  return WL_OK;
}

// Warm start of the walk-degree solve from the network: features, x_an and
// x0 = x_an * exp(y) on the device, kept as the handle's starting guess.
int wl_mlp_warm_start(wl_handle* h, const float* params, wl_stats* st) {
  NvtxRange nvtx__("wl_mlp_warm_start");
  CallScope cs__(h ? &h->retired : nullptr);
  if (st) memset(st, 0, sizeof(*st));
  if (!h || !params) return WL_ERR_INVALID_ARG;
  if (h->prm.f != WL_F_RESOLVENT) return WL_ERR_UNSUPPORTED;
  if (h->n == 0) return WL_OK;
  begin_timer(h);
  const size_t n = (size_t)h->n;
  const int np = wl_mlp_param_count();
  WL_TRY(ensure(h->ptmp, std::max(h->ptmp.bytes, features_tmp_bytes(h->n, h->nnz))));
  WL_TRY(ensure(h->stage_b, n * 4 * sizeof(float) + n * 8 + (size_t)np * sizeof(float) + 256));
  WL_TRY(ensure(h->warm, std::max<size_t>(n, 1) * 8));
  float* F = (float*)h->stage_b.p;
  double* X = (double*)((char*)h->stage_b.p + n * 4 * sizeof(float));
  float* P = (float*)((char*)X + n * 8);
  WL_CU(cudaMemcpyAsync(P, params, (size_t)np * sizeof(float), cudaMemcpyDefault, S(h)));
  counted(h, 9);
  WL_CU(launch_features(h->g.row_ptr, h->g.col, h->n, h->nnz, h->alpha, h->mu, nullptr, h->perm, F, X, h->ptmp.p,
                        S(h)));
  WL_CU(launch_mlp_predict(P, F, h->n, X, (double*)h->warm.p, S(h)));
  const double ms = end_timer(h);
  h->have_warm = true;
  h->have_Df = false;
  h->have_dfdf = false;
  if (st) {
    st->time_ms = ms;
    st->launches = h->launches;
  }
  prof_reset(h);
  return WL_OK;
}

int wl_degrees(wl_handle* h, double* Df, wl_stats* st) {
  NvtxRange nvtx__("wl_degrees");
  CallScope cs__(h ? &h->retired : nullptr);
  if (!h || (!Df && h->n > 0)) return WL_ERR_INVALID_ARG;
  SolveInfo info;
  begin_timer(h);
  int rc = WL_OK;
  if (h->n > 0) {
    h->have_Df = false;
  h->have_dfdf = false;
    rc = compute_Df(h, info);
    if (rc == WL_OK) rc = copy_out_vec(h, (const double*)h->Df.p, Df);
  }
  const double ms = end_timer(h);
  if (rc == WL_OK) rc = info.status;
  fill_stats(h, st, info, rc, ms, 0);
  return rc;
}

int wl_apply(wl_handle* h, const double* V, int64_t ldv, int k, double* W, int64_t ldw, wl_stats* st) {
  NvtxRange nvtx__("wl_apply");
  CallScope cs__(h ? &h->retired : nullptr);
  if (!h || k < 0 || (k > 0 && h->n > 0 && (!V || !W || ldv < k || ldw < k))) return WL_ERR_INVALID_ARG;
  SolveInfo info;
  begin_timer(h);
  int rc = WL_OK;
  if (k == 0 || h->n == 0) {
    fill_stats(h, st, info, WL_OK, end_timer(h), 0);
    return WL_OK;
  }
  const int64_t n = h->n;
  const bool w_dev = is_device_ptr(W);
  const double* Vd = nullptr;
  double* Wd = W;
  do {
    if (!h->have_Df && (rc = compute_Df(h, info)) != WL_OK) break;
    if ((rc = stage_in(h, h->stage_a, V, (size_t)n * ldv * 8, (const void**)&Vd)) != WL_OK) break;
    if (!w_dev) {
      if ((rc = ensure(h->stage_b, (size_t)n * ldw * 8)) != WL_OK) break;
      Wd = (double*)h->stage_b.p;
      if (ldw != k) cudaMemcpyAsync(Wd, W, (size_t)n * ldw * 8, cudaMemcpyHostToDevice, S(h));
    }
    int c0 = 0;
    for (int K : column_blocks(k)) {
      if ((rc = ensure(h->packV, (size_t)n * K * 8)) != WL_OK) break;
      if ((rc = ensure(h->packX, (size_t)n * K * 8)) != WL_OK) break;
      counted(h);
      cudaError_t e = h->perm ? launch_pack_perm(Vd, ldv, c0, K, n, 1.0, h->perm, (double*)h->packV.p, S(h))
                              : launch_pack(Vd, ldv, c0, K, n, 1.0, h->packV.p, false, S(h));
      if (e != cudaSuccess) { rc = set_cuda_error(e, "pack"); break; }
      if (h->prm.f == WL_F_IDENTITY) {
        PartDev* pd;
        int Tw, Tc;
        thresholds_f64(K, &Tw, &Tc);
        if ((rc = get_part(h, lanczos_step_grid(K), Tw, Tc, &pd, K, 8)) != WL_OK) break;
        counted(h);
        e = launch_laplacian_apply(h->g, *pd, (const double*)h->packV.p, K, c0, h->perm, Wd, ldw, S(h));
        info.nnz_rhs += (double)h->nnz * K;
        info.iters += 1;
      } else {
        if ((rc = phi_apply(h, (const double*)h->packV.p, (double*)h->packX.p, K, info)) != WL_OK) break;
        counted(h);
        e = h->perm ? launch_apply_out_perm((const double*)h->packV.p, (const double*)h->packX.p,
                                            (const double*)h->Df.p, n, K, c0, h->perm, Wd, ldw, S(h))
                    : launch_apply_out(Vd, ldv, (const double*)h->packX.p, (const double*)h->Df.p, n, K, c0, Wd,
                                       ldw, S(h));
      }
      if (e != cudaSuccess) { rc = set_cuda_error(e, "apply"); break; }
      c0 += K;
    }
    if (rc != WL_OK) break;
    if (!w_dev) {
      cudaError_t e = cudaMemcpyAsync(W, Wd, (size_t)n * ldw * 8, cudaMemcpyDeviceToHost, S(h));
      if (e != cudaSuccess) { rc = set_cuda_error(e, "copy W"); break; }
    }
  } while (0);
  const double ms = end_timer(h);
  if (rc == WL_OK) rc = info.status;
  fill_stats(h, st, info, rc, ms, 0);
  return rc;
}

int wl_expmv(wl_handle* h, const double* U0, int64_t ldu, int k, const double* taus, int ntau, double* U,
             int64_t ldo, wl_stats* st) {
  NvtxRange nvtx__("wl_expmv");
  CallScope cs__(h ? &h->retired : nullptr);
  if (!h || k < 0 || ntau < 0 || ntau > kMaxTau) return WL_ERR_INVALID_ARG;
  if (k > 0 && h->n > 0 && (!U0 || !U || !taus || ldu < k || ldo < k)) return WL_ERR_INVALID_ARG;
  for (int t = 0; t < ntau; ++t)
    if (!(taus[t] >= 0.0) || !std::isfinite(taus[t])) return WL_ERR_INVALID_ARG;
  SolveInfo info;
  begin_timer(h);
  if (k == 0 || ntau == 0 || h->n == 0) {
    fill_stats(h, st, info, WL_OK, end_timer(h), 0);
    return WL_OK;
  }
  const int64_t n = h->n;
  int rc = WL_OK;
  int outer_total = 0;
  const bool u_dev = is_device_ptr(U);
  const double* U0d = nullptr;
  double* Ud = U;
  do {
    if ((rc = stage_in(h, h->stage_a, U0, (size_t)n * ldu * 8, (const void**)&U0d)) != WL_OK) break;
    if (!u_dev) {
      if ((rc = ensure(h->stage_b, (size_t)ntau * n * ldo * 8)) != WL_OK) break;
      Ud = (double*)h->stage_b.p;
      if (ldo != k) cudaMemcpyAsync(Ud, U, (size_t)ntau * n * ldo * 8, cudaMemcpyHostToDevice, S(h));
    }
    const double* dtaus = nullptr;
    if ((rc = stage_taus(h, taus, ntau, &dtaus)) != WL_OK) break;
    int c0 = 0;
    bool capped = false;  // a column block reached max_outer: every block is still evaluated
    for (int K : column_blocks(k)) {
      if ((rc = ensure(h->packX, (size_t)n * K * 8)) != WL_OK) break;
      counted(h);
      cudaError_t e = h->perm ? launch_pack_perm(U0d, ldu, c0, K, n, 1.0, h->perm, (double*)h->packX.p, S(h))
                              : launch_pack(U0d, ldu, c0, K, n, 1.0, h->packX.p, false, S(h));
      if (e != cudaSuccess) { rc = set_cuda_error(e, "expmv pack"); break; }
      OuterRun o;
      if ((rc = outer_run(h, K, dtaus, ntau, info, o, outer_total)) != WL_OK) break;
      if (info.status != WL_OK) break;
      if ((rc = outer_combine(h, o, 0, ntau, Ud, ldo, n * ldo, c0, h->perm)) != WL_OK) break;
      if (!o.converged) capped = true;
      c0 += K;
    }
    if (rc != WL_OK) break;
    if (capped && info.status == WL_OK) info.status = WL_ERR_NO_CONVERGENCE;
    if (!u_dev) {
      cudaError_t e = cudaMemcpyAsync(U, Ud, (size_t)ntau * n * ldo * 8, cudaMemcpyDeviceToHost, S(h));
      if (e != cudaSuccess) { rc = set_cuda_error(e, "copy U"); break; }
    }
  } while (0);
  const double ms = end_timer(h);
  if (rc == WL_OK) rc = info.status;
  fill_stats(h, st, info, rc, ms, outer_total);
  return rc;
}

int wl_markov(wl_handle* h, const double* P0, int64_t ldp, int k, const int* steps, int nsteps, double* out,
              int64_t ldo, wl_stats* st) {
  NvtxRange nvtx__("wl_markov");
  CallScope cs__(h ? &h->retired : nullptr);
  if (!h || k < 0 || nsteps < 1 || nsteps > 64 || !steps) return WL_ERR_INVALID_ARG;
  if (k > 0 && h->n > 0 && (!P0 || !out || ldp < k || ldo < k)) return WL_ERR_INVALID_ARG;
  for (int t = 0; t < nsteps; ++t)
    if (steps[t] < 0 || (t > 0 && steps[t] < steps[t - 1])) return WL_ERR_INVALID_ARG;
  SolveInfo info;
  begin_timer(h);
  if (k == 0 || h->n == 0) {
    fill_stats(h, st, info, WL_OK, end_timer(h), 0);
    return WL_OK;
  }
  const int64_t n = h->n;
  int rc = WL_OK;
  const bool o_dev = is_device_ptr(out);
  const double* P0d = nullptr;
  double* Od = out;
  int nstep = 0;  // chain steps of the last column block
  do {
    if (!h->have_Df && (rc = compute_Df(h, info)) != WL_OK) break;
    if ((rc = stage_in(h, h->stage_a, P0, (size_t)n * ldp * 8, (const void**)&P0d)) != WL_OK) break;
    if (!o_dev) {
      if ((rc = ensure(h->stage_b, (size_t)nsteps * n * ldo * 8)) != WL_OK) break;
      Od = (double*)h->stage_b.p;
      if (ldo != k) cudaMemcpyAsync(Od, out, (size_t)nsteps * n * ldo * 8, cudaMemcpyHostToDevice, S(h));
    }
    int c0 = 0;
    for (int K : column_blocks(k)) {
      if ((rc = ensure(h->packV, (size_t)n * K * 8)) != WL_OK) break;
      if ((rc = ensure(h->packX, (size_t)n * K * 8)) != WL_OK) break;
      double* cur = (double*)h->packX.p;  // p_s of this block (internal node order)
      double* y = (double*)h->packV.p;    // p_s / D_f
      counted(h);
      cudaError_t e = h->perm ? launch_pack_perm(P0d, ldp, c0, K, n, 1.0, h->perm, cur, S(h))
                              : launch_pack(P0d, ldp, c0, K, n, 1.0, cur, false, S(h));
      if (e != cudaSuccess) { rc = set_cuda_error(e, "markov pack"); break; }
      int s = 0;
      nstep = 0;
      for (int t = 0; t < nsteps && rc == WL_OK; ++t) {
        for (; s < steps[t]; ++s) {
          counted(h);
          if ((e = launch_row_div(cur, (const double*)h->Df.p, n, K, y, S(h))) != cudaSuccess) {
            rc = set_cuda_error(e, "markov scale");
            break;
          }
          if (h->prm.f == WL_F_IDENTITY) {
            counted(h);
            if ((e = launch_adj_apply(h->g, y, K, cur, S(h))) != cudaSuccess) {
              rc = set_cuda_error(e, "markov step");
              break;
            }
            info.nnz_rhs += (double)h->nnz * K;
            info.iters += 1;
          } else {
            if ((rc = phi_apply(h, y, cur, K, info)) != WL_OK) break;
            if (info.status != WL_OK) break;
          }
          ++nstep;
        }
        if (rc != WL_OK || info.status != WL_OK) break;
        counted(h);
        e = launch_unpack(cur, n, K, c0, h->perm, Od + (size_t)t * n * ldo, ldo, S(h));
        if (e != cudaSuccess) { rc = set_cuda_error(e, "markov out"); break; }
      }
      if (rc != WL_OK || info.status != WL_OK) break;
      c0 += K;
    }
    if (rc != WL_OK) break;
    if (!o_dev) {
      cudaError_t e = cudaMemcpyAsync(out, Od, (size_t)nsteps * n * ldo * 8, cudaMemcpyDeviceToHost, S(h));
      if (e != cudaSuccess) { rc = set_cuda_error(e, "copy out"); break; }
    }
  } while (0);
  const double ms = end_timer(h);
  if (rc == WL_OK) rc = info.status;
  fill_stats(h, st, info, rc, ms, nstep);
  return rc;
}

int wl_trace(wl_handle* h, int M, uint64_t seed, double* est, double* err_est, uint16_t* omega_out, wl_stats* st) {
  NvtxRange nvtx__("wl_trace");
  CallScope cs__(h ? &h->retired : nullptr);
  if (!h || !est || !err_est || M < 2 || M > kMaxSketch) return WL_ERR_INVALID_ARG;
  if (h->prm.f != WL_F_RESOLVENT) return WL_ERR_UNSUPPORTED;
  SolveInfo info;
  begin_timer(h);
  *est = 0.0;
  *err_est = 0.0;
  if (h->n == 0) {
    fill_stats(h, st, info, WL_OK, end_timer(h), 0);
    return WL_OK;
  }
  const int64_t n = h->n;
  int K = 1;
  while (K < M) K <<= 1;
  int rc = WL_OK;
  do {
    const size_t nk = (size_t)n * K;
    if ((rc = ensure(h->omega, (size_t)n * M * sizeof(uint16_t))) != WL_OK) break;
    if ((rc = ensure(h->x, nk * 4)) != WL_OK) break;      // Y (FP32)
    if ((rc = ensure(h->r32, nk * 4)) != WL_OK) break;    // right-hand side / residual
    if ((rc = ensure(h->p, nk * 4)) != WL_OK) break;
    if ((rc = ensure(h->q, nk * 4)) != WL_OK) break;
    const int Gg = gram_grid(n);
    if ((rc = ensure(h->gram, (size_t)Gg * 2 * kMaxSketch * kMaxSketch * 4 + 2 * kMaxSketch * kMaxSketch * 8 +
                                 128 * 8)) != WL_OK) break;
    uint16_t* omega = (uint16_t*)h->omega.p;
    float* partial = (float*)h->gram.p;
    double* gout = (double*)((char*)h->gram.p + (size_t)Gg * 2 * kMaxSketch * kMaxSketch * 4);
    double* core = gout + 2 * kMaxSketch * kMaxSketch;
    counted(h, 2);
    cudaError_t e = launch_philox_sketch(omega, n, M, seed, S(h));
    uint16_t* om_int = omega;  // sketch rows in the internal node order
    if (e == cudaSuccess && h->perm) {
      if ((rc = ensure(h->omega_int, (size_t)n * M * sizeof(uint16_t))) != WL_OK) break;
      om_int = (uint16_t*)h->omega_int.p;
      counted(h);
      e = launch_permute_rows_u16(omega, n, M, h->perm, om_int, S(h));
    }
    if (h->prm.prec != WL_SKETCH) {
      // Y = phi Omega by the solve of the handle's form (FP64 n x K), Gram in FP64
      if (e == cudaSuccess && (rc = ensure(h->packV, nk * 8)) != WL_OK) break;
      if (e == cudaSuccess && (rc = ensure(h->packX, nk * 8)) != WL_OK) break;
      if (e == cudaSuccess && (rc = ensure(h->gram, (size_t)Gg * 2 * kMaxSketch * kMaxSketch * 8 +
                                                     2 * kMaxSketch * kMaxSketch * 8 + 128 * 8)) != WL_OK) break;
      counted(h);
      if (e == cudaSuccess) e = launch_sketch_block_f64(om_int, n, M, K, (double*)h->packV.p, S(h));
      if (e != cudaSuccess) { rc = set_cuda_error(e, "sketch"); break; }
      if ((rc = phi_apply(h, (const double*)h->packV.p, (double*)h->packX.p, K, info)) != WL_OK) break;
      if (info.status != WL_OK) break;
      double* part64 = (double*)h->gram.p;
      gout = part64 + (size_t)Gg * 2 * kMaxSketch * kMaxSketch;
      core = gout + 2 * kMaxSketch * kMaxSketch;
      counted(h, 3);
      e = launch_gram_f64(om_int, (const double*)h->packX.p, n, M, K, part64, Gg, gout, S(h));
      if (e == cudaSuccess) e = launch_nys_core(gout, M, core, S(h));
      if (e != cudaSuccess) { rc = set_cuda_error(e, "gram/core"); break; }
      double* hp = h->h_pin;
      WL_CU(cudaMemcpyAsync(hp, core, 8 * 8, cudaMemcpyDeviceToHost, S(h)));
      WL_CU(cudaStreamSynchronize(S(h)));
      if (hp[2] != 0.0) { rc = WL_ERR_NOT_SPD; break; }
      *est = hp[0];
      *err_est = hp[1];
      if (omega_out) {
        e = cudaMemcpyAsync(omega_out, omega, (size_t)n * M * sizeof(uint16_t), cudaMemcpyDefault, S(h));
        if (e != cudaSuccess) { rc = set_cuda_error(e, "copy omega"); break; }
      }
      break;
    }
    if (e == cudaSuccess) e = launch_sketch_rhs(om_int, n, M, K, h->a_scale, (float*)h->r32.p, S(h));
    if (e == cudaSuccess) e = cudaMemsetAsync(h->x.p, 0, nk * 4, S(h));
    if (e != cudaSuccess) { rc = set_cuda_error(e, "sketch"); break; }
    // Y = M^{-1} (a Omega) in FP32 lockstep CG
    const int grid_u = phase_blocks_f32(K), grid_s = grid_u + h->nhub;
    if ((rc = ensure_phase_buffers(h, grid_s)) != WL_OK) break;
    Smalls sm = smalls(h);
    CgState* st = h->cgst();
    WL_CU(cudaMemsetAsync(st, 0, sizeof(CgState), S(h)));
    const double tol = std::max(h->prm.tol, 1e-7);
    PhaseArgs<float> a{phase_graph_mid(h, grid_u), (float*)h->x.p, (float*)h->r32.p, (float*)h->p.p,
                       (float*)h->q.p, h->ca, h->cA, h->cD, nullptr, nullptr, (double*)h->part.p, st,
                       h->prm.max_iter, tol * tol};
    if ((rc = run_cg<float>(h, K, a, grid_s, grid_u, info, 4)) != WL_OK) break;
    (void)sm;
    counted(h, 3);
    int* gerr = (int*)((double*)h->small.p + 1000);
    e = cudaMemsetAsync(gerr, 0, sizeof(int), S(h));
    if (e == cudaSuccess) e = launch_gram(om_int, (const float*)h->x.p, n, M, K, partial, Gg, gout, h->gram_tc, gerr, S(h));
    if (e == cudaSuccess) e = launch_nys_core(gout, M, core, S(h));
    if (e != cudaSuccess) { rc = set_cuda_error(e, "gram/core"); break; }
    double* hp = h->h_pin;
    WL_CU(cudaMemcpyAsync(hp, core, 8 * 8, cudaMemcpyDeviceToHost, S(h)));
    WL_CU(cudaStreamSynchronize(S(h)));
    if (h->gram_tc) {
      int herr = 0;
      WL_CU(cudaMemcpy(&herr, gerr, sizeof(int), cudaMemcpyDeviceToHost));
      if (herr != 0) { rc = herr; break; }
    }
    if (hp[2] != 0.0) { rc = WL_ERR_NOT_SPD; break; }
    *est = hp[0];
    *err_est = hp[1];
    if (omega_out) {
      e = cudaMemcpyAsync(omega_out, omega, (size_t)n * M * sizeof(uint16_t), cudaMemcpyDefault, S(h));
      if (e != cudaSuccess) { rc = set_cuda_error(e, "copy omega"); break; }
    }
  } while (0);
  const double ms = end_timer(h);
  if (rc == WL_OK) rc = info.status;
  fill_stats(h, st, info, rc, ms, 0);
  return rc;
}

int wl_return_prob(wl_handle* h, int M, uint64_t seed, const double* ts, int nt, double* p_est, double* p_err,
                   wl_stats* st) {
  NvtxRange nvtx__("wl_return_prob");
  CallScope cs__(h ? &h->retired : nullptr);
  if (!h || !ts || !p_est || !p_err || M < 2 || M > kMaxSketch || nt < 1 || nt > kMaxReturnT) return WL_ERR_INVALID_ARG;
  for (int t = 0; t < nt; ++t)
    if (!(ts[t] >= 0.0) || !std::isfinite(ts[t])) return WL_ERR_INVALID_ARG;
  SolveInfo info;
  begin_timer(h);
  for (int t = 0; t < nt; ++t) p_est[t] = p_err[t] = 0.0;
  if (h->n == 0) {
    fill_stats(h, st, info, WL_OK, end_timer(h), 0);
    return WL_OK;
  }
  const int64_t n = h->n;
  int K = 1;
  while (K < M) K <<= 1;
  int rc = WL_OK;
  int outer_total = 0;
  do {
    const size_t nk = (size_t)n * K;
    if ((rc = ensure(h->omega, (size_t)n * M * sizeof(uint16_t))) != WL_OK) break;
    if ((rc = ensure(h->x, nk * 4)) != WL_OK) break;      // Y(t) in FP32 for the Gram
    if ((rc = ensure(h->packX, nk * 8)) != WL_OK) break;  // Omega as the FP64 start block
    if ((rc = ensure(h->ybig, (size_t)kMaxTau * nk * 8)) != WL_OK) break;
    const int Gg = gram_grid(n);
    const bool sketch = h->prm.prec == WL_SKETCH;  // FP32 Gram on the tensor cores; else FP64
    const size_t pbytes = (size_t)Gg * 2 * kMaxSketch * kMaxSketch * (sketch ? 4 : 8);
    if ((rc = ensure(h->gram, pbytes + 2 * kMaxSketch * kMaxSketch * 8 + 128 * 8)) != WL_OK) break;
    uint16_t* omega = (uint16_t*)h->omega.p;
    float* partial = (float*)h->gram.p;
    double* gout = (double*)((char*)h->gram.p + pbytes);
    double* core = gout + 2 * kMaxSketch * kMaxSketch;
    counted(h, 2);
    cudaError_t e = launch_philox_sketch(omega, n, M, seed, S(h));
    uint16_t* om_int = omega;  // sketch rows in the internal node order
    if (e == cudaSuccess && h->perm) {
      if ((rc = ensure(h->omega_int, (size_t)n * M * sizeof(uint16_t))) != WL_OK) break;
      om_int = (uint16_t*)h->omega_int.p;
      counted(h);
      e = launch_permute_rows_u16(omega, n, M, h->perm, om_int, S(h));
    }
    if (e == cudaSuccess) e = launch_sketch_block_f64(om_int, n, M, K, (double*)h->packX.p, S(h));
    if (e != cudaSuccess) { rc = set_cuda_error(e, "sketch"); break; }
    const double* dtaus = nullptr;
    if ((rc = stage_taus(h, ts, nt, &dtaus)) != WL_OK) break;
    // Y(t) = exp(-t L) Omega for every t from one Lanczos run per column
    OuterRun o;
    if ((rc = outer_run(h, K, dtaus, nt, info, o, outer_total)) != WL_OK) break;
    if (info.status != WL_OK) break;
    if (!o.converged) info.status = WL_ERR_NO_CONVERGENCE;
    int* gerr = (int*)((double*)h->small.p + 1000);
    double* hp = h->h_pin;
    double* Y = (double*)h->ybig.p;
    for (int t0 = 0; t0 < nt && rc == WL_OK; t0 += kMaxTau) {
      const int nb = std::min(kMaxTau, nt - t0);
      if ((rc = outer_combine(h, o, t0, nb, Y, K, (int64_t)nk, 0, nullptr)) != WL_OK) break;
      for (int i = 0; i < nb; ++i) {
        // XNysTrace of exp(-t L) from Y(t) and Omega (Alg. 1, last step)
        counted(h, 3);
        e = cudaMemsetAsync(gerr, 0, sizeof(int), S(h));
        if (!sketch) {
          if (e == cudaSuccess)
            e = launch_gram_f64(om_int, Y + (size_t)i * nk, n, M, K, (double*)h->gram.p, Gg, gout, S(h));
        } else {
          if (e == cudaSuccess) e = launch_to_f32(Y + (size_t)i * nk, (int64_t)nk, (float*)h->x.p, S(h));
          if (e == cudaSuccess)
            e = launch_gram(om_int, (const float*)h->x.p, n, M, K, partial, Gg, gout, h->gram_tc, gerr, S(h));
        }
        if (e == cudaSuccess) e = launch_nys_core(gout, M, core, S(h));
        if (e != cudaSuccess) { rc = set_cuda_error(e, "return probability gram/core"); break; }
        WL_CU(cudaMemcpyAsync(hp, core, 8 * 8, cudaMemcpyDeviceToHost, S(h)));
        WL_CU(cudaMemcpyAsync(hp + 8, gerr, sizeof(int), cudaMemcpyDeviceToHost, S(h)));
        WL_CU(cudaStreamSynchronize(S(h)));
        if (sketch && h->gram_tc && *(int*)(hp + 8) != 0) { rc = *(int*)(hp + 8); break; }
        if (hp[2] != 0.0 && info.status == WL_OK) info.status = WL_ERR_NOT_SPD;
        p_est[t0 + i] = hp[0] / (double)n;
        p_err[t0 + i] = hp[1] / (double)n;
      }
    }
  } while (0);
  const double ms = end_timer(h);
  if (rc == WL_OK) rc = info.status;
  fill_stats(h, st, info, rc, ms, outer_total);
  return rc;
}

void wl_destroy(wl_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  free_handle(h);
}

int wl_selftest_bounded_wait(int missing, void* stream) {
  if (missing < 0 || missing > 1024) return WL_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  GridBar* bar = nullptr;
  if (cudaMalloc(&bar, sizeof(GridBar)) != cudaSuccess) {
    (void)cudaGetLastError();
    return WL_ERR_OOM;
  }
  int err = 0;
  cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(GridBar), s);
  if (e == cudaSuccess) e = launch_selftest_wait(bar, 1u + (unsigned)missing, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&err, &bar->err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(bar);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return WL_ERR_CUDA;
  }
  return err != 0 ? err : WL_OK;
}

}  // extern "C"

namespace wl {

int report_cuda_error(cudaError_t e, const char* where) { return set_cuda_error(e, where); }
void report_error(const std::string& msg) { g_last_error = msg; }
std::string last_error_copy() { return g_last_error; }

namespace {
// A second search context on the graph of h, for a search that runs beside
// others: it borrows h's graph, row lists and stream and owns its Lanczos
// basis and state, which start as copies of h's (so its first run starts
// from h's last Ritz vector).
int sp_clone(wl_handle* h, wl_handle** out) {
  wl_handle* c = new wl_handle();
  c->n = h->n;
  c->nnz = h->nnz;
  c->variant = h->variant;
  c->prm = h->prm;
  c->stream = h->stream;
  c->g = h->g;
  c->hubs = h->hubs;  // borrowed: cleared before the clone is freed
  c->mid = h->mid;
  c->nhub = h->nhub;
  c->nmid = h->nmid;
  c->nmid_blk = h->nmid_blk;
  c->lmax = h->lmax;
  c->sp_c0 = h->sp_c0;
  c->sp_cD = h->sp_cD;
  c->sp_theta = h->sp_theta;
  c->sp_ritz_ready = h->sp_ritz_ready;
  c->sp_ritz_uu = h->sp_ritz_uu;
  c->sp_ritz_udu = h->sp_ritz_udu;
  auto fail = [&](int rc) {
    c->hubs = Buf{};
    c->mid = Buf{};
    free_handle(c);
    return rc;
  };
  // no pinned staging: a context's runs go through the batch, which reads
  // the states back itself
  int rc = sp_buffers(c, sp_grid(c) + c->nhub + c->nmid_blk);
  if (rc != WL_OK) return fail(rc);
  cudaError_t e = cudaMemcpyAsync(c->spW.p, h->spW.p, (size_t)2 * h->n * 8, cudaMemcpyDeviceToDevice, S(h));
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->spstate.p, h->spstate.p, sizeof(SpState), cudaMemcpyDeviceToDevice, S(h));
  if (e == cudaSuccess) e = cudaStreamSynchronize(S(h));
  if (e != cudaSuccess) return fail(set_cuda_error(e, "search context copy"));
  *out = c;
  return WL_OK;
}

void sp_clone_free(wl_handle* c) {
  if (!c) return;
  c->hubs = Buf{};
  c->mid = Buf{};
  free_handle(c);
}
}  // namespace

// Spectral scale of one graph for several mu values (Sec. 4.1): validates
// the CSR as wl_build does, then lambda_max(A) and rho(Z_mu) for each mu
// (rho(Z_0) = lambda_max(A)). Inside a batched build (the calling thread
// bound to an SpBatch) the searches of the mu values > 0 run side by side,
// each on its own thread and search context started from the Ritz vector of
// the lambda_max(A) run, so that the batch's rounds advance them together;
// elsewhere they run one after another, each from the previous one's Ritz
// vector.
int graph_spectral(const wl_csr* A, const double* mus, int nmu, void* stream, double* lmax, double* rho,
                   double rtol) {
  struct RtolScope {
    double old;
    explicit RtolScope(double r) : old(t_spec_rtol) { t_spec_rtol = r; }
    ~RtolScope() { t_spec_rtol = old; }
  } rs(rtol);
  for (int i = 0; i < nmu; ++i)
    if (!(mus[i] >= 0.0 && mus[i] <= 1.0)) return WL_ERR_INVALID_ARG;
  wl_params p;
  memset(&p, 0, sizeof(p));
  p.f = WL_F_IDENTITY;
  p.prec = WL_FP64;
  p.stream = stream;
  p.reorder = 0;  // the searches need no node relabelling
  wl_handle* h = nullptr;
  int rc = wl_build(A, WL_ALLWALK, &p, &h, nullptr);
  if (rc != WL_OK) return rc;
  *lmax = h->lmax;
  std::vector<int> todo;
  for (int i = 0; i < nmu; ++i) {
    if (h->n == 0 || h->nnz == 0 || mus[i] == 0.0)
      rho[i] = (h->n == 0 || h->nnz == 0) ? 0.0 : h->lmax;
    else
      todo.push_back(i);
  }
  SpBatch* bt = sp_batch_current();
  if (!bt || todo.size() <= 1) {
    for (int i : todo) {
      rc = rho_companion(h, mus[i], h->lmax, &rho[i]);
      if (rc != WL_OK) break;
    }
    wl_destroy(h);
    return rc;
  }
  // the Ritz vector of the lambda_max(A) run, then one context per search
  // (the first search runs on h itself, the others on copies made first)
  double q = 0.0, uAu = 0.0;
  rc = sp_ritz_q(h, &q, &uAu);
  std::vector<wl_handle*> ctx(todo.size(), nullptr);
  ctx[0] = h;
  for (size_t k = 1; k < todo.size() && rc == WL_OK; ++k) rc = sp_clone(h, &ctx[k]);
  if (rc != WL_OK) {
    for (size_t k = 1; k < ctx.size(); ++k) sp_clone_free(ctx[k]);
    wl_destroy(h);
    return rc;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  std::vector<int> rcs(todo.size(), WL_OK);
  std::vector<std::string> msgs(todo.size());
  sp_batch_join(bt, (int)todo.size());  // the searches join before this thread leaves
  std::vector<std::thread> th;
  for (size_t k = 0; k < todo.size(); ++k)
    th.emplace_back([&, k]() {
      struct Leave {
        SpBatch* b;
        ~Leave() {
          sp_batch_bind(nullptr);
          sp_batch_leave(b);
        }
      } leave{bt};
      cudaSetDevice(dev);
      sp_batch_bind(bt);
      RtolScope r2(rtol);
      rcs[k] = rho_companion(ctx[k], mus[todo[k]], h->lmax, &rho[todo[k]]);
      if (rcs[k] != WL_OK) msgs[k] = last_error_copy();
    });
  sp_batch_leave(bt);  // this thread submits nothing while it waits
  for (auto& x : th) x.join();
  sp_batch_join(bt, 1);
  for (size_t k = 0; k < todo.size(); ++k) {
    if (rc == WL_OK && rcs[k] != WL_OK) {
      rc = rcs[k];
      report_error(msgs[k]);
    }
    if (k > 0) sp_clone_free(ctx[k]);
  }
  wl_destroy(h);
  return rc;
}

}  // namespace wl
