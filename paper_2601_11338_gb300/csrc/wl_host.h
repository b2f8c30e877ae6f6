// Host-side launchers shared by the translation units of libwl.so.
// Every kernel is launched from the translation unit that defines it; the
// API code in wl_api.cu reaches them through these declarations.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <nvtx3/nvToolsExt.h>

#include <string>

#include "wl_cg2.cuh"
#include "wl_common.cuh"
#include "wl_lanczos.cuh"
#include "wl_expdf.cuh"
#include "wl_res.cuh"
#include "wl_exps.cuh"
#include "wl_spec.cuh"
#include "wl_reorth.cuh"

namespace wl {

// An NVTX range for the lifetime of a scope: API calls and solver phases show
// up by name on a profiler timeline (a no-op when no tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

struct PartDev {
  int G = 0;
  int Tw = 0, Tc = 0;
  int row_bytes = 0, entry_bytes = 0;  // partition cost model (bytes per row / per entry)
  int32_t* rb = nullptr;
  int32_t* seg = nullptr;
  int4* meta = nullptr;
  Part view() const { return Part{rb, seg, meta}; }
};

// ---- wl_k_misc.cu
// rb/seg/order for G CTAs with class thresholds Tw, Tc (arrays allocated by caller)
cudaError_t launch_partition(const Graph& g, PartDev& p, cudaStream_t s);
// flags[0] bit0: row_ptr not monotone / bounds; bit1: column out of range or
// unsorted/duplicate; bit2: self loop; bit3: asymmetric
cudaError_t launch_validate(const Graph& g, int* flags, cudaStream_t s);
// dst (n x kb, contiguous, double or float) = scale * src[:, c0:c0+kb] (leading dim ld)
cudaError_t launch_pack(const double* src, int64_t ld, int c0, int kb, int64_t n, double scale, void* dst,
                        bool to_f32, cudaStream_t s);
// W[:, c0:c0+K] = Df (.) V[:, c0:c0+K] - X  (X contiguous n x K)
cudaError_t launch_apply_out(const double* V, int64_t ldv, const double* X, const double* Df, int64_t n, int K,
                             int c0, double* W, int64_t ldw, cudaStream_t s);
// W[:, c0:c0+K] = Df (.) V[:, c0:c0+K] - V[:, c0:c0+K] * 0 - X where Df = d (identity case uses gather)
cudaError_t launch_fill(double* dst, double v, int64_t count, cudaStream_t s);
cudaError_t launch_degree_vector(const Graph& g, double* out, cudaStream_t s);
// out[c] = |X[:, c]|_2 (X contiguous n x K), deterministic
// column 2-norms of X (n x K, K a power of two <= 64); scratch: 304 x K doubles
cudaError_t launch_colnorms(const double* X, int64_t n, int K, double* out, double* scratch, cudaStream_t s);
// Y[:, c] = X[:, c] * inv[c]
cudaError_t launch_scale_cols(const double* X, int64_t n, int K, const double* inv, double* Y, cudaStream_t s);
cudaError_t launch_f2d_acc(const float* src, double* dst, int64_t count, cudaStream_t s);
// discrete-time chain: Y = X / D_f per row; Y = A X; scatter a packed block into caller columns
cudaError_t launch_row_div(const double* X, const double* Df, int64_t n, int K, double* Y, cudaStream_t s);
cudaError_t launch_adj_apply(const Graph& g, const double* X, int K, double* Y, cudaStream_t s);
cudaError_t launch_unpack(const double* src, int64_t n, int K, int c0, const int32_t* perm, double* dst, int64_t ld,
                          cudaStream_t s);
// identity-function apply: W[:, c0:c0+K] = d (.) V - A V for V packed n x K
cudaError_t launch_laplacian_apply(const Graph& g, const PartDev& p, const double* Vp, int K, int c0,
                                   const int32_t* perm, double* W, int64_t ldw, cudaStream_t s);

// node relabelling by decreasing degree: perm[new] = old, iperm[old] = new,
// relabelled CSR in new_rp / new_col; tmp holds relabel_tmp_i64(n) int64
cudaError_t launch_relabel(const Graph& g, int32_t* perm, int32_t* iperm, int32_t* new_rp, int32_t* new_col,
                           int64_t* tmp, cudaStream_t s);
size_t relabel_tmp_i64(int64_t n);
// the relabelled CSR for a given device perm[new] = old (iperm, new_rp, new_col);
// tmp holds at least 2 (n + 1) + n / 1024 + 4 int64 (relabel_tmp_i64(n) suffices)
cudaError_t launch_relabel_apply(const Graph& g, const int32_t* perm, int32_t* iperm, int32_t* new_rp,
                                 int32_t* new_col, int64_t* tmp, cudaStream_t s);
// reverse Cuthill-McKee order of a host CSR: perm[new] = old (host arrays)
int rcm_order(const int32_t* rp, const int32_t* col, int64_t n, int32_t* perm);
cudaError_t launch_scan(const int64_t* in, int64_t n, int64_t* out, int64_t* tmp, cudaStream_t s);
// partition by prefix of cost(row) = deg + kRowCost (hub rows weighted x3); tmp: 2 (n + 1) + n / 1024 + 4 int64
cudaError_t launch_partition_weighted(const Graph& g, PartDev& p, int64_t* tmp, cudaStream_t s);
cudaError_t launch_pack_perm(const double* src, int64_t ld, int c0, int kb, int64_t n, double scale,
                             const int32_t* perm, double* dst, cudaStream_t s);
cudaError_t launch_apply_out_perm(const double* Vp, const double* X, const double* Df, int64_t n, int K, int c0,
                                  const int32_t* perm, double* W, int64_t ldw, cudaStream_t s);
cudaError_t launch_permute_vec(const double* in, int64_t n, const int32_t* perm, bool scatter, double* out,
                               cudaStream_t s);

// ---- wl_k_cg64.cu / wl_k_cg32.cu: CG phase kernels
// mode 0: init (gamma_0, flags); 1: `chunk` iterations (S, U pairs); 2: final x += alpha p
// a solve's start from the residual norms already in st->gamma (no pass over r)
cudaError_t launch_cg_state_restart(CgState* st, const int* skip, int K, cudaStream_t s);
cudaError_t launch_cg_phases_f32(int K, const PhaseArgs<float>& a, int grid_s, int grid_u, int mode, int chunk,
                                 cudaStream_t s);
cudaError_t launch_cg_phases_f64(int K, const PhaseArgs<double>& a, int grid_s, int grid_u, int mode, int chunk,
                                 cudaStream_t s);
// one CTA waiting in the bounded grid barrier for nblocks CTAs (failure-detection self-test)
cudaError_t launch_selftest_wait(GridBar* bar, unsigned nblocks, cudaStream_t s);
// FP64 residual r = b - M x of a warm start, norms into st->gamma / st->b2
cudaError_t launch_res_phases(int K, const ResPhaseArgs& a, int grid, cudaStream_t s);
// x (n K doubles) -> (xh, xl) FP32 terms, or (join) xh + xl -> xout
cudaError_t launch_split_x(const double* x, int64_t total, float* xh, float* xl, bool join, double* xout,
                           cudaStream_t s);
// ---- wl_k_res.cu: double-float residual of the refined form
// r_out = r_in - M y (y gathered: the correction d; x += d) or, full, r_out = b - M x (x = yh + yl)
cudaError_t launch_df_res(int K, const DfResArgs& a, int grid, bool full, cudaStream_t s);
// (bh, bl) = scale * b (b: n x K FP64, contiguous), r32 = bh (if not NULL), |b|^2 per column -> b2
cudaError_t launch_df_from_f64(int K, const double* b, double scale, int64_t n, float* bh, float* bl, float* r32,
                               double* part, CgState* st, double* b2, int grid, cudaStream_t s);
int df_res_blocks(int K);
// outer Lanczos of the refined form on double-float vectors (cooperative launch)
int df_lanczos_grid(int K);
cudaError_t launch_df_lanczos_step(int K, const DfLanczosArgs& a, int G, cudaStream_t s);
cudaError_t launch_df_combine(int K, const DfCombineArgs& a, cudaStream_t s);
// hi + lo = X[:, c] / nrm[c] (X: n x K FP64, contiguous)
cudaError_t launch_df_scale_cols(const double* X, int64_t n, int K, const double* nrm, float* hi, float* lo,
                                 cudaStream_t s);
// one term of the exponential series (the kernel returns at once once st->active is 0)
cudaError_t launch_exp_term(int K, const ExpArgs& a, int grid, cudaStream_t s);
int exp_blocks(int K);
// hi + lo = x (total FP64 values)
cudaError_t launch_df_split(const double* x, size_t total, float* hi, float* lo, cudaStream_t s);
int phase_blocks_f32(int K);  // resident CTAs of the S kernel (all SMs)
int phase_blocks_f64(int K);
int res_blocks(int K);
void thresholds_f64(int K, int* Tw, int* Tc);  // class thresholds of Cfg<T, K>
void thresholds_f32(int K, int* Tw, int* Tc);
// rows with deg > kHubDeg in increasing order; *count (host, pinned) set after the stream syncs;
// tmp: 3 (n + 1) + n / 1024 + 4 int64
// rows with lo < deg <= hi in increasing order; *count (host, pinned) after a sync
cudaError_t launch_row_list(const int32_t* row_ptr, int64_t n, int lo, int hi, int32_t* rows, int64_t* tmp,
                            int64_t* count, cudaStream_t s);

// sum of the degrees of the listed rows into *out (device)
cudaError_t launch_list_entries(const int32_t* row_ptr, const int32_t* rows, int64_t count, unsigned long long* out,
                                cudaStream_t s);

// ---- wl_k_si.cu: shift-and-invert Lanczos (shifted solves with M - a (D_f + sigma)^{-1})
cudaError_t launch_si_prep(const double* Df, int64_t n, double a, double sigma, double* dsh64, float* dsh_h,
                           float* dsh_l, double* inv64, float* inv_h, float* inv_l, cudaStream_t s);
cudaError_t launch_si_rhs64(const double* V, const double* inv, int64_t n, int K, double* B, cudaStream_t s);
int si_rhs_blocks(int64_t n, int K);
// (bh, bl) = (vh, vl) / (D_f + sigma) row-wise; |B|^2 per column -> bn2; part: si_rhs_blocks * K doubles
cudaError_t launch_si_rhs_df(const float* vh, const float* vl, const float* inv_h, const float* inv_l, int64_t n,
                             int K, float* bh, float* bl, double* part, double* bn2, cudaStream_t s);
// -M z = -((B - r) + a (D_f + sigma)^{-1} z) from the shifted solve's residual r (no gather); y may alias r
cudaError_t launch_si_mz_df(const float* bh, const float* bl, const float* rh, const float* rl, const float* zh,
                            const float* zl, const float* inv_h, const float* inv_l, double a, int64_t n, int K,
                            float* yh, float* yl, cudaStream_t s);
cudaError_t launch_si_mz64(const double* B, const double* R, const double* Z, const double* inv, double a, int64_t n,
                           int K, double* X, cudaStream_t s);

// ---- wl_k_reorth.cu: basis reorthogonalisation of the outer Lanczos
int reorth_chunks(int nb, size_t blk);
size_t reorth_part_doubles(int nb, int K, size_t blk);
cudaError_t launch_reorth(ReorthArgs a, bool df, cudaStream_t s);

// ---- wl_k_lanczos.cu
int lanczos_step_grid(int K);
cudaError_t launch_lanczos_step(int K, const LanczosStepArgs& a, int G, cudaStream_t s);
// y = exp(-tau T_m) e_1 per (column, tau); mmax bounds the steps of every column
cudaError_t launch_tridiag_exp(const TridiagArgs& a, int K, int mmax, cudaStream_t s);
cudaError_t launch_combine(int K, const CombineArgs& a, cudaStream_t s);

// ---- wl_k_spec.cu: spectral-scale Lanczos (double-float basis, k = 1)
int sp_blocks();  // resident CTAs of the step kernels (all SMs)
// mode 0: a fresh run from the seeded start vector; 1: a new run from the
// vector in W[1] (a Ritz vector); 2: continue the current run
cudaError_t launch_sp_start(const SpArgs& a, int mode, int grid_u, cudaStream_t s);
// steps j0..j1-1 (the run stops by itself at cap - 1, on breakdown, or when the
// error bound checked every `check` steps and at j1 is below rtol |theta_1|)
cudaError_t launch_sp_steps(const SpArgs& a, int j0, int j1, int cap, int check, double rtol, int grid_s,
                            int grid_u, cudaStream_t s);
// Ritz vector of the run into W[1], |u|^2 and u^T D u into st->out[5], out[6]
cudaError_t launch_sp_ritz(const SpArgs& a, int grid_u, cudaStream_t s);
// One round of the batched spectral searches: the np jobs (device array) with
// their CTA offsets in the S kernel (off_s, np + 1 entries, off_s[np] =
// grid_s) and in the other row kernels (off_u, grid_u); `steps` Lanczos
// steps (a job runs those of its j0 .. j1 - 1), the eigen step every `check`
// steps and at j1, launched after the steps whose bit is set in eig_mask
// (those where some job has one); each job's state into out[np].
cudaError_t launch_sp_round(const SpJob* jobs, const int* off_s, const int* off_u, int np, int grid_s, int grid_u,
                            int steps, int check, unsigned eig_mask, bool any_ritz, bool any_init, SpOut* out,
                            cudaStream_t s);

// ---- wl_k_trace.cu
cudaError_t launch_philox_sketch(uint16_t* omega, int64_t n, int M, uint64_t seed, cudaStream_t s);
// dst[r * M + j] = src[perm[r] * M + j]
cudaError_t launch_permute_rows_u16(const uint16_t* src, int64_t n, int M, const int32_t* perm, uint16_t* dst,
                                    cudaStream_t s);
cudaError_t launch_sketch_rhs(const uint16_t* omega, int64_t n, int M, int K, double a, float* B, cudaStream_t s);
// Omega (bf16, n x M) as FP64 n x K with zero columns M..K-1; FP64 -> FP32 copy
cudaError_t launch_sketch_block_f64(const uint16_t* omega, int64_t n, int M, int K, double* B, cudaStream_t s);
cudaError_t launch_to_f32(const double* X, int64_t total, float* Y, cudaStream_t s);
int gram_grid(int64_t n);
// H = Omega^T Y and G = Y^T Y into out (128 x 64 doubles); partial holds G x 128 x 64 floats
cudaError_t launch_gram(const uint16_t* omega, const float* Y, int64_t n, int M, int K, float* partial, int G,
                        double* out, bool tensor_cores, int* err, cudaStream_t s);
// out[0] estimate, out[1] error estimate, out[2] status, out[8 + i] = t_i
cudaError_t launch_nys_core(const double* gram, int M, double* out, cudaStream_t s);
// [Omega Y]^T Y from an FP64 Y (n x K, first M columns), FP64 throughout; partial: G x 2 x 64 x 64 doubles
cudaError_t launch_gram_f64(const uint16_t* omega, const double* Y, int64_t n, int M, int K, double* partial, int G,
                            double* out, cudaStream_t s);

// cooperative launch helper (all CTAs co-resident; required by grid_sync)
template <typename Args>
inline cudaError_t coop_launch(const void* fn, int G, const Args& a, cudaStream_t s) {
  void* params[] = {const_cast<Args*>(&a)};
  return cudaLaunchCooperativeKernel(fn, dim3(G), dim3(kBlock), params, 0, s);
}

// grid size: CTAs per SM from the occupancy calculator (capped) times SMs
inline int coop_grid(const void* fn, int cap_per_sm) {
  int dev = 0, sms = 0, nb = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kBlock, 0);
  if (nb > cap_per_sm) nb = cap_per_sm;
  if (nb < 1) nb = 1;
  return nb * sms;
}

// ---- wl_pool.cu: caching allocator (free only blocks no queued work can touch)
cudaError_t pool_malloc(void** out, size_t bytes);
void pool_free(void* p);
cudaError_t pool_malloc_host(void** out, size_t bytes);
void pool_free_host(void* p);

// ---- wl_mlp.cu
// node features (n x 4, FP32, row perm[i] for internal row i, perm NULL: i)
// and the analytic guess x_an (n, FP64); perm_key: the caller's index of
// each internal node (NULL when not relabelled), the order of the columns
// in each row; tmp holds features_tmp_bytes(n, nnz)
cudaError_t launch_features(const int32_t* rp, const int32_t* col, int64_t n, int64_t nnz, double alpha, double mu,
                            const int32_t* perm, const int32_t* perm_key, float* F, double* xan, void* tmp,
                            cudaStream_t s);
size_t features_tmp_bytes(int64_t n, int64_t nnz);
// out = x_an * exp(y) per row (xan NULL: out = y)
cudaError_t launch_mlp_predict(const float* P, const float* F, int64_t rows, const double* xan, double* out,
                               cudaStream_t s);

// ---- wl_api.cu (shared with the batched executor)
int report_cuda_error(cudaError_t e, const char* where);
void report_error(const std::string& msg);

// Batched spectral searches (wl_api.cu): `participants` host threads each
// bind the batch, run their graphs' searches (every Lanczos round waits until
// all bound threads have one, then all run as shared launches on the batch's
// stream) and leave it when done; free after all have left.
struct SpBatch;
SpBatch* sp_batch_new(int participants);
void sp_batch_bind(SpBatch* b);  // the calling thread's searches go through b (nullptr: its own stream)
void sp_batch_join(SpBatch* b, int k);  // k more participants (called by a participant that is not waiting)
void sp_batch_leave(SpBatch* b);
SpBatch* sp_batch_current();  // the calling thread's batch, or nullptr
int sp_batch_rounds(const SpBatch* b);
void sp_batch_free(SpBatch* b);
std::string last_error_copy();
// rtol: relative accuracy of lambda_max(A) and rho(Z_mu) (0: wl_build's defaults)
int graph_spectral(const wl_csr* A, const double* mus, int nmu, void* stream, double* lmax, double* rho,
                   double rtol);

}  // namespace wl
