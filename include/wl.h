/*
 * wl.h - C ABI of the GB300 walk-based Laplacian library (libwl.so).
 *
 * Computes, for a simple undirected graph with 0/1 adjacency A and degree
 * matrix D (Sec. 2 of Arrigo and Durastante, "Walk based Laplacians for
 * Modeling Diffusion on Complex Networks"):
 *
 *   phi    = phi(A, c) = sum_k c_k q_k(A)          (Def. BDTW-Laplacian)
 *   D_f    = diag(phi 1)                            (walk degrees, Sec. 3.1)
 *   L V    = D_f V - phi V                          (Eq. weighted_laplacian)
 *   U(tau) = exp(-tau L) U0                         (Eq. diffusion_on_G_with_downweighted_walk)
 *   tr(phi) estimated by XNysTrace                  (Alg. 1, last step)
 *
 * with q_k the backtrack-downweighted walk counts of Eq. qrec (mu = 0: all
 * walks, Def. transformedlaplacian; mu = 1: nonbacktracking walks, Eq. Br).
 * For the resolvent c = (1, alpha, alpha^2, ...), phi = (1 - mu^2 alpha^2) *
 * M^{-1} with the sparse symmetric matrix
 *
 *   M = M_mu(alpha) = (1 - mu^2 alpha^2) I - alpha A + alpha^2 mu D,
 *
 * which is Eq. deformed for mu = 1 and its general-mu extension (remark after
 * Prop. CGworks); M is positive definite for 0 <= alpha < 1 / rho(Z_mu)
 * (Prop. CGworks, Eq. Zdef), so every phi V is one conjugate-gradient solve
 * (Sec. 4.2).
 *
 * Conventions shared by every entry point
 *  - Status: 0 (WL_OK) or a negative WL_ERR_* code; wl_status_string()
 *    describes it. On error no output is guaranteed unless stated.
 *  - Pointers: every array argument may be a device pointer or a host
 *    pointer (pageable or pinned); the library detects which with
 *    cudaPointerGetAttributes and stages host data through its own device
 *    workspace. Every call returns after its device work has completed
 *    (the solvers read per-column scalars back to decide convergence).
 *  - Blocks of vectors are row-major n x k with a leading dimension
 *    (elements between consecutive rows) ld >= k: element (i, j) is at
 *    ptr[i * ld + j].
 *  - Ownership: the caller owns every buffer it passes; the handle owns its
 *    copy of the graph and all workspace, released by wl_destroy().
 *  - A handle must not be used from two host threads at once.
 */
#ifndef WL_H
#define WL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define WL_OK                  0
#define WL_ERR_INVALID_ARG    -1  /* null pointer, negative size, bad enum, ld < k ... */
#define WL_ERR_NOT_SYMMETRIC  -2  /* CSR pattern is not symmetric */
#define WL_ERR_SELF_LOOP      -3  /* a diagonal entry is stored */
#define WL_ERR_UNSORTED       -4  /* row_ptr not monotone, columns unsorted/duplicated/out of range */
#define WL_ERR_ALPHA_RANGE    -5  /* alpha * rho(Z_mu) >= 1 or alpha < 0: phi undefined (Prop. whe-we-converge) */
#define WL_ERR_NOT_SPD        -6  /* CG breakdown p^T M p <= 0: M not positive definite */
#define WL_ERR_NONFINITE      -7  /* NaN / Inf met in inputs or iterates */
#define WL_ERR_NO_CONVERGENCE -8  /* iteration cap reached; outputs hold the last iterate */
#define WL_ERR_TIMEOUT        -9  /* a bounded device-side wait expired; kernel returned early */
#define WL_ERR_OOM           -10  /* device allocation failed */
#define WL_ERR_CUDA          -11  /* other CUDA runtime error (message via wl_last_error) */
#define WL_ERR_UNSUPPORTED   -12  /* combination not provided (e.g. the trace of the exponential) */

/* ------------------------------------------------------------ enums */
typedef enum {
  WL_ALLWALK = 0, /* mu = 0: q_k = A^k (Def. transformedlaplacian) */
  WL_NBT     = 1, /* mu = 1: nonbacktracking counts p_k (Eq. Br) */
  WL_BTDW    = 2  /* mu from wl_params.mu, backtrack weight theta = 1 - mu (Eq. qrec) */
} wl_variant;

typedef enum {
  WL_F_RESOLVENT = 0, /* c_k = alpha^k, f(x) = (1 - alpha x)^{-1}  (Sec. 3.2.1) */
  WL_F_EXP       = 1, /* c_k = beta^k / k!, f(x) = exp(beta x) (Def. BDTW-Laplacian), any mu:
                         phi V is summed term by term over the walk counts of Eq. qrec */
  WL_F_IDENTITY  = 2  /* c = (0, 1, 0, ...): phi = A, L = D - A (Sec. 3.1) */
} wl_func;

typedef enum {
  WL_FP64    = 0, /* every vector operation in FP64 ("plain FP64 Krylov") */
  WL_REFINED = 1, /* inner CG in FP32; residual and update in double-float (FP32 pairs), FP64-level accuracy */
  WL_SKETCH  = 2  /* the fast form of the randomized estimators (wl_trace, wl_return_prob): Y enters the Gram
                     in FP32 on the tensor cores, and wl_trace solves Y = phi Omega by FP32 CG alone (relative
                     residual max(tol, 1e-7)); about 1e-5 relative agreement with the exact-Y estimate. Every
                     other call treats it as WL_REFINED. */
} wl_precision;

/* ------------------------------------------------------------ structs */
/* Simple undirected graph: symmetric 0/1 pattern, no self-loops, strictly
 * increasing column indices within each row, row_ptr[0] = 0,
 * row_ptr[n] = nnz < 2^31. Values are implicit (all ones). */
typedef struct {
  int64_t n;
  int64_t nnz;
  const int32_t* row_ptr; /* n + 1 entries, host or device */
  const int32_t* col_idx; /* nnz entries, host or device */
} wl_csr;

typedef struct {
  wl_func f;
  double alpha;      /* resolvent scale, used when alpha_rel <= 0 */
  double alpha_rel;  /* > 0: alpha = alpha_rel / rho(Z_mu), rho computed by wl_build */
  double beta;       /* exp scale; <= 0: beta = 1 / lambda_max(A) (Sec. 4.1.2) */
  double mu;         /* WL_BTDW only: mu in [0, 1]; theta = 1 - mu */
  wl_precision prec;
  double tol;        /* relative residual target of each solve (<= 0: 1e-12) */
  int max_iter;      /* CG iteration cap per solve (<= 0: 2000) */
  int max_outer;     /* Lanczos step cap of wl_expmv (<= 0: 400; at most 1000) */
  double outer_tol;  /* wl_expmv: relative change of exp(-tau T_m) e_1 between checks (<= 0: 1e-10) */
  void* stream;      /* cudaStream_t the handle works on; NULL: legacy default stream */
  int reorder;       /* 0: keep the caller's node order internally; 1: relabel nodes by
                        decreasing degree inside the handle (better gather locality);
                        2: reverse Cuthill-McKee order (wl_rcm_order, computed on the host
                        at build time; for graphs with geometric locality such as road
                        networks and grids). Results are always returned in the caller's
                        node order. Other values: WL_ERR_INVALID_ARG. */
  int reorth;        /* outer Lanczos of wl_expmv and wl_return_prob (Sec. 4.1): 0 none (the plain
                        three-term recurrence); 1 full: every new basis block is made orthogonal
                        to all earlier blocks of its column by two classical Gram-Schmidt passes
                        (cost of step j: four reads of j basis blocks). A basis kept orthogonal
                        needs fewer steps for the same change of exp(-tau T_m) e_1 between checks;
                        without it the steps still converge (more slowly) to the same result.
                        Other values: WL_ERR_INVALID_ARG. */
  double shift;      /* outer Krylov space of wl_expmv and wl_return_prob (Sec. 4.4, rational
                        Krylov): 0 the polynomial Lanczos process on L (one apply of L per step);
                        sigma > 0 the shift-and-invert Lanczos process on (L + sigma I)^{-1}
                        (resolvent only): each step is one CG solve with the sparse positive
                        definite M - a (D_f + sigma I)^{-1} and one product with M, and
                        exp(-tau L) u0 ~ |u0| V_m exp(-tau (T_m^{-1} - sigma I)) e_1 with the
                        eigendecomposition of the small T_m. Its step count does not grow with
                        |L| (walk degrees near the pole, large tau). Negative or non-finite:
                        WL_ERR_INVALID_ARG. */
  int gram;          /* Gram [Omega Y]^T Y of the sketch form of wl_trace and wl_return_prob
                        (Sec. 4.4): 0 on the CUDA cores in FP32 (per-CTA partials summed in
                        FP64); 1 on the tensor cores (tcgen05.mma kind::tf32 with Y split into
                        two TF32 terms, accumulator in tensor memory). Both agree to about 1e-5
                        relative; measured on 4.2e6 x 64, the CUDA-core kernel takes 1.9 ms and
                        the tensor-core one 2.3 ms. Other values: WL_ERR_INVALID_ARG. */
} wl_params;

typedef struct {
  int status;         /* status of the call */
  int iters;          /* operator SpMM applications (lockstep blocks) in the call */
  int outer_iters;    /* Lanczos steps (wl_expmv) */
  int refinements;    /* residual evaluations of the refinement (WL_REFINED) */
  double rel_res;     /* largest final relative residual over the call's solves */
  double time_ms;     /* device time of the call (CUDA events on the handle's stream) */
  double nnz_rhs_iters; /* sum over SpMM applications of nnz * columns */
  double bytes_alg;   /* algorithmic bytes of the CG iterations (4 nnz + 4 (n+1) + 6 n k s each) */
  double alpha, beta, mu, rho, lambda_max; /* parameters in force */
  int launches;       /* CUDA kernels launched by the call */
  /* device time of the call's kernels by family, from CUDA events recorded
   * on the handle's stream around each launch */
  int k_cg_launches;  /* persistent CG kernels (FP32 in WL_REFINED, FP64 otherwise) */
  int k_cg_iters;     /* CG iterations executed by those launches */
  double k_cg_ms;
  double k_cg_bytes;  /* algorithmic bytes of those iterations */
  int k_res_launches; /* refinement residual kernels (double-float) */
  double k_res_ms;
  int k_lan_launches; /* Lanczos step (and basis reorthogonalisation) kernels */
  double k_lan_ms;
  int reorth_blocks;  /* outer Lanczos basis blocks reorthogonalised (wl_params.reorth) */
} wl_stats;

typedef struct wl_handle wl_handle;

/* ------------------------------------------------------------ core calls */

/* Copies and validates the graph (sorted rows, indices in range, no
 * self-loops, symmetric pattern), estimates lambda_max(A) and rho(Z_mu)
 * by Lanczos (Prop. whe-we-converge, Alg. 1 "approximate the spectral
 * radius"), fixes alpha (and beta), and checks alpha * rho(Z_mu) < 1.
 * `A` and its arrays may be freed after the call. *out receives the handle
 * (NULL on error). `st` may be NULL. */
int wl_build(const wl_csr* A, wl_variant v, const wl_params* p, wl_handle** out, wl_stats* st);

/* Updates the per-call settings of a handle: prec, tol, max_iter,
 * max_outer, outer_tol, reorth, shift and stream (the operator parameters
 * stay fixed). */
int wl_set_params(wl_handle* h, const wl_params* p);

/* Walk degrees D_f = phi 1 (total communicability, Sec. 3.1), n FP64
 * values. The result is also cached in the handle for wl_apply/wl_expmv.
 * Resolvent: one CG solve M x = (1 - mu^2 alpha^2) 1 (Sec. 4.2). */
int wl_degrees(wl_handle* h, double* Df, wl_stats* st);

/* W = L V = D_f (.) V - phi V for k columns (Eq. weighted_laplacian); V
 * and W are n x k FP64 blocks with leading dimensions ldv, ldw (>= k).
 * Computes D_f first if it is not cached. k = 0 is a no-op. */
int wl_apply(wl_handle* h, const double* V, int64_t ldv, int k, double* W, int64_t ldw, wl_stats* st);

/* U(tau_t) = exp(-tau_t L) U0 for t = 0..ntau-1 (diffusion equation in
 * column form; L = L^T), by Lanczos on L with one apply per step
 * (Sec. 4.1, Krylov evaluation of f(A)v). U0 is n x k (ld ldu); U holds
 * ntau blocks, block t at U + t * n * ldo, each n x k with leading dimension
 * ldo. taus is a host array of ntau values >= 0. Every 4 steps y(tau) =
 * exp(-tau T_m) e_1 is evaluated; a column stops when, for every tau, y
 * changed by at most outer_tol |y| since the previous evaluation (a y that
 * underflowed to zero does not count as converged: the exact result keeps
 * the mass of U0). WL_ERR_NO_CONVERGENCE when max_outer steps do not
 * suffice (U then holds the last approximation). */
int wl_expmv(wl_handle* h, const double* U0, int64_t ldu, int k, const double* taus, int ntau,
             double* U, int64_t ldo, wl_stats* st);

/* Discrete-time diffusion (Sec. 3.3, Eq. let_there_be_markov): the chain
 * p_{s+1} = p_s P with P = I - D^{-1} L = D^{-1} phi, where D = diag(phi 1)
 * holds the walk degrees D_f (the reading under which the chain needs one
 * evaluation of the matrix function and reproduces the stationary
 * distributions printed in Fig. 1: pi = D_f / 1^T D_f). In column form one
 * step is p <- phi (p / D_f): a diagonal scale and one resolvent solve for
 * all k columns (for WL_F_IDENTITY, phi = A: the simple random walk).
 * P0 is n x k (ld ldp, columns are start distributions, host or device);
 * steps is a host array of nsteps non-decreasing step counts >= 0; out
 * (host or device) holds nsteps blocks, block t at out + t * n * ldo, each
 * n x k with leading dimension ldo: the distributions after steps[t] steps.
 * 1 <= nsteps <= 64. */
int wl_markov(wl_handle* h, const double* P0, int64_t ldp, int k, const int* steps, int nsteps, double* out,
              int64_t ldo, wl_stats* st);

/* XNysTrace estimate of tr(phi) with M Gaussian test vectors (Alg. 1,
 * "XNysTrace(Y, Omega)"). Omega (n x M) is drawn on the device by
 * Philox4x32-10 from `seed` (element e = i M + j uses block e / 4, see the
 * library documentation), rounded to bfloat16. Y = phi Omega and the Gram
 * matrices [Omega Y]^T Y depend on the handle's prec:
 *   WL_FP64, WL_REFINED: Y by the CG solve of that form (to tol), the Gram
 *     in FP64 on CUDA cores (estimate as accurate as Y);
 *   WL_SKETCH: Y by FP32 CG, the Gram in TF32 on the tensor cores with Y
 *     split in two terms and FP32 sums per node chunk.
 * The leave-one-out core runs in FP64. Writes the estimate and the error
 * estimate std(t_i)/sqrt(M) to the host scalars. omega_out (optional,
 * n x M uint16 bf16 bits, host or device) receives Omega. 2 <= M <= 64. */
int wl_trace(wl_handle* h, int M, uint64_t seed, double* est, double* err_est, uint16_t* omega_out,
             wl_stats* st);

/* Average return probability p(t) = tr(exp(-t L)) / n (Sec. 4.4, Eq.
 * average_return_probabilities) with its randomized estimate, Alg. 1
 * ("XNysTrace-exp"): the M Gaussian test vectors Omega are drawn as in
 * wl_trace (Philox4x32-10 from `seed`, rounded to bfloat16); Y(t) =
 * exp(-t L) Omega comes from one lockstep Lanczos run on L per column
 * (Sec. 4.1) evaluated at every t; XNysTrace(Y(t), Omega) / n gives
 * p_est[t] and the error estimate p_err[t] (host arrays of nt values).
 * The Gram takes Y(t) in FP64 (WL_FP64, WL_REFINED) or rounded to FP32 on
 * the tensor cores (WL_SKETCH). ts: host array of nt time points >= 0,
 * 1 <= nt <= 256; 2 <= M <= 64.
 * A polynomial Krylov basis replaces the paper's block rational one (one
 * apply of L per step instead of shifted solves with L). */
int wl_return_prob(wl_handle* h, int M, uint64_t seed, const double* ts, int nt, double* p_est, double* p_err,
                   wl_stats* st);

/* Optional starting guess x0 (n FP64 values, host or device) for the D_f
 * solve of wl_degrees; NULL clears it (start from 0). Copied. */
int wl_set_warm_start(wl_handle* h, const double* x0);

/* Parameters in force: alpha, beta, mu, rho(Z_mu), lambda_max(A) (host). */
int wl_get_info(const wl_handle* h, wl_stats* info);

void wl_destroy(wl_handle* h);

const char* wl_status_string(int status);

/* Text of the last CUDA error seen by the calling thread (or ""). */
const char* wl_last_error(void);

/* ------------------------------------------------------------ device memory cache */
/* The library keeps freed device and pinned host blocks for reuse by later
 * handles (building and destroying handles then costs no cudaMalloc /
 * cudaFree). wl_pool_release returns every cached block to the driver;
 * wl_pool_cached_bytes reports how much is held. Live handles keep theirs. */
void wl_pool_release(void);
size_t wl_pool_cached_bytes(void);

/* ------------------------------------------------------------ no-allocation variant */
/* Walk degrees D_f = phi 1 for the resolvent (the computation of wl_degrees
 * with prec = WL_FP64, without spectral-radius estimation and without node
 * relabelling) for callers that cannot allocate GPU memory: code that runs
 * inside a framework step whose memory planner forbids allocation, hosts
 * that reserve all device memory up front, and plug-ins that only receive
 * pre-allocated buffers. The paper has no counterpart to this entry point.
 *
 * It calls no cudaMalloc, cudaFree or allocating library routine: every
 * intermediate vector lives in one fixed array compiled into libwl.so
 * (about 12 MB of device memory, held by every GPU that loads the library
 * until the process exits). Limits and rules:
 *  - A->n must not exceed 262144 nodes; larger graphs return
 *    WL_ERR_INVALID_ARG because the fixed array cannot hold their vectors.
 *  - A (row_ptr, col_idx) and Df are DEVICE pointers owned by the caller; Df
 *    receives n FP64 values. mu is used only with WL_BTDW. alpha is taken
 *    as given and the call does not estimate rho(Z_mu): the caller must keep
 *    alpha < 1 / rho(Z_mu), the range where M is positive definite.
 *    WL_ERR_NOT_SPD is returned only when CG meets a non-positive curvature
 *    (p, M p); for an indefinite M it may instead stop on max_iter or return
 *    a finite vector that is not the walk series. tol <= 0 means 1e-12,
 *    max_iter <= 0 means 2000.
 *  - The first call on each device looks up the array's device address with
 *    cudaGetSymbolAddress (that device must be current) and caches it; make
 *    that first call before any stream capture begins.
 *  - All calls share the one array and each call resets what must start at
 *    zero. Calls that overlap on the GPU (different streams or host threads
 *    at the same time) race on the array and corrupt each other's results;
 *    serialise them.
 *  - Every call synchronises `stream` before it returns (it reads the
 *    validation flags and the CG state back into host memory), so its device
 *    work has completed on return. st->status equals the return code on every
 *    exit. `st` may be NULL. */
int wl_degrees_noalloc(const wl_csr* A, wl_variant v, double mu, double alpha, double tol, int max_iter,
                       double* Df, void* stream, wl_stats* st);

/* Gram [Omega Y]^T Y of the XNysTrace core (Alg. 1): omega n x M BF16 bit
 * patterns, Y n x ldy FP32 (first M columns used), M <= 64; DEVICE pointers.
 * out (device, 128 x 64 FP64): rows 0..63 = Omega^T Y, rows 64..127 =
 * Y^T Y, entries beyond M zero. tensor_cores = 1: tcgen05 MMA (kind::tf32,
 * FP32 accumulation in tensor memory) with Y split into two TF32 terms;
 * 0: FP32 CUDA cores. FP64 sum across node chunks either way. Synchronous;
 * WL_ERR_TIMEOUT if a bounded tensor-core wait gave up. */
int wl_sketch_gram(const uint16_t* omega, const float* Y, int64_t n, int M, int ldy, int tensor_cores, double* out,
                   void* stream);

/* ------------------------------------------------------------ learned warm start */
/* A small perceptron supplies the starting guess of the walk-degree solve
 * (wl_degrees); the paper has no learned part. Features per node i:
 *   f0 = log(1 + d_i), f1 = log(1 + (A d)_i), f2 = log(1 + t_i) (triangles
 *   through i), f3 = log(1 + (A d - d)_i) (nonbacktracking 2-walks).
 * Guess: x0 = x_an * exp(y), x_an = 1 + B 1 + B^2 1 with
 * B = (alpha A - alpha^2 mu D) / (1 - mu^2 alpha^2) (two terms of the
 * Neumann series of D_f), y = W3 tanh(W2 tanh(W1 s + b1) + b2) + b3 on the
 * standardised features s = (f - mean) / std.
 * Parameter vector (wl_mlp_param_count() = 4553 floats): mean[4], std[4],
 * W1[64][4], b1[64], W2[64][64], b2[64], W3[64], b3. */
int wl_mlp_param_count(void);

/* Checkpoint of the network (host arrays of wl_mlp_param_count() floats):
 * a 32-byte header (magic "WLMLP001", inputs, hidden width, outputs,
 * parameter count, FNV-1a hash of the parameter bytes) and the parameters as
 * little-endian FP32. wl_mlp_load rejects a file of another shape, length or
 * magic (WL_ERR_INVALID_ARG) and one whose hash does not match its
 * parameters (WL_ERR_NONFINITE); params is left untouched then. The paper has
 * no counterpart (its method has no learned part). */
int wl_mlp_save(const char* path, const float* params);
int wl_mlp_load(const char* path, float* params);

/* Features (n x 4 FP32, row-major) and x_an (n FP64) of the handle's graph
 * and parameters (f = WL_F_RESOLVENT), in the caller's node order; either
 * output may be NULL; host or device pointers. Synchronous. */
int wl_mlp_features(wl_handle* h, float* feats, double* xan, wl_stats* st);

/* Trains the network on rows (feats[r], target[r]) with the MSE loss and
 * Adam (beta1 0.9, beta2 0.999, eps 1e-8, step size lr): `steps` updates on
 * consecutive slices of `batch` rows (batch <= 0: all rows). standardize = 1
 * first sets mean/std from the rows. params: in = initial values, out =
 * trained values (host or device). final_loss: MSE of the trained network
 * over all rows. Synchronous. */
int wl_mlp_train(float* params, const float* feats, const float* target, int64_t rows, int steps, int64_t batch,
                 float lr, int standardize, double* final_loss, void* stream);

/* MSE loss over all rows and its gradient (layout of the parameter vector,
 * zero for mean/std), FP32 accumulation per 128 rows, FP64 across them. */
int wl_mlp_loss_grad(const float* params, const float* feats, const float* target, int64_t rows, double* loss,
                     float* grad, void* stream);

/* out[r] = xan[r] * exp(y_r) (xan NULL: out[r] = y_r). */
int wl_mlp_predict(const float* params, const float* feats, int64_t rows, const double* xan, double* out,
                   void* stream);

/* Training target[r] = log(Df[r] / xan[r]) (FP32). */
int wl_mlp_targets(const double* Df, const double* xan, int64_t rows, float* target, void* stream);

/* Features, x_an and x0 on the device for the handle's graph; x0 becomes
 * the starting guess of the next wl_degrees (as wl_set_warm_start). */
int wl_mlp_warm_start(wl_handle* h, const float* params, wl_stats* st);

/* ------------------------------------------------------------ batched executor */
/* Walk degrees and walk-Laplacian applies for a collection of graphs and a
 * sweep of backtrack weights, all problems at once (Sec. 4.2 applied to
 * every (graph, mu) pair; Def. BDTW-Laplacian with theta = 1 - mu, so
 * mu = 1 is the non-backtracking and mu = 0 the all-walk resolvent).
 * A problem is one (graph g, mu_j) pair; problem index p = j * ngraph + g. */
typedef struct wl_batch wl_batch;

/* graphs[0 .. ngraph): CSR graphs as in wl_build (host or device arrays,
 * copied; each validated like wl_build). mus[0 .. nmu): mu values in [0, 1].
 * p: f must be WL_F_RESOLVENT; alpha_rel > 0 gives alpha = alpha_rel /
 * rho(Z_mu) per problem (a graph with no edges gets alpha = 0), otherwise
 * p->alpha is used for all; every problem must have alpha rho(Z_mu) < 1
 * (else WL_ERR_ALPHA_RANGE). p->prec is WL_FP64 or WL_REFINED; tol,
 * max_iter, max_outer and stream as in wl_build. Synchronous. The spectral
 * searches (lambda_max(A) and rho(Z_mu) to 1e-10 relative) of all graphs run
 * together: each round of Lanczos steps is one launch per kernel and step
 * over every search in flight, and the searches of a graph's mu values > 0
 * run side by side, each from the Ritz vector of its lambda_max(A) run. st
 * may be NULL: time_ms, status, outer_iters = the rounds of those shared
 * searches. */
int wl_batch_build(const wl_csr* graphs, int ngraph, const double* mus, int nmu, const wl_params* p,
                   wl_batch** out, wl_stats* st);

/* For every problem p = (g, mu_j):
 *   Df[j][row]        = D_f of graph g at mu_j       (nmu x n, n = total rows)
 *   W[j][row][c]      = (L_mu_j V_g)[row][c]          (nmu x n x k)
 * V: n x k row-major FP64 (rows of the graphs concatenated in order); the
 * same V serves every mu. k in {1, 2, 4, 8, 16, 32, 64}. V, Df and W may be
 * host or device pointers. stepped = 0 runs the whole computation as one
 * CUDA graph launch (captured on the first call for this k and form, then
 * replayed); stepped = 1 launches the same kernels one by one with a host
 * read per iteration (for checking; the results are identical).
 * Returns the first non-OK problem status (WL_ERR_NO_CONVERGENCE, ...);
 * outputs hold the last iterates then. Synchronous. st may be NULL:
 * time_ms, rel_res (largest relative residual), nnz_rhs_iters, launches. */
int wl_batch_run(wl_batch* b, const double* V, int k, double* Df, double* W, int stepped, wl_stats* st);

/* Per-problem figures of the build and the last run (any pointer may be NULL):
 * alpha, rho(Z_mu), lambda_max(A), the CG iterations of the D_f solve and of
 * the K-column solve (summed over refinement steps), the problem's status. */
int wl_batch_info(const wl_batch* b, int graph, int mu_index, double* alpha, double* rho, double* lambda_max,
                  int* iters_df, int* iters_v, int* status);

/* Rows per plain tile chosen by the autotuner for width k (0 before the first run). */
int wl_batch_tile_rows(const wl_batch* b, int k);

void wl_batch_destroy(wl_batch* b);

/* Reverse Cuthill-McKee order of a simple graph (host arrays, the CSR of
 * wl_csr; the relabelling of reorder = 2): perm[new] = old, a permutation of
 * 0..n-1. Each connected component is numbered breadth-first from a
 * pseudo-peripheral node with neighbours by increasing degree (ties by id),
 * components in order of their lowest-degree node, and the numbering is then
 * reversed. Deterministic. The CSR is not validated here (wl_build does);
 * indices must be in range. WL_ERR_INVALID_ARG for n < 0 or NULL arrays. */
int wl_rcm_order(const int32_t* row_ptr, const int32_t* col_idx, int64_t n, int32_t* perm);

/* ---------------------------------------------------------------- self-test
 * Failure detection of the device-side waits. One CTA enters the grid barrier
 * that the cooperative kernels use (Lanczos step, spectral search), told to
 * expect 1 + missing CTAs. missing = 0: the barrier completes; WL_OK.
 * missing > 0: no other CTA ever arrives, the wait gives up after its limit
 * (2 s of GPU time), records WL_ERR_TIMEOUT and the kernel returns normally,
 * so the context stays usable; the call returns WL_ERR_TIMEOUT. stream: a
 * cudaStream_t or NULL (default stream). Synchronous. WL_ERR_INVALID_ARG for
 * missing < 0 or missing > 1024. */
int wl_selftest_bounded_wait(int missing, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* WL_H */
