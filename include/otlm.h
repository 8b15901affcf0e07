/*
 * otlm.h -- C ABI of the GB300 solver for Optimal Transport Linear Models (OTLM).
 *
 * The solver runs the Scaling Algorithm for OTLM (Algorithm 1 of Kacprzak et al.,
 * "Scalable Approximate Algorithms for Optimal Transport Linear Models", arXiv 2504.04609):
 * per iteration a Gibbs-kernel apply a = K u1, one majorisation-minimisation (MM) step on the
 * dictionary weights w (Table 2), the source scaling u2 = X w / a, a second apply b = K^T u2,
 * and the datafit proximal step u1 = prox_L(b | y) / b (Table 1).  K = exp(-C/eps) with the
 * squared-distance cost C_ij = (x_i - x_j)^2 on a 1-D grid x (Sec. 2.2, Gibbs kernel), or the
 * absolute distance |x_i - x_j| (otlm_config.cost).
 *
 * Conventions shared by every entry point
 *  - Every array argument is a DEVICE pointer owned by the caller, except where a function
 *    says "host".  The library never frees caller memory.  A handle owns only its workspace.
 *  - Element type: `double` when the handle was created with OTLM_PREC_FP64, otherwise `float`.
 *    Integer outputs are int32.
 *  - Layouts are row-major and dense: x [n]; D [n][k] (the paper's X, one column per atom,
 *    shared by every problem of the batch); y, g, t [batch][n]; w [batch][k].
 *  - Calls are asynchronous on the stream given at create time (NULL = the legacy default
 *    stream); results are valid once that stream has been synchronised.  The host blocks only
 *    for the short convergence polls that `otlm_solve` makes every few iterations.
 *  - Return value: OTLM_OK (0) or a negative OTLM_E* code; otlm_strerror() names it.  No C++
 *    exception crosses the ABI.  Arguments are validated before any work is queued.
 *  - Potentials: g = eps log u1 (target side), f = eps log u2 (source side).
 *  - Readings of passages the paper leaves open (used throughout):
 *      Q_ij = u2_i K_ij u1_j; the objective is eps KL(Q||K) + lam L(Q^T 1|y) + alpha R(w)
 *      (Eq. OTLM without the duplicated <C,Q> term); Table 2's l1 shift is alpha/(eps x_j) and
 *      its squared-l2 update is w_j = W0(c_j e^{nu_j})/c_j, c_j = alpha/(eps x_j) (App. A);
 *      "not converged" (Algorithm 1) means e = ||u2*(K u1) - X w||_1 / ||X w||_1 > tol,
 *      measured with the u1 of the following iteration.
 */
#ifndef OTLM_H
#define OTLM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------------------ */
#define OTLM_OK            0
#define OTLM_EINVAL       -1  /* an argument is out of range or inconsistent with the handle */
#define OTLM_ECUDA        -2  /* a CUDA runtime call failed (the CUDA error is not cleared)  */
#define OTLM_ENOMEM       -3  /* workspace allocation failed                                  */
#define OTLM_EUNSUPPORTED -4  /* valid request this build does not implement                  */
#define OTLM_ESCRATCH     -5  /* problem too large for otlm_solve_noalloc's static scratch    */
#define OTLM_ETIMEOUT     -6  /* a bounded device-side wait expired (tensor-core path)        */

/* per-problem status written to status_out[] */
#define OTLM_CONVERGED     0  /* e <= tol                                                     */
#define OTLM_MAX_ITER      1  /* stopped at max_iter                                          */
#define OTLM_NONFINITE     2  /* a NaN/Inf appeared in the violation e; state left as is      */
#define OTLM_INVALID       3  /* otlm_solve_ragged: the problem's sizes or offsets fall outside
                                 the packed arrays; the problem was not touched                */

/* ---- problem options ----------------------------------------------------------------------- */
typedef enum {            /* marginal datafit L(. | y), Table 1 */
  OTLM_DATAFIT_BALANCED = 0,  /* indicator {Q^T 1 = y}: prox = y                               */
  OTLM_DATAFIT_KL       = 1,  /* lam KL(s|y): prox = s^{eps/(eps+lam)} y^{lam/(eps+lam)}        */
  OTLM_DATAFIT_TV       = 2,  /* lam ||s-y||_1: prox = min(s e^{lam/eps}, max(s e^{-lam/eps},y)) */
  OTLM_DATAFIT_L2       = 3,  /* (lam/2)||s-y||^2: prox = (eps/lam) W0((lam/eps) s e^{lam y/eps}) */
  OTLM_DATAFIT_POISSON  = 4   /* lam sum (s - y log s): prox = (lam y/eps) / W0((lam y/(eps s))
                                 e^{lam/eps}), s e^{-lam/eps} where y = 0 (Table 1's last row; its
                                 "W0^{-1}" read as 1/W0, re-derived from the stationarity
                                 condition of App. B) */
} otlm_datafit;

typedef enum {            /* weight penalty R(w), Table 2 */
  OTLM_PENALTY_NONE = 0,
  OTLM_PENALTY_L1   = 1,      /* alpha sum w                                                 */
  OTLM_PENALTY_L2SQ = 2,      /* (alpha/2) ||w||^2                                           */
  OTLM_PENALTY_ELASTIC = 3    /* alpha sum w + (beta/2) ||w||^2, beta from otlm_config; update
                                 w_j = W0(g_j e^{nu_j - alpha/(eps x_j)})/g_j, g_j = beta/(eps x_j)
                                 (App. A's stationarity condition; Table 2 prints alpha/beta)   */
} otlm_penalty;

typedef enum {            /* grid cost of otlm_solve / otlm_solve_host / otlm_objective (Sec. 2.2) */
  OTLM_COST_GRID_SQ  = 0,     /* C_ij = (x_i - x_j)^2 (the default)                              */
  OTLM_COST_GRID_ABS = 1      /* C_ij = |x_i - x_j|: the cost of the paper's demonstrations and
                                 scalability tests, C = rho |x_i - x_j| (pass x scaled by rho)    */
} otlm_cost_kind;

typedef enum {
  OTLM_PREC_FP32_LOG = 0,     /* FP32, scalings carried as log2 potentials (stable at small eps) */
  OTLM_PREC_FP64     = 1,     /* FP64 throughout, same log-domain arithmetic                   */
  OTLM_PREC_BF16_TC  = 2      /* kernel applies as tensor-core GEMMs K V^T: BF16 hi/lo operands
                                 (three products, ~16 mantissa bits), FP32 accumulation, a
                                 per-problem max shift; potentials and updates in FP32.  Element
                                 type float.  Rows whose sum underflows (all significant terms
                                 below 2^-126 of the problem's largest) are recomputed exactly in
                                 the log domain.  otlm_objective on such a handle runs FP32 applies
                                 (the in-solve objective of check_every runs tensor-core ones). */
} otlm_precision;

typedef struct otlm_config {
  int    n_max;        /* largest grid size a solve on this handle may use (>= 2)             */
  int    k_max;        /* largest dictionary size (1..256)                                    */
  int    batch_max;    /* largest number of problems per solve (>= 1)                         */
  int    precision;    /* otlm_precision                                                      */
  int    datafit;      /* otlm_datafit                                                        */
  int    penalty;      /* otlm_penalty                                                        */
  int    max_iter;     /* iteration cap (>= 1)                                                */
  double tol;          /* stop a problem once e <= tol; tol <= 0 runs exactly max_iter        */
  int    poll_every;   /* host polls the number of unfinished problems every this many
                          iterations (>= 1); larger = fewer host syncs, more idle launches   */
  double beta;         /* squared-l2 weight of OTLM_PENALTY_ELASTIC (> 0 there; ignored by the
                          other penalties)                                                     */
  int    mm_steps;     /* MM steps of the weight update per iteration, all with the same
                          a = K u1 (Sec. 4.2: Algorithm 1 takes one; more approach
                          prox_{alpha P}(K u1 | X)); 0 or 1 = one step, at most 64             */
  /* Further stopping criteria (Algorithm 1 leaves "converged" open; reading: every enabled
   * criterion must hold at the same iteration, tol's violation test being the first).  Fields
   * added after mm_steps; zero-initialise the struct to leave them off. */
  int    check_every;  /* >= 0.  > 0: every this many iterations, and for every problem at the end,
                          the FP64 primal and dual of the state the solve would return (Eq. OTLM and
                          its Fenchel dual, as otlm_objective) are reduced on the GPU, with one extra
                          kernel apply per check in the handle's own arithmetic (tensor cores on a
                          BF16 handle); read them with otlm_solve_stats.  0: never (no extra memory
                          or work).  otlm_solve, otlm_solve_cost, otlm_solve_host only.          */
  double gap_tol;      /* >= 0, finite.  > 0 (needs check_every > 0): a problem stops only at a check
                          where primal - dual <= gap_tol |primal|                               */
  double dw_tol;       /* >= 0, finite.  > 0: a problem stops only where the last weight update's
                          ||w_new - w_old||_1 / ||w_new||_1 <= dw_tol (the weights converge far more
                          slowly than the marginals: reading A8).  otlm_solve, otlm_solve_cost,
                          otlm_solve_host only.                                                  */
  /* Tile shapes of otlm_solve_ragged, as otlm_tune_ragged reports them (0 everywhere = defaults) */
  int    ragged_cta;   /* threads per CTA: 128, 256 or 512; 0 = 256                             */
  int    ragged_rows_log2[16];  /* rows per thread for problems with n in (256 b, 256 (b + 1)],
                          b = 0..15 (the last bucket also takes larger n), as log2: 1..5 (2..32 rows),
                          raised where needed to cover n; 0 = the fewest that cover n          */
  double bf16_single_until;  /* OTLM_PREC_BF16_TC only, in [0, 1).  0 (default): the kernel applies
                          always take the three BF16 hi/lo products.  > 0: a precision schedule: the
                          applies take the single product hi x hi (one third of the tensor work)
                          until some problem's violation e is <= this value, then hi/lo to the end.
                          Early errors of ~2^-9 per apply are contracted away for the squared-error
                          datafit (the measured workload stays at the 1e-5 bar: tests), but persist
                          in w where the weights converge slowly (e.g. KL + l1 at eps = 5e-3: ~2e-5),
                          so it is off by default.                                              */
  int    cost;         /* otlm_cost_kind of the grid solves (0 = squared distance).  otlm_solve_cost
                          (dense C) and otlm_solve_banded (cost diagonals) take their cost as given
                          and ignore it; otlm_solve_ragged and otlm_tune_ragged support the squared
                          distance only (OTLM_EUNSUPPORTED otherwise).                          */
} otlm_config;

typedef struct otlm_ctx* otlm_handle;

/* Create a handle and its device workspace (about (8 n_max + 2 k_max + 16) * batch_max
 * elements).  `cuda_stream` is a cudaStream_t (NULL = default stream).  The workspace is
 * owned by the handle and released by otlm_destroy.
 * With check_every > 0 the workspace also holds the objective scratch (3 batch_max n_max elements
 * and 20 batch_max bytes).
 * Errors: OTLM_EINVAL (null pointers, sizes out of range, unknown enum, ELASTIC without a
 * finite beta > 0, mm_steps outside 0..64, check_every < 0, gap_tol or dw_tol negative or not
 * finite, gap_tol > 0 with check_every == 0, ragged_cta not 0/128/256/512, a ragged_rows_log2
 * entry outside 0..5), OTLM_ENOMEM, OTLM_ECUDA.  On error *h is set to NULL. */
int otlm_create(otlm_handle* h, const otlm_config* cfg, void* cuda_stream);

/* Release the workspace.  Waits for the handle's stream.  NULL is ignored. */
void otlm_destroy(otlm_handle h);

/* Solve `batch` independent OTLM problems sharing one grid and one dictionary
 * (Algorithm 1; cfg.mm_steps MM steps per iteration, one by default as in Sec. 4.2).
 *   x      [n]          grid; cost C_ij = (x_i - x_j)^2, or |x_i - x_j| with OTLM_COST_GRID_ABS
 *   D      [n][k]       dictionary X of the paper; entries >= 0, every column sum > 0
 *   y      [batch][n]   targets, >= 0
 *   eps, lam, alpha     entropic weight (> 0), datafit weight (> 0; ignored for BALANCED),
 *                       penalty weight (>= 0; > 0 for L2SQ)
 *   w      [batch][k]   in: initial weights (every entry > 0: zero weights stay zero);
 *                       out: weights after the last completed iteration
 *   g      [batch][n]   in: initial target potential g = eps log u1 (warm start), or NULL for
 *                       u1 = 1; out (when not NULL): final g
 *   t_out  [batch][n]   transported target marginal Q^T 1 of the returned state, or NULL
 *   iters_out  [batch]  completed iterations (device int32, may be NULL)
 *   err_out    [batch]  last measured violation e (device; float for an FP32 handle, double
 *                       for FP64; may be NULL)
 *   status_out [batch]  OTLM_CONVERGED / OTLM_MAX_ITER / OTLM_NONFINITE (device int32, may be NULL)
 * Problems stop independently (once every enabled criterion holds: e <= tol, and the weight change
 * and the FP64 gap when dw_tol / gap_tol are set); finished problems drop out of the remaining
 * launches.
 * Errors: OTLM_EINVAL (batch/n/k beyond the handle, n < 2, k < 1, eps <= 0, lam <= 0 for a
 * soft datafit, alpha < 0, alpha == 0 with L2SQ, a NULL required pointer), OTLM_ECUDA. */
int otlm_solve(otlm_handle h, int batch, int n, int k,
               const void* x, const void* D, const void* y,
               double eps, double lam, double alpha,
               void* w, void* g, void* t_out,
               int* iters_out, void* err_out, int* status_out);

/* Same as otlm_solve for a cost given as a dense matrix instead of a grid: C [n][n] (device,
 * row-major, the handle's element type) is the cost of moving mass from source bin i (row) to
 * target bin j (column), shared by the batch; it need not be symmetric (e.g. the non-stationary
 * cost rho (x_i - x_j)^2 / x_i^2 of the muonic X-ray spectra appendix), and +inf forbids a pair (a
 * truncated cost; NaN and -inf are not allowed).  Both kernel applies of Algorithm 1 follow
 * Q_ij = u2_i K_ij u1_j with K = exp(-C / eps): the source apply sums row i of K, the target apply
 * column j.  Tensor-core handles build K and K^T once per call (BF16 hi/lo) in the workspace; FP32
 * and FP64 handles read C in tiles through shared memory in every apply (log domain, as the grid
 * solves; check_every and the stopping criteria as otlm_solve).  Errors as otlm_solve.
 * otlm_objective covers the grid costs only. */
int otlm_solve_cost(otlm_handle h, int batch, int n, int k,
                    const void* C, const void* D, const void* y,
                    double eps, double lam, double alpha,
                    void* w, void* g, void* t_out,
                    int* iters_out, void* err_out, int* status_out);

/* Same as otlm_solve, with x, D, y, w (in/out), g (in/out, may be NULL) and t_out (may be
 * NULL) in HOST memory (pageable or pinned), and iters_out / status_out / err_out as host
 * arrays (may be NULL).  The host<->device copies run on the handle's stream through the
 * handle's workspace; the call returns after the results are in host memory. */
int otlm_solve_host(otlm_handle h, int batch, int n, int k,
                    const void* x, const void* D, const void* y,
                    double eps, double lam, double alpha,
                    void* w, void* g, void* t_out,
                    int* iters_out, void* err_out, int* status_out);

/* Solve `batch` problems sharing a BANDED cost and a SPARSE dictionary (Algorithm 1, FP32 log
 * domain; the form of the paper's scalability test, App. "Performance Scalability Tests": a cost
 * truncated to +inf beyond a distance, so K_ij = 0 off a band, and k = n/10 truncated basis
 * functions).  K is never formed; both applies are log-sum-exps over the band.
 *   Cd       [2hw+1][n]  cost in diagonal storage: Cd[d][i] = C(i, i + d - hw); +inf marks a
 *                        forbidden pair (K = 0) and pads the diagonals where i + d - hw falls
 *                        outside [0, n) (entries there are ignored).  No NaN or -inf.
 *   hw                   half-width of the band, 0..64 and < n
 *   col_ptr [k+1], row_idx [nnz], val [nnz]   the dictionary X [n][k] in CSC form (int32 and
 *                        float, device memory): column m holds rows row_idx[col_ptr[m] ..
 *                        col_ptr[m+1]) with values >= 0; col_ptr[0] = 0, col_ptr[k] = nnz; every
 *                        column sum > 0.  Not modified; a CSR copy is built in the workspace.
 *   y [batch][n], w [batch][k] (in/out), g [batch][n] (in/out or NULL), t_out, iters_out,
 *   err_out, status_out: as otlm_solve (float, device memory).
 * The handle must be OTLM_PREC_FP32_LOG with mm_steps <= 1 (else OTLM_EUNSUPPORTED); datafit,
 * penalty, beta, max_iter, tol and poll_every come from it; batch <= batch_max, while n and k are
 * not bounded by n_max and k_max: the banded workspace (about 4 (6 batch n + batch k + (2hw+1) n
 * + 2 nnz + 3 n) bytes) is allocated on the first call and grown when a later call needs more.
 * The band and dictionary are validated on the device before use (one host synchronisation).
 * Errors: OTLM_EINVAL (sizes, eps, lam, alpha as otlm_solve, hw out of range, NULL pointers, a
 * malformed band or dictionary), OTLM_EUNSUPPORTED, OTLM_ENOMEM, OTLM_ECUDA. */
int otlm_solve_banded(otlm_handle h, int batch, int n, int hw, const float* Cd,
                      int k, int nnz, const int* col_ptr, const int* row_idx, const float* val,
                      const float* y, double eps, double lam, double alpha,
                      float* w, float* g, float* t_out, int* iters_out, float* err_out,
                      int* status_out);

/* Solve an UNEVEN batch in one persistent launch (Algorithm 1 per problem, FP32 log domain):
 * problem p has its own grid size n[p] (2..n_max, n_max <= 4096), dictionary size k[p]
 * (1..k_max), eps[p] > 0, grid, dictionary and target.  Arrays are concatenated over problems:
 *   x, y, g, t_out  [sum n]     problem p at offset off_n[p]
 *   D               [sum n k]   problem p at offset off_D[p], row-major [n[p]][k[p]]
 *   w               [sum k]     problem p at offset off_k[p]; in: initial weights (> 0), out: result
 *   n, k, eps, off_* , iters_out, err_out, status_out: [batch], device memory
 * g: in/out potentials (NULL = cold start, no output); t_out may be NULL.  lam and alpha as in
 * otlm_solve; datafit, penalty, beta, mm_steps, max_iter and tol come from the handle, which
 * must be OTLM_PREC_FP32_LOG.  One CTA solves one problem at a time with its state in shared memory; CTAs
 * take problems largest-first from a device queue; the launch is captured in a CUDA graph (on an
 * internal stream ordered after the handle's stream) and replayed while the arguments repeat.
 * The host copies n, k, eps and the three offset arrays once to validate and order the batch
 * (synchronous copies): every problem's range must lie inside the packed lengths sum n, sum n k
 * and sum k (offsets may come in any order).
 * Errors: OTLM_EINVAL (sizes beyond the handle, eps <= 0, an offset range outside the packed
 * arrays, NULL pointers), OTLM_EUNSUPPORTED (handle not FP32), OTLM_ENOMEM, OTLM_ECUDA. */
int otlm_solve_ragged(otlm_handle h, int batch, const int* n, const int* k, const float* eps,
                      const long long* off_n, const long long* off_D, const long long* off_k,
                      const float* x, const float* D, const float* y, double lam, double alpha,
                      float* w, float* g, float* t_out, int* iters_out, float* err_out,
                      int* status_out);

/* Autotuner for otlm_solve_ragged (the paper has no counterpart): chooses the tile shape of the
 * persistent kernel, i.e. the CTA size (128, 256 or 512 threads) and, for each size bucket of
 * otlm_config.ragged_rows_log2, the rows each thread owns (more rows reuse each staged column for
 * more exponentials; fewer keep more threads busy).  Every sample_every-th problem of the
 * largest-first order joins its bucket's sample; for each CTA size, each bucket times its feasible
 * choices (the fewest rows that cover the bucket and up to four times as many) on its sample
 * repeated over two waves of CTAs, `iters` iterations each, and keeps the fastest; the CTA size
 * with the smallest total wins.  The choice is kept on the handle; *cta_threads_out (may be NULL)
 * and rows_log2_out [16] (may be NULL) receive it in otlm_config's form, so that a later
 * otlm_create can take it without tuning.  Caller buffers are not modified (w is copied).  Same
 * argument rules as otlm_solve_ragged. */
int otlm_tune_ragged(otlm_handle h, int batch, const int* n, const int* k, const float* eps,
                     const long long* off_n, const long long* off_D, const long long* off_k,
                     const float* x, const float* D, const float* y, double lam, double alpha,
                     const float* w, int sample_every, int iters, int* cta_threads_out, int* rows_log2_out);

/* ---- learned warm start (an extension: the paper starts every solve from u1 = 1) -------------
 * A 4-layer MLP maps a target y [n] to an initial state for Algorithm 1: features
 * [n y / sum(y), log sum(y)] -> 3 x (Linear + GELU, width H) -> Linear -> [g/eps (n), log w (k)],
 * with outputs normalised per coordinate by (mean, std).  Weights: FP32 masters updated by AdamW
 * (beta 0.9 / 0.999, eps 1e-8, decoupled weight decay) and BF16 copies for the forward pass; all
 * accumulation in FP32.  Parameters are one flat FP32 vector: for each layer W [out][in] then
 * b [out].  All pointers are device pointers; calls are asynchronous on the stream given at
 * create time.  Errors: OTLM_EINVAL, OTLM_ENOMEM, OTLM_ECUDA. */
typedef struct otlm_ws_ctx* otlm_ws;

/* Create a network for grids of n bins and k atoms, hidden width H, at most batch_max rows per
 * call; weights uniform(+-sqrt(6/(fan_in+fan_out))) from a counter-based hash of `seed`. */
int otlm_ws_create(otlm_ws* out, int n, int k, int width, int batch_max, unsigned long long seed,
                   void* cuda_stream);
void otlm_ws_destroy(otlm_ws w);
long long otlm_ws_num_params(otlm_ws w);
/* Output normalisation: mean, std [n + k] (device). */
int otlm_ws_set_normalization(otlm_ws w, const float* mean, const float* std);
int otlm_ws_get_params(otlm_ws w, float* params_out);
int otlm_ws_set_params(otlm_ws w, const float* params);
/* Loss and its gradient for y [batch][n] and targets [batch][n + k] (g/eps, log w of solved
 * problems; non-finite entries are masked): loss = mean over unmasked entries of
 * (z - (t - mean)/std)^2.  grad_out [num_params] and loss_out [1] may be NULL. */
int otlm_ws_gradients(otlm_ws w, int batch, const float* y, const float* target, float* grad_out,
                      float* loss_out);
/* One AdamW step on that loss (learning rate lr, weight decay wd); loss_out may be NULL. */
int otlm_ws_train_step(otlm_ws w, int batch, const float* y, const float* target, double lr,
                       double weight_decay, float* loss_out);
/* Training targets from solved problems: targets [batch][n + k] = [g / eps, log w] for g [batch][n]
 * and w [batch][k] as returned by otlm_solve; g / eps is clipped below at g_floor, and a
 * non-finite g or a weight <= 0 gives -inf (masked by the loss).  batch is not bounded by
 * batch_max.  Errors: OTLM_EINVAL (NULL pointers, batch < 1, eps not finite and > 0, g_floor NaN),
 * OTLM_ECUDA. */
int otlm_ws_make_targets(otlm_ws w, int batch, const float* g, const float* wts, double eps, double g_floor,
                         float* targets);
/* Output normalisation fitted to training targets [rows][n + k]: per output, the mean and the
 * standard deviation (floored at 1e-3) over the finite entries, two passes with FP64 sums; stored
 * on the network (as otlm_ws_set_normalization) and copied to mean_out / std_out [n + k] when not
 * NULL.  rows is not bounded by batch_max.  Errors: OTLM_EINVAL, OTLM_ECUDA. */
int otlm_ws_fit_normalization(otlm_ws w, int rows, const float* targets, float* mean_out, float* std_out);
/* Warm start for otlm_solve: g0 [batch][n] = eps * predicted g/eps, w0 [batch][k] = exp(predicted
 * log w); a non-finite prediction falls back to the cold start (g0 = 0, w0 = cold_w).  The forward
 * pass runs on the tensor cores (BF16 weights times activations carried as BF16 hi/lo pairs, FP32
 * accumulation: ~16 bits, against the FP32-activation forward pass of training); if one of its
 * GEMMs gives up a bounded wait, every row falls back to the cold start. */
int otlm_ws_predict(otlm_ws w, int batch, const float* y, double eps, const float* cold_w, float* g0,
                    float* w0);

/* Per-problem diagnostics of the handle's last otlm_solve / otlm_solve_cost / otlm_solve_host call
 * (the paper has no counterpart; they support the stopping criteria of reading A8):
 *   dw_out [batch]      ||w_new - w_old||_1 / ||w_new||_1 of each problem's last weight update
 *                       (element type of the handle; NaN if it made none); may be NULL
 *   primal_out, dual_out [batch]  FP64 primal and Fenchel dual of the returned state (w, g), as
 *                       otlm_objective defines them, computed at the end of the solve; need a
 *                       handle created with check_every > 0; may be NULL
 * Device pointers; asynchronous on the handle's stream; batch must not exceed the last solve's.
 * Errors: OTLM_EINVAL (NULL handle, batch out of range, primal/dual asked of a handle with
 * check_every == 0), OTLM_ECUDA. */
int otlm_solve_stats(otlm_handle h, int batch, void* dw_out, double* primal_out, double* dual_out);

/* Cold start of Algorithm 1 on the device: w_out [batch][k] = sum_i y_pi / (k x_j), x_j = sum_i D_ij
 * (Algorithm 1 leaves the initial w open; this reading spreads the target's mass evenly over the
 * atoms; the matching initial potential is u1 = 1, i.e. g = NULL in otlm_solve).  D [n][k] and
 * y [batch][n] as in otlm_solve, element type of the handle; sums in FP64.  Uses the handle's
 * stream and workspace (column masses); asynchronous.
 * Errors: OTLM_EINVAL (NULL pointers, batch/n/k beyond the handle), OTLM_ECUDA. */
int otlm_initial_weights(otlm_handle h, int batch, int n, int k, const void* D, const void* y, void* w_out);

/* Objective of a solver state (w, g), in FP64 (Eq. OTLM with the reading above).
 * From (w, g): a = K u1, s = D w, f = eps log(s/a); the plan Q = diag(e^{f/eps}) K diag(e^{g/eps})
 * satisfies Q 1 = D w, so primal_out = eps KL(Q||K) + lam L(Q^T 1|y) + alpha R(w) is the value
 * of a feasible point (ELASTIC: alpha sum w + (beta/2)||w||^2 in place of alpha R(w)).  dual_out is the Fenchel dual
 *   -F1*(-f') - F2*(-g') - eps sum_ij K_ij (e^{(f'_i+g'_j)/eps} - 1)
 * at g' = the datafit step from K^T e^{f/eps} and f' = f shifted by the smallest constant that
 * makes it dual-feasible (l1 / no penalty), so dual_out <= optimum <= primal_out and
 * primal_out - dual_out is a duality gap.  BALANCED datafit: primal_out is +inf unless Q^T 1 = y.
 * POISSON: the dual takes g' = lam y / v' - lam (v' the prox value, -lam where y = 0), the datafit
 * step written so that lam + g' keeps its precision.
 * The two kernel applies run in FP32 (FP32 and BF16 handles) or FP64; all sums are FP64.
 *   w [batch][k], g [batch][n] as returned by otlm_solve; primal_out, dual_out [batch] device
 *   doubles.  Errors as otlm_solve. */
int otlm_objective(otlm_handle h, int batch, int n, int k,
                   const void* x, const void* D, const void* y,
                   double eps, double lam, double alpha,
                   const void* w, const void* g,
                   double* primal_out, double* dual_out);

/* Number of kernel launches the handle has queued since creation (instrumentation; the paper
 * has no counterpart).  NULL handle: -1. */
long long otlm_launch_count(otlm_handle h);

/* Device-time instrumentation (the paper has no counterpart).  When enabled, every launch a
 * solve or objective call queues is bracketed by two CUDA events on the handle's stream, and
 * the elapsed device time is accumulated per kernel kind: [0] kernel apply (a = K u1 and
 * b = K^T u2), [1] MM weight update + source step, [2] batch compaction, [3] set-up / finalize
 * / objective reductions.  otlm_get_timing writes the sums (milliseconds) and launch counts
 * into ms[4] and launches[4] (host arrays) and resets them; it waits for pending events.
 * Errors: OTLM_EINVAL (NULL arguments), OTLM_ECUDA (event creation or query failed). */
int otlm_set_timing(otlm_handle h, int enable);
int otlm_get_timing(otlm_handle h, double* ms, long long* launches);

/* FP32 solve that allocates nothing.  The paper has no counterpart: this entry point exists for
 * callers that cannot allocate device memory themselves -- code living inside a host framework
 * whose allocator owns the GPU's memory budget (an extra cudaMalloc could fail against the
 * framework's quota or fragment its pool), or latency-critical loops in which cudaMalloc/cudaFree
 * would synchronise the device.  It needs no handle: the caller passes inputs and outputs
 * (device pointers, same meaning and layout as otlm_solve, float only) plus the options a handle
 * would hold (datafit, penalty, max_iter, tol) and a cudaStream_t (NULL = default stream).
 * All workspace comes from one statically allocated 16 MiB __device__ array that every GPU
 * loading the library reserves until process exit; no cudaMalloc, cudaFree or allocating
 * library routine is called.  The problem fits when its workspace (about 4 * (5 batch*n + n*k
 * + batch*k + 8 batch) bytes) is at most 16 MiB, e.g. batch 64 at n = 4096 and k = 128;
 * larger problems return OTLM_ESCRATCH before any work is queued.
 * The first call on a device looks up the array's device address (with that device current)
 * and caches it; make that first call before any stream capture.  Every call on a device
 * shares the one array and it keeps the previous call's contents (each solve re-initialises
 * what it reads), so calls whose GPU work overlaps -- two streams, two host threads -- race.
 * The host waits at the convergence polls (every 8 iterations) like otlm_solve.
 * One MM step per iteration; the penalty is NONE, L1 or L2SQ (ELASTIC needs a beta this call
 * does not take).
 * Errors: OTLM_EINVAL (as otlm_solve, plus unknown datafit/penalty, ELASTIC, max_iter < 1),
 * OTLM_ESCRATCH, OTLM_ECUDA. */
int otlm_solve_noalloc(int batch, int n, int k, const float* x, const float* D, const float* y,
                       double eps, double lam, double alpha, int datafit, int penalty, int max_iter,
                       double tol, float* w, float* g, float* t_out, int* iters_out, float* err_out,
                       int* status_out, void* cuda_stream);

/* Static description of a status code; never NULL. */
/* Self-check of the tensor-core kernels' bounded waits (no fault and no hang: the waits are what is
 * exercised).  Runs one small BF16 GEMM (256 x 256 x 256, zero operands) on the one-SM kernel
 * (two_sm = 0) or the two-SM kernel (two_sm != 0) with a 20 ms wait limit, whose first CTA arms its
 * first ring stage but never issues the copies: the waits on that stage and the ones behind it run
 * out, the kernel records an error code and leaves after releasing its tensor memory, and the device
 * stays usable.  Returns OTLM_ETIMEOUT with the first recorded code in *code_out (1: operand copies,
 * 2: ring stage release, 3: accumulator), OTLM_OK if no expiry was detected (a defect),
 * OTLM_ENOMEM / OTLM_ECUDA, OTLM_EINVAL for a null code_out.  Allocates and frees about 1 MB and
 * a stream of its own. */
int otlm_check_wait_expiry(int two_sm, int* code_out);

const char* otlm_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* OTLM_H */
