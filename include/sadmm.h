/*
 * sadmm.h -- C ABI of the GB300 sharing-ADMM radar-imaging library.
 *
 * The library runs the per-iteration hot path of accelerated sharing ADMM
 * (ASADMM, "Distributed Radar Imaging Based on Accelerated ADMM", Section III)
 * on one GPU: for Q sensors with complex operators A_q (KM x N, Eq. 1) and
 * measurements y_q it iterates
 *
 *   x_q,J  <- (rho I + mu B_J^T B_J)^{-1} (mu B_J^T y'_q + rho v_J)      Eq. 3, x_q-update
 *             v = x_q - x_bar + z_bar - s, on the active set J_q only
 *   z_bar  <- soft(x_bar + s, lambda / rho)                               Eq. 3, x_G-update
 *   s      <- s + x_bar - z_bar                                           Eq. 3, dual update
 *   J_q    <- SSC(last Kp updates, eps_p) when ||eta_pri|| <= eps_pri       Eq. 3, selector update; Algorithm 1
 *
 * with B = [Re A; Im A] the real form of A, x_bar = mean_q x_q, x_G = Q z_bar
 * the output image and s the scaled dual (the paper's sigma = rho s, its
 * beta = rho).  Removed pixels keep their value (freeze_mode 0) and are folded
 * into y'_q = y_q - A_q,E x_q,E, or are set to zero (freeze_mode 1).
 *
 * Conventions
 *   - Complex data are interleaved float pairs (re, im): "complex64".
 *   - A_q is PIXEL-MAJOR: element (row r, pixel n) is at float offset
 *     2 * (n * K * M + r) (re) and 2 * (n * K * M + r) + 1 (im); row r = m K + k.
 *   - x vectors are float32, length N, pixel n = iy * nx + ix.
 *   - Pointers documented "host or device" may be either (unified virtual
 *     addressing, cudaMemcpyDefault); host memory may be pageable or pinned.
 *   - Every function returns SADMM_OK (0) or a negative status; no C++
 *     exception crosses this boundary.  sadmm_last_error() gives a message.
 *   - Work is issued on the context's stream (sadmm_set_stream); calls that
 *     return host-visible results synchronise that stream.
 *   - Memory: device buffers come from the allocator installed with
 *     sadmm_set_allocator (default cudaMalloc / cudaFree).
 */
#ifndef SADMM_H
#define SADMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SADMM_OK          0
#define SADMM_EINVAL     -1   /* invalid argument or size                     */
#define SADMM_ENOMEM     -2   /* device or host allocation failed             */
#define SADMM_ECUDA      -3   /* a CUDA runtime call or kernel launch failed  */
#define SADMM_ETIMEOUT   -4   /* a bounded device-side wait gave up           */
#define SADMM_ENOTREADY  -5   /* an operator has not been set                 */
#define SADMM_ENONFINITE -6   /* NaN or Inf in an input or an iterate         */

typedef struct sadmm_ctx* sadmm_t;

/* Method knobs.  Defaults (sadmm_default_criterion) are the paper's values
 * (Section IV): Kp = 5, eps_p = 1e-5, eps_abs = 1e-4, eps_rel = 1e-2; mu = 1. */
typedef struct {
  double mu;          /* data-fidelity weight of Eq. 2                                  */
  int    Kp;          /* Algorithm 1 window: number of past updates averaged (1..64)    */
  double eps_p;       /* Algorithm 1 tolerance: keep pixel i iff zeta_i >= eps_p         */
  double eps_abs;     /* absolute feasibility tolerance (gate of Algorithm 1, stop)      */
  double eps_rel;     /* relative feasibility tolerance                                 */
  int    elim;        /* 0 = plain SADMM, 1 = pixel elimination (ASADMM), 2 = ASADMM plus
                         the learned proposal and re-admission (sadmm_set_eliminator)   */
  int    freeze_mode; /* 0 = removed pixels keep their value, 1 = removed pixels set to 0 */
  int    stop;        /* 0 = ||X^{k+1}-X^k||_F <= tol ||X^{k+1}||_F; 1 = primal & dual
                         residuals below eps_pri and eps_dual (Boyd Sec. 3.3.1)          */
  int    precision;   /* operator used by the per-iteration products:
                         0 = complex64 (FP32), 1 = BF16 hi/lo pairs, 2 = FP16 hi/lo pairs,
                         3 = BF16 hi plane with the lo-plane products refreshed every
                         correct_every iterations, 4 = the same with FP16 planes.  With
                         planes, the method is solved for the pair operator hi + lo (exact
                         in FP32, within 2^-16 (BF16) or 2^-22 (FP16) of each entry): the
                         factor, its updates and the fold use it too, and the primal-form
                         adjoint passes g to the factor apply as an exact pair.  Changing
                         the operator form (sadmm_set_criterion) refactors on the next
                         solve. */
  int    correct_every; /* precision 3/4: lo-plane refresh period (>= 1)                    */
  /* elim = 2 (an extension; the paper has no counterpart).  Every learn_every
     iterations (once k >= max(Kp, 4)), before Algorithm 1's pass:
       - re-admission: a pixel i frozen in sensor q re-enters J_q when the step
         |mu Re(a_qi^H (A_q x_q - y_q)) + rho s_i| / (mu ||a_qi||^2 + rho) that a
         single-coordinate x-update would take exceeds readmit * eps_p (the pixel's
         entry of the optimality condition of Eq. 2 is then far from zero);
       - proposal: the network set by sadmm_set_eliminator maps six per-pixel
         features (sadmm_features) to p_i; p_i > learn_theta drops pixel i from
         every J_q, in addition to (and independently of the gate of) Algorithm 1.
     Re-admitted pixels are unfolded from y', their last Kp updates are set to
     2 eps_p, and the factors gain their columns.  Without a network, elim = 2
     runs as elim = 1. */
  int    learn_every;   /* default 10                                                   */
  double learn_theta;   /* default 0.5, in [0, 1]                                       */
  double readmit;       /* default 10 (>= 0); elim = 2 also needs eps_p > 0               */
  /* Removal policy (an extension; the paper runs Algorithm 1 every iteration):
     Algorithm 1's pass runs after iteration k only when k is a multiple of
     ssc_every (default 1), so that each factor update takes a batch of columns. */
  int    ssc_every;
  /* Formulation (an option; the paper's method is the sharing form of Eq. 2-3):
     0 = sharing ADMM (SADMM / ASADMM; output x_G = sum_q x_q);
     1 = consensus ADMM (CADMM / ACADMM, the sibling formulation of Section I,
     read as global consensus, Boyd et al. 2011 Sec. 7.1): every sensor images
     one common z, min sum_q mu/2 ||y_q - A_q x_q||^2 + lambda ||z||_1 with
     x_q = z, scaled duals u_q per sensor; x-update with v = z - u_q (the same
     system), z = soft(mean_q (x_q + u_q), lambda / (Q rho)), u_q += x_q - z,
     residuals of Boyd Sec. 7.1, Algorithm 1 per sensor as in the sharing form;
     output z.  elim = 2 needs the sharing form. */
  int    consensus;
} sadmm_criterion;

/* Per-solve summary. */
typedef struct {
  int    iters;        /* iterations run                                              */
  int    stop_reason;  /* 0 = iteration limit, 1 = relative change, 2 = residuals      */
  int    refreshes;    /* factor refreshes after active-set changes                    */
  int    active_total; /* sum_q |J_q| at the end                                       */
  int    learned_steps;/* learned proposal steps run (elim = 2)                        */
  int    readmitted;   /* (sensor, pixel) pairs re-admitted over the solve (elim = 2)  */
  double r_pri, eps_pri, d, eps_dual, relchange;   /* last iteration                    */
  double ms_total;     /* host wall time of the solve                                  */
  double ms_refresh;   /* of which: fold + factor refresh after set changes            */
  double bytes_iter;   /* algorithmic bytes read by the iteration kernels, summed      */
  int    proposed;     /* (sensor, pixel) pairs the learned proposal removed that
                          Algorithm 1 alone would have kept (elim = 2), since the start  */
  int    proposed_readmitted; /* of those, re-admitted later: the proposal's false
                          eliminations caught by the re-admission test                  */
} sadmm_stats;

/* One record per iteration of the last solve. */
typedef struct {
  int    k;            /* iterations completed                                         */
  int    gate;         /* 1 if Algorithm 1's test ran (elim on, k >= Kp, k a multiple of
                          ssc_every, r_pri <= eps_pri)                                  */
  int    changed;      /* number of sensors whose active set shrank                    */
  int    active_total; /* sum_q |J_q| after this iteration                             */
  int    learned;      /* 1 if the learned proposal ran in this iteration (elim = 2)   */
  int    readmitted;   /* (sensor, pixel) pairs re-admitted in this iteration          */
  double r_pri, eps_pri, d, eps_dual, relchange;
} sadmm_iter_record;

typedef void* (*sadmm_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void  (*sadmm_free_fn)(void* ptr, void* stream, void* user);

/* Fills *c with the defaults above. */
void sadmm_default_criterion(sadmm_criterion* c);

/* Installs the device allocator used by contexts created afterwards
 * (NULL, NULL restores cudaMalloc / cudaFree).  The functions are called with
 * the context's stream.  Not thread-safe against concurrent sadmm_create. */
int sadmm_set_allocator(sadmm_alloc_fn alloc, sadmm_free_fn release, void* user);

/* Creates a solver for Q sensors, M receivers, K fast-time samples and N pixels
 * on the current CUDA device (Eq. 1 sizes, Eq. 2 weights rho = beta, lambda).
 * Requirements: 1 <= Q <= 64, K*M a multiple of 32 and <= 16384, 1 <= N, rho > 0,
 * lambda >= 0, crit->mu > 0, 1 <= crit->Kp <= 64.  Allocates the device
 * state: about (8 K M N + 20 n^2) Q bytes with n = min(N, 2KM) (the operator,
 * the FP64 full-set factor with its scratch, its packed pair copy), 16 n^2 Q
 * more for the factors of shrunken sets when elim > 0 (allocated on first
 * need otherwise), 8 K M N Q more for split-precision planes, plus
 * O((Kp + 4) Q N).
 * crit may be NULL (defaults).  On failure *out is NULL. */
int sadmm_create(int Q, int M, int K, int N, double rho, double lambda,
                 const sadmm_criterion* crit, sadmm_t* out);

/* Replaces the method knobs of an existing context between solves (same
 * validity rules as sadmm_create), keeping its operators and its full-set
 * factors (refactored on the next solve only if mu or the operator form --
 * FP32 or BF16 / FP16 pairs -- changed), so that one
 * factorisation serves several forms of the method (plain, elimination,
 * split precision, learned).  Buffers the new knobs need are allocated on
 * first use; switching between BF16 and FP16 planes reconverts them.  The next
 * sadmm_solve starts from zero as usual (sadmm_resume after a change is not
 * supported).  SADMM_EINVAL for an invalid criterion, SADMM_ENOMEM if a
 * buffer cannot be allocated (the context keeps its previous criterion). */
int sadmm_set_criterion(sadmm_t ctx, const sadmm_criterion* crit);

/* Replaces lambda (Eq. 2) for the next solves; the factors do not depend on
 * it, so several scenes of one geometry (different measurements and lambda)
 * share one factorisation.  SADMM_EINVAL unless lambda is finite and >= 0. */
int sadmm_set_lambda(sadmm_t ctx, double lambda);

/* Uses `stream` (a cudaStream_t, may be NULL for the legacy default stream)
 * for all later work of this context. */
int sadmm_set_stream(sadmm_t ctx, void* stream);

/* Copies operator A_q (pixel-major complex64, N*K*M complex values; host or
 * device pointer) into the context and invalidates sensor q's factor. */
int sadmm_set_operator(sadmm_t ctx, int q, const float* A_q);

/* Operator A_q from the signal model of Section II (Eq. 1) instead of its
 * entries: receiver m, fast-time sample k and pixel n with round-trip delay
 * tau[m][n] (seconds; M x N doubles, host or device, copied) give
 * A_q[(m, k), n] = exp(j 2 pi tau[m][n] (f0 + k df)), row m K + k (f0 the chirp
 * start frequency, df = BW / K the frequency step per sample).  The library
 * forms A_q itself (phases in FP64, entries rounded to complex64, as
 * sadmm_set_operator would take them; the factor and the fold use it) and
 * the factors C[m][a][n] = exp(j 2 pi tau (f0 + 16 a df)) and
 * D[m][b][n] = exp(j 2 pi tau b df), whose products are the entries
 * k = 16 a + b.  While every sensor's operator was set this way (and the
 * criterion's precision is 0), the per-iteration forward and adjoint products
 * read C and D ((K/16 + 16) M N complex values instead of K M N) and form the
 * entries on the fly; see sadmm_set_products.  Requires K = 16, 32, 64, 128,
 * 256 or 512 (SADMM_EINVAL otherwise); invalidates sensor q's factor. */
int sadmm_set_operator_delays(sadmm_t ctx, int q, const double* tau, double f0, double df);

/* Composite back-projection image out[n] = sum_q |a_{q,n}^H y_q| (N floats,
 * host or device) from measurements y[0..Q-1] (K*M complex64 each, host or
 * device): the BP comparison images of Section IV (Fig. 1), read as each
 * sensor's matched filter taken in magnitude and added over the sensors.  It
 * uses the operator representation the per-iteration products use (see
 * sadmm_set_products) and leaves the solver state untouched.  Returns
 * SADMM_ENOTREADY if an operator is missing. */
int sadmm_backprojection(sadmm_t ctx, const float* const* y, float* out);

/* Which operator representation the per-iteration products read:
 * SADMM_PRODUCTS_AUTO (default): the factored tables when every sensor's
 * operator came from sadmm_set_operator_delays and precision is 0, else the
 * stored operator; SADMM_PRODUCTS_STORED: always the stored operator;
 * SADMM_PRODUCTS_FACTORED: the tables (a solve returns SADMM_ENOTREADY if a
 * sensor has none, SADMM_EINVAL if precision > 0).  SADMM_EINVAL for any
 * other mode. */
#define SADMM_PRODUCTS_AUTO 0
#define SADMM_PRODUCTS_STORED 1
#define SADMM_PRODUCTS_FACTORED 2
int sadmm_set_products(sadmm_t ctx, int mode);

/* Computes the full-active-set factor of every sensor whose operator changed:
 * (rho I + mu B B^T)^{-1} if N > 2KM, else (rho I + mu B^T B)^{-1}, in FP64
 * (Gram, Cholesky, explicit inverse).  It is kept and reused by later solves.
 * Called implicitly by sadmm_solve; returns SADMM_ENOTREADY if an operator
 * is missing. */
int sadmm_prepare(sadmm_t ctx);

/* Runs at most `iters` iterations from zero on measurements y[0..Q-1] (each
 * K*M complex64 values, host or device) and writes x_G = Q z_bar (N floats,
 * host or device; may be NULL).  tol is the stop-mode-0 relative-change
 * tolerance (<= 0 disables it).  st may be NULL. */
int sadmm_solve(sadmm_t ctx, const float* const* y, float* x_out, int iters, double tol,
                sadmm_stats* st);

/* Continues from the current state for at most `iters` more iterations
 * (same outputs as sadmm_solve). */
int sadmm_resume(sadmm_t ctx, float* x_out, int iters, double tol, sadmm_stats* st);

/* Copies x_q (N floats) to `out` (host or device). */
int sadmm_get_xq(sadmm_t ctx, int q, float* out);

/* Copies the active set J_q (sorted pixel indices, host or device int32 array
 * of capacity N) to idx and its size to *count (host). */
int sadmm_get_active(sadmm_t ctx, int q, int* idx, int* count);

/* Iteration records of the last solve/resume: copies up to cap records and
 * returns how many were written (or a negative status). */
int sadmm_history(sadmm_t ctx, sadmm_iter_record* out, int cap);

/* Checkpoint: serialises (k, x, x_bar, z_bar, s, the Kp-deep update ring, the
 * active sets and y', and in the consensus form the duals u) into host memory.
 * With buf == NULL only *bytes is set. */
int sadmm_get_state(sadmm_t ctx, void* buf, size_t* bytes);

/* Restores a checkpoint made by sadmm_get_state (same sizes and Kp).  Factors
 * are recomputed for active sets that are not full. */
int sadmm_set_state(sadmm_t ctx, const void* buf, size_t bytes);

/* Learned proposal network for elim = 2 (an extension; the paper has no
 * counterpart): params are sadmm_cnn_num_params() FP32 values (host or
 * device) in the flat layout of sadmm_cnn_set_params, for the H x W pixel grid
 * (H * W = N, pixel i at row i / W, column i % W).  The context keeps its own
 * copy (allocated with cudaMalloc, not the allocator hooks).  params = NULL
 * removes the network. */
int sadmm_set_eliminator(sadmm_t ctx, const float* params, int H, int W);

/* The six per-pixel features the network reads, at the current state after k
 * iterations: out (host or device) is 6 x N floats (NCHW with one image):
 *   c0 = log(1 + sum_q |x_qi|),  c1 = log(1 + max_q |x_qi|),
 *   c(2+j) = log10(||dx_i^(k-j)||_2 / eps_p + 1e-4) / 4,  j = 0..3,
 * dx^(t) being the update of iteration t over the sensors (zero when t < 1 or
 * j >= Kp; frozen pixels' updates are zero). */
int sadmm_features(sadmm_t ctx, float* out);

/* Profiling (tracing): when on, every kernel group of the iteration is
 * bracketed by CUDA events on the context's stream and its device time is
 * accumulated per phase.  Phases: 0 forward product (partials + reduction),
 * 1 Woodbury SPD apply, 2 adjoint + x-update (Woodbury form), 3 adjoint
 * (primal form), 4 SPD apply + x-update (primal form), 5 prox/dual/residuals,
 * 6 Algorithm 1 compaction (with the learned step's re-admission test and
 * network), 7 fold + factor refresh (and re-admission).  Turning it on resets
 * the totals. */
#define SADMM_NUM_PHASES 8
int sadmm_set_profiling(sadmm_t ctx, int on);

/* Copies min(cap, SADMM_NUM_PHASES) accumulated phase times (ms) and launch
 * counts; returns the number of phases copied. */
int sadmm_profile(sadmm_t ctx, double* ms, long long* launches, int cap);

/* Number of kernels this library has launched in this process. */
long long sadmm_launch_count(void);

/* Releases all device memory of the context. */
void sadmm_destroy(sadmm_t ctx);

const char* sadmm_strerror(int status);
const char* sadmm_last_error(void);

/* ------------------------------------------------------------------------
 * Batched form: S = 16 scenes sharing one geometry (the operators A_q, hence
 * the factors) iterate together; the forward and adjoint products become
 * GEMMs with 16 right-hand sides, so each operator byte read serves 16
 * scenes.  Plain SADMM (Eq. 3 without pixel elimination: every scene keeps
 * the full active set and the shared full-set factor), fixed iteration
 * count, one captured CUDA graph replayed per iteration.
 * ---------------------------------------------------------------------- */
typedef struct sadmm_batch_ctx* sadmm_batch_t;

/* S must be 16; lambda: S per-scene l1 weights; criterion as for
 * sadmm_create (elim and precision are ignored; consensus must be 0: SADMM_EINVAL). */
int sadmm_batch_create(int Q, int M, int K, int N, int S, double rho, const double* lambda,
                       const sadmm_criterion* crit, sadmm_batch_t* out);
int sadmm_batch_set_stream(sadmm_batch_t b, void* stream);
int sadmm_batch_set_operator(sadmm_batch_t b, int q, const float* A_q);
/* y: S x Q x KM complex64 (scene-major, host or device); x_out: S x N floats
 * (x_G of each scene, host or device, may be NULL). */
int sadmm_batch_solve(sadmm_batch_t b, const float* y, float* x_out, int iters, sadmm_stats* st);
int sadmm_batch_get_xq(sadmm_batch_t b, int scene, int q, float* out);
void sadmm_batch_destroy(sadmm_batch_t b);

/* Autotuner for the batched products' work decomposition (an extension; the
 * paper has no batched form).  The tensor-core GEMM tiles are fixed (128
 * operator rows or pixels x 16 scenes x 32-row K slabs); what is tuned is
 * how each GEMM's K range is split across persistent CTAs: the forward
 * product's pixel splits and the adjoint's real-row splits.  Each candidate
 * (up to eight per product, from a quarter to four times the default) is
 * launched `reps` times on the batch's stream with CUDA events around the
 * launches; the fastest is kept for every later solve and the captured graph
 * is rebuilt.  The operators must be set; the batch's state is reset by the
 * next solve.  out (may be NULL) receives the candidates, their mean times
 * per launch and the choice.  Errors: SADMM_EINVAL for reps < 1. */
typedef struct {
  int n_fwd, n_adj;              /* candidates tried */
  int fwd_splits[8], adj_splits[8];
  double fwd_ms[8], adj_ms[8];   /* mean time per launch (GEMM + its reduction) */
  int fwd_choice, adj_choice;    /* the splits kept */
  int fwd_default, adj_default;  /* the splits a batch starts with (always among the candidates) */
} sadmm_batch_tuning;
/* Returns SADMM_EINVAL for a NULL batch or reps < 1, SADMM_ENOTREADY if an
 * operator is missing, SADMM_ETIMEOUT if a tensor-core pipeline wait ran out
 * during the timed launches. */
int sadmm_batch_tune(sadmm_batch_t b, int reps, sadmm_batch_tuning* out);

/* A group of batches with different geometries (Q, M, K, N may all differ),
 * iterated together: one CUDA graph holds one iteration of every batch, each
 * batch on its own branch, so the GPU runs the batches' kernels side by side
 * and one graph launch advances every scene of every geometry by one
 * iteration.  The caller keeps ownership of the batches and must not destroy
 * one while the group exists; changing a batch (operator, stream, tuning)
 * makes the group rebuild its graph at the next solve.  At most 64 batches. */
typedef struct sadmm_batch_group_ctx* sadmm_batch_group_t;
int sadmm_batch_group_create(const sadmm_batch_t* batches, int n, sadmm_batch_group_t* out);
int sadmm_batch_group_set_stream(sadmm_batch_group_t g, void* stream);
/* y[i], x_out[i] and st[i] as for sadmm_batch_solve of batch i (x_out and st
 * may be NULL, and so may any x_out[i]); every batch runs `iters` iterations. */
int sadmm_batch_group_solve(sadmm_batch_group_t g, const float* const* y, float* const* x_out, int iters,
                            sadmm_stats* st);
void sadmm_batch_group_destroy(sadmm_batch_group_t g);

/* ------------------------------------------------------------------------
 * Learned elimination proposal (an extension; the paper has no counterpart):
 * a CNN over the H x W pixel grid with five 3x3 convolutions (6 -> 32, then
 * 32 -> 32, zero padding), GELU after each, a 1x1 head (32 -> 1) and a
 * sigmoid.  Weights are BF16-rounded copies of FP32 master parameters; sums
 * are FP32.  Flat parameter order: W1[32][6][3][3] b1[32] W2[32][32][3][3]
 * b2[32] ... W5 b5 Wh[32] bh[1] (sadmm_cnn_num_params() = 38785 floats).
 * Inputs are NCHW float32 (6 feature channels), outputs H x W probabilities.
 * ---------------------------------------------------------------------- */
typedef struct sadmm_cnn_ctx* sadmm_cnn_t;
int sadmm_cnn_create(int H, int W, int max_batch, sadmm_cnn_t* out);
int sadmm_cnn_num_params(void);
/* params: host or device FP32; resets the Adam state. */
int sadmm_cnn_set_params(sadmm_cnn_t c, const float* params);
/* rounded = 1: the BF16-rounded weights the kernels use; 0: FP32 masters. */
int sadmm_cnn_get_params(sadmm_cnn_t c, float* params, int rounded);
/* prob (device, B x H x W) = CNN(in) for in (device, B x 6 x H x W). */
int sadmm_cnn_forward(sadmm_cnn_t c, const float* in, int B, float* prob, void* stream);
/* Gradient (device, num_params floats) of the mean weighted binary
 * cross-entropy  -mean(w_i [y_i log p_i + (1-y_i) log(1-p_i)]),  w_i = pos_weight
 * for y_i = 1 else 1, with respect to the (rounded) weights; *loss (host) the
 * loss, may be NULL.  labels: device, B x H x W in {0, 1}. */
int sadmm_cnn_backward(sadmm_cnn_t c, const float* in, const float* labels, int B, double pos_weight,
                       float* grad, double* loss, void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the FP32 masters. */
int sadmm_cnn_adam_step(sadmm_cnn_t c, const float* grad, double lr, void* stream);
void sadmm_cnn_destroy(sadmm_cnn_t c);

/* ------------------------------------------------------------------------
 * Kernel-level entry points on DEVICE pointers (used by parity tests and for
 * composing other pipelines).  All work is on `stream`; none synchronises.
 * ---------------------------------------------------------------------- */

/* r = base - A_J v_J  (Eq. 1 forward product over the listed columns).
 * A: pixel-major complex64 (N x KM), idx: nidx pixel indices in [0, N)
 * (any order, repeats allowed), v: N floats indexed by pixel, base and r:
 * KM complex64 (base may be NULL for 0; r may alias base). */
int sadmm_forward(const float* A, int KM, int N, const int* idx, int nidx, const float* v,
                  const float* base, float* r, void* stream);

/* Same result as sadmm_forward, for callers that cannot allocate device
 * memory while they run (for example a real-time radar front end with a fixed
 * per-frame latency budget, where cudaMalloc/cudaFree may synchronise the
 * device, or a process whose device memory is rationed by another allocator).
 * The paper has no counterpart: this is a library-interface variant.
 * It allocates nothing: the partial sums go to one fixed 8 MiB device array
 * that every GPU loading this library holds until the process exits.  Sizes
 * whose partial sums (chunks x KM x 16 bytes: double-float pairs) exceed
 * 8 MiB are rejected with SADMM_EINVAL and a message naming the sizes.  Every
 * call looks up the array's device address on the calling device (a lookup
 * that allocates nothing), so the entry stays valid across a device reset.
 * All calls on a device share
 * the array and it keeps the last call's contents; every entry a call reads is
 * written earlier in the same call, so nothing needs clearing, but calls whose
 * work overlaps on the GPU (different streams, or different host threads) race
 * on it and must be serialised by the caller. */
int sadmm_forward_noalloc(const float* A, int KM, int N, const int* idx, int nidx,
                          const float* v, const float* base, float* r, void* stream);

/* g[p] = Re(a_{idx[p]}^H w) for p < nidx (adjoint of the real-input forward
 * product).  w: KM complex64 (KM even, <= 16384); g: nidx floats. */
int sadmm_adjoint(const float* A, int KM, int N, const int* idx, int nidx, const float* w,
                  float* g, void* stream);

/* The factored representation of sadmm_set_operator_delays at kernel level
 * (Section II, Eq. 1; all pointers are device pointers owned by the caller,
 * work is queued on `stream` and the call returns without synchronising).
 * sadmm_operator_tables: from tau (M x N doubles, row m holds the delays of
 * receiver m) writes A (N x KM complex64, pixel-major as sadmm_set_operator
 * takes it; may be NULL), C (M x K/16 x N complex64: C[m][a][n] =
 * exp(j 2 pi tau (f0 + 16 a df))) and D (M x 16 x N complex64: D[m][b][n] =
 * exp(j 2 pi tau b df)); C and D may both be NULL.  Phases are formed in
 * FP64 and rounded once.  K = 16, 32, ..., 512 (a power of two) for C and D;
 * SADMM_EINVAL for bad sizes, a NULL tau, or non-finite f0 / df. */
int sadmm_operator_tables(const double* tau, int M, int K, int N, double f0, double df, float* A, float* C,
                          float* D, void* stream);
/* r = base - A_J v_J with A given by its factors C, D (the layouts above; the
 * other arguments as for sadmm_forward).  Partial sums use stream-ordered
 * scratch that the call allocates and frees. */
int sadmm_forward_factored(const float* C, const float* D, int M, int K, int N, const int* idx, int nidx,
                           const float* v, const float* base, float* r, void* stream);
/* g[p] = Re(a_{idx[p]}^H w) with A given by its factors C, D (the layouts
 * above; the other arguments as for sadmm_adjoint; M K <= 16384, since w is
 * staged in shared memory). */
int sadmm_adjoint_factored(const float* C, const float* D, int M, int K, int N, const int* idx, int nidx,
                           const float* w, float* g, void* stream);

/* Factor of the x-update (Eq. 3, x_q-update) for the listed columns, in FP64:
 * if nidx > 2KM, F = (rho I + mu B_J B_J^T)^{-1} with B_J rows interleaved
 * (re, im) per sample (dimension n = 2KM, *form = 1); otherwise
 * F = (rho I + mu B_J^T B_J)^{-1} (n = nidx, *form = 0).  F is n x n,
 * row-major with leading dimension ldf >= roundup(n, 64), capacity
 * ldf * ldf doubles; the padding is overwritten.  form is a host pointer. */
int sadmm_factor(const float* A, int KM, int N, const int* idx, int nidx, double mu,
                 double rho, double* F, int ldf, int* form, void* stream);

/* The first step of sadmm_factor alone: F = mu G + rho I, the matrix of the
 * x-update system (Eq. 3, x_q-update), with G = B_J^T B_J (primal form, n =
 * nidx, when nidx <= 2KM) or G = B_J B_J^T (Woodbury form, n = 2KM), rows
 * interleaved (re, im) as in sadmm_factor; F row-major FP64 with leading
 * dimension ldf = roundup(n, 64), both triangles written, padding set to the
 * identity.  method 0 (what the solver's factor uses): tensor cores on exact
 * BF16 digit slices of the operator (each Gram row scaled by a power of two,
 * four 8-bit digits per entry, the ten digit products of orders 2..5, exact
 * integer chunk sums drained to double-float totals): within about 2^-36 of
 * each entry's row and column scale 2^(e_i + e_j), e_i the least exponent
 * with max |row i| <= 2^e_i; transient scratch of 4 x 2 bytes per padded
 * operand entry from the stream-ordered pool.  method 1: FP64 SIMT (KM a
 * multiple of 8).  Synchronises `stream`.  SADMM_EINVAL for bad sizes,
 * SADMM_ENOMEM without scratch, SADMM_ETIMEOUT if a bounded device wait
 * gave up.  form (host pointer, may be NULL) receives 1 for the Woodbury form. */
int sadmm_gram(const float* A, int KM, int N, const int* idx, int nidx, double mu, double rho, int method,
               double* F, int ldf, int* form, void* stream);

/* The batched form's factor apply with 16 right-hand sides (Eq. 3, x_q-update:
 * U = W R in the Woodbury form, H G in the primal form) on the tensor cores:
 * out[i][s] = sum_{j < n} F[i][j] U[j][s], i < n, s < 16.  F: device, n x n
 * FP64, row-major, leading dimension ld >= n (read, not modified); U: device,
 * n x 16 FP32 [row][s]; out: device, n x 16 FP64 [row][s].  Each row of F
 * and each column of U is scaled by a power of two (2^-e_i, 2^-f_s: the least
 * exponents with max_j |F_ij| <= 2^e_i and max_j |U_js| <= 2^f_s) and cut into
 * four exact 8-bit BF16 digits; the ten digit GEMMs of orders 0..3 run as
 * tcgen05 MMAs whose 256-term chunk sums are exact integers, drained to
 * double-float totals.  Error per entry at most about 5 * 2^-32 * n *
 * 2^(e_i + f_s); integer-valued F and U with |F_ij|, |U_js| <= 128 give the
 * exact product (up to 2^48).  Allocates and frees its scratch (cudaMalloc,
 * about 8 bytes per padded entry of F) and synchronises `stream`.
 * SADMM_EINVAL for bad arguments, SADMM_ETIMEOUT if a bounded device wait
 * gave up. */
int sadmm_digit_apply16(const double* F, int ld, int n, const float* U, double* out, void* stream);

/* Split-precision operator planes: for each of the 2 n_complex floats a of A,
 * hi = round(a) and lo = round(a - hi) in BF16 (kind 1) or FP16 (kind 2),
 * round-to-nearest; hi + lo is exact in FP32.  hi and lo: device arrays of
 * 2 n_complex 16-bit values in A's layout (pixel-major (re, im) pairs). */
int sadmm_split_operator(const float* A, size_t n_complex, int kind, void* hi, void* lo, void* stream);

/* r = base - P_idx v_idx with P = hi (planes 1), lo (planes 2) or hi + lo
 * (planes 3), FP32 accumulation (as sadmm_forward; KM a multiple of 4). */
int sadmm_forward_split(const void* hi, const void* lo, int kind, int planes, int KM, int N, const int* idx,
                        int nidx, const float* v, const float* base, float* r, void* stream);

/* g[p] = Re(P[:, idx[p]]^H w) with P as in sadmm_forward_split (KM <= 16384). */
int sadmm_adjoint_split(const void* hi, const void* lo, int kind, int planes, int KM, int N, const int* idx,
                        int nidx, const float* w, float* g, void* stream);

/* In-place rank-e downdate of a Woodbury-form factor after removing the e
 * columns E (pixel indices) from its active set (Eq. 3, x_q-update, with those
 * pixels frozen): W <- (W^{-1} - mu B_E B_E^T)^{-1} = W + mu T T^T with
 * P = W B_E, S = I - mu B_E^T P = L L^T, T = P L^{-T} (Woodbury identity),
 * in FP64, in passes of at most 32 columns.  W: 2KM x 2KM row-major FP64
 * (leading dimension 2KM), rows interleaved (re, im) as in sadmm_factor.
 * Returns SADMM_ENONFINITE if S is not numerically positive definite. */
int sadmm_factor_downdate(const float* A, int KM, const int* E, int e, double mu, double* W,
                          void* stream);

/* In-place rank-e update of a Woodbury-form factor.  sign = +1 removes the e
 * columns E (exactly sadmm_factor_downdate); sign = -1 adds them (pixels
 * re-admitted to the active set): W <- (W^{-1} + mu B_E B_E^T)^{-1} = W - mu T T^T
 * with P = W B_E, S = I + mu B_E^T P = L L^T, T = P L^{-T} (Woodbury identity).
 * Same layout, passes and errors as sadmm_factor_downdate. */
int sadmm_factor_update(const float* A, int KM, const int* E, int e, double mu, int sign, double* W,
                        void* stream);

/* out = F u for a symmetric n x n FP64 matrix (row-major, leading dimension
 * ldf even and >= n, n <= 49152; only the upper triangle is read) and FP32 u;
 * out rounded to FP32.  As in the solver, the upper triangle is first packed
 * into 64 x 64 tiles of FP32 pairs (hi, lo), and the products are formed
 * exactly and summed as FP32 pairs with the error-free two-sum (about 48
 * significant bits).  Allocates the packed copy and partial sums on `stream`
 * and synchronises it.  SADMM_ETIMEOUT if a tile copy did not complete. */
int sadmm_spd_apply(const double* F, int n, int ldf, const float* u, float* out, void* stream);

/* Failure-handling test hook (the paper has no counterpart).  Sets how many
 * times the symmetric factor apply (sadmm_spd_apply and the solver's x-update)
 * polls the barrier of each tile copy before it gives up and reports
 * SADMM_ETIMEOUT; polls < 0 restores the default (2^26).  A CTA that gives up
 * still waits, with the default limit, for the copy in flight into its shared
 * memory before it exits, so a short limit ends the apply early without
 * leaving work on the GPU.  It applies to the current device and to every
 * later launch until changed.  SADMM_ECUDA if the device value cannot be set. */
int sadmm_set_wait_limit(long long polls);

/* G = Re(A^H W) for one sensor and 16 right-hand sides on the tensor cores:
 * the adjoint product of the batched form (Eq. 3, x_q-update for 16 scenes),
 * the paper has no batched form.  A: device complex64, N x KM pixel-major (as
 * sadmm_set_operator); W: device complex64, KM x 16 ([row][scene]); G: device
 * float, N x 16 ([pixel][scene]).  Each operand is split into TF32 hi + lo and
 * hi*hi + hi*lo + lo*hi is accumulated in FP32 (tcgen05.mma kind::tf32), which
 * is within a few FP32 roundings of the FP32 product.  2KM must be a multiple
 * of 32.  Allocates a few bytes of scratch on `stream` and synchronises it;
 * SADMM_ETIMEOUT if a tensor-core wait timed out. */
int sadmm_adjoint16_tc(const float* A, int KM, int N, const float* W, float* G, void* stream);

/* The batched form's forward product on the tensor cores (Eq. 3, x_q-update:
 * the B v of r = y' - B v for 16 right-hand sides): R[m][s] = sum_p
 * A[p][m] V[p][s] (complex A, real V), m < KM, s < 16.  A: device,
 * pixel-major complex64 (N x KM); V: device, N x 16 FP32 [pixel][s]; R:
 * device, KM x 16 complex64 [m][s].  3xTF32 products (each within 2^-21 of
 * the FP32 one) accumulated in FP32 over the N pixels.  2KM must be a
 * multiple of 16.  Synchronises `stream`; SADMM_EINVAL for bad arguments,
 * SADMM_ETIMEOUT if a bounded device wait gave up. */
int sadmm_forward16_tc(const float* A, int KM, int N, const float* V, float* R, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SADMM_H */
